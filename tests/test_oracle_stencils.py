"""Pins of the oracle's operator tables against mathematics and the paper.

Table 1 stencils are pinned by polynomial exactness (Taylor order); the
Fourier symbols are pinned to the stencils by a direct DFT of the stencil and
to the continuum operator at small k; Table 2 fluxes by telescoping to
Table 1; Lagrange weights by polynomial reproduction; and the paper's
printed attenuation numbers at k_Ny/2 (Sec. 3.4.1) by a golden fixture.
"""

import os

import numpy as np
import pytest

from oracle import stencils as st

ORDERS = (2, 4, 6)


@pytest.mark.parametrize("order", ORDERS)
def test_laplacian_taylor_order(order):
    # exact on x^p for p <= order + 1 (even stencil: odd terms vanish), wrong at p = order + 2
    w = st.LAPLACIAN_1D[order]
    g = order // 2
    offs = np.arange(-g, g + 1, dtype=np.float64)
    x0 = 0.37
    for p in range(order + 2):
        val = np.sum(w * (x0 + offs) ** p)
        exact = p * (p - 1) * x0 ** (p - 2) if p >= 2 else 0.0
        assert val == pytest.approx(exact, abs=1e-9), (order, p)
    p = order + 2
    val = np.sum(w * (x0 + offs) ** p)
    assert abs(val - p * (p - 1) * x0 ** (p - 2)) > 1e-6


@pytest.mark.parametrize("order", ORDERS)
def test_gradient_taylor_order(order):
    w = st.GRADIENT_1D[order]
    g = order // 2
    offs = np.arange(-g, g + 1, dtype=np.float64)
    x0 = -0.21
    for p in range(order + 1):
        val = np.sum(w * (x0 + offs) ** p)
        exact = p * x0 ** (p - 1) if p >= 1 else 0.0
        assert val == pytest.approx(exact, abs=1e-9), (order, p)
    p = order + 1
    assert abs(np.sum(w * (x0 + offs) ** p) - p * x0 ** (p - 1)) > 1e-6


@pytest.mark.parametrize("order", ORDERS)
def test_symbols_are_dft_of_stencils(order):
    g = order // 2
    offs = np.arange(-g, g + 1)
    theta = np.linspace(-np.pi, np.pi, 41)
    # numpy convention: a mode exp(+i theta x) is multiplied by sum_s w_s exp(+i theta s)
    lap = np.array([np.sum(st.LAPLACIAN_1D[order] * np.exp(1j * t * offs)) for t in theta])
    grad = np.array([np.sum(st.GRADIENT_1D[order] * np.exp(1j * t * offs)) for t in theta])
    np.testing.assert_allclose(lap.real, st.laplacian_symbol_1d(order, theta), atol=1e-12)
    np.testing.assert_allclose(lap.imag, 0.0, atol=1e-12)
    np.testing.assert_allclose(grad.imag, st.gradient_symbol_1d(order, theta), atol=1e-12)
    np.testing.assert_allclose(grad.real, 0.0, atol=1e-12)


@pytest.mark.parametrize("order", ORDERS)
def test_symbols_match_continuum_at_small_k(order):
    t = 1e-2
    # -k^2 and k up to O(theta^(n+2)) and O(theta^(n+1))
    assert abs(st.laplacian_symbol_1d(order, t) + t * t) < 10 * t ** (order + 2)
    assert abs(st.gradient_symbol_1d(order, t) - t) < 10 * t ** (order + 1)


@pytest.mark.parametrize("order", ORDERS)
def test_flux_telescopes_to_laplacian(order):
    F = st.FLUX_1D[order]
    g = order // 2
    # F_{i+1/2} on cells i-g+1..i+g ; F_{i-1/2} on cells i-g..i+g-1 ; difference on i-g..i+g
    lap = np.zeros(2 * g + 1)
    lap[1:] += F
    lap[:-1] -= F
    np.testing.assert_allclose(lap, st.LAPLACIAN_1D[order], atol=1e-14)
    # a face gradient: exact slope for a linear profile
    cells = np.arange(-g + 1, g + 1, dtype=np.float64)
    assert np.sum(F * (3.0 * cells + 1.0)) == pytest.approx(3.0, abs=1e-13)


def test_printed_flux_rows_have_mixed_signs():
    # Table 2 as printed: [-1 1], [-1 15 -15 1]/12, [2 -25 245 -245 25 -2]/180.
    printed = {2: np.array([-1.0, 1.0]), 4: np.array([-1.0, 15, -15, 1]) / 12,
               6: np.array([2.0, -25, 245, -245, 25, -2]) / 180}
    for order, row in printed.items():
        lap = np.convolve([-1.0, 1.0], row)
        sign = 1.0 if order == 2 else -1.0
        np.testing.assert_allclose(lap, sign * st.LAPLACIAN_1D[order][::-1], atol=1e-14)
        np.testing.assert_allclose(st.FLUX_1D[order], sign * row, atol=1e-15)


@pytest.mark.parametrize("order", ORDERS)
def test_lagrange_weights_reproduce_polynomials(order):
    tw = st.tangential_weights(order)
    half = order // 2
    nodes = np.arange(-half, half + 1, dtype=np.float64)
    for parity, x in ((0, -0.25), (1, 0.25)):
        for p in range(order + 1):
            assert np.sum(tw[parity] * nodes ** p) == pytest.approx(x ** p, abs=1e-13)
    cw, fw = st.normal_weights(order)
    cn = np.array([-(2.0 * m + 1) for m in range(half)])
    fn = np.array([q + 0.5 for q in range(half + 1)])
    for m in range(half):
        x = -(m + 0.5)
        for p in range(order + 1):
            val = np.sum(cw[m] * cn ** p) + np.sum(fw[m] * fn ** p)
            assert val == pytest.approx(x ** p, abs=1e-11)


def test_order2_normal_weights_are_martin_cartwright_quadratic():
    # one coarse point at -h (fine units -1), fine points at 1/2, 3/2, ghost at -1/2
    cw, fw = st.normal_weights(2)
    np.testing.assert_allclose(cw[0], [8.0 / 15.0], atol=1e-15)
    np.testing.assert_allclose(fw[0], [2.0 / 3.0, -1.0 / 5.0], atol=1e-15)


def _golden(name):
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_attenuation_at_half_nyquist_matches_paper():
    rows = _golden("attenuation_kny_half.txt")
    theta = np.pi / 2
    for order_s, lo, hi in rows:
        order = int(order_s)
        # from the stencils themselves (a sampled mode), not from the symbol formulas
        g = order // 2
        offs = np.arange(-g, g + 1)
        lap = np.sum(st.LAPLACIAN_1D[order] * np.cos(theta * offs))
        grad = np.sum(st.GRADIENT_1D[order] * np.sin(theta * offs))
        ratio = (grad / abs(lap)) / (1.0 / theta)
        assert float(lo) <= ratio <= float(hi), (order, ratio)
    # and the closed-form values quoted in the design notes
    for order, expect in ((2, 0.7854), (4, 0.8976), (6, 0.9511)):
        r = st.gradient_symbol_1d(order, theta) * theta / abs(st.laplacian_symbol_1d(order, theta))
        assert r == pytest.approx(expect, abs=1e-4)
