"""Planted mistakes in the oracle must fail at least one pin.

Each test patches one plausible error into the oracle (on the CPU, for the
duration of the test only) and checks that the pin written for that part of
the method catches it: a transposed interpolation weight, a dropped flux
term, a wrong restriction, a shifted injection, a reversed gradient, a wrong
mixed derivative, a wrong smoother diagonal, a cubic volume in the composite mean,
edge ghosts without their tensor cross-terms.
"""

import numpy as np
import pytest

import oracle.hierarchy as hy
import oracle.lpt as lpt
import oracle.multigrid as mg
import oracle.stencils as st
from tests import test_oracle_lpt as t_lpt
from tests import test_oracle_nested as t_nested
from tests import test_oracle_single_level as t_single


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_swapped_tangential_parity_is_caught(monkeypatch):
    good = st.tangential_weights

    def swapped(order):
        w = good(order)
        return {0: w[1], 1: w[0]}

    monkeypatch.setattr(hy, "tangential_weights", swapped)
    _fails(t_nested.test_ghost_interpolation_exact_on_polynomials, 4)


def test_reversed_normal_layers_are_caught(monkeypatch):
    good = st.normal_weights

    def reversed_layers(order):
        cw, fw = good(order)
        return cw[::-1].copy(), fw[::-1].copy()

    monkeypatch.setattr(hy, "normal_weights", reversed_layers)
    _fails(t_nested.test_ghost_interpolation_exact_on_polynomials, 6)


def test_dropped_flux_term_is_caught(monkeypatch):
    table = dict(st.FLUX_1D)
    table[4] = np.array([0.0, -15.0, 15.0, 0.0]) / 12.0
    monkeypatch.setattr(hy, "FLUX_1D", table)
    _fails(t_nested.test_flux_matching_and_conservation, 4, ((16, 4),))


def test_flux_shift_on_wrong_side_is_caught(monkeypatch):
    original = hy.fill_coarse_fine

    def no_fix(hier, l, edges=False, flux_fix=True):
        return original(hier, l, edges=edges, flux_fix=False)

    monkeypatch.setattr(hy, "fill_coarse_fine", no_fix)
    _fails(t_nested.test_flux_matching_and_conservation, 2, ((16, 4),))


def test_first_child_restriction_is_caught(monkeypatch):
    def first_child(fine):
        return fine[::2, ::2, ::2].copy()

    monkeypatch.setattr(mg, "restrict", first_child)
    _fails(t_single.test_fas_reaches_exact_dft_solve, 2, 24)


def test_shifted_injection_is_caught(monkeypatch):
    good = hy.inject

    def shifted(coarse):
        return np.roll(good(coarse), 1, axis=0)

    monkeypatch.setattr(mg, "inject", shifted)
    _fails(t_single.test_fas_reaches_exact_dft_solve, 4, 24)


def test_wrong_smoother_diagonal_is_caught(monkeypatch):
    table = dict(st.LAPLACIAN_1D)
    bad = table[6].copy()
    bad[3] *= 0.5
    table[6] = bad
    monkeypatch.setattr(mg, "LAPLACIAN_1D", table)
    with np.errstate(over="ignore", invalid="ignore"):   # the mutated iteration diverges
        _fails(t_single.test_fas_reaches_exact_dft_solve, 6, 24)


def test_reversed_gradient_is_caught(monkeypatch):
    table = {k: v[::-1].copy() for k, v in st.GRADIENT_1D.items()}
    monkeypatch.setattr(lpt, "GRADIENT_1D", table)
    _fails(t_single.test_gradient_matches_symbol, 4)


def test_mixed_derivative_as_product_is_caught(monkeypatch):
    good = lpt.second_derivatives

    def product_of_gradients(lev):
        diag, mixed = good(lev)
        w = st.GRADIENT_1D[lev.order]
        grads = []
        for a in range(3):
            acc = np.zeros(lev.n)
            for s in range(-lev.g, lev.g + 1):
                acc += w[s + lev.g] * lev.shifted(a, s)
            grads.append(acc / lev.h)
        bad = {(a, b): grads[a] * grads[b] for (a, b) in mixed}
        return diag, bad

    monkeypatch.setattr(lpt, "second_derivatives", product_of_gradients)
    _fails(t_lpt.test_tau_diagonal_mode_closed_form, 2)


def test_cubic_volume_in_composite_mean_is_caught(monkeypatch):
    """The composite mean divided by box^3 instead of the base's volume h^3 n0 n1 n2
    agrees on cubic bases only; the non-cubic pins catch it."""
    def box_cubed(hier, fields):
        total = 0.0
        for l, fld in zip(hier.leaf_levels(), fields):
            total += hier.levels[l].h ** 3 * float(np.sum(fld[hier.uncovered_mask(l)]))
        return total / hier.box ** 3

    monkeypatch.setattr(mg, "composite_mean", box_cubed)
    _fails(t_nested.test_constant_source_vanishes_on_noncubic_base, 4)
    _fails(t_nested.test_prepared_source_has_zero_composite_integral_on_noncubic_base, 2)


def _additive_edges(lev, U, tw, half):
    """Edge and corner ghosts from the neighbouring face ghosts and interior cells,
    u(x) = sum_a u(x with the other outside axes clamped) - (m - 1) u(all clamped):
    exact for affine fields, wrong by the cross-terms of a product field."""
    g, n = lev.g, lev.n
    idx = [np.arange(-g, n[a] + g) for a in range(3)]
    I = np.meshgrid(*idx, indexing="ij")
    out = [(I[a] < 0) | (I[a] >= n[a]) for a in range(3)]
    cl = [np.clip(I[a], 0, n[a] - 1) for a in range(3)]
    count = out[0].astype(int) + out[1] + out[2]
    sel = count >= 2
    u = lev.u.copy()
    acc = np.zeros(u.shape)
    for a in range(3):
        pos = [np.where(out[b] & (b != a), cl[b], I[b]) + g for b in range(3)]
        acc += np.where(out[a], u[pos[0], pos[1], pos[2]], 0.0)
    allc = [cl[b] + g for b in range(3)]
    acc -= (count - 1) * u[allc[0], allc[1], allc[2]]
    lev.u[sel] = acc[sel]


def test_additive_edge_rule_is_caught(monkeypatch):
    """Edges that drop the tensor cross-terms pass the affine pin but fail the
    product-field pin."""
    monkeypatch.setattr(hy, "_fill_edges", _additive_edges)
    t_nested.test_edge_ghosts_exact_on_separable_polynomials(4)   # affine: still exact
    _fails(t_nested.test_edge_ghosts_exact_on_tensor_linear_field, 4, False)
    _fails(t_nested.test_edge_ghosts_exact_on_tensor_linear_field, 2, True)
