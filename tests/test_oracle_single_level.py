"""Single periodic level: the oracle's FAS iteration against plain definitions.

* the exact DFT solve is checked by applying the STENCIL (not the symbol)
  to its result, and against a single Fourier mode in closed form;
* the FAS V-cycle reaches the exact DFT solve (Sec. 3.2: it solves
  L u = f; the first step fixes the mean);
* at least one order of magnitude of residual reduction per V-cycle
  (Sec. 3.2, closing paragraph; golden fixture);
* the observed order of accuracy against the continuum solution equals the
  order of the FD operators (Table 1);
* the gradient agrees with its Fourier symbol.
"""

import os

import numpy as np
import pytest

from oracle.fft_solve import exact_solve, laplacian_symbol, spectral_gradient
from oracle.hierarchy import Level, fill_periodic, laplacian
from oracle.lpt import gradient
from oracle.hierarchy import Hierarchy
from oracle.multigrid import solve
from oracle.stencils import laplacian_symbol_1d
from synthetic import Geometry, make_delta_powerlaw

ORDERS = (2, 4, 6)


def _claims():
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_claims.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def _apply_stencil(phi, h, order):
    lev = Level(phi.shape, h, order, True)
    lev.interior[...] = phi
    fill_periodic(lev)
    return laplacian(lev)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 20, 8), (9, 10, 11)])
def test_exact_solve_satisfies_stencil(order, shape):
    rng = np.random.default_rng(3)
    f = rng.standard_normal(shape)
    f -= f.mean()
    h = 0.7
    phi = exact_solve(f, h, order)
    assert abs(phi.mean()) < 1e-14
    r = f - _apply_stencil(phi, h, order)
    assert np.max(np.abs(r)) < 1e-11 * np.max(np.abs(f))


@pytest.mark.parametrize("order", ORDERS)
def test_single_mode_closed_form(order):
    n, box = 24, 2.0
    h = box / n
    x = (np.arange(n) + 0.5) * h
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    k = 2 * np.pi / box * np.array([3, 1, 5])
    f = np.cos(k[0] * X + k[1] * Y + k[2] * Z)
    lam = sum(laplacian_symbol_1d(order, kk * h) for kk in k) / h ** 2
    phi = exact_solve(f, h, order)
    np.testing.assert_allclose(phi, f / lam, atol=1e-14 * np.max(np.abs(f / lam)) * 50)
    # the FAS iteration reaches the same closed form
    g = Geometry((n, n, n), box, order, ())
    phis, info = solve(g, [f], tol=1e-13, max_cycles=40)
    np.testing.assert_allclose(phis[0], f / lam, rtol=0, atol=1e-11 * np.max(np.abs(f / lam)))


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("n", [32, 24])
def test_fas_reaches_exact_dft_solve(order, n):
    d = make_delta_powerlaw((n,) * 3, 1)
    g = Geometry((n,) * 3, 1.0, order, ())
    phis, info = solve(g, [d], tol=1e-13, max_cycles=40)
    ex = exact_solve(d - d.mean(), 1.0 / n, order)
    rel = np.sqrt(np.mean((phis[0] - ex) ** 2) / np.mean(ex ** 2))
    assert rel < 1e-12
    hist = info["history"]
    reduction = _claims()["min_reduction_per_cycle"]
    for a, b in zip(hist[:-1], hist[1:]):
        assert a / b >= reduction, hist


def test_unigrid64_order2_reference_case():
    # the 64^3, 7-point, unit-RMS k^-2 case to 1e-10 relative residual
    d = make_delta_powerlaw((64,) * 3, 1)
    g = Geometry((64,) * 3, 1.0, 2, ())
    phis, info = solve(g, [d], tol=1e-10, max_cycles=30)
    assert info["rel_residual"] <= 1e-10
    assert info["cycles"] <= 10
    ex = exact_solve(d - d.mean(), 1.0 / 64, 2)
    rel = np.sqrt(np.mean((phis[0] - ex) ** 2) / np.mean(ex ** 2))
    assert rel < 1e-9


def _cell_avg_mode(n, box):
    h = box / n
    x = (np.arange(n) + 0.5) * h
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    k = 2 * np.pi / box
    fac = np.sin(k * h / 2) / (k * h / 2)
    sol = fac ** 3 * np.sin(k * X) * np.cos(k * Y) * np.sin(k * Z)
    return sol, -3 * k * k * sol


@pytest.mark.parametrize("order", ORDERS)
def test_observed_order_of_accuracy(order):
    errs = []
    sizes = (8, 16, 32) if order == 6 else (16, 32, 64)
    for n in sizes:
        sol, src = _cell_avg_mode(n, 1.0)
        phi = exact_solve(src, 1.0 / n, order)
        errs.append(np.sqrt(np.mean((phi - sol) ** 2)))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > order - 0.2), slopes
    assert np.all(slopes < order + 0.5), slopes


@pytest.mark.parametrize("order", ORDERS)
def test_gradient_matches_symbol(order):
    n = 20
    d = make_delta_powerlaw((n,) * 3, 4)
    h = 1.0 / n
    phi = exact_solve(d - d.mean(), h, order)
    g = Geometry((n,) * 3, 1.0, order, ())
    psi = gradient(Hierarchy(g), [phi])[0]
    ref = spectral_gradient(phi, h, order)
    for a in range(3):
        np.testing.assert_allclose(psi[a], ref[a], atol=1e-12 * np.max(np.abs(ref[a])))


def test_symbol_has_single_null_mode():
    lam = laplacian_symbol((8, 6, 10), 1.0, 6)
    assert np.sum(np.abs(lam) < 1e-12) == 1
    assert np.all(lam.flat[1:] < 0)
