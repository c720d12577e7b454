"""2LPT source and displacements of the oracle against closed forms (Sec. 3.1).

With phi = A cos(k1 x) + B cos(k2 y) the FD second derivatives are
phi_,xx = A lam(k1 h)/h^2 cos(k1 x), phi_,yy likewise, phi_,xy = 0, so
tau = A B lam1 lam2 / h^4 cos(k1 x) cos(k2 y).  With phi = cos(k (x + y)),
phi_,xx = phi_,yy = lam/h^2 cos and G_x G_y multiplies the mode by
(i g/h)^2, so tau = (lam^2/h^4 - g^4/h^4) cos^2: not zero, although the
continuum value is.  The trace of the FD Hessian is the FD Laplacian.
"""

import numpy as np
import pytest

from oracle.fft_solve import exact_solve
from oracle.hierarchy import Hierarchy, fill_ghosts, laplacian
from oracle.lpt import load_potential, lpt2_source, second_derivatives, solve_2lpt
from oracle.stencils import gradient_symbol_1d, laplacian_symbol_1d
from synthetic import Geometry, make_delta, make_delta_powerlaw, small_zoom

ORDERS = (2, 4, 6)


def _grid(n, box):
    h = box / n
    x = (np.arange(n) + 0.5) * h
    return h, np.meshgrid(x, x, x, indexing="ij")


@pytest.mark.parametrize("order", ORDERS)
def test_tau_two_mode_closed_form(order):
    n, box = 16, 1.0
    h, (X, Y, Z) = _grid(n, box)
    k1, k2 = 2 * np.pi * 3, 2 * np.pi * 2
    A, B = 0.7, -1.3
    phi = A * np.cos(k1 * X) + B * np.cos(k2 * Y)
    geom = Geometry((n,) * 3, box, order, ())
    tau = lpt2_source(Hierarchy(geom), [phi])[0]
    l1 = laplacian_symbol_1d(order, k1 * h) / h ** 2
    l2 = laplacian_symbol_1d(order, k2 * h) / h ** 2
    expect = A * B * l1 * l2 * np.cos(k1 * X) * np.cos(k2 * Y)
    np.testing.assert_allclose(tau, expect, atol=1e-9 * np.abs(expect).max())


@pytest.mark.parametrize("order", ORDERS)
def test_tau_diagonal_mode_closed_form(order):
    n, box = 16, 1.0
    h, (X, Y, Z) = _grid(n, box)
    k = 2 * np.pi * 3
    phi = np.cos(k * (X + Z))
    geom = Geometry((n,) * 3, box, order, ())
    tau = lpt2_source(Hierarchy(geom), [phi])[0]
    lam = laplacian_symbol_1d(order, k * h) / h ** 2
    gam = gradient_symbol_1d(order, k * h) / h
    expect = (lam * lam - gam ** 4) * np.cos(k * (X + Z)) ** 2
    np.testing.assert_allclose(tau, expect, atol=1e-9 * np.abs(expect).max())
    assert np.abs(expect).max() > 1.0  # the FD value differs from the continuum's 0


@pytest.mark.parametrize("order", ORDERS)
def test_hessian_trace_is_laplacian(order):
    geom = small_zoom(24, ((20, 7),), order=order, box=10.0)
    hier = Hierarchy(geom)
    rng = np.random.default_rng(2)
    phis = [rng.standard_normal(hier.levels[l].n) for l in hier.leaf_levels()]
    load_potential(hier, phis)
    for l in hier.leaf_levels():
        fill_ghosts(hier, l, edges=True)
        diag, mixed = second_derivatives(hier.levels[l])
        np.testing.assert_allclose(diag[0] + diag[1] + diag[2], laplacian(hier.levels[l]),
                                   atol=1e-9)


@pytest.mark.parametrize("order", ORDERS)
def test_second_solve_single_level_equals_dft(order):
    n = 16
    d = make_delta_powerlaw((n,) * 3, 3)
    h = 1.0 / n
    phi1 = exact_solve(d - d.mean(), h, order)
    geom = Geometry((n,) * 3, 1.0, order, ())
    tau = lpt2_source(Hierarchy(geom), [phi1])[0]
    phi2, info = solve_2lpt(geom, [phi1], tol=1e-13, max_cycles=40)
    ex = exact_solve(tau - tau.mean(), h, order)
    np.testing.assert_allclose(phi2[0], ex, atol=1e-11 * np.abs(ex).max())


def test_tau_is_invariant_under_sign_and_constant():
    geom = small_zoom(24, ((16, 6),), order=4, box=20.0)
    d = make_delta(geom, 9)
    t1 = lpt2_source(Hierarchy(geom), d)
    t2 = lpt2_source(Hierarchy(geom), [-x + 3.0 for x in d])
    for a, b in zip(t1, t2):
        np.testing.assert_allclose(a, b, atol=1e-12 * np.abs(a).max())
