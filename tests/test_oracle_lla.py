"""Pins of the local-Lagrangian-approximation oracle (Sec. 5.3): closed forms for
single Fourier modes of the potential (through the Table-1 symbols), the linear
limit rho - 1 -> -div L = L Phi, and mass conservation on a nested hierarchy."""

import numpy as np
import pytest

from oracle.hierarchy import Hierarchy, restrict
from oracle.lpt import lla_density
from oracle.multigrid import composite_mean, solve
from synthetic import Geometry, make_delta, small_zoom

N = 32


def _lap_symbol(order, t):
    """-(1D second-difference symbol) at phase t, from Table 1 (units 1/h^2)."""
    if order == 2:
        return 2.0 * (1.0 - np.cos(t))
    if order == 4:
        return (np.cos(2 * t) - 16.0 * np.cos(t) + 15.0) / 6.0
    return (-2.0 * np.cos(3 * t) + 27.0 * np.cos(2 * t) - 270.0 * np.cos(t) + 245.0) / 90.0


def _grad_symbol(order, t):
    """|1D gradient symbol| at phase t, from Table 1."""
    if order == 2:
        return np.sin(t)
    if order == 4:
        return (8.0 * np.sin(t) - np.sin(2 * t)) / 6.0
    return (45.0 * np.sin(t) - 9.0 * np.sin(2 * t) + np.sin(3 * t)) / 30.0


def _grid(n):
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return i, j, k


def test_zero_potential_gives_mean_density():
    geom = small_zoom(16, ((16, 4),), order=4, box=10.0)
    zero = [np.zeros(n) for n in [geom.base_n] + [ns.n for ns in geom.nests]]
    for rho in lla_density(Hierarchy(geom), zero):
        np.testing.assert_array_equal(rho, 1.0)


@pytest.mark.parametrize("order", (2, 4, 6))
def test_plane_wave(order):
    geom = Geometry((N,) * 3, 1.0, order, ())
    h = 1.0 / N
    i, _, _ = _grid(N)
    m = 3
    t = 2 * np.pi * m / N
    amp = 0.2 * h * h / _lap_symbol(order, t)     # Phi_,xx amplitude 0.2
    phi = amp * np.cos(t * i)
    raw = 1.0 / (1.0 + 0.2 * np.cos(t * i))       # det[1 - Phi_,xx] = 1 + 0.2 cos
    rho = lla_density(Hierarchy(geom), [phi])[0]
    np.testing.assert_allclose(rho, raw + (1.0 - raw.mean()), rtol=0, atol=1e-12)
    assert abs(rho.mean() - 1.0) < 1e-13


@pytest.mark.parametrize("order", (2, 6))
def test_diagonal_mode(order):
    geom = Geometry((N,) * 3, 1.0, order, ())
    h = 1.0 / N
    i, j, _ = _grid(N)
    t = 2 * np.pi * 2 / N
    a = 0.05
    phi = a * np.cos(t * (i + j))
    c = np.cos(t * (i + j))
    hxx = -a * _lap_symbol(order, t) / (h * h) * c   # = Phi_,yy
    hxy = -a * (_grad_symbol(order, t) / h) ** 2 * c
    raw = 1.0 / ((1.0 - hxx) ** 2 - hxy ** 2)
    rho = lla_density(Hierarchy(geom), [phi])[0]
    np.testing.assert_allclose(rho, raw + (1.0 - raw.mean()), rtol=0, atol=1e-11)


def test_linear_limit_is_the_laplacian():
    geom = Geometry((N,) * 3, 1.0, 4, ())
    rng = np.random.Generator(np.random.PCG64(5))
    d = rng.standard_normal((N,) * 3)
    phi, _ = solve(geom, [d], tol=1e-12)
    errs = []
    for eps in (1e-4, 5e-5):
        rho = lla_density(Hierarchy(geom), [eps * phi[0]])[0]
        # first order: 1/det(I - H) = 1 + tr H + O(H^2), tr H = L Phi = eps * (d - <d>)
        errs.append(np.abs(rho - 1.0 - eps * (d - d.mean())).max())
    assert errs[0] / errs[1] > 3.5   # second order in eps


def test_two_potentials_combine_linearly_and_mass_is_conserved():
    geom = small_zoom(24, ((20, 7),), order=6, box=50.0)
    deltas = make_delta(geom, 9)
    phi1, _ = solve(geom, deltas, tol=1e-10)
    phi2, _ = solve(geom, [0.3 * x for x in deltas], tol=1e-10)
    h = Hierarchy(geom)
    a = lla_density(h, phi1, phi2, 0.02, 0.01)
    b = lla_density(Hierarchy(geom), [0.02 * p + 0.01 * q for p, q in zip(phi1, phi2)])
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-14)
    hh = Hierarchy(geom)
    assert abs(composite_mean(hh, a) - 1.0) < 1e-13
    # covered parent cells hold the mean of their children
    np.testing.assert_allclose(a[0][hh.covered_region(hh.base + 1)], restrict(a[1]), atol=1e-14)
    assert np.std(a[1]) > 1e-3
