"""Nested (composite) grids: the oracle against invariants of Sec. 3.3.

* ghost interpolation is exact on polynomials of degree <= n (Sec. 3.3: the
  interpolating polynomial has the order of the FD scheme), with and without
  the flux step for fields the parent flux already matches;
* after a ghost fill the mean of the 4 fine fluxes under each parent face
  element equals the parent flux (flux matching, Sec. 3.3);
* hence the composite operator is conservative: sum over leaf cells of
  h^3 L u vanishes for ANY u on a periodic base (divergence theorem, Sec. 3.3);
* >= 10x residual reduction per V-cycle with nests of any depth (Sec. 3.3,
  last paragraph); without flux matching the residual stalls (Sec. 3.3);
* the nested solution agrees with a unigrid solve of the degraded source
  (Sec. 4.4: restriction + re-injection makes the solve independent of the
  refinement) away from the coarse-fine boundary.
"""

import os

import numpy as np
import pytest

from oracle.fft_solve import exact_solve, spectral_gradient
from oracle.hierarchy import Hierarchy, fill_ghosts, inject, laplacian
from oracle.lpt import gradient
from oracle.multigrid import leaf_residual_norms, solve, sync_covered
from oracle.stencils import FLUX_1D
from synthetic import make_delta, small_zoom

ORDERS = (2, 4, 6)
CHAINS = [((16, 4),), ((20, 7), (16, 6)), ((12, 6),)]


def _claims():
    out = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_claims.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


def _poly(X, Y, Z, degree):
    rng = np.random.default_rng(degree)
    out = np.zeros_like(X)
    for i in range(degree + 1):
        for j in range(degree + 1 - i):
            for k in range(degree + 1 - i - j):
                out += rng.uniform(-1, 1) * X ** i * Y ** j * Z ** k
    return out


def _centres(lev, origin, extra=0):
    g = lev.g
    ax = [origin[a] + (np.arange(-extra, lev.n[a] + extra) + 0.5) * lev.h for a in range(3)]
    return np.meshgrid(*ax, indexing="ij")


def _fill_with(hier, l, fun):
    """Write fun(centres) into level l's interior (parent coordinates built from offsets)."""
    origin = np.zeros(3)
    for m in range(hier.base + 1, l + 1):
        origin = origin + np.array(hier.levels[m].off) * hier.levels[m - 1].h
    X, Y, Z = _centres(hier.levels[l], origin)
    hier.levels[l].interior[...] = fun(X, Y, Z)
    return origin


@pytest.mark.parametrize("order", ORDERS)
def test_ghost_interpolation_exact_on_polynomials(order):
    geom = small_zoom(24, ((20, 7),), order=order, box=1.0)
    hier = Hierarchy(geom)
    fun = lambda X, Y, Z: _poly(X, Y, Z, order)  # noqa: E731
    _fill_with(hier, hier.base, fun)
    origin = _fill_with(hier, hier.finest, fun)
    lev = hier.levels[hier.finest]
    fill_ghosts(hier, hier.finest, edges=True, flux_fix=False)
    X, Y, Z = _centres(lev, origin, extra=lev.g)
    expect = fun(X, Y, Z)
    # the parent's covered cells were overwritten by child averages; ghosts read uncovered
    # parent cells for faces, so only face ghosts are exact here
    g, n = lev.g, lev.n
    outside = np.zeros(lev.u.shape, dtype=int)
    for a in range(3):
        idx = np.arange(-g, n[a] + g)
        sh = [1, 1, 1]
        sh[a] = -1
        outside = outside + ((idx < 0) | (idx >= n[a])).reshape(sh)
    face = outside == 1
    np.testing.assert_allclose(lev.u[face], expect[face], atol=1e-11)


@pytest.mark.parametrize("order", ORDERS)
def test_edge_ghosts_exact_on_separable_polynomials(order):
    geom = small_zoom(24, ((20, 7),), order=order, box=1.0)
    hier = Hierarchy(geom)
    # a tensor-degree-n polynomial whose 8-child averages equal the parent's samples
    # only for degree <= 1; use an affine field so covered parent cells stay exact
    fun = lambda X, Y, Z: 0.3 + 1.1 * X - 0.7 * Y + 0.2 * Z  # noqa: E731
    _fill_with(hier, hier.base, fun)
    origin = _fill_with(hier, hier.finest, fun)
    lev = hier.levels[hier.finest]
    fill_ghosts(hier, hier.finest, edges=True, flux_fix=True)
    X, Y, Z = _centres(lev, origin, extra=lev.g)
    expect = fun(X, Y, Z)
    np.testing.assert_allclose(lev.u, expect, atol=1e-12)


def _face_fluxes(hier, l):
    """(mean of 4 fine fluxes, parent flux) for every face element of nest l."""
    lev, par = hier.levels[l], hier.levels[l - 1]
    F = FLUX_1D[lev.order]
    half, g, n, off = lev.order // 2, lev.g, lev.n, lev.off
    U = par.interior
    out = []
    for a in range(3):
        b, c = [x for x in range(3) if x != a]
        for side in (0, 1):
            face = g if side == 0 else g + n[a]
            ff = 0.0
            for s in range(lev.order):
                sl = [slice(g, g + n[0]), slice(g, g + n[1]), slice(g, g + n[2])]
                sl[a] = face - half + s
                ff = ff + F[s] * lev.u[tuple(sl)]
            ff = ff / lev.h
            pface = off[a] if side == 0 else off[a] + n[a] // 2
            fc = 0.0
            for s in range(lev.order):
                plane = np.take(U, pface - half + s, axis=a)
                fc = fc + F[s] * plane[off[b]:off[b] + n[b] // 2, off[c]:off[c] + n[c] // 2]
            fc = fc / par.h
            mean = ff.reshape(n[b] // 2, 2, n[c] // 2, 2).mean(axis=(1, 3))
            out.append((mean, fc))
    return out


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("chain", CHAINS)
def test_flux_matching_and_conservation(order, chain):
    geom = small_zoom(24, chain, order=order, box=3.0)
    hier = Hierarchy(geom)
    rng = np.random.default_rng(11)
    for l in hier.leaf_levels():
        hier.levels[l].interior[...] = rng.standard_normal(hier.levels[l].n)
    sync_covered(hier)
    total = 0.0
    scale = 0.0
    for l in hier.leaf_levels():
        fill_ghosts(hier, l)
        if l > hier.base:
            for mean, fc in _face_fluxes(hier, l):
                np.testing.assert_allclose(mean, fc, atol=1e-12 * np.max(np.abs(fc)))
    for l in hier.leaf_levels():
        lev = hier.levels[l]
        lu = laplacian(lev)
        mask = hier.uncovered_mask(l)
        total += lev.h ** 3 * np.sum(lu[mask])
        scale += lev.h ** 3 * np.sum(np.abs(lu[mask]))
    assert abs(total) < 1e-13 * scale


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("chain", CHAINS)
def test_nested_convergence_rate(order, chain):
    geom = small_zoom(24, chain, order=order, box=50.0)
    d = make_delta(geom, 5)
    phis, info = solve(geom, d, tol=1e-12, max_cycles=30)
    hist = info["history"]
    assert info["rel_residual"] <= 1e-12
    reduction = _claims()["min_reduction_per_cycle_nested"]
    for a, b in zip(hist[:-1], hist[1:]):
        assert a / b >= reduction, hist
    # gauge: zero mean over the base level (covered cells hold child averages)
    hier = info["hierarchy"]
    base = hier.levels[hier.base].interior
    assert abs(base.mean()) < 1e-12 * np.abs(base).max()


def test_no_flux_matching_stalls():
    geom = small_zoom(24, ((16, 4),), order=2, box=50.0)
    d = make_delta(geom, 5)
    phis, info = solve(geom, d, cycles=12, flux_fix=False)
    floor = _claims()["noflux_residual_floor"]
    assert min(info["history"]) > floor
    phis, info = solve(geom, d, cycles=12, flux_fix=True)
    assert info["history"][-1] < 1e-11


@pytest.mark.parametrize("order", (2, 6))
def test_degraded_unigrid_agreement(order):
    n = 32
    geom = small_zoom(n, ((n, n // 4),), order=order, box=100.0)
    d = make_delta(geom, 5)
    phis, info = solve(geom, d, tol=1e-13, max_cycles=40)
    psi = gradient(Hierarchy(geom), phis)
    fine = inject(d[0])
    o = n // 2
    fine[o:o + n, o:o + n, o:o + n] = d[1]
    h = 100.0 / (2 * n)
    ex = exact_solve(fine - fine.mean(), h, order)
    gex = spectral_gradient(ex, h, order)
    for a in range(3):
        ref = gex[a][o:o + n, o:o + n, o:o + n]
        diff = psi[1][a] - ref
        whole = np.sqrt(np.mean(diff ** 2)) / np.std(ref)
        inner = np.sqrt(np.mean(diff[6:-6, 6:-6, 6:-6] ** 2)) / np.std(ref)
        assert whole < 5e-2, whole
        assert inner < 1e-2, inner
        assert inner < whole / 4  # errors are concentrated at the coarse-fine boundary


def _cellavg_fields(n, h, origin):
    k = 2 * np.pi
    ax = [origin + (np.arange(n) + 0.5) * h for _ in range(3)]
    X, Y, Z = np.meshgrid(*ax, indexing="ij")
    fac = np.sin(k * h / 2) / (k * h / 2)
    sol = fac ** 2 * np.sin(k * X) * np.cos(k * Y)
    return sol, -2 * k * k * sol


@pytest.mark.parametrize("order,min_slope", [(2, 1.8), (4, 2.8), (6, 2.5)])
def test_composite_observed_order(order, min_slope):
    errs = []
    for n in (16, 32, 64):
        # nest of n/2 cells (n/4 parent cells) at offset 3n/8: margin >= 6 parent cells
        geom = small_zoom(n, ((n // 2, 3 * n // 8),), order=order, box=1.0)
        sb, fb = _cellavg_fields(n, 1.0 / n, 0.0)
        sn, fn = _cellavg_fields(n // 2, 0.5 / n, (3 * n // 8) / n)
        phis, _ = solve(geom, [fb, fn], tol=1e-13, max_cycles=40)
        errs.append(max(np.sqrt(np.mean((phis[0] - sb) ** 2)), np.sqrt(np.mean((phis[1] - sn) ** 2))))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(slopes > min_slope), slopes


def test_residual_norm_counts_leaf_cells_only():
    geom = small_zoom(16, ((16, 4),), order=2, box=1.0)
    hier = Hierarchy(geom)
    for l in hier.leaf_levels():
        hier.levels[l].f[...] = 1.0
    # a source only on covered base cells must not enter the norm
    hier.levels[hier.base].f[...] = 0.0
    hier.levels[hier.base].f[hier.covered_region(hier.finest)] = 5.0
    hier.levels[hier.finest].f[...] = 0.0
    rn, fn = leaf_residual_norms(hier)
    assert fn == 0.0 and rn == 0.0


def _smooth_source(n, box):
    h = box / n
    x = (np.arange(n) + 0.5) * h
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    t = 2 * np.pi / box
    return (np.cos(t * X) * np.cos(2 * t * Y) + 0.5 * np.sin(3 * t * Z + 0.3)
            + 0.3 * np.cos(t * (X + Z)))


@pytest.mark.parametrize("order,bound", [(2, 1e-2), (4, 5e-4)])
def test_nested_solution_tends_to_unigrid_as_the_patch_grows(order, bound):
    """A smooth source sampled on a periodic grid of spacing h/2 and solved exactly
    there (the unigrid solution) against the composite solve on a base of spacing h
    (source: the children means) with a centred nest at h/2 (source: the fine samples):
    inside the nest the two agree better the larger the nest (Sec. 3.3: the nest only
    sees the coarse discretisation through its boundary), and better at order 4."""
    from synthetic import Geometry, NestSpec
    n, box = 32, 1.0
    fine = _smooth_source(2 * n, box)
    uni = exact_solve(fine - fine.mean(), box / (2 * n), order)
    base = fine.reshape(n, 2, n, 2, n, 2).mean(axis=(1, 3, 5))
    errs = []
    for side in (8, 16, 24):           # nest extent in parent cells, centred
        off = (n - side) // 2
        sl = tuple(slice(2 * off, 2 * (off + side)) for _ in range(3))
        geom = Geometry((n,) * 3, box, order, (NestSpec((2 * side,) * 3, (off,) * 3),))
        phis, info = solve(geom, [base, fine[sl]], tol=1e-11)
        assert info["rel_residual"] <= 1e-11
        ref = uni[sl]
        d = phis[1] - ref
        d -= d.mean()                   # the two gauges differ by a constant
        errs.append(np.sqrt(np.mean(d ** 2) / np.mean((ref - ref.mean()) ** 2)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[0] < bound


# ---- non-cubic periodic base (the base's volume is h^3 n0 n1 n2, not box^3) --------

def _noncubic(order, nest=True):
    """24 x 32 x 40 periodic base (box = length of axis 0); optionally a nest of
    16 x 20 x 24 cells (8 x 10 x 12 parent cells) with a margin of >= 6 parent cells."""
    from synthetic import Geometry, NestSpec
    nests = (NestSpec((16, 20, 24), (8, 11, 14)),) if nest else ()
    return Geometry((24, 32, 40), 30.0, order, nests)


@pytest.mark.parametrize("order", ORDERS)
def test_prepared_source_has_zero_composite_integral_on_noncubic_base(order):
    """After the mean removal (solvability of the periodic composite problem, reading
    of Sec. 3.2) the volume-weighted sum of f over leaf cells vanishes, whatever the
    aspect ratio of the base."""
    from oracle.multigrid import prepare_source
    geom = _noncubic(order)
    hier = Hierarchy(geom)
    rng = np.random.default_rng(21)
    src = [rng.standard_normal(hier.levels[l].n) + 0.7 for l in hier.leaf_levels()]
    mean = prepare_source(hier, src)
    total = scale = 0.0
    for l in hier.leaf_levels():
        lev = hier.levels[l]
        mask = hier.uncovered_mask(l)
        total += lev.h ** 3 * np.sum(lev.f[mask])
        scale += lev.h ** 3 * np.sum(np.abs(lev.f[mask]))
    assert abs(total) < 1e-13 * scale
    assert 0.5 < mean < 0.9   # the +0.7 offset, up to the noise's own mean


@pytest.mark.parametrize("order", ORDERS)
def test_constant_source_vanishes_on_noncubic_base(order):
    """A constant source is its own composite mean: the prepared source is zero on
    every level and the solve returns phi = 0 (to rounding)."""
    from oracle.multigrid import prepare_source
    geom = _noncubic(order)
    hier = Hierarchy(geom)
    c = 2.5
    mean = prepare_source(hier, [np.full(hier.levels[l].n, c) for l in hier.leaf_levels()])
    assert abs(mean - c) < 1e-14 * c
    for l in hier.leaf_levels():
        assert np.max(np.abs(hier.levels[l].f)) < 1e-13 * c
    phis, _ = solve(geom, [np.full(hier.levels[l].n, c) for l in hier.leaf_levels()], cycles=2)
    for p in phis:
        assert np.max(np.abs(p)) < 1e-10


@pytest.mark.parametrize("order", ORDERS)
def test_noncubic_single_level_fas_reaches_exact_dft_solve(order):
    """On one periodic 24 x 32 x 40 level the FAS iteration reaches the DFT solve of
    the same discrete operator (the plain definition of the result)."""
    geom = _noncubic(order, nest=False)
    rng = np.random.default_rng(5)
    f = rng.standard_normal(geom.base_n) + 0.3
    phis, info = solve(geom, [f], tol=1e-13, max_cycles=40)
    ex = exact_solve(f - f.mean(), geom.box / geom.base_n[0], order)
    rel = np.sqrt(np.mean((phis[0] - ex) ** 2) / np.mean(ex ** 2))
    assert rel < 1e-12
    hier = info["hierarchy"]
    assert abs(hier.levels[hier.base].f.mean()) < 1e-14


@pytest.mark.parametrize("order", ORDERS)
def test_noncubic_nested_convergence_rate(order):
    geom = _noncubic(order)
    d = make_delta(geom, 9)
    phis, info = solve(geom, d, tol=1e-12, max_cycles=30)
    assert info["rel_residual"] <= 1e-12
    reduction = _claims()["min_reduction_per_cycle_nested"]
    hist = info["history"]
    for a, b in zip(hist[:-1], hist[1:]):
        assert a / b >= reduction, hist


# ---- edge and corner ghosts on a field with tensor cross-terms ---------------------

def _tensor_linear(X, Y, Z):
    """A product of per-axis linear factors: its 8-child mean equals its value at the
    parent centre, so covered parent cells stay exact after the two-way sync, while the
    cross-terms xy, yz, xz, xyz are non-zero (an additive edge rule is not exact)."""
    return (0.4 + 1.3 * X) * (0.9 - 1.1 * Y) * (-0.6 + 0.8 * Z)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("noncubic", [False, True])
def test_edge_ghosts_exact_on_tensor_linear_field(order, noncubic):
    """Every ghost of a nest (faces after the flux step, edges and corners by tensor
    interpolation of parent data, reading R10) reproduces a field that is linear along
    each axis, including its mixed terms, which the mixed derivatives of the 2LPT source
    (Sec. 3.1.2) read at the edges."""
    geom = _noncubic(order) if noncubic else small_zoom(24, ((20, 7),), order=order, box=1.0)
    hier = Hierarchy(geom)
    _fill_with(hier, hier.base, _tensor_linear)
    origin = _fill_with(hier, hier.finest, _tensor_linear)
    lev = hier.levels[hier.finest]
    fill_ghosts(hier, hier.finest, edges=True, flux_fix=True)
    X, Y, Z = _centres(lev, origin, extra=lev.g)
    expect = _tensor_linear(X, Y, Z)
    np.testing.assert_allclose(lev.u, expect, atol=1e-12)


def test_per_level_residual_norms_add_up_to_the_leaf_norm():
    """The per-level sums of the leaf residual norm (reading of the Sec. 3.2 stopping
    rule, level by level) add up to the composite norm, and a residual that lives on
    one level's leaf cells shows up on that level only."""
    from oracle.multigrid import level_relative_residuals
    geom = small_zoom(24, ((20, 7), (16, 6)), order=4, box=50.0)
    hier = Hierarchy(geom)
    rng = np.random.default_rng(4)
    for l in hier.leaf_levels():
        hier.levels[l].f[...] = rng.standard_normal(hier.levels[l].n)
        hier.levels[l].interior[...] = rng.standard_normal(hier.levels[l].n)
    pairs = []
    rn, fn = leaf_residual_norms(hier, per_level=pairs)
    assert len(pairs) == 3
    assert abs(np.sqrt(sum(p[0] for p in pairs)) - rn) < 1e-13 * rn
    assert abs(np.sqrt(sum(p[1] for p in pairs)) - fn) < 1e-13 * fn
    # u = 0 and a source on the finest level only: relative residual 1 there, 0 elsewhere
    for l in hier.leaf_levels():
        hier.levels[l].u[...] = 0.0
        hier.levels[l].f[...] = 0.0
    hier.levels[hier.finest].f[...] = 1.0
    pairs = []
    leaf_residual_norms(hier, per_level=pairs)
    rel = level_relative_residuals(pairs)
    assert rel[0] == 0.0 and rel[1] == 0.0
    assert abs(rel[2] - 1.0) < 1e-14
