"""FAS multigrid V-cycle on the composite grid (Sec. 3.2 and 3.3).

Steps per level l, starting at the finest (Sec. 3.2, enumerated algorithm):
coarsest level: exact solve; otherwise nu1 smoothing sweeps, residual
r = f_fas - L u, restriction of r and of u to the covered part of the parent,
tau-correction f_fas(l-1) = I r + L I u there (the parent's own source
elsewhere), recursion, correction u += inject(u(l-1) - I u), nu2 sweeps.

Readings where the paper is silent or ambiguous:
* smoother: red-black Gauss-Seidel with colour (i+j+k) mod 2 in the level's
  own indices, red first; within one colour every cell reads the values from
  before the half-sweep (exact red-black GS for the 7-point stencil; for the
  13/19-point stencils same-colour cells couple and this fixes the order);
* ghosts are refilled before every half-sweep and every residual;
* after each cycle every covered parent cell is set to the average of its
  children (finest first), then the convergence norm is taken: the
  volume-weighted L2 norm of f - L u over leaf cells (cells not covered by a
  finer level) divided by the same norm of f;
* the source is shifted by its composite leaf mean, the solvability
  condition of the periodic composite problem; covered cells of f hold the
  average of their children (they are never used by the iteration).
"""

import numpy as np

from .fft_solve import exact_solve
from .hierarchy import (Hierarchy, fill_ghosts, fill_periodic, inject,
                        laplacian, restrict)
from .stencils import LAPLACIAN_1D


def half_sweep(hier, l, colour, flux_fix=True):
    """One colour of red-black Gauss-Seidel on level l with source ffas."""
    lev = hier.levels[l]
    fill_ghosts(hier, l, flux_fix=flux_fix)
    w = LAPLACIAN_1D[lev.order]
    g = lev.g
    centre = 3.0 * w[g]
    offdiag = np.zeros(lev.n)
    for axis in range(3):
        for s in range(-g, g + 1):
            if s != 0:
                offdiag += w[s + g] * lev.shifted(axis, s)
    new = (lev.h * lev.h * lev.ffas - offdiag) / centre
    sel = lev.colour == colour
    lev.interior[sel] = new[sel]


def smooth(hier, l, sweeps, flux_fix=True):
    for _ in range(sweeps):
        half_sweep(hier, l, 0, flux_fix)
        half_sweep(hier, l, 1, flux_fix)


def coarsest_solve(hier):
    lev = hier.levels[0]
    lev.interior[...] = exact_solve(lev.ffas, lev.h, lev.order)
    fill_periodic(lev)


def vcycle(hier, l, nu1=2, nu2=2, flux_fix=True):
    if l == 0:
        coarsest_solve(hier)
        return
    lev = hier.levels[l]
    par = hier.levels[l - 1]
    smooth(hier, l, nu1, flux_fix)
    fill_ghosts(hier, l, flux_fix=flux_fix)
    r = lev.ffas - laplacian(lev)
    region = hier.covered_region(l)
    ubar = restrict(lev.interior)
    rbar = restrict(r)
    par.interior[region] = ubar
    lev.ubar = ubar
    if par.periodic:
        fill_periodic(par)
    lu = laplacian(par)
    if par.f is not None:
        par.ffas[...] = par.f
    par.ffas[region] = rbar + lu[region]
    vcycle(hier, l - 1, nu1, nu2, flux_fix)
    lev.interior[...] += inject(par.interior[region] - lev.ubar)
    smooth(hier, l, nu2, flux_fix)


def sync_covered(hier):
    """Covered parent cells := average of their children, finest level first."""
    for l in range(hier.finest, hier.base, -1):
        hier.levels[l - 1].interior[hier.covered_region(l)] = restrict(hier.levels[l].interior)


def leaf_residual_norms(hier, flux_fix=True, per_level=None):
    """(sqrt(sum h^3 r^2), sqrt(sum h^3 f^2)) over leaf cells, after sync.

    If per_level is a list, the pair (sum h^3 r^2, sum h^3 f^2) of every leaf level
    (base first) is appended to it: the per-level view of the same norm (reading of
    the "norm of the residual" stopping rule, Sec. 3.2)."""
    sync_covered(hier)
    num = den = 0.0
    for l in hier.leaf_levels():
        lev = hier.levels[l]
        fill_ghosts(hier, l, flux_fix=flux_fix)
        r = lev.f - laplacian(lev)
        mask = hier.uncovered_mask(l)
        vol = lev.h ** 3
        rr = vol * float(np.sum(r[mask] ** 2))
        ff = vol * float(np.sum(lev.f[mask] ** 2))
        num += rr
        den += ff
        if per_level is not None:
            per_level.append((rr, ff))
    return np.sqrt(num), np.sqrt(den)


def level_relative_residuals(pairs):
    """sqrt(rr) / sqrt(ff) per leaf level (the residual norm itself where ff = 0)."""
    return [np.sqrt(rr) / np.sqrt(ff) if ff > 0 else np.sqrt(rr) for rr, ff in pairs]


def composite_mean(hier, fields):
    total = 0.0
    for l, fld in zip(hier.leaf_levels(), fields):
        total += hier.levels[l].h ** 3 * float(np.sum(fld[hier.uncovered_mask(l)]))
    base = hier.levels[hier.base]
    return total / (base.h ** 3 * np.prod(base.n))


def prepare_source(hier, sources):
    """f on base and nests: given values, covered cells averaged from their
    children, minus the composite leaf mean."""
    leaf = list(hier.leaf_levels())
    fields = [np.array(s, dtype=np.float64, copy=True) for s in sources]
    for i in range(len(leaf) - 1, 0, -1):
        fields[i - 1][hier.covered_region(leaf[i])] = restrict(fields[i])
    mean = composite_mean(hier, fields)
    for l, fld in zip(leaf, fields):
        hier.levels[l].f[...] = fld - mean
    return mean


def solve(geom_or_hier, sources, tol=1e-10, max_cycles=50, nu1=2, nu2=2, cycles=None,
          flux_fix=True):
    """Solve L phi = f on the composite grid.

    sources: f on base and nests (base first).  With `cycles` set, exactly that
    many V-cycles run (matched-cycle parity); otherwise V-cycles run until the
    relative leaf residual is <= tol or max_cycles is reached.
    Returns (phi per leaf level, info dict)."""
    hier = geom_or_hier if isinstance(geom_or_hier, Hierarchy) else Hierarchy(geom_or_hier)
    prepare_source(hier, sources)
    for lev in hier.levels:
        lev.u[...] = 0.0
    hier.levels[hier.finest].ffas[...] = hier.levels[hier.finest].f
    history = []
    limit = cycles if cycles is not None else max_cycles
    rel = np.inf
    levels = []
    for _ in range(limit):
        vcycle(hier, hier.finest, nu1, nu2, flux_fix)
        pairs = []
        rnorm, fnorm = leaf_residual_norms(hier, flux_fix, per_level=pairs)
        rel = rnorm / fnorm if fnorm > 0 else rnorm
        history.append(rel)
        levels = level_relative_residuals(pairs)
        if cycles is None and rel <= tol:
            break
    phis = [hier.levels[l].interior.copy() for l in hier.leaf_levels()]
    return phis, {"cycles": len(history), "rel_residual": rel, "history": history,
                  "level_rel_residual": levels, "hierarchy": hier}
