"""Autotuner for the mixed-precision schedule and the smoother tile.

For MG_MIXED the float32 V-cycles are only the inner solver of a float64
iterative refinement whose stopping test (the float64 leaf residual) fixes the
accuracy, so their schedule is free: float32 V-cycles per refinement step
(inner_cycles), pre/post smoothing sweeps of those cycles (nu1, nu2), and the
smoother's thread-block tile (32 z-pairs x tile_rows rows).  The tuner times the
whole step (1LPT, 2LPT, displacements) of a representative hierarchy of each
size class for every candidate and keeps the fastest that converges.
"""

import statistics
import time

from . import mg

DEFAULT_SPACE = tuple((inner, nu1, nu2, rows)
                      for inner in (2, 3, 4)
                      for (nu1, nu2) in ((1, 1), (2, 1), (2, 2))
                      for rows in (2, 4, 8))

# Size classes by level-cells (upper bounds).
CLASSES = (("xs", 3e5), ("s", 1e6), ("m", 3e6), ("l", float("inf")))


def size_class(geom):
    cells = geom.level_cells()
    for name, bound in CLASSES:
        if cells < bound:
            return name
    return CLASSES[-1][0]


def config(geom, params, tol, max_cycles=50):
    inner, nu1, nu2, rows = params
    return mg.config_from_geometry(geom, tol=tol, max_cycles=max_cycles, precision=mg.MG_MIXED,
                                   inner_cycles=inner, nu1=nu1, nu2=nu2, tile_rows=rows)


def time_candidate(geom, deltas, params, tol, reps=2):
    """Median ms of the whole step with these parameters (None if it did not converge)."""
    import torch
    h = mg.Hierarchy(config(geom, params, tol))
    try:
        out, i1, i2 = h.pipeline(deltas, allow_noconv=True)
        if i1["rel_residual"] > tol or i2["rel_residual"] > tol:
            return None
        times = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h.pipeline(deltas, out)
            torch.cuda.synchronize()
            times.append((time.perf_counter() - t0) * 1e3)
        return statistics.median(times)
    finally:
        h.close()


def tune(geom, deltas, tol, space=DEFAULT_SPACE, reps=2):
    """(best parameters, {parameters: ms}) for one hierarchy."""
    table = {}
    for params in space:
        table[params] = time_candidate(geom, deltas, params, tol, reps)
    ok = {p: t for p, t in table.items() if t is not None}
    if not ok:
        raise RuntimeError("no candidate schedule converged")
    return min(ok, key=ok.get), table


def representatives(geoms):
    """Index of the median-size member of every size class present."""
    by = {}
    for i, g in enumerate(geoms):
        by.setdefault(size_class(g), []).append(i)
    reps = {}
    for name, idx in by.items():
        idx = sorted(idx, key=lambda i: geoms[i].level_cells())
        reps[name] = idx[len(idx) // 2]
    return reps


def tune_batch(geoms, deltas, tol, space=DEFAULT_SPACE, reps=2):
    """{size class: best parameters}, tuned on one representative per class."""
    best = {}
    for name, i in representatives(geoms).items():
        best[name], _ = tune(geoms[i], deltas[i], tol, space, reps)
    return best


def batch_configs(geoms, best, tol):
    return [config(g, best[size_class(g)], tol) for g in geoms]
