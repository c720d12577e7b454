"""Autotuner for the mixed-precision schedule, the smoother tile and the batch's
launch mode.

For MG_MIXED the float32 V-cycles are only the inner solver of a float64
iterative refinement whose stopping test (the float64 leaf residual) fixes the
accuracy, so their schedule is free: float32 V-cycles per refinement step
(inner_cycles), pre/post smoothing sweeps of those cycles (nu1, nu2), and the
smoother's thread-block tile (32 z-pairs x tile_rows rows).

Two tuners:
* tune_batch: per size class, the whole step (1LPT, 2LPT, displacements) of the
  class's median hierarchy timed alone for every candidate; the fastest that
  converges.  Cheap, but a hierarchy alone is not a hierarchy in a batch, where
  small members' launches overlap the large members' work.
* tune_batch_joint: coordinate descent on the batch itself: starting from the
  default schedule, each size class in turn (largest total work first) tries
  each candidate schedule while the others keep theirs, and each launch mode of
  the batch (per-operation graphs, or the persistent launch for the classes up to
  a size at a grid of k blocks per SM) is tried; a change is kept only if the
  whole batch's measured step time falls by more than `gain`.
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


JOINT_SPACE = ((2, 2, 2, 4), (3, 2, 2, 4), (4, 2, 1, 4), (3, 1, 1, 4), (6, 1, 1, 4),
               (4, 2, 2, 2), (4, 2, 2, 8))
DEFAULT_PARAMS = (4, 2, 2, 4)
# launch modes: (name, classes whose members join the persistent launch, blocks per SM)
LAUNCH_MODES = (("graphs", (), 0), ("persistent_xs_s", ("xs", "s"), 3),
                ("persistent_xs", ("xs",), 2))


def time_batch(geoms, deltas, sched, tol, mode=LAUNCH_MODES[0], reps=2):
    """Median seconds of the whole batched step with schedule sched ({class: params})
    and launch mode `mode`; None if a member did not converge."""
    import torch
    _, pers, bps = mode
    hs = []
    try:
        for g in geoms:
            c = size_class(g)
            inner, nu1, nu2, rows = sched[c]
            hs.append(mg.Hierarchy(mg.config_from_geometry(
                g, tol=tol, max_cycles=50, precision=mg.MG_MIXED, inner_cycles=inner, nu1=nu1,
                nu2=nu2, tile_rows=rows, persistent=c in pers)))
        b = mg.Batch(hs)
        b.set_persistent_blocks(bps)
        outs, i1, i2 = b.pipeline(deltas, allow_noconv=True)
        if any(x["rel_residual"] > tol for x in i1 + i2):
            b.close()
            return None
        times = []
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            b.pipeline(deltas, outs)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        b.close()
        return statistics.median(times)
    finally:
        for h in hs:
            h.close()


def tune_batch_joint(geoms, deltas, tol, space=JOINT_SPACE, modes=LAUNCH_MODES, reps=2,
                     gain=0.02, budget_s=90.0):
    """(schedule {class: params}, launch mode, log of (what, seconds)) by coordinate
    descent on the batch's measured step time; stops trying once budget_s has passed."""
    t_start = time.perf_counter()
    classes = sorted({size_class(g) for g in geoms},
                     key=lambda c: -sum(g.level_cells() for g in geoms if size_class(g) == c))
    sched = {c: DEFAULT_PARAMS for c in classes}
    mode = modes[0]
    best = time_batch(geoms, deltas, sched, tol, mode, reps)
    log = [("default", best)]
    for c in classes:
        for cand in space:
            if cand == sched[c] or time.perf_counter() - t_start > budget_s:
                continue
            trial = dict(sched)
            trial[c] = cand
            t = time_batch(geoms, deltas, trial, tol, mode, reps)
            log.append(("%s=%s" % (c, cand), t))
            if t is not None and t < best * (1.0 - gain):
                sched, best = trial, t
    for m in modes[1:]:
        if time.perf_counter() - t_start > budget_s:
            break
        t = time_batch(geoms, deltas, sched, tol, m, reps)
        log.append(("mode=%s" % m[0], t))
        if t is not None and t < best * (1.0 - gain):
            mode, best = m, t
    return sched, mode, log

