#!/usr/bin/env python
"""Benchmark of the nested-grid initial-conditions step on GB300.

One step = the whole hot path on one hierarchy: 1LPT solve of L phi1 = delta,
2LPT source tau(phi1), 2LPT solve of L phi2 = tau, displacements -G phi1 and
-G phi2 (float64, order-6 operators).  Workload: 128^3 periodic base of a
100 Mpc/h box plus one centred 128^3 nest at twice the resolution (4,194,304
level-cells), BBKS density at z = 50 from seeded white noise.  Each solve
stops at a relative leaf residual of 1e-7, which gives <= 1e-6 RMS relative
error in phi and in the displacements (checked by the GPU tests).

Default: N = 1, 10 timed steps after 3 warm-up steps.  Under torchrun every
rank solves its own hierarchy (replicas, no collective in the data path);
value = level-cells of all ranks / max-over-ranks time.

--impl reference times the CPU oracle on a bounded sample of the same
workload (one V-cycle per step, scaled to the cycles of a full step).
"""

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "level-cells solved/s to 1e-6 rel. error; % HBM peak; p50/p99 solve latency"
UNIT = "level-cells/s"
SOLVE_TOL = 1e-7
SEED = 2
BATCH_SEED = 1000
SERVE_SEED = 5
# float32 V-cycles per float64 refinement step in the mixed-precision variant
MIXED_INNER_CYCLES = 4
# V-cycles of one full step (1LPT + 2LPT; unigrid64: 1LPT) at each workload's
# stopping rule, as the GPU arm reports them; the oracle arm scales its one-cycle
# sample by this.
CYCLES_PER_STEP = {"zoom2": 14, "unigrid64": 9, "deep_zoom": 14, "zoom256": 14}
FP64_PEAK_GOPS = 625.0   # nominal 1.25 TFLOP/s FP64 = 625 G FP64 instructions/s
HBM_PEAK_GBS = 6765.0    # measured copy bandwidth of the GB300s
L2_FLUSH_BYTES = 256 << 20

# smoother: FP64 instructions per updated cell (three 6-neighbour sums: 15 adds,
# a_f * f: 1 multiply, 3 fused multiply-adds) for the order-6 stencil
SMOOTH_OPS_PER_UPDATE = {2: 7, 4: 13, 6: 19}
# in-place algorithmic bytes of one colour half-sweep per level-cell: read u of
# both colours (8 B), f of the updated colour (4 B), write the updated colour (4 B)
SMOOTH_BYTES_PER_CELL = 16.0
# DRAM bytes (read + write) per updated cell of k_smooth_half<6,double> from one ncu
# capture of the 128^3 launch; scaled per launch by
# the updated cells.  Set to None whenever the kernel changes.
SMOOTH_TRAFFIC_PER_UPDATE = 35.8
# the same for k_smooth_half<6,float> (ncu capture of the 128^3 nest launch) and for
# k_smooth_half_tma<6,float> (capture of the 256^3 nest launch)
SMOOTH_F32_TRAFFIC_PER_UPDATE = 17.8
SMOOTH_TMA_F32_TRAFFIC_PER_UPDATE = 22.3
# float32 levels of at least this many cells that are not periodic take the
# TMA-staged smoother by default
TMA_MIN_CELLS = 1 << 23


# Workloads: zoom2 is the headline; the others are the single-level and deep-zoom
# configurations, measured with --workload.  Seeds and stopping rules per workload.
WORKLOADS = ("zoom2", "unigrid64", "deep_zoom", "zoom256")
WORKLOAD_SEED = {"zoom2": SEED, "unigrid64": 1, "deep_zoom": 3, "zoom256": 4}
WORKLOAD_TOL = {"zoom2": SOLVE_TOL, "unigrid64": 1e-10, "deep_zoom": SOLVE_TOL,
                "zoom256": SOLVE_TOL}
WORKLOAD_TEXT = {
    "zoom2": "zoom2: 128^3 periodic base (100 Mpc/h) + centred 128^3 nest at 2x, order-6 FD, "
             "FP64, 1LPT+2LPT+displacements, BBKS z=50, seed 2",
    "unigrid64": "unigrid64: 64^3 periodic, 7-point Laplacian, FP64, 1LPT (phi and -grad phi) "
                 "to 1e-10 relative residual, power law P ~ k^-2 at unit RMS, seed 1",
    "deep_zoom": "deep zoom: 128^3 periodic base (100 Mpc/h) + 4 nests of 128^3, centred with "
                 "+-16 jitter (seed 3), order-6 FD, FP64, 1LPT+2LPT+displacements, BBKS z=50",
    "zoom256": "zoom256: 256^3 periodic base (200 Mpc/h) + centred 256^3 nest at 2x, order-6 FD, "
               "FP64, 1LPT+2LPT+displacements, BBKS z=50, seed 4 (the size of the serving "
               "configuration's large levels; its float32 nest takes the TMA-staged smoother)",
}


def workload(name="zoom2"):
    from synthetic import config_deep_zoom, config_unigrid64, config_zoom2
    return {"zoom2": config_zoom2, "unigrid64": config_unigrid64, "deep_zoom": config_deep_zoom,
            "zoom256": lambda: config_zoom2(base=256, nest=256, box=200.0)}[name]()


def workload_inputs(name, geom):
    from synthetic import make_delta, make_delta_powerlaw
    if name == "unigrid64":
        return [make_delta_powerlaw(tuple(geom.base_n), WORKLOAD_SEED[name])]
    return make_delta(geom, WORKLOAD_SEED[name])


def workload_config(geom, name="zoom2"):
    return {"workload": WORKLOAD_TEXT[name],
            "level_cells": geom.level_cells(), "order": geom.order, "levels": geom.n_levels,
            "solve_tol": WORKLOAD_TOL[name], "precision": "fp64",
            "l2": "256 MiB flush written between timed steps, outside the per-step events"}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(value, dist, device):
    """Max over ranks of a float (identity when not distributed)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(value, dist, device):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate(local_ms_total, local_units, steps, dist, device):
    """Whole-job throughput: units of all ranks / max-over-ranks timed span."""
    span_ms = reduce_max(local_ms_total, dist, device)
    units = reduce_sum(local_units, dist, device)
    return units / (span_ms / 1e3), span_ms / steps


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline(geom, deltas, cycles_per_step, lpt2=True):
    """The oracle on the host cores: one V-cycle, tau and one gradient of the
    same hierarchy, scaled to a full step (cycles_per_step cycles, tau, two
    gradients; without the 2LPT part: the cycles and one gradient)."""
    from oracle.hierarchy import Hierarchy
    from oracle.lpt import gradient, lpt2_source
    from oracle.multigrid import solve
    t0 = time.perf_counter()
    phis, _ = solve(geom, deltas, tol=0.0, cycles=1)
    t_cycle = time.perf_counter() - t0
    t0 = time.perf_counter()
    lpt2_source(Hierarchy(geom), phis)
    t_tau = time.perf_counter() - t0
    t0 = time.perf_counter()
    gradient(Hierarchy(geom), phis)
    t_grad = time.perf_counter() - t0
    if lpt2:
        t_step = cycles_per_step * t_cycle + t_tau + 2 * t_grad
        rest = "tau + 2 gradients"
    else:
        t_step = cycles_per_step * t_cycle + t_grad
        rest = "1 gradient"
    return {"value": geom.level_cells() / t_step, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "1 V-cycle (%.1f s) + tau (%.1f s) + 1 gradient (%.1f s) of the same "
                      "hierarchy on one host core (numpy), scaled to %d cycles + %s"
                      % (t_cycle, t_tau, t_grad, cycles_per_step, rest)}


_BARRIER = None


def _oracle_worker_init(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_worker(name):
    """One process of the all-cores oracle run: builds the workload's inputs, waits
    for every other process, then times the same sample as cpu_baseline."""
    from oracle.hierarchy import Hierarchy
    from oracle.lpt import gradient, lpt2_source
    from oracle.multigrid import solve
    geom = workload(name)
    deltas = workload_inputs(name, geom)
    _BARRIER.wait(timeout=600)  # a process that failed breaks the barrier for all
    t0 = time.perf_counter()
    phis, _ = solve(geom, deltas, tol=0.0, cycles=1)
    t1 = time.perf_counter()
    if name != "unigrid64":
        lpt2_source(Hierarchy(geom), phis)
    t2 = time.perf_counter()
    gradient(Hierarchy(geom), phis)
    t3 = time.perf_counter()
    return t1 - t0, t2 - t1, t3 - t2


def cpu_baseline_all_cores(name, geom, cycles_per_step, lpt2=True):
    """The oracle on every host core: one process per core (spawned, one thread
    each), each timing the cpu_baseline sample on its own copy of the hierarchy at
    the same moment; value = processes x level-cells / the slowest process's
    scaled step time."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        barrier = ctx.Barrier(cores)
        t0 = time.perf_counter()
        with ctx.Pool(cores, initializer=_oracle_worker_init, initargs=(barrier,)) as pool:
            times = pool.map(_oracle_worker, [name] * cores, chunksize=1)
        wall = time.perf_counter() - t0
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    t_cycle = max(t[0] for t in times)
    t_tau = max(t[1] for t in times)
    t_grad = max(t[2] for t in times)
    t_step = cycles_per_step * t_cycle + (t_tau + 2 * t_grad if lpt2 else t_grad)
    return {"value": cores * geom.level_cells() / t_step, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": "%d processes (one per host core, one thread each) each timing 1 V-cycle "
                      "(slowest %.1f s) + tau (%.1f s) + 1 gradient (%.1f s) of its own copy of "
                      "the hierarchy at once, scaled like the one-core figure (%.0f s wall with "
                      "input generation)" % (cores, t_cycle, t_tau, t_grad, wall)}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np  # noqa: F401
    from oracle.hierarchy import Hierarchy
    from oracle.lpt import gradient, lpt2_source
    from oracle.multigrid import solve
    from synthetic import make_delta
    name = args.workload
    geom = workload(name)
    deltas = workload_inputs(name, geom)
    lpt2 = name != "unigrid64"
    extra = 0.0
    for w in range(args.warmup):
        phis, _ = solve(geom, deltas, tol=0.0, cycles=1)
        if w == 0:
            t0 = time.perf_counter()
            if lpt2:
                lpt2_source(Hierarchy(geom), phis)
                gradient(Hierarchy(geom), phis)
            gradient(Hierarchy(geom), phis)
            extra = time.perf_counter() - t0
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        solve(geom, deltas, tol=0.0, cycles=1)
        times.append(time.perf_counter() - t0)
    t_cycle = statistics.mean(times)
    cycles = CYCLES_PER_STEP[name]
    t_step = cycles * t_cycle + extra
    value = geom.level_cells() / t_step
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(geom, name), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "each step: 1 V-cycle of the FP64 numpy oracle (mean %.2f s); "
                                       "reported per full step = %d cycles + %s "
                                       "(%.1f s, timed once in warm-up)"
                                       % (t_cycle, cycles,
                                          "tau + 2 gradients" if lpt2 else "1 gradient", extra)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _batch_delta(job):
    """Input of one batch member (runs in a spawned worker process)."""
    i, geom = job
    import numpy as np
    from synthetic import make_delta
    return [np.ascontiguousarray(x) for x in make_delta(geom, BATCH_SEED + i)]


def serve_large_geometry(side):
    """Large request class of the serving mix: side^3 base + 3 nests of side^3."""
    from synthetic import config_deep_zoom
    return config_deep_zoom(seed=SERVE_SEED, base=side, nest=side, levels=3,
                            jitter=max(1, side // 8))


def batch_inputs(large_side=None):
    """The 64-hierarchy batched workload (and, if asked, the large serving
    class) with inputs generated by a spawned process pool, before the first
    CUDA call of this process."""
    import multiprocessing as mp
    from synthetic import config_batch
    geoms = config_batch()
    jobs = list(enumerate(geoms))
    if large_side:
        jobs.append((len(geoms), serve_large_geometry(large_side)))
    workers = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        deltas = pool.map(_batch_delta, jobs)
    large = (jobs[-1][1], deltas[-1]) if large_side else None
    return geoms, deltas[:len(geoms)], large


def serving_measure(pkg, geoms, deltas_np, large, seconds, rate, workers, native=True):
    """Open-loop Poisson arrivals (mean `rate`/s for `seconds`): 90% draws from the
    batched workload's hierarchies, 10% the large class; mixed precision, host
    buffers in and out, admission by HBM budget, device-resident hierarchies.
    native: the C++ scheduler (mg_server_*, `workers` requests on the GPU at
    once); else the Python server with `workers` threads."""
    import numpy as np
    import torch
    from paper_1103_6031_gb300 import serve
    rng = np.random.Generator(np.random.PCG64(SERVE_SEED))
    pinned = [[torch.from_numpy(x).pin_memory() for x in d] for d in deltas_np]
    large_in = [torch.from_numpy(x).pin_memory() for x in large[1]]
    kw = dict(tol=SOLVE_TOL, max_cycles=50, precision=pkg.MG_MIXED, inner_cycles=MIXED_INNER_CYCLES)
    cfg_small = [pkg.config_from_geometry(g, **kw) for g in geoms]
    cfg_large = pkg.config_from_geometry(large[0], **kw)
    def draw(count, rng, first_id=0):
        out, cells = [], 0
        for k in range(count):
            if rng.uniform() < 0.1:
                out.append(serve.Request(first_id + k, cfg_large, large_in))
                out[-1].cls = "large"
                cells += large[0].level_cells()
            else:
                i = int(rng.integers(len(geoms)))
                out.append(serve.Request(first_id + k, cfg_small[i], pinned[i]))
                out[-1].cls = "batch_draw"
                cells += geoms[i].level_cells()
        return out, cells

    n = int(seconds * rate)
    reqs, cells = draw(n, rng)
    if native:
        server = serve.NativeServer(max_active=workers, hbm_budget=64 << 30, keep_outputs=False)
    else:
        server = serve.Server(workers=workers, hbm_budget=64 << 30, keep_outputs=False)
    # warm server: one untimed request per configuration first, so that the timed
    # window sees resident hierarchies with captured graphs (steady state), not the
    # first-use allocation and capture of 65 configurations
    t0 = time.perf_counter()
    warm = [serve.Request(-1 - i, c, pinned[i]) for i, c in enumerate(cfg_small)]
    warm.append(serve.Request(-1 - len(cfg_small), cfg_large, large_in))
    for r in warm:
        server.submit(r)
    server.drain()
    # then one untimed second of the same arrival process (other seed): the steady
    # state has the pinned output buffers cached and the busiest configurations with
    # a second resident hierarchy
    pre, _ = draw(int(rate), np.random.Generator(np.random.PCG64(SERVE_SEED + 1)), n)
    serve.run_open_loop(server, pre, rate, seed=SERVE_SEED + 1)
    warm_s = time.perf_counter() - t0
    server.completed.clear()
    wall = serve.run_open_loop(server, reqs, rate, seed=SERVE_SEED)
    errors = [r for r in reqs if r.error is not None]
    if native:
        st = server.stats()
        peak_gb, evictions = st["peak_bytes"] / 2 ** 30, st["evictions"]
    else:
        peak_gb, evictions = server.admission.peak / 2 ** 30, server.admission.evictions
    stats = serve.latency_stats(reqs)
    by_class = {}
    for c in ("batch_draw", "large"):
        sub = [r for r in reqs if r.cls == c]
        if sub:
            st = serve.latency_stats(sub)
            by_class[c] = {"count": st["count"], "p50": st["p50_ms"], "p99": st["p99_ms"]}
    out = {"offered_rate_per_s": rate, "requests": n, "seconds_of_arrivals": seconds,
           "completed_per_s": n / wall, "level_cells_per_s": cells / wall,
           "latency_ms": {"p50": stats["p50_ms"], "p99": stats["p99_ms"], "mean": stats["mean_ms"],
                          "max": stats["max_ms"]},
           "latency_ms_by_class": by_class,
           "server": ("native: one C++ scheduler thread, non-blocking pipelines (mg_server_*)"
                      if native else "python: one thread per request in flight"),
           "workers": workers, "peak_inflight": server.peak_inflight,
           "warmup": {"requests": len(warm) + len(pre), "seconds": warm_s,
                      "what": "one untimed request per configuration, then one untimed second "
                              "of the same arrival process, before the timed window"},
           "peak_resident_gb": peak_gb, "evictions": evictions, "errors": len(errors),
           "mix": "90%% draws from the 64 batched hierarchies, 10%% %d^3 base + 3 nests of %d^3 "
                  "(%.1f M level-cells); mixed precision; pinned host buffers in and out; "
                  "latency from arrival to results in host memory" % (
                      large[0].base_n[0], large[0].base_n[0], large[0].level_cells() / 1e6)}
    server.close()
    return out


def generator_measure(pkg, steps, with_oracle):
    """Periodic BBKS density fields on the GPU (Philox white noise + cuFFT
    convolution, mg_field_generate) for 128^3 and 256^3 base grids of a 100 Mpc/h
    box, CUDA-event timed; the numpy oracle of the same field on one host core
    beside it (128^3 only)."""
    import numpy as np
    import torch
    from synthetic.spectra import BBKSPower
    res = {}
    for side in (128, 256):
        h = 100.0 / side
        nt = 8192
        dk = 2 * np.pi / h * np.sqrt(3) * 0.5 * 1.01 / (nt - 1)
        k = np.arange(nt) * dk
        amp = np.sqrt(BBKSPower()(np.maximum(k, 1e-12)) / h ** 3)
        amp[0] = 0.0
        f = pkg.Field((side,) * 3, h, amp, dk)
        out = torch.empty((side,) * 3, dtype=torch.float64, device="cuda")
        s = torch.cuda.current_stream()
        for w in range(3):
            f.generate(w, out)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        for i in range(steps):
            f.generate(100 + i, out)
        b.record(s)
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        entry = {"ms_per_field": ms, "cells_per_s": side ** 3 / (ms * 1e-3)}
        if side == 128 and with_oracle:
            from oracle.noise import gaussian_field, white_noise
            t0 = time.perf_counter()
            gaussian_field(white_noise(7, side ** 3).reshape((side,) * 3), h, amp, dk)
            t = time.perf_counter() - t0
            entry["cpu_oracle"] = {"cells_per_s": side ** 3 / t, "cores": 1, "kind": "oracle",
                                   "sample": "one 128^3 field (numpy: Philox, Box-Muller, FFT)"}
        res["%d^3" % side] = entry
        f.close()
    res["what"] = ("white noise (Philox4x32-10 + Box-Muller) and its periodic convolution with "
                   "a BBKS amplitude table (cuFFT D2Z, amplitude kernel, Z2D), in place")
    # the multi-scale field of the zoom2 hierarchy (128^3 base + 128^3 nest): noise per
    # level, Hoffman-Ribak, periodic and zero-padded convolutions, carried outside field
    from synthetic import config_zoom2
    geom = config_zoom2()
    nt = 8192
    h = geom.box / geom.base_n[0] / 2
    dk = 2 * np.pi / h * np.sqrt(3) * 0.5 * 1.01 / (nt - 1)
    k = np.arange(nt) * dk
    sqrt_p = np.sqrt(BBKSPower()(np.maximum(k, 1e-12)))
    sqrt_p[0] = 0.0
    cfg = pkg.config_from_geometry(geom)
    from paper_1103_6031_gb300 import mg as _mg
    outs = _mg.density_multiscale(cfg, 1, sqrt_p, dk)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(3):
        _mg.density_multiscale(cfg, 2 + i, sqrt_p, dk, outs)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) / 3 * 1e3
    res["multiscale_zoom2"] = {"ms_per_hierarchy": ms, "level_cells_per_s": geom.level_cells() / (ms * 1e-3),
                               "includes": "work-array allocation and cuFFT plan creation per call"}
    return res


def batched_measure(pkg, geoms, deltas_np, steps, device):
    """Hierarchies/s on the batched workload: the float64 solve one hierarchy at a
    time against the mixed-precision batch (one graph launch per iteration)."""
    import torch
    deltas = [[torch.from_numpy(x).to(device) for x in d] for d in deltas_np]
    cells = sum(g.level_cells() for g in geoms)
    res = {}
    for name, prec, batched in (("fp64_one_at_a_time", pkg.MG_FP64, False),
                                ("mixed_batched", pkg.MG_MIXED, True)):
        kw = dict(tol=SOLVE_TOL, max_cycles=50)
        if prec == pkg.MG_MIXED:
            kw.update(precision=prec, inner_cycles=MIXED_INNER_CYCLES)
        hs = [pkg.Hierarchy(pkg.config_from_geometry(g, **kw)) for g in geoms]
        if batched:
            runner = pkg.Batch(hs)
            outs, _, _ = runner.pipeline(deltas)
            step = lambda: runner.pipeline(deltas, outs)  # noqa: E731
        else:
            outs = [h.pipeline(d)[0] for h, d in zip(hs, deltas)]

            def step():
                for h, d, o in zip(hs, deltas, outs):
                    h.pipeline(d, o)
        step()
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            t0 = time.perf_counter()
            step()
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        dt = statistics.mean(times)
        res[name] = {"hierarchies_per_s": len(geoms) / dt, "level_cells_per_s": cells / dt,
                     "ms_per_batch": dt * 1e3}
        if batched:
            runner.close()
        for h in hs:
            h.close()
        del outs
        torch.cuda.empty_cache()
    # the same batch with the schedule and tile the autotuner picks per size class
    from paper_1103_6031_gb300 import autotune
    t0 = time.perf_counter()
    best = autotune.tune_batch(geoms, deltas, SOLVE_TOL)
    tune_s = time.perf_counter() - t0
    hs = [pkg.Hierarchy(c) for c in autotune.batch_configs(geoms, best, SOLVE_TOL)]
    runner = pkg.Batch(hs)
    outs, _, _ = runner.pipeline(deltas)
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        runner.pipeline(deltas, outs)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    dt = statistics.mean(times)
    res["mixed_batched_tuned"] = {"hierarchies_per_s": len(geoms) / dt, "level_cells_per_s": cells / dt,
                                  "ms_per_batch": dt * 1e3, "tuning_s": tune_s,
                                  "schedule": {k: {"inner_cycles": v[0], "nu1": v[1], "nu2": v[2],
                                                   "tile_rows": v[3]} for k, v in best.items()}}
    runner.close()
    for h in hs:
        h.close()
    del outs
    torch.cuda.empty_cache()
    res["workload"] = ("64 hierarchies: base side uniform in {32,48,64,96,128}, 0-3 nests of "
                       "0.5-1.0 x base side (seed 4), order 6, BBKS z=50, 1LPT+2LPT+displacements, "
                       "%.1f M level-cells per batch" % (cells / 1e6))
    res["steps"] = steps
    res["speedup_mixed_batched_vs_fp64"] = (res["mixed_batched"]["hierarchies_per_s"]
                                            / res["fp64_one_at_a_time"]["hierarchies_per_s"])
    res["speedup_tuned_vs_fp64"] = (res["mixed_batched_tuned"]["hierarchies_per_s"]
                                    / res["fp64_one_at_a_time"]["hierarchies_per_s"])
    return res


def run_ours(args):
    world, rank, local = dist_env()
    batch = None
    name = args.workload
    if not args.profile_run and not args.no_batch and name == "zoom2":
        batch = batch_inputs(args.serve_large_side if args.serve_seconds > 0 else None)
    import torch
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
        dist = tdist
    else:
        torch.cuda.set_device(0)
    device = torch.device("cuda", torch.cuda.current_device())
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_6031_gb300 as pkg

    geom = workload(name)
    deltas_np = workload_inputs(name, geom)
    tol = WORKLOAD_TOL[name]
    lpt2 = name != "unigrid64"
    # the dominant smoother launches: half-sweeps of the largest level
    from synthetic.geometry import level_shapes
    dominant = max(n[0] * n[1] * n[2] for n in level_shapes(geom)) // 2
    big = "%d^3" % round((2 * dominant) ** (1.0 / 3.0))
    if args.profile_run and args.precision == "mixed":
        cfg = pkg.config_from_geometry(geom, tol=tol, max_cycles=50, precision=pkg.MG_MIXED,
                                       inner_cycles=MIXED_INNER_CYCLES)
    else:
        # both solves' iteration loops on the device: the whole step is queued at once
        # and the host waits once per step (the steps that carry profiling events fall
        # back to the host loop)
        cfg = pkg.config_from_geometry(geom, tol=tol, max_cycles=50,
                                       device_loop=not args.profile_run)
    h = pkg.Hierarchy(cfg)
    stream = h.stream
    deltas = [torch.from_numpy(x).to(device) for x in deltas_np]
    shapes = h.shapes
    out = {"phi1": [torch.empty(s, dtype=torch.float64, device=device) for s in shapes],
           "phi2": [torch.empty(s, dtype=torch.float64, device=device) for s in shapes],
           "disp1": [torch.empty(s, dtype=torch.float64, device=device) for s in shapes for _ in range(3)],
           "disp2": [torch.empty(s, dtype=torch.float64, device=device) for s in shapes for _ in range(3)]}
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def step(hh):
        """One whole step on hierarchy hh; returns the infos of its solves."""
        if lpt2:
            _, i1, i2 = hh.pipeline(deltas, out)
            return i1, i2
        phis, i1 = hh.solve_1lpt(deltas)
        hh.displacements(phis)
        return i1, None

    info1 = info2 = None
    for w in range(args.warmup):
        info1, info2 = step(h)
    h.stats(reset=True)
    h.set_profiling(["smooth"], min_cells=dominant)
    sampler = ClockSampler(device.index)
    sampler.start()
    time.sleep(0.4)
    barrier()
    evs = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        info1, info2 = step(h)
        b.record(stream)
        evs.append((a, b))
    barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    stats = h.stats(reset=True)
    value, ms_per_step = aggregate(sum(step_ms), geom.level_cells() * args.steps, args.steps,
                                   dist, device)
    launches = sum(v["launches"] for v in stats.values())
    sm = stats["smooth"]
    # dominant launches (the largest level), timed in the first cycle of each solve
    updates_per_launch = sm["timed_cells"] / max(sm["timed"], 1)
    ms_per_launch = sm["event_ms"] / max(sm["timed"], 1)
    ops = SMOOTH_OPS_PER_UPDATE[geom.order] * updates_per_launch
    achieved_gops = ops / (ms_per_launch * 1e-3) / 1e9
    smooth_gbs = SMOOTH_BYTES_PER_CELL * 2 * updates_per_launch / (ms_per_launch * 1e-3) / 1e9
    # every level: one more step with every launch of every kernel family timed in the
    # first cycle of each solve (and every launch outside the cycle loops)
    from paper_1103_6031_gb300.mg import FAMILY_NAMES
    h.set_profiling(list(FAMILY_NAMES), min_cells=0)
    step(h)
    fam = h.stats(reset=True)
    h.set_profiling([])
    sa = fam["smooth"]

    # open-loop serving, measured early in the process: measured after the batched
    # and autotuning sections (hundreds of hierarchies made and destroyed), its p50
    # latency was 15x worse than in a fresh process
    serving = None
    if batch is not None and args.serve_seconds > 0 and world == 1:
        serving = serving_measure(pkg, batch[0], batch[1], batch[2], args.serve_seconds,
                                  args.serve_rate, args.serve_workers,
                                  native=args.serve_impl == "native")
    all_ms = sa["event_ms"] / max(sa["timed"], 1)
    all_updates = sa["timed_cells"] / max(sa["timed"], 1)
    all_gops = SMOOTH_OPS_PER_UPDATE[geom.order] * all_updates / (all_ms * 1e-3) / 1e9
    # the sampled launches stand for all launches of their family in the step
    est = {k: v["event_ms"] / max(v["timed"], 1) * v["launches"] for k, v in fam.items() if v["timed"]}
    total_smooth_ms = est.get("smooth", 0.0)
    # share of kernel time with every launch carrying the same event nodes: the figure
    # to compare with an ncu launch list (which serialises launches without events)
    share_kernel_time = total_smooth_ms / max(sum(est.values()), 1e-12)

    # mixed precision on the same workload and stopping rule (float32 V-cycles
    # inside float64 iterative refinement), device-resident like the headline
    mixed = None
    if not args.profile_run:
        cfg_m = pkg.config_from_geometry(geom, tol=tol, max_cycles=50,
                                         precision=pkg.MG_MIXED, inner_cycles=MIXED_INNER_CYCLES)
        hm = pkg.Hierarchy(cfg_m)
        for w in range(args.warmup):
            m1, m2 = step(hm)
        hm.stats(reset=True)
        barrier()
        evm = []
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            m1, m2 = step(hm)
            b.record(stream)
            evm.append((a, b))
        barrier()
        mixed_ms = [a.elapsed_time(b) for a, b in evm]
        mstats = hm.stats(reset=True)
        mixed_value, mixed_ms_step = aggregate(sum(mixed_ms), geom.level_cells() * args.steps,
                                               args.steps, dist, device)
        # roofline of the float32 smoother from 3 more steps with CUDA events around
        # its 128^3 launches (event nodes cost ~1 us each against ~10 us launches,
        # so the value above is taken without them)
        hm.set_profiling(["smooth"], min_cells=dominant)
        for i in range(3):
            step(hm)
        msm = hm.stats(reset=True)["smooth"]
        hm.set_profiling([])
        m_ms = msm["event_ms"] / max(msm["timed"], 1)
        m_upd = msm["timed_cells"] / max(msm["timed"], 1)
        # float32 in place: 8 B per level-cell (read u of both colours 4 B, f of the
        # updated colour 2 B, write the updated colour 2 B)
        m_gbs = 8.0 * 2 * m_upd / (m_ms * 1e-3) / 1e9
        # which kernel the timed launches ran: the plain one on the periodic base and
        # on smaller nests, the TMA-staged one on float32 nests of >= 2^23 cells
        shapes = level_shapes(geom)
        tma_nests = [n for n in shapes[1:] if n[0] * n[1] * n[2] // 2 == dominant
                     and n[0] * n[1] * n[2] >= TMA_MIN_CELLS]
        base_big = shapes[0][0] * shapes[0][1] * shapes[0][2] // 2 == dominant
        if not tma_nests:
            m_kernel = "k_smooth_half<%d,float> (%s levels)" % (geom.order, big)
            m_traffic = SMOOTH_F32_TRAFFIC_PER_UPDATE * m_upd if geom.order == 6 else None
        elif not base_big:
            m_kernel = "k_smooth_half_tma<%d,float> (%s nests)" % (geom.order, big)
            m_traffic = SMOOTH_TMA_F32_TRAFFIC_PER_UPDATE * m_upd if geom.order == 6 else None
        else:
            m_kernel = ("k_smooth_half<%d,float> (%s periodic base) and k_smooth_half_tma<%d,"
                        "float> (%s nests)" % (geom.order, big, geom.order, big))
            m_traffic = None
        mixed = {"value": mixed_value, "unit": UNIT, "ms_per_step": mixed_ms_step,
                 "latency_ms": {"p50": statistics.median(mixed_ms),
                                "p99": sorted(mixed_ms)[max(0, int(round(0.99 * len(mixed_ms))) - 1)]},
                 "precision": "float32 V-cycles (smoothing, transfers, coarse-fine ghosts) inside "
                              "float64 refinement (residual, coarsest solve, update)",
                 "inner_cycles": MIXED_INNER_CYCLES,
                 "outer": {"1lpt": m1["cycles"], "2lpt": m2["cycles"] if m2 else None},
                 "rel_residual": {"1lpt": m1["rel_residual"],
                                  "2lpt": m2["rel_residual"] if m2 else None},
                 "gpu_launches": sum(v["launches"] for v in mstats.values()),
                 "roofline": {"bound": "hbm", "achieved": m_gbs, "peak": HBM_PEAK_GBS,
                              "unit": "GB/s", "frac": m_gbs / HBM_PEAK_GBS, "traffic": m_traffic,
                              "traffic_unit": "bytes per launch (ncu, scaled by updated cells)",
                              "kernel": m_kernel,
                              "peak_source": "measured copy bandwidth (of measured)",
                              "ms_per_launch": m_ms, "updates_per_launch": m_upd,
                              "bytes_per_cell": 8.0},
                 "error_bound": "<= 1e-6 RMS relative vs float64 (tests/test_gpu_parity.py)"}
        hm.close()

    generator = None
    if not args.profile_run and name == "zoom2":
        generator = generator_measure(pkg, args.steps, world == 1 and not args.skip_baseline)

    batched = None
    if batch is not None:
        batched = batched_measure(pkg, batch[0], batch[1], min(args.steps, 3), device)

    if args.profile_run:
        if rank == 0:
            print(json.dumps({"profile_run": True, "value": value, "ms_per_step": ms_per_step,
                              "gpu_launches": launches,
                              "cycles": [info1["cycles"], info2["cycles"] if info2 else 0]}))
        h.close()
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # end to end through the C ABI with pinned host buffers
    host_in = [torch.from_numpy(x).pin_memory() for x in deltas_np]
    host_out = {"phi1": [torch.empty(s, dtype=torch.float64, pin_memory=True) for s in shapes],
                "phi2": [torch.empty(s, dtype=torch.float64, pin_memory=True) for s in shapes],
                "disp1": [torch.empty(s, dtype=torch.float64, pin_memory=True) for s in shapes for _ in range(3)],
                "disp2": [torch.empty(s, dtype=torch.float64, pin_memory=True) for s in shapes for _ in range(3)]}
    if not lpt2:
        # 1LPT only: phi and -grad phi come back (the C ABI's host-buffer entry point
        # is the whole 2LPT step, so the copies are issued here)
        host_out = {"phi1": host_out["phi1"], "disp1": host_out["disp1"]}

    def e2e_step():
        if lpt2:
            h.pipeline(host_in, host_out, host=True)
            return
        with torch.cuda.stream(stream):
            for d, x in zip(deltas, host_in):
                d.copy_(x, non_blocking=True)
            phis, _ = h.solve_1lpt(deltas)
            disp = h.displacements(phis)
            for x, y in zip(host_out["phi1"], phis):
                x.copy_(y, non_blocking=True)
            for x, y in zip(host_out["disp1"], [c for lv in disp for c in lv]):
                x.copy_(y, non_blocking=True)
        stream.synchronize()

    e2e_step()
    barrier()
    e2e_ms = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        torch.cuda.synchronize()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    barrier()
    e2e_value, _ = aggregate(sum(e2e_ms), geom.level_cells() * args.steps, args.steps, dist, device)
    h2d = sum(x.numel() * 8 for x in host_in)
    d2h = sum(x.numel() * 8 for k in host_out for x in host_out[k])

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(geom, name),
            "latency_ms": {"p50": statistics.median(step_ms),
                           "p99": sorted(step_ms)[max(0, int(round(0.99 * len(step_ms))) - 1)]},
            "cycles": {"1lpt": info1["cycles"], "2lpt": info2["cycles"] if info2 else None,
                       "rel_residual_1lpt": info1["rel_residual"],
                       "rel_residual_2lpt": info2["rel_residual"] if info2 else None},
            "roofline": {"bound": "alu", "achieved": achieved_gops, "peak": FP64_PEAK_GOPS,
                         "unit": "G FP64 instr/s", "frac": achieved_gops / FP64_PEAK_GOPS,
                         "traffic": (SMOOTH_TRAFFIC_PER_UPDATE * updates_per_launch
                                     if SMOOTH_TRAFFIC_PER_UPDATE and geom.order == 6 else None),
                         "traffic_unit": "bytes per launch (ncu, scaled by updated cells)",
                         "kernel": "k_smooth_half<%d,double> (%s levels)" % (geom.order, big),
                         "peak_source": "nominal FP64 1.25 TFLOP/s (recipe) = 625 G FMA/s",
                         "ms_per_launch": ms_per_launch, "updates_per_launch": updates_per_launch,
                         "hbm_view": {"achieved_gbs": smooth_gbs, "peak_gbs": HBM_PEAK_GBS,
                                      "frac": smooth_gbs / HBM_PEAK_GBS,
                                      "bytes_per_cell": SMOOTH_BYTES_PER_CELL},
                         "all_levels": {"ms_per_launch": all_ms, "updates_per_launch": all_updates,
                                        "achieved": all_gops, "frac": all_gops / FP64_PEAK_GOPS},
                         "share_of_step": total_smooth_ms / max(sum(step_ms) / len(step_ms), 1e-9),
                         "share_of_kernel_time": share_kernel_time},
            "gpu_launches": launches,
            "iteration_loop": ("host (profiling run)" if args.profile_run else
                               "on the device (MG_FLAG_DEVICE_LOOP): one host wait per step"),
            "clocks": clocks,
            "mixed_precision": mixed,
            "batched": batched,
            "serving": serving,
            "generator": generator,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "ms_per_step": statistics.mean(e2e_ms)},
        }
        if not args.skip_baseline and world == 1:
            cycles = info1["cycles"] + (info2["cycles"] if info2 else 0)
            line["cpu_baseline"] = cpu_baseline(geom, deltas_np, cycles, lpt2)
            if not args.skip_all_cores:
                line["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(
                    args.workload, geom, cycles, lpt2)
        print(json.dumps(line))
    h.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=WORKLOADS, default="zoom2",
                    help="zoom2 (default, the headline), unigrid64, deep_zoom or zoom256")
    ap.add_argument("--skip-baseline", action="store_true",
                    help="leave out the CPU-oracle baseline")
    ap.add_argument("--skip-all-cores", action="store_true",
                    help="leave out the all-cores run of the CPU-oracle baseline")
    ap.add_argument("--profile-run", action="store_true",
                    help="timed steps only: no end-to-end pass, no CPU baseline (for ncu)")
    ap.add_argument("--no-batch", action="store_true",
                    help="leave out the 64-hierarchy batched and the serving measurements")
    ap.add_argument("--serve-seconds", type=float, default=5.0,
                    help="seconds of open-loop arrivals in the serving measurement (0: none)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="mean arrivals per second")
    ap.add_argument("--serve-workers", type=int, default=16, help="concurrent requests at most")
    ap.add_argument("--serve-impl", choices=["native", "python"], default="native",
                    help="serving runtime: the C++ scheduler (mg_server_*) or Python threads")
    ap.add_argument("--serve-large-side", type=int, default=128,
                    help="side of the large request class (base and 3 nests); 256 is full size")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="precision of the timed steps of a --profile-run")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
