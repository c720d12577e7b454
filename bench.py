#!/usr/bin/env python
"""Benchmark of the nested-grid initial-conditions step on GB300.

One step = the whole hot path on one hierarchy: 1LPT solve of L phi1 = delta,
2LPT source tau(phi1), 2LPT solve of L phi2 = tau, displacements -G phi1 and
-G phi2 (float64, order-6 operators).  Default workload (the largest single
hierarchy): a 128^3 periodic base of a 100 Mpc/h box plus 4 nests of 128^3, each
at twice its parent's resolution, centred with a seeded +-16-cell jitter
(10,485,760 level-cells), BBKS density at z = 50 from seeded white noise.  Each
float64 solve stops at a relative leaf residual of 3e-8 (mixed precision: 1e-8),
the tolerances that kept every output of the benchmark's hierarchies within 1e-6
RMS relative error; the error of every output against a float64 solve to 1e-12 is
measured in the run and printed.

Default: N = 1, 10 timed steps after 3 warm-up steps.  Under torchrun every
rank solves its own hierarchy (replicas, no collective in the data path);
value = level-cells of all ranks / max-over-ranks time.

--impl reference times the CPU oracle: whole steps (both solves to the same
stopping rule, tau, both displacement fields) of a bounded sample of the
workload, the same hierarchy shape at 32^3 cells per level.
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
# stopping tolerances (relative leaf residual): the largest that kept every output
# (phi1, phi2, both displacement fields, every level) of the 64 batched hierarchies,
# the serving mix's large class, zoom2 and the deep zoom within 1e-6 RMS relative error
# of float64 solves to 1e-12 (largest errors measured: 3.9e-7 and 3.7e-7; at 1e-7 they
# reached 1.0e-6 in float64 and 1.8e-6 in mixed precision)
SOLVE_TOL = 3e-8
MIXED_TOL = 1e-8
# resident hierarchies per configuration in the serving measurement (the warm-up
# creates them all before the timed window)
SERVE_INSTANCES = 3
REF_TOL = 1e-12        # float64 solve the measured errors are taken against
BATCH_SEED = 1000
SERVE_SEED = 5
# float32 V-cycles per float64 refinement step in the mixed-precision variant: 3 on the
# large single hierarchies (measured on the deep zoom: 3, 4, 5, 6, 8 cycles all take 3 + 3
# outer iterations, in 22.2, 25.6, 29.6, 33.7, 40.5 ms), 4 on the batched workload's
# small hierarchies (the batch autotuner's default schedule)
MIXED_INNER_CYCLES = 3
BATCH_INNER_CYCLES = 4
HBM_PEAK_GBS = 6765.0    # measured copy bandwidth of the GB300s
L2_FLUSH_BYTES = 256 << 20

# smoother: FP64 instructions per updated cell (three 6-neighbour sums: 15 adds,
# a_f * f: 1 multiply, 3 fused multiply-adds) for the order-6 stencil
SMOOTH_OPS_PER_UPDATE = {2: 7, 4: 13, 6: 19}
# in-place algorithmic bytes of one colour half-sweep per level-cell: read u of
# both colours (8 B), f of the updated colour (4 B), write the updated colour (4 B)
SMOOTH_BYTES_PER_CELL = 16.0
# DRAM bytes (read + write) per updated cell of k_smooth_half<6,double> from one ncu
# capture of the 128^3 launch; scaled per launch by the updated cells.  Set to None
# whenever the kernel changes.
SMOOTH_TRAFFIC_PER_UPDATE = 35.8
# the same for k_smooth_half<6,float> (ncu capture of the 128^3 nest launch) and for
# k_smooth_half_tma<6,float> (capture of the 256^3 nest launch)
SMOOTH_F32_TRAFFIC_PER_UPDATE = 17.8
SMOOTH_TMA_F32_TRAFFIC_PER_UPDATE = 22.3
# k_smooth_quad<6> (float32 levels whose rows are a multiple of 4 long; capture of the
# 128^3 nest launch)
SMOOTH_QUAD_F32_TRAFFIC_PER_UPDATE = 17.8
# float32 levels of at least this many cells that are not periodic take the
# TMA-staged smoother by default
TMA_MIN_CELLS = 1 << 23

# Workloads: deep_zoom is the headline; zoom2 runs beside it (extra key) and alone
# with --workload; unigrid64 and zoom256 with --workload.
WORKLOADS = ("deep_zoom", "zoom2", "unigrid64", "zoom256")
WORKLOAD_SEED = {"zoom2": 2, "unigrid64": 1, "deep_zoom": 3, "zoom256": 4}
WORKLOAD_TOL = {"zoom2": SOLVE_TOL, "unigrid64": 1e-10, "deep_zoom": SOLVE_TOL,
                "zoom256": SOLVE_TOL}
WORKLOAD_TEXT = {
    "zoom2": "zoom2: 128^3 periodic base (100 Mpc/h) + centred 128^3 nest at 2x, order-6 FD, "
             "FP64, 1LPT+2LPT+displacements, BBKS z=50, seed 2",
    "unigrid64": "unigrid64: 64^3 periodic, 7-point Laplacian, FP64, 1LPT (phi and -grad phi) "
                 "to 1e-10 relative residual, power law P ~ k^-2 at unit RMS, seed 1",
    "deep_zoom": "deep zoom: 128^3 periodic base (100 Mpc/h) + 4 nests of 128^3, each at 2x its "
                 "parent, centred with +-16 jitter (seed 3), order-6 FD, FP64, "
                 "1LPT+2LPT+displacements, BBKS z=50",
    "zoom256": "zoom256: 256^3 periodic base (200 Mpc/h) + centred 256^3 nest at 2x, order-6 FD, "
               "FP64, 1LPT+2LPT+displacements, BBKS z=50, seed 4",
}


def workload(name="deep_zoom"):
    from synthetic import config_deep_zoom, config_unigrid64, config_zoom2
    return {"zoom2": config_zoom2, "unigrid64": config_unigrid64, "deep_zoom": config_deep_zoom,
            "zoom256": lambda: config_zoom2(base=256, nest=256, box=200.0)}[name]()


def workload_inputs(name, geom):
    from synthetic import make_delta, make_delta_powerlaw
    if name == "unigrid64":
        return [make_delta_powerlaw(tuple(geom.base_n), WORKLOAD_SEED[name])]
    return make_delta(geom, WORKLOAD_SEED[name])


def workload_config(geom, name):
    return {"workload": WORKLOAD_TEXT[name],
            "level_cells": geom.level_cells(), "order": geom.order, "levels": geom.n_levels,
            "solve_tol": WORKLOAD_TOL[name], "mixed_tol": MIXED_TOL, "precision": "fp64",
            "l2": "256 MiB flush written between timed steps, outside the per-step events"}


# ---- the CPU oracle on a bounded sample --------------------------------------------

def oracle_sample(name):
    """The hierarchy the oracle is timed on: the workload's shape with 32^3 cells per
    level for the deep zoom, 48^3 for the two-level zooms (64^3 for unigrid64, the
    workload itself), so that one whole step takes a few seconds on one host core."""
    from synthetic import config_deep_zoom, config_zoom2, Geometry
    if name == "unigrid64":
        geom = Geometry((64,) * 3, 1.0, 2, ())
        what = "the workload itself (64^3, order 2, 1LPT to 1e-10)"
    elif name == "deep_zoom":
        geom = config_deep_zoom(seed=3, base=32, nest=32, jitter=4)
        what = "32^3 base + 4 nests of 32^3 (+-4 jitter), order 6, 1LPT+2LPT to 3e-8"
    elif name == "zoom256":
        geom = config_zoom2(base=64, nest=64, box=50.0)
        what = "64^3 base + centred 64^3 nest, order 6, 1LPT+2LPT to 3e-8"
    else:
        geom = config_zoom2(base=48, nest=48, box=37.5)
        what = "48^3 base + centred 48^3 nest, order 6, 1LPT+2LPT to 3e-8"
    return geom, what


def _sample_inputs(name, geom):
    from synthetic import make_delta, make_delta_powerlaw
    if name == "unigrid64":
        return [make_delta_powerlaw(tuple(geom.base_n), WORKLOAD_SEED[name])]
    return make_delta(geom, WORKLOAD_SEED[name])


def oracle_step(name, geom, deltas):
    """One whole step of the oracle, as the library's step: both solves to the
    workload's stopping rule, tau, both displacement fields (1LPT only for
    unigrid64); returns the total V-cycles."""
    from oracle.hierarchy import Hierarchy
    from oracle.lpt import gradient, lpt_pipeline
    from oracle.multigrid import solve
    tol = WORKLOAD_TOL[name]
    if name == "unigrid64":
        phis, info = solve(geom, deltas, tol=tol)
        gradient(Hierarchy(geom), phis)
        return info["cycles"]
    out = lpt_pipeline(geom, deltas, tol=tol)
    return out["info1"]["cycles"] + out["info2"]["cycles"]


def cpu_baseline(name, min_seconds=10.0, max_steps=5):
    """The oracle on one host core: whole steps of the bounded sample until
    min_seconds have passed (at least 2, at most max_steps)."""
    geom, what = oracle_sample(name)
    deltas = _sample_inputs(name, geom)
    times, cycles = [], 0
    t_all = time.perf_counter()
    while len(times) < max_steps and (len(times) < 2 or time.perf_counter() - t_all < min_seconds):
        t0 = time.perf_counter()
        cycles = oracle_step(name, geom, deltas)
        times.append(time.perf_counter() - t0)
    t = statistics.mean(times)
    return {"value": geom.level_cells() / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d whole steps (%d V-cycles each, mean %.2f s) of %s (%d level-cells), "
                      "numpy float64 on one host core" % (len(times), cycles, t, what,
                                                          geom.level_cells())}


_BARRIER = None


def _oracle_worker_init(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_worker(name):
    """One process of the all-cores oracle run: builds the sample's inputs, waits
    for every other process, then times one whole step."""
    geom, _ = oracle_sample(name)
    deltas = _sample_inputs(name, geom)
    _BARRIER.wait(timeout=600)  # a process that failed breaks the barrier for all
    t0 = time.perf_counter()
    oracle_step(name, geom, deltas)
    return time.perf_counter() - t0


def cpu_baseline_all_cores(name):
    """The oracle on every host core: one spawned process per core (one thread
    each), each timing one whole step of its own copy of the sample at the same
    moment; value = processes x level-cells / the slowest process's step time."""
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
    geom, what = oracle_sample(name)
    return {"value": cores * geom.level_cells() / max(times), "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": "%d processes (one per host core, one thread each), each one whole step of "
                      "its own copy of %s at once (slowest %.1f s; %.0f s wall with input "
                      "generation)" % (cores, what, max(times), wall)}


def run_reference(args):
    """The reference arm: the oracle as it stands, timed on the host cores, whole
    steps of the bounded sample (warm-up steps untimed)."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    name = args.workload
    geom, what = oracle_sample(name)
    deltas = _sample_inputs(name, geom)
    for _ in range(args.warmup):
        oracle_step(name, geom, deltas)
    times = []
    cycles = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        cycles = oracle_step(name, geom, deltas)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = geom.level_cells() * len(times) / total
    big = workload(name)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / len(times) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(big, name), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "every step one whole step (%d V-cycles) of %s (%d "
                                       "level-cells), numpy float64 on one host core; "
                                       "ms_per_step is that sample's step time"
                                       % (cycles, what, geom.level_cells())},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---- helpers ------------------------------------------------------------------------

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


def p99(xs):
    s = sorted(xs)
    return s[max(0, int(round(0.99 * len(s))) - 1)]


def sig(x, digits=4):
    """x rounded to `digits` significant digits (compact JSON)."""
    if x is None or isinstance(x, (bool, int, str)):
        return x
    if x != x or x == 0:
        return x
    return float("%.*g" % (digits, x))


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


def rms_rel(a, b):
    """RMS relative error of a against b (device tensors)."""
    num = float(((a - b) ** 2).sum())
    den = float((b * b).sum())
    return (num / den) ** 0.5 if den > 0 else num ** 0.5


def output_errors(out, ref, n_levels):
    """Per output field, the largest RMS relative error over the levels (displacements:
    over levels and components) of `out` against `ref` (dicts of device lists)."""
    errs = {}
    for key in ("phi1", "phi2", "disp1", "disp2"):
        if key in out and key in ref:
            errs[key] = max(rms_rel(a, b) for a, b in zip(out[key], ref[key]))
    errs["max"] = max(errs.values())
    return errs


def clone_outputs(out):
    return {k: [x.clone() for x in v] for k, v in out.items()}


# ---- GPU sections -------------------------------------------------------------------

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


def batch_inputs(large_side=None, extra=()):
    """The 64-hierarchy batched workload (and, if asked, the large serving class and
    the `extra` named workloads' inputs) generated by a spawned process pool, before
    the first CUDA call of this process."""
    import multiprocessing as mp
    from synthetic import config_batch
    geoms = config_batch()
    jobs = list(enumerate(geoms))
    if large_side:
        jobs.append((len(geoms), serve_large_geometry(large_side)))
    workers = max(1, min(16, os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        deltas = pool.map(_batch_delta, jobs)
        named = pool.map(_named_inputs, list(extra))
    large = (jobs[-1][1], deltas[-1]) if large_side else None
    return geoms, deltas[:len(geoms)], large, dict(zip(extra, named))


def _named_inputs(name):
    import numpy as np
    geom = workload(name)
    return [np.ascontiguousarray(x) for x in workload_inputs(name, geom)]


def time_steps(step, steps, stream, flush, barrier):
    """CUDA-event times (ms) of `steps` calls of step() on `stream`, the L2 flush
    written before each one outside its events."""
    import torch
    barrier()
    evs = []
    for i in range(steps):
        flush.fill_(i & 0xFF)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        evs.append((a, b))
    barrier()
    return [a.elapsed_time(b) for a, b in evs]


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
    kw = dict(tol=MIXED_TOL, max_cycles=50, precision=pkg.MG_MIXED)
    cfg_small = [pkg.config_from_geometry(g, inner_cycles=BATCH_INNER_CYCLES, **kw) for g in geoms]
    cfg_large = pkg.config_from_geometry(large[0], inner_cycles=MIXED_INNER_CYCLES, **kw)

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
        # an output set per request in flight (no shared sets): the warm-up at full
        # concurrency below grows the pool to the window's needs (27 GB of pinned sets
        # with the 128^3 large class); with the 256^3 class a set is 4.3 GB, so its
        # requests beyond two share sets as before
        small_large = large[0].level_cells() < (1 << 24)
        server = serve.NativeServer(max_active=workers, hbm_budget=64 << 30, keep_outputs=False,
                                    dropped_sets=None if small_large else 2)
        # at most 3 resident hierarchies per configuration: creating one stalls the
        # device, and uncapped the server kept creating instances under load (20-54 inside
        # a 5 s window), which cut its capacity by up to half from run to run
        server.set_max_instances(SERVE_INSTANCES)
        # pinned output sets of the large class up front (0.5 GB each at 128^3, 4.3 GB at
        # 256^3); the others come from the warm-up below and are recycled from then on
        server.reserve_outputs(cfg_large, 8 if small_large else 2)
    else:
        server = serve.Server(workers=workers, hbm_budget=64 << 30, keep_outputs=False)
    # warm server: every configuration served as many times at once as it may have
    # resident instances (untimed), so that the timed window sees resident hierarchies
    # with captured graphs (steady state), not the first-use allocation and capture
    copies = SERVE_INSTANCES if native else 1
    t0 = time.perf_counter()
    warm = [serve.Request(-1 - copies * i - c, cf, pinned[i])
            for i, cf in enumerate(cfg_small) for c in range(copies)]
    warm += [serve.Request(-1 - copies * len(cfg_small) - c, cfg_large, large_in)
             for c in range(copies)]
    for r in warm:
        server.submit(r)
    server.drain()
    def closed_loop(reqs_):
        """Keeps `workers` requests in the server until every request has run; seconds
        from the first submission to the last result."""
        t_b = time.perf_counter()
        for r in reqs_:
            while len(server.inflight) >= workers:
                time.sleep(2e-4)
            r.arrival = time.perf_counter()
            server.submit(r)
        server.drain()
        return max(r.done for r in reqs_) - t_b

    # then an untimed closed loop over the mix at full concurrency (the server creates
    # the extra resident instances that overlapping requests of one configuration need,
    # with their captured graphs, before the timed window: creating them inside it
    # stalled the GPU) and one untimed second of the same arrival process (other seeds)
    if native:
        pre0, _ = draw(int(1.5 * rate), np.random.Generator(np.random.PCG64(SERVE_SEED + 3)), 20 * n)
        closed_loop(pre0)
    pre, _ = draw(int(rate), np.random.Generator(np.random.PCG64(SERVE_SEED + 1)), n)
    serve.run_open_loop(server, pre, rate, seed=SERVE_SEED + 1)
    warm_s = time.perf_counter() - t0
    created0 = server.stats()["created"] if native else None
    sets0 = sum(len(v) for v in server._owned.values()) if native else None
    server.completed.clear()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    st0 = server.stats() if native else None
    cpu0 = time.process_time()
    wall = serve.run_open_loop(server, reqs, rate, seed=SERVE_SEED)
    cpu_window = time.process_time() - cpu0
    st1 = server.stats() if native else None
    clocks = sampler.stop()
    errors = [r for r in reqs if r.error is not None]
    # capacity: a closed loop over the same mix (other seed) that keeps `workers`
    # requests in the server, completions per second until the last result; utilisation
    # = offered work / that capacity (at ~0.9 and above, queueing makes p50/p99 vary from
    # run to run)
    capacity, util, created_in_window = None, None, None
    sets_in_window = None
    if native:
        created_in_window = server.stats()["created"] - created0
        sets_in_window = sum(len(v) for v in server._owned.values()) - sets0
        burst, bcells = draw(int(1.5 * rate), np.random.Generator(np.random.PCG64(SERVE_SEED + 2)),
                             10 * n)
        st2 = server.stats()
        wall_b = closed_loop(burst)
        st3 = server.stats()
        capacity = {"requests_per_s": sig(len(burst) / wall_b),
                    "level_cells_per_s": sig(bcells / wall_b), "requests": len(burst),
                    "in_server": workers}
        util = sig((cells / seconds) / (bcells / wall_b), 3)
    def sched(a, b, count):
        """Scheduler thread between two stats snapshots: CPU share, share of wall time
        in passes that moved a job, CPU ms per request."""
        dt = b["uptime_s"] - a["uptime_s"]
        return {"cpu_share": sig((b["sched_cpu_s"] - a["sched_cpu_s"]) / dt, 3),
                "busy_share": sig((b["sched_busy_s"] - a["sched_busy_s"]) / dt, 3),
                "passes_per_s": sig((b["passes"] - a["passes"]) / dt),
                "cpu_ms_per_request": sig(1e3 * (b["sched_cpu_s"] - a["sched_cpu_s"]) / count)}
    scheduler = None
    if native:
        scheduler = {"window": sched(st0, st1, n), "capacity": sched(st2, st3, len(burst))}
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
            sc = serve.latency_stats(sub)
            by_class[c] = {"count": sc["count"], "p50": sig(sc["p50_ms"]), "p99": sig(sc["p99_ms"])}
    # time the requests spent waiting for admission and on the GPU (native clock)
    queue = [r.admitted - r.arrival for r in reqs if r.admitted is not None]
    out = {"offered_rate_per_s": rate, "requests": n, "seconds_of_arrivals": seconds,
           "completed_per_s": sig(n / wall), "level_cells_per_s": sig(cells / wall),
           "offered_level_cells_per_s": sig(cells / seconds),
           "capacity": capacity,
           "hierarchies_created_in_window": created_in_window,
           "output_sets_allocated_in_window": sets_in_window,
           "pinned_output_gb": (sig(sum(8 * t.numel() for sets in server._owned.values()
                                         for st in sets for v in st.values() for t in v) / 2 ** 30)
                                if native else None),
           "utilisation": util,
           "scheduler_thread": scheduler,
           "process_cpu_s_in_window": sig(cpu_window),
           "clocks_in_window": clocks,
           "latency_ms": {"p50": sig(stats["p50_ms"]), "p99": sig(stats["p99_ms"]),
                          "mean": sig(stats["mean_ms"]), "max": sig(stats["max_ms"])},
           "queue_wait_ms_p50": sig(1e3 * statistics.median(queue)) if queue else None,
           "latency_ms_by_class": by_class,
           "server": ("native: one C++ scheduler thread, non-blocking pipelines (mg_server_*)"
                      if native else "python: one thread per request in flight"),
           "workers": workers, "peak_inflight": server.peak_inflight,
           "warmup": {"requests": len(warm) + len(pre) + (len(pre0) if native else 0),
                      "seconds": sig(warm_s),
                      "instances_per_config": copies},
           "peak_resident_gb": sig(peak_gb), "evictions": evictions, "errors": len(errors),
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
        entry = {"ms_per_field": sig(ms), "cells_per_s": sig(side ** 3 / (ms * 1e-3))}
        if side == 128 and with_oracle:
            from oracle.noise import gaussian_field, white_noise
            t0 = time.perf_counter()
            gaussian_field(white_noise(7, side ** 3).reshape((side,) * 3), h, amp, dk)
            t = time.perf_counter() - t0
            entry["cpu_oracle_cells_per_s"] = sig(side ** 3 / t)
        res["%d^3" % side] = entry
        f.close()
    return res


def batched_measure(pkg, geoms, deltas_np, steps, device):
    """Hierarchies/s on the batched workload: the float64 solve one hierarchy at a
    time against the mixed-precision batch (one graph launch per iteration), untuned
    and autotuned; the RMS relative error of every member's mixed-precision result
    against its float64 solve to 1e-12."""
    import torch
    deltas = [[torch.from_numpy(x).to(device) for x in d] for d in deltas_np]
    cells = sum(g.level_cells() for g in geoms)
    # reference results for the error of each member
    refs = []
    for g, d in zip(geoms, deltas):
        h = pkg.Hierarchy(pkg.config_from_geometry(g, tol=REF_TOL, max_cycles=60))
        refs.append(clone_outputs(h.pipeline(d)[0]))
        h.close()
    res = {}
    member_err = None
    for name, prec, batched in (("fp64_one_at_a_time", pkg.MG_FP64, False),
                                ("mixed_batched", pkg.MG_MIXED, True)):
        kw = dict(tol=SOLVE_TOL, max_cycles=50)
        if prec == pkg.MG_MIXED:
            kw.update(tol=MIXED_TOL, precision=prec, inner_cycles=BATCH_INNER_CYCLES)
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
        res[name] = {"hierarchies_per_s": sig(len(geoms) / dt), "level_cells_per_s": sig(cells / dt),
                     "ms_per_batch": sig(dt * 1e3)}
        if batched:
            member_err = [output_errors(o, r, g.n_levels)["max"] for o, r, g in zip(outs, refs, geoms)]
            runner.close()
        for h in hs:
            h.close()
        del outs
        torch.cuda.empty_cache()
    # the same float32 V-cycles of every member as one persistent launch per outer
    # iteration over a (hierarchy, level operation, block range) work list
    hs = [pkg.Hierarchy(pkg.config_from_geometry(g, tol=MIXED_TOL, max_cycles=50,
                                                 precision=pkg.MG_MIXED,
                                                 inner_cycles=BATCH_INNER_CYCLES, persistent=True))
          for g in geoms]
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
    pers_err = [output_errors(o, r, g.n_levels)["max"] for o, r, g in zip(outs, refs, geoms)]
    res["mixed_persistent"] = {"hierarchies_per_s": sig(len(geoms) / dt),
                               "level_cells_per_s": sig(cells / dt), "ms_per_batch": sig(dt * 1e3)}
    runner.close()
    for h in hs:
        h.close()
    del outs
    torch.cuda.empty_cache()
    # the autotuner on the batch itself: coordinate descent over each size class's
    # schedule and the launch mode, objective the measured batch step time
    from paper_1103_6031_gb300 import autotune
    t0 = time.perf_counter()
    sched, mode, log = autotune.tune_batch_joint(geoms, deltas, MIXED_TOL, budget_s=60.0)
    tune_s = time.perf_counter() - t0
    t_tuned = autotune.time_batch(geoms, deltas, sched, MIXED_TOL, mode, reps=max(steps, 2))
    ok = [t for _, t in log if t is not None]
    res["mixed_batched_tuned"] = {"hierarchies_per_s": sig(len(geoms) / t_tuned),
                                  "ms_per_batch": sig(t_tuned * 1e3), "tuning_s": sig(tune_s),
                                  "schedule": {k: list(v) for k, v in sched.items()},
                                  "launch_mode": mode[0], "candidates": len(log),
                                  "candidate_ms": [sig(min(ok) * 1e3), sig(max(ok) * 1e3)],
                                  "default_ms": sig(log[0][1] * 1e3) if log[0][1] else None}
    torch.cuda.empty_cache()
    res["workload"] = ("64 hierarchies: base side uniform in {32,48,64,96,128}, 0-3 nests of "
                       "0.5-1.0 x base side (seed 4), order 6, BBKS z=50, 1LPT+2LPT+displacements, "
                       "%.1f M level-cells per batch" % (cells / 1e6))
    res["steps"] = steps
    res["mixed_error_per_member"] = {"max": sig(max(member_err)),
                                     "median": sig(statistics.median(member_err)),
                                     "persistent_max": sig(max(pers_err)),
                                     "against": "each member's float64 solve to 1e-12"}
    return res


def net_frac(frac, ms_per_launch, floor_us):
    """The roofline fraction with the event-pair floor taken off the event-timed launch
    duration: an upper bound of the kernel's own fraction (the raw one is a lower bound)."""
    if floor_us is None or not ms_per_launch or 1e3 * ms_per_launch <= floor_us:
        return None
    return frac * (1e3 * ms_per_launch) / (1e3 * ms_per_launch - floor_us)


def fp64_peak(pkg, device):
    """Measured FP64 FMA issue rate (G/s) of this GPU, best of three probes of ~0.3 s
    each, with the SM clock sampled meanwhile; (rate, clocks)."""
    from paper_1103_6031_gb300 import mg as _mg
    sampler = ClockSampler(device.index)
    sampler.start()
    time.sleep(0.3)
    rate = max(_mg.fp64_fma_rate(65536) for _ in range(3)) / 1e9
    clocks = sampler.stop()
    return rate, clocks


def solve_workload(pkg, name, deltas_np, steps, warmup, device, flush, barrier, dist, geom=None,
                   mixed_too=True, profile=True, profile_run=False, precision="fp64"):
    """The whole-step measurements of one workload on the GPU: float64 (device-side
    iteration loops) with the smoother's dominant launches event-timed, the RMS
    relative error of every output against a float64 solve to 1e-12, and (mixed_too)
    the mixed-precision variant with its own error and float32 smoother roofline."""
    import torch
    from synthetic.geometry import level_shapes
    geom = geom or workload(name)
    tol = WORKLOAD_TOL[name]
    mixed_tol = MIXED_TOL if name != "unigrid64" else tol
    lpt2 = name != "unigrid64"
    deltas = [torch.from_numpy(x).to(device) for x in deltas_np]
    dominant = max(n[0] * n[1] * n[2] for n in level_shapes(geom)) // 2
    big = "%d^3" % round((2 * dominant) ** (1.0 / 3.0))

    def make(cfg):
        h = pkg.Hierarchy(cfg)
        shapes = h.shapes
        out = {"phi1": [torch.empty(s, dtype=torch.float64, device=device) for s in shapes],
               "disp1": [torch.empty(s, dtype=torch.float64, device=device) for s in shapes for _ in range(3)]}
        if lpt2:
            out["phi2"] = [torch.empty(s, dtype=torch.float64, device=device) for s in shapes]
            out["disp2"] = [torch.empty(s, dtype=torch.float64, device=device) for s in shapes for _ in range(3)]
        return h, out

    def stepper(hh, out):
        def step():
            if lpt2:
                _, i1, i2 = hh.pipeline(deltas, out)
                return i1, i2
            phis, i1 = hh.solve_1lpt(deltas)
            disp = hh.displacements(phis)
            with torch.cuda.stream(hh.stream):
                for x, y in zip(out["phi1"], phis):
                    x.copy_(y)
                for x, y in zip(out["disp1"], [c for lv in disp for c in lv]):
                    x.copy_(y)
            return i1, None
        return step

    res = {"geom": geom, "dominant": dominant, "big": big}
    ref = None
    if not profile_run:
        hr, outr = make(pkg.config_from_geometry(geom, tol=REF_TOL, max_cycles=60))
        stepper(hr, outr)()
        torch.cuda.synchronize()
        ref = clone_outputs(outr)
        hr.close()
        del outr

    # ---- float64 ----
    if profile_run and precision == "mixed":
        cfg = pkg.config_from_geometry(geom, tol=mixed_tol, max_cycles=50, precision=pkg.MG_MIXED,
                                       inner_cycles=MIXED_INNER_CYCLES)
    else:
        # with the smoother's launches event-timed inside the timed steps the iteration
        # loops run on the host (one record read per V-cycle; a device-side loop cannot
        # carry event nodes); without events, on the device (the whole step is queued at
        # once and the host waits once per step)
        cfg = pkg.config_from_geometry(geom, tol=tol, max_cycles=50,
                                       device_loop=not profile and not profile_run)
    h, out = make(cfg)
    step = stepper(h, out)
    info = [None, None]

    def run():
        info[0], info[1] = step()
    for _ in range(warmup):
        run()
    h.stats(reset=True)
    if profile:
        h.set_profiling(["smooth"], min_cells=dominant)
    sampler = ClockSampler(device.index)
    sampler.start()
    time.sleep(0.4)
    step_ms = time_steps(run, steps, h.stream, flush, barrier)
    res["clocks"] = sampler.stop()
    stats = h.stats(reset=True)
    res["value"], res["ms_per_step"] = aggregate(sum(step_ms), geom.level_cells() * steps, steps,
                                                 dist, device)
    res["step_ms"] = step_ms
    res["launches"] = sum(v["launches"] for v in stats.values())
    res["info"] = list(info)
    res["smooth"] = stats["smooth"]
    res["error"] = output_errors(out, ref, geom.n_levels) if ref is not None else None
    res["h"], res["out"], res["step"], res["deltas"] = h, out, step, deltas
    res["loop"] = "host" if (profile or profile_run) else "device"
    if profile and not profile_run:
        # every level: one more step with every launch of every kernel family timed in
        # the first cycle of each solve
        from paper_1103_6031_gb300.mg import FAMILY_NAMES
        h.set_profiling(list(FAMILY_NAMES), min_cells=0)
        step()
        res["families"] = h.stats(reset=True)
        h.set_profiling([])
        # the same steps without events, iteration loops on the device
        hd, outd = make(pkg.config_from_geometry(geom, tol=tol, max_cycles=50, device_loop=True))
        stepd = stepper(hd, outd)
        for _ in range(warmup):
            stepd()
        dl_ms = time_steps(stepd, steps, hd.stream, flush, barrier)
        res["device_loop"] = {"ms_per_step": statistics.mean(dl_ms), "p99_ms": p99(dl_ms),
                              "value": geom.level_cells() / (statistics.mean(dl_ms) * 1e-3)}
        hd.close()
        del outd
    if not mixed_too or profile_run:
        return res

    # ---- mixed precision: same workload and stopping rule ----
    cfg_m = pkg.config_from_geometry(geom, tol=mixed_tol, max_cycles=50, precision=pkg.MG_MIXED,
                                     inner_cycles=MIXED_INNER_CYCLES)
    hm, outm = make(cfg_m)
    stepm = stepper(hm, outm)
    minfo = [None, None]

    def runm():
        minfo[0], minfo[1] = stepm()
    for _ in range(warmup):
        runm()
    hm.stats(reset=True)
    mixed_ms = time_steps(runm, steps, hm.stream, flush, barrier)
    mstats = hm.stats(reset=True)
    mv, mms = aggregate(sum(mixed_ms), geom.level_cells() * steps, steps, dist, device)
    merr = output_errors(outm, ref, geom.n_levels)
    # roofline of the float32 smoother from 3 more steps with CUDA events around its
    # largest launches (event nodes cost ~1 us each against ~10 us launches, so the
    # value above is taken without them)
    hm.set_profiling(["smooth"], min_cells=dominant)
    for _ in range(3):
        stepm()
    msm = hm.stats(reset=True)["smooth"]
    hm.set_profiling([])
    m_ms = msm["event_ms"] / max(msm["timed"], 1)
    m_upd = msm["timed_cells"] / max(msm["timed"], 1)
    # float32 in place: 8 B per level-cell (read u of both colours 4 B, f of the
    # updated colour 2 B, write the updated colour 2 B)
    m_gbs = 8.0 * 2 * m_upd / (m_ms * 1e-3) / 1e9
    shapes = level_shapes(geom)
    tma_nests = [n for n in shapes[1:] if n[0] * n[1] * n[2] // 2 == dominant
                 and n[0] * n[1] * n[2] >= TMA_MIN_CELLS]
    if not tma_nests and all(n[2] % 4 == 0 for n in shapes
                             if n[0] * n[1] * n[2] // 2 == dominant):
        m_kernel = "k_smooth_quad<%d> (%s levels)" % (geom.order, big)
        m_traffic = (SMOOTH_QUAD_F32_TRAFFIC_PER_UPDATE * m_upd
                     if geom.order == 6 and SMOOTH_QUAD_F32_TRAFFIC_PER_UPDATE else None)
    elif not tma_nests:
        m_kernel = "k_smooth_half<%d,float> (%s levels)" % (geom.order, big)
        m_traffic = SMOOTH_F32_TRAFFIC_PER_UPDATE * m_upd if geom.order == 6 else None
    else:
        m_kernel = "k_smooth_half_tma<%d,float> (%s nests)" % (geom.order, big)
        m_traffic = SMOOTH_TMA_F32_TRAFFIC_PER_UPDATE * m_upd if geom.order == 6 else None
    res["mixed"] = {
        "value": mv, "ms_per_step": mms,
        "latency_ms": {"p50": statistics.median(mixed_ms), "p99": p99(mixed_ms)},
        "outer": [minfo[0]["cycles"], minfo[1]["cycles"] if minfo[1] else None],
        "inner": [minfo[0]["inner_cycles"], minfo[1]["inner_cycles"] if minfo[1] else None],
        "launches": sum(v["launches"] for v in mstats.values()),
        "error": merr,
        "roofline": {"bound": "hbm", "achieved": m_gbs, "peak": HBM_PEAK_GBS, "unit": "GB/s",
                     "frac": m_gbs / HBM_PEAK_GBS, "traffic": m_traffic, "kernel": m_kernel,
                     "ms_per_launch": m_ms, "updates_per_launch": m_upd}}
    hm.close()
    return res


def run_serving_only(args):
    """Only the open-loop serving measurement (e.g. the large class at full size,
    --serve-large-side 256, at a given arrival rate); one JSON line."""
    pre = batch_inputs(args.serve_large_side, ())
    import torch
    torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_6031_gb300 as pkg
    r = serving_measure(pkg, pre[0], pre[1], pre[2], args.serve_seconds, args.serve_rate,
                        args.serve_workers, native=args.serve_impl == "native")
    print(json.dumps({"serving_only": True, "metric": "p50/p99 latency and completions/s of "
                      "open-loop Poisson arrivals", "serving": r}))
    return 0


def run_ours(args):
    world, rank, local = dist_env()
    name = args.workload
    do_batch = not args.profile_run and not args.no_batch
    extra = ("zoom2",) if (not args.profile_run and name == "deep_zoom") else ()
    pre = batch_inputs(args.serve_large_side if args.serve_seconds > 0 else None, extra) \
        if do_batch else None
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
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # open-loop serving first, in a fresh process: measured after the other sections
    # (hundreds of hierarchies made and destroyed, graphs cached), its p50 latency was
    # 6-15x worse than in a fresh process
    serving = None
    if pre is not None and args.serve_seconds > 0 and world == 1:
        serving = serving_measure(pkg, pre[0], pre[1], pre[2], args.serve_seconds,
                                  args.serve_rate, args.serve_workers,
                                  native=args.serve_impl == "native")
        torch.cuda.empty_cache()

    peak_fma, peak_clocks = fp64_peak(pkg, device) if not args.profile_run else (None, None)
    # what an event pair reads around an empty kernel node of a graph: the fixed cost in
    # every event-timed launch below (reported beside the raw fractions, not taken off them)
    from paper_1103_6031_gb300 import mg as _mg
    floor_us = None if args.profile_run else min(_mg.event_pair_floor(200) for _ in range(3))
    R = solve_workload(pkg, name, deltas_np, args.steps, args.warmup, device, flush, barrier, dist,
                       geom=geom, mixed_too=not args.profile_run, profile_run=args.profile_run,
                       precision=args.precision)
    h = R["h"]
    sm = R["smooth"]
    updates_per_launch = sm["timed_cells"] / max(sm["timed"], 1)
    ms_per_launch = sm["event_ms"] / max(sm["timed"], 1)
    ops = SMOOTH_OPS_PER_UPDATE[geom.order] * updates_per_launch
    achieved_gops = ops / (ms_per_launch * 1e-3) / 1e9
    smooth_gbs = SMOOTH_BYTES_PER_CELL * 2 * updates_per_launch / (ms_per_launch * 1e-3) / 1e9

    if args.profile_run:
        if rank == 0:
            print(json.dumps({"profile_run": True, "value": R["value"], "ms_per_step": R["ms_per_step"],
                              "gpu_launches": R["launches"],
                              "cycles": [R["info"][0]["cycles"],
                                         R["info"][1]["cycles"] if R["info"][1] else 0]}))
        h.close()
        if dist is not None:
            dist.destroy_process_group()
        return 0

    fam = R["families"]
    sa = fam["smooth"]
    all_ms = sa["event_ms"] / max(sa["timed"], 1)
    all_updates = sa["timed_cells"] / max(sa["timed"], 1)
    all_gops = SMOOTH_OPS_PER_UPDATE[geom.order] * all_updates / (all_ms * 1e-3) / 1e9
    est = {k: v["event_ms"] / max(v["timed"], 1) * v["launches"] for k, v in fam.items() if v["timed"]}
    share_kernel_time = est.get("smooth", 0.0) / max(sum(est.values()), 1e-12)

    # zoom2 beside the deep-zoom headline
    zoom2 = None
    if pre is not None and "zoom2" in pre[3]:
        Z = solve_workload(pkg, "zoom2", pre[3]["zoom2"], args.steps, args.warmup, device, flush,
                           barrier, dist, profile=False)
        zoom2 = {"level_cells": Z["geom"].level_cells(), "fp64": sig(Z["value"]),
                 "fp64_error": sig(Z["error"]["max"]), "mixed": sig(Z["mixed"]["value"]),
                 "mixed_error": sig(Z["mixed"]["error"]["max"]),
                 "mixed_smoother_frac": sig(Z["mixed"]["roofline"]["frac"], 3)}
        Z["h"].close()
        del Z

    generator = None
    if pre is not None:
        generator = generator_measure(pkg, args.steps, world == 1 and not args.skip_baseline)

    batched = None
    if pre is not None:
        batched = batched_measure(pkg, pre[0], pre[1], min(args.steps, 3), device)

    # end to end through the C ABI with pinned host buffers
    lpt2 = name != "unigrid64"
    shapes = h.shapes
    stream = h.stream
    host_in = [torch.from_numpy(x).pin_memory() for x in deltas_np]
    host_out = {"phi1": [torch.empty(s, dtype=torch.float64, pin_memory=True) for s in shapes],
                "disp1": [torch.empty(s, dtype=torch.float64, pin_memory=True) for s in shapes for _ in range(3)]}
    if lpt2:
        host_out["phi2"] = [torch.empty(s, dtype=torch.float64, pin_memory=True) for s in shapes]
        host_out["disp2"] = [torch.empty(s, dtype=torch.float64, pin_memory=True) for s in shapes for _ in range(3)]
    deltas = R["deltas"]

    def e2e_step():
        if lpt2:
            h.pipeline(host_in, host_out, host=True)
            return
        # 1LPT only: phi and -grad phi come back (the C ABI's host-buffer entry point
        # is the whole 2LPT step, so the copies are issued here)
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
        info1, info2 = R["info"]
        M = R["mixed"]
        peak = peak_fma
        line = {
            "metric": METRIC, "value": R["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": R["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(geom, name),
            "gpu_launches": R["launches"],
            "clocks": R["clocks"],
            "iteration_loop": ("host: one convergence-record read per V-cycle; the dominant "
                               "smoother launches of each solve's first cycle carry CUDA events"),
            "device_loop": {k: sig(v) for k, v in R["device_loop"].items()},
            "details": {
                "generator": generator,
                "batched_tuned": batched["mixed_batched_tuned"] if batched else None,
                "serving_full": serving,
                "roofline_all_levels": {"ms_per_launch": sig(all_ms), "updates_per_launch": all_updates,
                                        "achieved": sig(all_gops), "frac": sig(all_gops / peak, 3)},
                "smoother_share_of_kernel_time": sig(share_kernel_time, 3),
                "mixed_roofline_detail": {k: sig(v) for k, v in M["roofline"].items()},
            },
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": sig(statistics.mean(e2e_ms))},
        }
        if not args.skip_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(name)
            if not args.skip_all_cores:
                line["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(name)
        # the evidence a reader of the last part of the line sees
        line["latency_ms"] = {"p50": sig(statistics.median(R["step_ms"])), "p99": sig(p99(R["step_ms"]))}
        line["cycles"] = {"1lpt": info1["cycles"], "2lpt": info2["cycles"] if info2 else None,
                          "level_rel_residual_max": sig(max(info1["level_rel_residual"]
                                                            + (info2["level_rel_residual"] if info2 else [])))}
        line["error"] = {k: sig(v, 3) for k, v in R["error"].items()}
        line["error"]["against"] = "float64 solve to 1e-12 (oracle parity in the GPU tests)"
        line["roofline"] = {
            "bound": "alu", "achieved": sig(achieved_gops), "peak": sig(peak), "unit": "G FP64 instr/s",
            "frac": sig(achieved_gops / peak, 3),
            "traffic": (SMOOTH_TRAFFIC_PER_UPDATE * updates_per_launch
                        if SMOOTH_TRAFFIC_PER_UPDATE and geom.order == 6 else None),
            "kernel": "k_smooth_half<%d,double> (%s levels)" % (geom.order, R["big"]),
            "peak_source": "measured FP64 FMA issue rate (mg_fp64_fma_rate, 3 x 0.3 s, SM clock "
                           "%s MHz), of measured" % (peak_clocks or {}).get("sm_mhz"),
            "frac_of_nominal": sig(achieved_gops / 625.0, 3),
            "ms_per_launch": sig(ms_per_launch), "updates_per_launch": updates_per_launch,
            "hbm_frac": sig(smooth_gbs / HBM_PEAK_GBS, 3),
            "event_pair_floor_us": sig(floor_us),
            "frac_net_of_event_floor": sig(net_frac(achieved_gops / peak, ms_per_launch, floor_us), 3)}
        line["mixed_precision"] = {
            "value": sig(M["value"]), "ms_per_step": sig(M["ms_per_step"]),
            "p99_ms": sig(M["latency_ms"]["p99"]), "outer": M["outer"], "inner": M["inner"],
            "gpu_launches": M["launches"],
            "error": {k: sig(v, 3) for k, v in M["error"].items()},
            "smoother_hbm_frac": sig(M["roofline"]["frac"], 3),
            "smoother_hbm_frac_net_of_event_floor": sig(net_frac(M["roofline"]["frac"],
                                                                 M["roofline"]["ms_per_launch"],
                                                                 floor_us), 3)}
        if zoom2:
            line["zoom2"] = zoom2
        if batched:
            tb = batched["mixed_batched_tuned"]
            line["batched"] = {"fp64_h_per_s": batched["fp64_one_at_a_time"]["hierarchies_per_s"],
                               "mixed_h_per_s": batched["mixed_batched"]["hierarchies_per_s"],
                               "persistent_h_per_s": batched["mixed_persistent"]["hierarchies_per_s"],
                               "tuned_h_per_s": tb["hierarchies_per_s"],
                               "tuned": "%s, %d candidates %s ms" % (tb["launch_mode"], tb["candidates"],
                                                                   tb["candidate_ms"]),
                               "mixed_error_max": batched["mixed_error_per_member"]["max"]}
        if serving:
            line["serving"] = {"rate": serving["offered_rate_per_s"],
                               "done_per_s": serving["completed_per_s"],
                               "p50_ms": serving["latency_ms"]["p50"],
                               "p99_ms": serving["latency_ms"]["p99"],
                               "capacity_per_s": (serving["capacity"] or {}).get("requests_per_s"),
                               "utilisation": serving["utilisation"],
                               "large": serving["mix"].split(" base")[0].split("10% ")[-1],
                               "errors": serving["errors"]}
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
    ap.add_argument("--workload", choices=WORKLOADS, default="deep_zoom",
                    help="deep_zoom (default, the headline), zoom2, unigrid64 or zoom256")
    ap.add_argument("--skip-baseline", action="store_true",
                    help="leave out the CPU-oracle baseline")
    ap.add_argument("--skip-all-cores", action="store_true",
                    help="leave out the all-cores run of the CPU-oracle baseline")
    ap.add_argument("--profile-run", action="store_true",
                    help="timed steps only: no end-to-end pass, no CPU baseline (for ncu)")
    ap.add_argument("--no-batch", action="store_true",
                    help="leave out the zoom2, batched, serving and generator measurements")
    ap.add_argument("--serve-seconds", type=float, default=5.0,
                    help="seconds of open-loop arrivals in the serving measurement (0: none)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="mean arrivals per second")
    ap.add_argument("--serve-workers", type=int, default=96, help="concurrent requests at most")
    ap.add_argument("--serve-impl", choices=["native", "python"], default="native",
                    help="serving runtime: the C++ scheduler (mg_server_*) or Python threads")
    ap.add_argument("--serve-large-side", type=int, default=128,
                    help="side of the large request class (base and 3 nests); 256 is full size")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="precision of the timed steps of a --profile-run")
    ap.add_argument("--serving-only", action="store_true",
                    help="only the serving measurement (with --serve-large-side, --serve-rate)")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.serving_only:
        return run_serving_only(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
