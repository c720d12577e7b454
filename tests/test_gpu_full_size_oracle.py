"""Full-size results against the converged CPU oracle.

The benchmark's claims are "<= 1e-6 RMS relative error" for the float64 step at its
stopping tolerance (relative leaf residual 3e-8) and for the mixed-precision step
(float32 V-cycles inside float64 refinement, stopping at 1e-8).  Here each claim meets an oracle array:
the oracle's whole step (both solves to a relative leaf residual of 1e-10, tau, both
displacement fields) on the zoom2 workload (128^3 base + 128^3 nest), the deep zoom
(128^3 base + 4 nests of 128^3), and the two request classes of the serving mix (a
hierarchy of the batched workload, and the large class, 128^3 base + 3 nests of
128^3), served through the native server.  The oracle runs in spawned worker
processes while the GPU work of the same test proceeds.
"""

import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ERR = 1e-6
ORACLE_TOL = 1e-10


def _case(name):
    from synthetic import config_batch, config_deep_zoom, config_zoom2, make_delta
    if name == "zoom2":
        geom, seed = config_zoom2(), 2
    elif name == "deep_zoom":
        geom, seed = config_deep_zoom(), 3
    elif name == "large":
        geom, seed = config_deep_zoom(seed=5, base=128, nest=128, levels=3, jitter=16), 5
    else:   # a member of the batched workload: 64^3 base with three nests
        geom = [g for g in config_batch() if g.base_n[0] == 64 and g.n_levels == 4][0]
        seed = 1000
    return geom, [np.ascontiguousarray(x) for x in make_delta(geom, seed)]


def _oracle_step(name):
    """Runs in a spawned process: the oracle's converged whole step."""
    from oracle.lpt import lpt_pipeline
    geom, deltas = _case(name)
    out = lpt_pipeline(geom, deltas, tol=ORACLE_TOL, max_cycles=40)
    return {"phi1": out["phi1"], "phi2": out["phi2"],
            "disp1": [c for lv in out["psi1"] for c in lv],
            "disp2": [c for lv in out["psi2"] for c in lv],
            "rel": (out["info1"]["rel_residual"], out["info2"]["rel_residual"])}


@pytest.fixture(scope="module")
def oracle():
    """Futures of the oracle's converged steps, computed in spawned processes."""
    ex = cf.ProcessPoolExecutor(max_workers=4, mp_context=mp.get_context("spawn"))
    futs = {n: ex.submit(_oracle_step, n) for n in ("deep_zoom", "large", "zoom2", "batch")}
    yield futs
    ex.shutdown(wait=True, cancel_futures=True)


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_6031_gb300 as pkg
    return pkg


def _rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b * b)))


def _check(out, ref, bound, what):
    worst = 0.0
    for key in ("phi1", "phi2", "disp1", "disp2"):
        for a, b in zip(out[key], ref[key]):
            e = _rel(a, b)
            worst = max(worst, e)
            assert e <= bound, (what, key, e)
    return worst


def _step(lib, geom, deltas, **kw):
    import torch
    h = lib.Hierarchy(lib.config_from_geometry(geom, max_cycles=50, **kw))
    out, i1, i2 = h.pipeline([torch.from_numpy(x).cuda() for x in deltas])
    out = {k: [x.cpu() for x in v] for k, v in out.items()}
    h.close()
    return out, i1, i2


@pytest.mark.parametrize("name", ["zoom2", "deep_zoom"])
def test_bench_workloads_within_1e6_of_converged_oracle(lib, oracle, name):
    """The benchmark's float64 and mixed-precision steps at its stopping tolerance:
    every output on every level within 1e-6 RMS relative of the converged oracle;
    float64 solved to 1e-12 within 1e-8 of it (both converge to one solution)."""
    import bench
    geom, deltas = _case(name)
    fp64, f1, f2 = _step(lib, geom, deltas, tol=bench.SOLVE_TOL)
    mixed, m1, m2 = _step(lib, geom, deltas, tol=bench.MIXED_TOL, precision=lib.MG_MIXED,
                          inner_cycles=bench.MIXED_INNER_CYCLES)
    tight, _, _ = _step(lib, geom, deltas, tol=1e-12)
    ref = oracle[name].result(timeout=1800)
    assert max(ref["rel"]) <= ORACLE_TOL
    assert max(f1["rel_residual"], f2["rel_residual"]) <= bench.SOLVE_TOL
    assert max(m1["rel_residual"], m2["rel_residual"]) <= bench.MIXED_TOL
    _check(fp64, ref, ERR, "fp64")
    _check(mixed, ref, ERR, "mixed")
    _check(tight, ref, 1e-8, "fp64 tight")


def test_served_results_of_each_request_class_within_1e6_of_oracle(lib, oracle):
    """One request of each class of the serving mix (mixed precision at the bench's
    stopping tolerance, pinned host buffers) through the native server, each output
    within 1e-6 RMS relative of the converged oracle."""
    import torch
    import bench
    from paper_1103_6031_gb300.serve import NativeServer, Request
    cases = {n: _case(n) for n in ("batch", "large")}
    server = NativeServer(max_active=4, hbm_budget=16 << 30, keep_outputs=True)
    reqs = {}
    for k, (n, (geom, deltas)) in enumerate(cases.items()):
        inner = bench.BATCH_INNER_CYCLES if n == "batch" else bench.MIXED_INNER_CYCLES
        cfg = lib.config_from_geometry(geom, tol=bench.MIXED_TOL, max_cycles=50, precision=lib.MG_MIXED,
                                       inner_cycles=inner)
        reqs[n] = Request(k, cfg, [torch.from_numpy(x).pin_memory() for x in deltas])
        server.submit(reqs[n])
    server.drain()
    server.close()
    for n, r in reqs.items():
        assert r.error is None, r.error
        ref = oracle[n].result(timeout=1800)
        _check(r.outputs, ref, ERR, "served " + n)
