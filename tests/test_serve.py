"""Serving loop: admission bookkeeping on the CPU, and on the GPU that every
request served in a concurrent mix (several workers, evictions forced by a small
HBM budget) returns exactly what the same request returns when served alone."""

import numpy as np
import pytest

from synthetic import Geometry, make_delta, small_zoom


def _adm(budget, sizes):
    from paper_1103_6031_gb300.serve import Admission
    closed = []
    adm = Admission(budget, workspace_bytes=lambda cfg: sizes[cfg], close=closed.append)
    return adm, closed


def test_admission_respects_budget_and_evicts_idle_lru():
    adm, closed = _adm(100, {"a": 40, "b": 40, "c": 40, "d": 90})
    ea = adm.reserve("A", "a")
    ea[0] = "hA"
    eb = adm.reserve("B", "b")
    eb[0] = "hB"
    assert adm.reserve("C", "c") is None          # 120 > 100 and nothing idle
    adm.release(ea)
    ec = adm.reserve("C", "c")                     # evicts the idle A
    assert ec is not None and closed == ["hA"] and adm.resident == 80
    assert adm.reserve("B", "b") is None           # B is busy
    adm.release(eb)
    assert adm.reserve("B", "b") is eb             # cached and idle: reused, no new bytes
    assert adm.resident == 80 and adm.peak <= 100
    adm.release(eb)
    adm.release(ec)
    ed = adm.reserve("D", "d")                     # needs both evicted, LRU first (C, then B)
    assert ed is not None and closed == ["hA", "hB"] and adm.resident == 90  # C had no handle yet
    assert adm.evictions == 3


def test_admission_never_evicts_busy_entries():
    adm, closed = _adm(50, {"a": 30, "b": 30})
    ea = adm.reserve("A", "a")
    assert adm.reserve("B", "b") is None
    assert closed == [] and adm.resident == 30
    adm.release(ea)
    assert adm.reserve("B", "b") is not None and adm.resident == 30


GEOMS = [
    (small_zoom(16, ((16, 4),), order=2, box=20.0), 0),
    (small_zoom(24, ((20, 7),), order=6, box=50.0), 1),
    (Geometry((32, 32, 32), 64.0, 4, ()), 1),
    (small_zoom(32, ((24, 8),), order=6, box=80.0), 0),
]


@pytest.mark.gpu
def test_results_are_identical_alone_and_in_the_mix():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_6031_gb300 as pkg
    from paper_1103_6031_gb300.serve import Request, Server, latency_stats, run_open_loop

    def cfg(i):
        g, mixed = GEOMS[i % len(GEOMS)]
        kw = dict(tol=1e-9, max_cycles=40)
        if mixed:
            kw.update(precision=pkg.MG_MIXED, inner_cycles=3)
        return pkg.config_from_geometry(g, **kw)

    inputs = [[torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
               for x in make_delta(g, 70 + i)] for i, (g, _) in enumerate(GEOMS)]
    n = 24
    reqs = [Request(k, cfg(k), inputs[k % len(GEOMS)]) for k in range(n)]
    # budget: room for about two hierarchies at once, so the mix forces evictions
    budget = 2 * max(pkg.workspace_bytes(cfg(i)) for i in range(len(GEOMS)))
    server = Server(workers=3, hbm_budget=budget)
    run_open_loop(server, reqs, rate=2000.0)
    stats = latency_stats(reqs)
    assert server.peak_inflight >= 2 and server.admission.evictions > 0
    assert server.admission.peak <= budget
    server.close()
    assert stats["count"] == n and stats["p99_ms"] >= stats["p50_ms"] > 0
    for k in range(len(GEOMS)):
        alone = pkg.Hierarchy(cfg(k))
        out, _, _ = alone.pipeline(inputs[k], host=True)
        alone.close()
        for r in reqs[k::len(GEOMS)]:
            assert r.error is None
            for key in ("phi1", "phi2", "disp1", "disp2"):
                for a, b in zip(r.outputs[key], out[key]):
                    assert torch.equal(a, b), (r.id, key)
