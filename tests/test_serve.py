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


def test_admission_runs_overlapping_requests_of_one_config_on_separate_instances():
    adm, closed = _adm(100, {"a": 40})
    e1 = adm.reserve("A", "a")
    e2 = adm.reserve("A", "a")                     # first instance busy: a second one
    assert e1 is not None and e2 is not None and e1 is not e2
    assert adm.instances("A") == 2 and adm.resident == 80
    assert adm.reserve("A", "a") is None           # a third would exceed the budget
    adm.release(e2)
    assert adm.reserve("A", "a") is e2             # idle instance reused
    adm.release(e1)
    adm.release(e2)
    adm.reserve("A", "a")
    assert adm.instances("A") == 2 and closed == [] and adm.evictions == 0


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


@pytest.mark.gpu
def test_concurrent_creation_from_one_shared_config():
    """Several worker threads create hierarchies from one shared config struct at
    once (the serving cache holds several instances of a busy configuration); the
    binding works on private copies, so the caller's struct is never written and
    every instance solves correctly."""
    import threading
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_6031_gb300 as pkg
    geom = small_zoom(24, ((20, 7),), order=6, box=50.0)
    cfg = pkg.config_from_geometry(geom, tol=1e-9, max_cycles=40)
    deltas = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in make_delta(geom, 91)]
    ref = pkg.Hierarchy(cfg)
    want, _, _ = ref.pipeline(deltas, host=True)
    ref.close()
    results, errors = [None] * 8, []

    def work(i):
        try:
            torch.cuda.set_device(0)
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                h = pkg.Hierarchy(cfg, stream=s)
                results[i], _, _ = h.pipeline(deltas, host=True)
                h.close()
        except Exception as exc:  # reported below
            errors.append(exc)

    threads = [threading.Thread(target=work, args=(i,)) for i in range(8)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    assert not cfg.dev_alloc and not cfg.dev_free
    for out in results:
        for key in ("phi1", "phi2", "disp1", "disp2"):
            for a, b in zip(out[key], want[key]):
                assert torch.equal(a, b), key


def _native_setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_6031_gb300 as pkg
    return torch, pkg


@pytest.mark.gpu
def test_native_server_results_equal_solo_runs_under_eviction():
    """mg_server_*: mixed float64 and mixed-precision requests of three
    configurations, several of each in flight at once, under a budget of about
    two hierarchies (so idle ones are closed to make room); every result equals a
    solo Hierarchy.pipeline(host=True) bit for bit."""
    torch, pkg = _native_setup()
    from paper_1103_6031_gb300.serve import NativeServer, Request, latency_stats, run_open_loop

    def cfg(i):
        g, mixed = GEOMS[i % len(GEOMS)]
        kw = dict(tol=1e-9, max_cycles=40)
        if mixed:
            kw.update(precision=pkg.MG_MIXED, inner_cycles=3)
        return pkg.config_from_geometry(g, **kw)

    inputs = [[torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
               for x in make_delta(g, 70 + i)] for i, (g, _) in enumerate(GEOMS)]
    n = 30
    reqs = [Request(k, cfg(k), inputs[k % len(GEOMS)]) for k in range(n)]
    budget = 2 * max(pkg.workspace_bytes(cfg(i)) for i in range(len(GEOMS)))
    server = NativeServer(max_active=4, hbm_budget=budget)
    run_open_loop(server, reqs, rate=3000.0)
    st = server.stats()
    server.close()
    stats = latency_stats(reqs)
    assert stats["count"] == n and stats["p99_ms"] >= stats["p50_ms"] > 0
    assert st["completed"] == n and st["pending"] == 0 and st["active"] == 0
    assert st["evictions"] > 0 and st["peak_bytes"] <= budget and st["peak_active"] >= 2
    for k in range(len(GEOMS)):
        alone = pkg.Hierarchy(cfg(k))
        out, i1, i2 = alone.pipeline(inputs[k], host=True)
        alone.close()
        for r in reqs[k::len(GEOMS)]:
            assert r.error is None, r.error
            assert r.info[0]["cycles"] == i1["cycles"] and r.info[1]["cycles"] == i2["cycles"]
            assert r.admitted is None or r.arrival <= r.admitted + 1e-3
            for key in ("phi1", "phi2", "disp1", "disp2"):
                for a, b in zip(r.outputs[key], out[key]):
                    assert torch.equal(a, b), (r.id, key)


@pytest.mark.gpu
def test_native_server_runs_overlapping_requests_of_one_config_concurrently():
    """Eight requests of one configuration at once get one hierarchy each (the
    budget holds them all) and run together."""
    torch, pkg = _native_setup()
    from paper_1103_6031_gb300.serve import NativeServer, Request
    geom = small_zoom(24, ((20, 7),), order=6, box=50.0)
    cfg = pkg.config_from_geometry(geom, tol=1e-9, max_cycles=40)
    deltas = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in make_delta(geom, 91)]
    server = NativeServer(max_active=8, hbm_budget=64 * pkg.workspace_bytes(cfg))
    reqs = [Request(k, cfg, deltas) for k in range(8)]
    for r in reqs:
        server.submit(r)
    assert server.drain(timeout=120)
    st = server.stats()
    server.close()
    assert st["instances"] == st["created"] >= 2 and st["evictions"] == 0
    first = reqs[0].outputs
    for r in reqs:
        assert r.error is None, r.error
        for key in ("phi1", "phi2", "disp1", "disp2"):
            for a, b in zip(r.outputs[key], first[key]):
                assert torch.equal(a, b), key


@pytest.mark.gpu
def test_native_server_rejects_invalid_and_oversized_requests():
    torch, pkg = _native_setup()
    from paper_1103_6031_gb300 import mg
    from paper_1103_6031_gb300.serve import NativeServer, Request
    geom = Geometry((32, 32, 32), 64.0, 2, ())
    good = pkg.config_from_geometry(geom, tol=1e-9, max_cycles=40)
    deltas = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in make_delta(geom, 5)]
    server = NativeServer(max_active=2, hbm_budget=pkg.workspace_bytes(good))
    bad = pkg.config_from_geometry(geom, tol=1e-9, max_cycles=40)
    bad.order = 5
    with pytest.raises(mg.MGError) as e1:
        server.submit(Request(0, bad, deltas))
    assert e1.value.status == 1
    big_geom = Geometry((64, 64, 64), 64.0, 2, ())
    big = pkg.config_from_geometry(big_geom, tol=1e-9, max_cycles=40)
    with pytest.raises(mg.MGError) as e2:
        server.submit(Request(1, big, deltas))
    assert e2.value.status == 2
    # the C entry point checks the same on its own
    import ctypes
    arr = ctypes.cast(mg._ptrs(deltas, [(32, 32, 32)], True), ctypes.POINTER(ctypes.c_void_p))
    assert server.lib.mg_server_submit(server.h, 98, ctypes.byref(bad), arr, None, None, None,
                                       None) == 1
    assert server.lib.mg_server_submit(server.h, 99, ctypes.byref(big), arr, None, None, None,
                                       None) == 2
    assert server.lib.mg_server_submit(server.h, 97, ctypes.byref(good), None, None, None, None,
                                       None) == 1
    r = Request(2, good, deltas)
    server.submit(r)
    assert server.drain(timeout=60)
    server.close()
    assert r.error is None and r.info[0]["rel_residual"] <= 1e-9


@pytest.mark.gpu
def test_native_server_recycles_output_sets_when_results_are_dropped():
    """With keep_outputs=False a finished request's pinned output set goes back to a
    pool and the next request of the same shapes reuses it (no pinned allocation in
    the submitting thread); a request kept after that still gets correct results."""
    torch, pkg = _native_setup()
    from paper_1103_6031_gb300.serve import NativeServer, Request
    geom, _ = GEOMS[1]
    cfg = pkg.config_from_geometry(geom, tol=1e-9, max_cycles=40)
    inputs = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in make_delta(geom, 5)]
    server = NativeServer(max_active=2, hbm_budget=8 << 30, keep_outputs=False)
    server.reserve_outputs(cfg, 1)
    key = next(iter(server._pool))
    first = server._pool[key][-1]
    r = Request(0, cfg, inputs)
    server.submit(r)
    assert len(server._pool[key]) == 0          # the reserved set is in use
    server.drain()
    assert r.error is None and r.outputs is None
    assert len(server._pool[key]) == 1 and server._pool[key][0] is first
    server.keep_outputs = True
    r2 = Request(1, cfg, inputs)
    server.submit(r2)
    server.drain()
    server.close()
    alone = pkg.Hierarchy(cfg)
    want, _, _ = alone.pipeline(inputs, host=True)
    alone.close()
    for k in ("phi1", "phi2", "disp1", "disp2"):
        for a, b in zip(r2.outputs[k], want[k]):
            assert torch.equal(a, b), k


@pytest.mark.gpu
def test_native_server_bounds_pinned_sets_for_dropped_results():
    """Requests whose results are dropped allocate at most `dropped_sets` pinned output
    sets per shape; more overlapping ones write into a set already in use (nobody reads
    it), so a burst allocates nothing in the submitting thread and still completes."""
    torch, pkg = _native_setup()
    from paper_1103_6031_gb300.serve import NativeServer, Request
    geom, _ = GEOMS[0]
    cfg = pkg.config_from_geometry(geom, tol=1e-9, max_cycles=40)
    inputs = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in make_delta(geom, 6)]
    server = NativeServer(max_active=8, hbm_budget=8 << 30, keep_outputs=False)
    reqs = [Request(k, cfg, inputs) for k in range(12)]
    for r in reqs:
        server.submit(r)
    server.drain()
    key = next(iter(server._owned))
    assert len(server._owned[key]) == server.dropped_sets
    assert all(r.error is None and r.done is not None for r in reqs)
    server.close()


@pytest.mark.gpu
def test_native_server_instance_cap():
    """With at most one hierarchy per configuration, overlapping requests of one
    configuration wait for it instead of getting new ones: one hierarchy is created,
    and every result equals the solo run bit for bit."""
    torch, pkg = _native_setup()
    from paper_1103_6031_gb300.serve import NativeServer, Request
    geom, _ = GEOMS[1]
    cfg = pkg.config_from_geometry(geom, tol=1e-9, max_cycles=40)
    inputs = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in make_delta(geom, 8)]
    server = NativeServer(max_active=8, hbm_budget=8 << 30)
    server.set_max_instances(1)
    reqs = [Request(k, cfg, inputs) for k in range(6)]
    for r in reqs:
        server.submit(r)
    assert server.drain(timeout=120)
    st = server.stats()
    server.close()
    assert st["created"] == 1 and st["completed"] == 6
    alone = pkg.Hierarchy(cfg)
    want, _, _ = alone.pipeline(inputs, host=True)
    alone.close()
    for r in reqs:
        assert r.error is None
        for k in ("phi1", "phi2", "disp1", "disp2"):
            for a, b in zip(r.outputs[k], want[k]):
                assert torch.equal(a, b), (r.id, k)


def test_output_set_views_tile_one_allocation():
    """NativeServer.output_set: phi1, phi2 (one per level), disp1, disp2 (three per level)
    are contiguous views of one allocation that tile it exactly, in that order, without
    overlap (host logic; pinning itself needs a GPU and is replaced here)."""
    import torch
    from paper_1103_6031_gb300.serve import NativeServer

    class _Torch:
        float64 = torch.float64

        @staticmethod
        def empty(*a, **k):
            k.pop("pin_memory", None)
            return torch.empty(*a, **k)

    fake = type("S", (), {"_torch": _Torch})()
    shapes = [(4, 6, 8), (10, 12, 16)]
    out = NativeServer.output_set(fake, shapes)
    order = out["phi1"] + out["phi2"] + out["disp1"] + out["disp2"]
    assert [tuple(v.shape) for v in out["phi1"]] == shapes == [tuple(v.shape) for v in out["phi2"]]
    assert [tuple(v.shape) for v in out["disp1"]] == [s for s in shapes for _ in range(3)]
    base = order[0].untyped_storage().data_ptr()
    pos = 0
    for v in order:
        assert v.is_contiguous() and v.untyped_storage().data_ptr() == base
        assert v.storage_offset() == pos
        pos += v.numel()
    assert pos == order[0].untyped_storage().nbytes() // 8
