"""Device-side iteration loop (MG_FLAG_DEVICE_LOOP): one CUDA graph per solve whose
while node repeats the iteration and whose last kernel applies the stopping rule
(and the mixed-precision inner-cycle plan) on the device.  It must give exactly the
host loop's results: the same iteration counts, residual histories, launches and
bit-identical outputs, alone, through the pipeline and through the native server.
The float64 results are also checked against the oracle at the matched cycle count.
"""

import numpy as np
import pytest

from oracle.multigrid import solve as oracle_solve
from synthetic import Geometry, make_delta, make_delta_powerlaw, small_zoom

pytestmark = pytest.mark.gpu

CASES = [
    ("unigrid32_o2_fp64", Geometry((32,) * 3, 1.0, 2, ()), False),
    ("zoom_o6_fp64", small_zoom(32, ((24, 8),), order=6, box=80.0), False),
    ("zoom2deep_o4_fp64", small_zoom(32, ((24, 8), (16, 8)), order=4, box=60.0), False),
    ("zoom_o6_mixed", small_zoom(32, ((24, 8),), order=6, box=80.0), True),
    ("zoom2deep_o6_mixed", small_zoom(32, ((24, 8), (16, 8)), order=6, box=60.0), True),
]


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_6031_gb300 as pkg
    return pkg


def _cfg(lib, geom, mixed, device_loop, **kw):
    args = dict(tol=1e-9, max_cycles=40)
    args.update(kw)
    if mixed:
        args.update(precision=lib.MG_MIXED, inner_cycles=4)
    return lib.config_from_geometry(geom, device_loop=device_loop, **args)


def _inputs(geom, seed):
    import torch
    if geom.nests:
        arrs = make_delta(geom, seed)
    else:
        arrs = [make_delta_powerlaw(tuple(geom.base_n), seed)]
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in arrs]


def _same_info(a, b):
    assert a["cycles"] == b["cycles"]
    assert a["inner_cycles"] == b["inner_cycles"]
    assert a["rel_residual"] == b["rel_residual"]
    assert a["source_mean"] == b["source_mean"]
    assert a["history"] == b["history"]
    assert a["level_rel_residual"] == b["level_rel_residual"]


@pytest.mark.parametrize("name,geom,mixed", CASES, ids=[c[0] for c in CASES])
def test_device_loop_equals_host_loop(lib, name, geom, mixed):
    import torch
    d = _inputs(geom, 11)
    outs, infos, launches = [], [], []
    for device_loop in (False, True):
        h = lib.Hierarchy(_cfg(lib, geom, mixed, device_loop))
        for _ in range(2):  # the second pass replays the cached graphs
            h.stats(reset=True)
            out, i1, i2 = h.pipeline(d)
        st = h.stats()
        h.close()
        outs.append(out)
        infos.append((i1, i2))
        launches.append({k: v["launches"] for k, v in st.items()})
    _same_info(infos[0][0], infos[1][0])
    _same_info(infos[0][1], infos[1][1])
    assert launches[0] == launches[1]
    for key in ("phi1", "phi2", "disp1", "disp2"):
        for a, b in zip(outs[0][key], outs[1][key]):
            assert torch.equal(a, b), key


def test_device_loop_fixed_cycle_count_matches_oracle(lib):
    """tol = 0: exactly max_cycles iterations on the device; the float64 result
    matches the oracle's at the same cycle count."""
    geom = small_zoom(32, ((24, 8),), order=6, box=80.0)
    deltas = make_delta(geom, 12)
    h = lib.Hierarchy(_cfg(lib, geom, False, True, tol=0.0, max_cycles=5))
    import torch
    phis, info = h.solve_1lpt([torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in deltas])
    h.close()
    assert info["cycles"] == 5 and len(info["history"]) == 5
    ref, _ = oracle_solve(geom, deltas, tol=0.0, cycles=5)
    for a, b in zip(phis, ref):
        a = a.cpu().numpy()
        assert np.sqrt(np.sum((a - b) ** 2) / np.sum(b * b)) < 1e-10


def test_device_loop_through_native_server(lib):
    import torch
    from paper_1103_6031_gb300.serve import NativeServer, Request
    geom = small_zoom(32, ((24, 8),), order=6, box=80.0)
    host = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in make_delta(geom, 13)]
    ref = lib.Hierarchy(_cfg(lib, geom, True, False))
    want, w1, w2 = ref.pipeline(host, host=True)
    ref.close()
    cfg = _cfg(lib, geom, True, True)
    server = NativeServer(max_active=4, hbm_budget=8 * lib.workspace_bytes(cfg))
    reqs = [Request(k, cfg, host) for k in range(6)]
    for r in reqs:
        server.submit(r)
    assert server.drain(timeout=120)
    server.close()
    for r in reqs:
        assert r.error is None, r.error
        _same_info(r.info[0], w1)
        _same_info(r.info[1], w2)
        for key in ("phi1", "phi2", "disp1", "disp2"):
            for a, b in zip(r.outputs[key], want[key]):
                assert torch.equal(a, b), key


def test_device_loops_in_a_batch_equal_solo_host_loops(lib):
    """A batch whose members all run device-side loops launches every member's loop
    graph on its own stream; each member's results equal its solo host-loop run."""
    import torch
    members = [(geom, mixed, _inputs(geom, 20 + i)) for i, (_, geom, mixed) in enumerate(CASES)]
    want = []
    for geom, mixed, d in members:
        h = lib.Hierarchy(_cfg(lib, geom, mixed, False))
        want.append(h.pipeline(d))
        h.close()
    hs = [lib.Hierarchy(_cfg(lib, geom, mixed, True)) for geom, mixed, _ in members]
    batch = lib.Batch(hs)
    outs, i1, i2 = batch.pipeline([d for _, _, d in members])
    batch.close()
    for h in hs:
        h.close()
    for k, (wout, w1, w2) in enumerate(want):
        _same_info(i1[k], w1)
        _same_info(i2[k], w2)
        for key in ("phi1", "phi2", "disp1", "disp2"):
            for a, b in zip(outs[k][key], wout[key]):
                assert torch.equal(a, b), (k, key)
