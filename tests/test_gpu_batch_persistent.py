"""The persistent batch kernel (MG_FLAG_PERSISTENT): the float32 V-cycles of every
mixed-precision member of a batch run as one launch over a work list of (hierarchy,
level operation, block range) items.  Every member's result is bit-identical to its
solo run (the same operation bodies on the same data in the same order per member),
one member meets the float64 oracle within 1e-6, uneven members (orders 2/4/6,
0-2 nests, anisotropic, different inner-cycle counts) mix in one launch, and the
bounded dependency wait reports MG_ETIMEOUT through its self-test."""

import numpy as np
import pytest

from oracle.lpt import lpt_pipeline
from synthetic import Geometry, NestSpec, config_batch, make_delta, small_zoom

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_6031_gb300 as pkg
    return pkg


MEMBERS = [
    small_zoom(24, ((20, 7), (16, 6)), order=6, box=50.0),
    Geometry((32, 32, 32), 64.0, 4, ()),
    small_zoom(32, ((24, 8),), order=6, box=80.0),
    Geometry((24, 32, 40), 24.0, 6, (NestSpec((14, 20, 18), (7, 6, 9)),)),
    small_zoom(16, ((16, 4),), order=2, box=20.0),
    small_zoom(32, ((28, 10),), order=4, box=30.0),
    Geometry((48, 48, 48), 10.0, 6, ()),
]


def _cfg(lib, geom, persistent, inner=3, tol=1e-9):
    return lib.config_from_geometry(geom, tol=tol, max_cycles=40, precision=lib.MG_MIXED,
                                    inner_cycles=inner, persistent=persistent)


def _dev(arrs):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in arrs]


def test_persistent_batch_equals_solo_runs(lib):
    import torch
    deltas = [_dev(make_delta(g, 60 + i)) for i, g in enumerate(MEMBERS)]
    inner = [3, 2, 4, 3, 2, 3, 4]
    solo = []
    for g, d, n in zip(MEMBERS, deltas, inner):
        h = lib.Hierarchy(_cfg(lib, g, False, n))
        solo.append(h.pipeline(d))
        h.close()
    members = [lib.Hierarchy(_cfg(lib, g, True, n)) for g, n in zip(MEMBERS, inner)]
    batch = lib.Batch(members)
    for rep in range(2):  # the second pass replays the cached launches
        outs, infos1, infos2 = batch.pipeline(deltas)
        for i, (out, i1, i2) in enumerate(solo):
            assert infos1[i]["cycles"] == i1["cycles"] and infos2[i]["cycles"] == i2["cycles"]
            assert infos1[i]["history"] == i1["history"]
            for key in ("phi1", "phi2", "disp1", "disp2"):
                for a, b in zip(outs[i][key], out[key]):
                    assert torch.equal(a, b), (i, key, rep)
    batch.close()
    for h in members:
        h.close()


def test_persistent_batch_member_matches_oracle(lib):
    geom = MEMBERS[0]
    deltas = make_delta(geom, 61)
    ref = lpt_pipeline(geom, deltas, tol=1e-12, max_cycles=40)
    members = [lib.Hierarchy(_cfg(lib, g, True, tol=1e-10)) for g in MEMBERS[:3]]
    ins = [_dev(make_delta(g, 61 + i)) for i, g in enumerate(MEMBERS[:3])]
    outs, i1, _ = lib.Batch(members).pipeline(ins)
    assert i1[0]["rel_residual"] <= 1e-10

    def rel(a, b):
        a = a.cpu().numpy()
        return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b * b)))
    for l in range(geom.n_levels):
        assert rel(outs[0]["phi1"][l], ref["phi1"][l]) <= 1e-6
        assert rel(outs[0]["phi2"][l], ref["phi2"][l]) <= 1e-6
        for a in range(3):
            assert rel(outs[0]["disp1"][3 * l + a], ref["psi1"][l][a]) <= 1e-6
            assert rel(outs[0]["disp2"][3 * l + a], ref["psi2"][l][a]) <= 1e-6


def test_persistent_batch_on_benchmark_members(lib):
    """Sixteen hierarchies of the 64-hierarchy workload (bases 32-128, 0-3 nests,
    order 6): persistent and per-operation batches give bit-identical results."""
    import torch
    geoms = config_batch()[:16]
    deltas = [_dev(make_delta(g, 1000 + i)) for i, g in enumerate(geoms)]
    res = []
    for persistent in (False, True):
        hs = [lib.Hierarchy(_cfg(lib, g, persistent, 4, 1e-8)) for g in geoms]
        b = lib.Batch(hs)
        outs, i1, i2 = b.pipeline(deltas)
        res.append((outs, i1, i2))
        b.close()
        for h in hs:
            h.close()
    (oa, a1, a2), (ob, b1, b2) = res
    for i in range(len(geoms)):
        assert a1[i]["history"] == b1[i]["history"] and a2[i]["history"] == b2[i]["history"]
        for key in ("phi1", "phi2", "disp1", "disp2"):
            for x, y in zip(oa[i][key], ob[i][key]):
                assert torch.equal(x, y), (i, key)


def test_persistent_wait_limit_selftest(lib):
    from paper_1103_6031_gb300 import mg
    assert mg.selftest_persist_wait() == "MG_ETIMEOUT"
    # the context stays usable: a persistent batch right after it is still correct
    test_persistent_batch_member_matches_oracle(lib)
