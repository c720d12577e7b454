"""Batched solves: every member of a batch gives exactly (bit for bit) what the
same hierarchy gives alone, for float64 and mixed-precision members of
different geometries and orders in one batch; and the batched mixed-precision
results stay within 1e-6 of the float64 oracle."""

import numpy as np
import pytest

from oracle.lpt import lpt_pipeline
from synthetic import Geometry, NestSpec, make_delta, small_zoom

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
    (small_zoom(16, ((16, 4),), order=2, box=20.0), "fp64"),
    (small_zoom(24, ((20, 7), (16, 6)), order=6, box=50.0), "mixed"),
    (Geometry((32, 32, 32), 64.0, 4, ()), "mixed"),
    (Geometry((24, 32, 40), 24.0, 6, (NestSpec((14, 20, 18), (7, 6, 9)),)), "fp64"),
    (small_zoom(32, ((24, 8),), order=6, box=80.0), "mixed"),
    (Geometry((48, 48, 48), 10.0, 6, ()), "fp64"),
    (small_zoom(32, ((32, 8),), order=6, box=30.0), "fp64"),
    (small_zoom(48, ((48, 12), (40, 10)), order=6, box=60.0), "fp64"),
    (small_zoom(32, ((28, 10),), order=4, box=30.0), "mixed"),
    (Geometry((64, 64, 64), 100.0, 6, ()), "fp64"),
]


def _cfg(lib, geom, prec):
    kw = dict(tol=1e-9, max_cycles=40)
    if prec == "mixed":
        kw.update(precision=lib.MG_MIXED, inner_cycles=3)
    return lib.config_from_geometry(geom, **kw)


def _dev(arrs):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in arrs]


def test_batch_members_equal_solo_runs(lib):
    import torch
    deltas = [_dev(make_delta(g, 40 + i)) for i, (g, _) in enumerate(MEMBERS)]
    solo = []
    for (g, prec), d in zip(MEMBERS, deltas):
        h = lib.Hierarchy(_cfg(lib, g, prec))
        out, i1, i2 = h.pipeline(d)
        solo.append((out, i1, i2))
        h.close()
    members = [lib.Hierarchy(_cfg(lib, g, prec)) for g, prec in MEMBERS]
    batch = lib.Batch(members)
    for rep in range(2):
        outs, infos1, infos2 = batch.pipeline(deltas)
        for i, (out, i1, i2) in enumerate(solo):
            assert infos1[i]["cycles"] == i1["cycles"] and infos2[i]["cycles"] == i2["cycles"]
            for key in ("phi1", "phi2", "disp1", "disp2"):
                for a, b in zip(outs[i][key], out[key]):
                    assert torch.equal(a, b), (i, key, rep)
    batch.close()


def test_batch_mixed_matches_oracle(lib):
    geom = MEMBERS[1][0]
    deltas = make_delta(geom, 41)
    ref = lpt_pipeline(geom, deltas, tol=1e-12, max_cycles=40)
    members = [lib.Hierarchy(_cfg(lib, g, p)) for g, p in MEMBERS[:3]]
    ins = [_dev(make_delta(g, 40 + i)) for i, (g, _) in enumerate(MEMBERS[:3])]
    outs, _, _ = lib.Batch(members).pipeline(ins)
    for l in range(geom.n_levels):
        a = outs[1]["phi1"][l].cpu().numpy()
        assert np.sqrt(np.sum((a - ref["phi1"][l]) ** 2) / np.sum(ref["phi1"][l] ** 2)) <= 1e-6
        a = outs[1]["disp2"][3 * l].cpu().numpy()
        b = ref["psi2"][l][0]
        assert np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)) <= 1e-6
