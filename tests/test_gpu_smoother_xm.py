"""GPU: the float32 smoother with shared-memory plane tiles and an x-march against
the plain smoother kernel.

Both compute the same colour half-sweep (Sec. 3.2) with the same arithmetic in the
same order, so mixed-precision pipelines with the tiled kernel on every eligible level
(sides multiples of 4, 8 and 64) and with the plain kernel everywhere (MG_FLAG_NO_TMA)
agree bit for bit: periodic bases and nests, orders 2/4/6, levels whose x extent is
several blocks of 4 planes."""

import numpy as np
import pytest

from synthetic import Geometry, NestSpec, config_zoom2, make_delta

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


GEOMS = [
    # 64 x 64 x 128 periodic base + a 64 x 64 x 128 nest (both eligible), order 6
    Geometry((64, 64, 128), 40.0, 6, (NestSpec((64, 64, 128), (16, 16, 32)),)),
    # eligible base 128 x 64 x 64 (x: 32 blocks of 4 planes), nest 40 x 48 x 64, order 4
    Geometry((128, 64, 64), 50.0, 4, (NestSpec((40, 48, 64), (40, 12, 12)),)),
    # order 2, cubic 64 with a 32 x 32 x 64 nest
    Geometry((64, 64, 64), 1.0, 2, (NestSpec((32, 32, 64), (20, 20, 12)),)),
]


@pytest.mark.parametrize("geom", GEOMS, ids=["o6", "o4_aniso", "o2"])
def test_tiled_float32_smoother_bit_identical_to_plain(lib, geom):
    import torch
    deltas = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in make_delta(geom, 77)]
    outs = []
    for tma in ("auto", "off"):
        h = lib.Hierarchy(lib.config_from_geometry(geom, tol=1e-9, max_cycles=40,
                                                   precision=lib.MG_MIXED, inner_cycles=3,
                                                   tma=tma))
        outs.append(h.pipeline(deltas))
        h.close()
    (a, a1, a2), (b, b1, b2) = outs
    assert a1["history"] == b1["history"] and a2["history"] == b2["history"]
    for key in ("phi1", "phi2", "disp1", "disp2"):
        for x, y in zip(a[key], b[key]):
            assert torch.equal(x, y), key


def test_tiled_float32_smoother_on_zoom2(lib):
    import torch
    geom = config_zoom2()
    deltas = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in make_delta(geom, 2)]
    outs = []
    for tma in ("auto", "off"):
        h = lib.Hierarchy(lib.config_from_geometry(geom, tol=1e-8, max_cycles=40,
                                                   precision=lib.MG_MIXED, inner_cycles=4,
                                                   tma=tma))
        outs.append(h.pipeline(deltas)[0])
        h.close()
    for key in ("phi1", "phi2", "disp1", "disp2"):
        for x, y in zip(outs[0][key], outs[1][key]):
            assert torch.equal(x, y), key
