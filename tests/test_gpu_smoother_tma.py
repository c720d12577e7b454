"""GPU: the TMA-staged smoother kernel against the plain smoother kernel and the
oracle.

The smoother kernels compute the same colour half-sweep (Sec. 3.2) with the
same arithmetic in the same order, so whole pipelines run with any of them
on every level must agree bit for bit, in float64 and in mixed precision.
The geometries span several z tiles (64 cells), y tiles (8 rows) and x chunks,
with ragged tails on each axis, all three stencil orders, periodic and nested
levels.
"""

import numpy as np
import pytest

from oracle.lpt import lpt_pipeline
from synthetic import Geometry, NestSpec, config_zoom2, make_delta, small_zoom

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_6031_gb300 as pkg
    return pkg


def to_dev(arrs):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in arrs]


def rel(a, b):
    a = a.detach().cpu().numpy()
    return float(np.sqrt(np.sum((a - b) ** 2) / max(np.sum(b * b), 1e-300)))


GEOMS = [
    # ragged on every axis: z 100 (2 tiles, second partial), y 44, x 36
    Geometry((36, 44, 100), 30.0, 6, (NestSpec((24, 18, 70), (6, 13, 15)),)),
    Geometry((40, 24, 136), 20.0, 4, (NestSpec((30, 20, 64), (5, 6, 30)),)),
    Geometry((34, 34, 34), 1.0, 2, (NestSpec((18, 18, 18), (9, 8, 11)),)),
    small_zoom(32, ((24, 8), (20, 6)), order=6, box=80.0),
]
IDS = ["o6_ragged", "o4_ragged", "o2_base34", "o6_L3"]


def run(lib, geom, deltas, tma, **kw):
    cfg = lib.config_from_geometry(geom, tma=tma, **kw)
    h = lib.Hierarchy(cfg)
    out, i1, i2 = h.pipeline(to_dev(deltas), allow_noconv=True)
    h.close()
    return out, i1, i2


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("geom", GEOMS, ids=IDS)
def test_smoother_kernels_bit_identical(lib, geom, precision):
    import torch
    deltas = make_delta(geom, 31)
    kw = dict(tol=0.0, max_cycles=3)
    if precision == "mixed":
        kw.update(precision=lib.MG_MIXED, inner_cycles=2)
    a, ai1, ai2 = run(lib, geom, deltas, "off", **kw)
    b, bi1, bi2 = run(lib, geom, deltas, "all", **kw)
    assert ai1["history"] == bi1["history"] and ai2["history"] == bi2["history"]
    for key in ("phi1", "phi2", "disp1", "disp2"):
        for x, y in zip(a[key], b[key]):
            assert torch.equal(x, y), key


@pytest.mark.parametrize("geom", GEOMS[:2], ids=IDS[:2])
def test_smoother_kernels_match_oracle(lib, geom):
    deltas = make_delta(geom, 17)
    cycles = 3
    ref = lpt_pipeline(geom, deltas, tol=0.0, cycles=cycles)
    out, i1, i2 = run(lib, geom, deltas, "all", tol=0.0, max_cycles=cycles)
    np.testing.assert_allclose(i1["history"], ref["info1"]["history"], rtol=1e-6, atol=1e-14)
    for l in range(geom.n_levels):
        assert rel(out["phi1"][l], ref["phi1"][l]) < TOL
        assert rel(out["phi2"][l], ref["phi2"][l]) < TOL
        for a in range(3):
            assert rel(out["disp2"][3 * l + a], ref["psi2"][l][a]) < TOL


def test_smoother_kernels_bench_workload_bit_identical(lib):
    """128^3 base + 128^3 nest, order 6: the TMA-staged kernel on every level
    against the plain kernel everywhere, mixed precision at the bench's stopping
    rule."""
    import torch
    geom = config_zoom2()
    deltas = make_delta(geom, 2)
    kw = dict(tol=1e-7, max_cycles=50, precision=lib.MG_MIXED, inner_cycles=4)
    a, ai1, ai2 = run(lib, geom, deltas, "off", **kw)
    b, bi1, bi2 = run(lib, geom, deltas, "all", **kw)
    assert ai1["cycles"] == bi1["cycles"] and ai2["cycles"] == bi2["cycles"]
    for key in ("phi1", "phi2", "disp1", "disp2"):
        for x, y in zip(a[key], b[key]):
            assert torch.equal(x, y), key


def test_tma_default_on_a_256_cube_nest_bit_identical(lib):
    """The size class the TMA-staged kernel is the default for: a 256^3 float32 nest
    (inside a 256^3 periodic base), mixed precision, order 6, against the plain kernel."""
    import torch
    from synthetic import Geometry, NestSpec
    geom = Geometry((256, 256, 256), 200.0, 6, (NestSpec((256, 256, 256), (64, 64, 64)),))
    rng = np.random.Generator(np.random.PCG64(8))
    deltas = [rng.standard_normal((256,) * 3), rng.standard_normal((256,) * 3)]
    kw = dict(tol=1e-7, max_cycles=30, precision=lib.MG_MIXED, inner_cycles=4)
    a, ai1, ai2 = run(lib, geom, deltas, "off", **kw)
    b, bi1, bi2 = run(lib, geom, deltas, "auto", **kw)
    assert ai1["cycles"] == bi1["cycles"] and ai2["cycles"] == bi2["cycles"]
    assert ai1["rel_residual"] <= 1e-7
    for key in ("phi1", "phi2", "disp1", "disp2"):
        for x, y in zip(a[key], b[key]):
            assert torch.equal(x, y), key


@pytest.mark.parametrize("geom", GEOMS, ids=IDS)
def test_quad_and_pair_smoothers_bit_identical(lib, geom):
    """float32 levels whose rows are a multiple of 4 cells long are smoothed by the
    z-quad kernel (the others by the z-pair kernel); forcing the z-pair kernel on every
    level changes no bit of any output or residual."""
    import torch
    deltas = make_delta(geom, 37)
    kw = dict(tol=0.0, max_cycles=3, precision=lib.MG_MIXED, inner_cycles=2)
    a, ai1, ai2 = run(lib, geom, deltas, "off", **kw)
    b, bi1, bi2 = run(lib, geom, deltas, "off", pair_smoother=True, **kw)
    assert ai1["history"] == bi1["history"] and ai2["history"] == bi2["history"]
    for key in ("phi1", "phi2", "disp1", "disp2"):
        for x, y in zip(a[key], b[key]):
            assert torch.equal(x, y), key
