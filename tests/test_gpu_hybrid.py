"""GPU hybrid Poisson correction (Sec. 3.5.2) against the oracle: the standalone
entry point on a periodic single level and on a zero-padded nest, and the
pipeline flag, whose finest-level displacements differ from the plain pipeline's
by exactly the correction of that level's (mean-removed) source, delta for psi1
and tau for psi2, while coarser levels are unchanged."""

import numpy as np
import pytest

from oracle.hierarchy import Hierarchy as OracleHierarchy
from oracle.hierarchy import restrict
from oracle.hybrid import hybrid_correction
from oracle.lpt import lpt2_source
from oracle.multigrid import composite_mean
from synthetic import Geometry, make_delta, small_zoom

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


def rel(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b * b)))


@pytest.mark.parametrize("geom,pad", [
    (Geometry((32, 32, 32), 16.0, 2, ()), False),
    (Geometry((24, 20, 28), 12.0, 6, ()), False),
    (small_zoom(24, ((20, 7),), order=4, box=50.0), True),
    (Geometry((24, 32, 40), 24.0, 6, (__import__("synthetic").NestSpec((14, 20, 18), (7, 6, 9)),)), True),
], ids=["periodic_o2", "periodic_o6_aniso", "nest_o4", "nest_o6_aniso"])
def test_entry_point_matches_oracle(lib, geom, pad):
    import torch
    h = lib.Hierarchy(lib.config_from_geometry(geom))
    shape = h.shapes[-1]
    rng = np.random.Generator(np.random.PCG64(3))
    f = rng.standard_normal(shape)
    psi = [torch.zeros(shape, dtype=torch.float64, device="cuda") for _ in range(3)]
    h.hybrid_correction(torch.from_numpy(f).cuda(), psi)
    hf = geom.box / geom.base_n[0] / 2 ** (geom.n_levels - 1)
    want = hybrid_correction(f, hf, geom.order, pad=pad)
    for a in range(3):
        assert rel(psi[a].cpu().numpy(), want[a]) < 1e-12
    h.close()


def _mean_removed(geom, fields):
    hier = OracleHierarchy(geom)
    leaf = list(hier.leaf_levels())
    fields = [np.array(x, dtype=np.float64) for x in fields]
    for i in range(len(leaf) - 1, 0, -1):
        fields[i - 1][hier.covered_region(leaf[i])] = restrict(fields[i])
    m = composite_mean(hier, fields)
    return [x - m for x in fields]


@pytest.mark.parametrize("mixed", [False, True], ids=["fp64", "mixed"])
def test_pipeline_flag_adds_the_correction_of_each_source(lib, mixed):
    import torch
    geom = small_zoom(32, ((24, 8),), order=6, box=80.0)
    deltas = make_delta(geom, 51)
    kw = dict(tol=1e-10)
    if mixed:
        kw.update(precision=lib.MG_MIXED, inner_cycles=3)
    dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in deltas]
    plain = lib.Hierarchy(lib.config_from_geometry(geom, **kw))
    hyb = lib.Hierarchy(lib.config_from_geometry(geom, hybrid=True, **kw))
    a, _, _ = plain.pipeline(dev)
    b, _, _ = hyb.pipeline(dev)
    for key in ("phi1", "phi2"):
        for x, y in zip(a[key], b[key]):
            assert torch.equal(x, y)
    for c in range(3):                                    # coarser level untouched
        assert torch.equal(a["disp1"][c], b["disp1"][c])
        assert torch.equal(a["disp2"][c], b["disp2"][c])
    hf = geom.box / geom.base_n[0] / 2
    f1 = _mean_removed(geom, deltas)[-1]
    tau = lpt2_source(OracleHierarchy(geom), [x.cpu().numpy() for x in a["phi1"]])
    f2 = _mean_removed(geom, tau)[-1]
    for key, f in (("disp1", f1), ("disp2", f2)):
        want = hybrid_correction(f, hf, geom.order, pad=True)
        for c in range(3):
            got = (b[key][3 + c] - a[key][3 + c]).cpu().numpy()
            assert rel(got, want[c]) < 1e-9, (key, c)
    plain.close()
    hyb.close()
