"""GPU local Lagrangian density (Sec. 5.3) against the oracle: the same
finite-difference Hessian of Phi = a1 phi1 + a2 phi2, 1/det[I - H], covered cells
as children's means and unit composite mean; <= 1e-10 RMS relative error in
rho - 1 on nested hierarchies of orders 2, 4 and 6, with one and two potentials,
in both precision modes of the hierarchy."""

import numpy as np
import pytest

from oracle.hierarchy import Hierarchy as OracleHierarchy
from oracle.lpt import lla_density, lpt_pipeline
from synthetic import make_delta, small_zoom

pytestmark = pytest.mark.gpu
TOL = 1e-10

GEOMS = [
    small_zoom(16, ((16, 4),), order=2, box=20.0),
    small_zoom(24, ((20, 7), (16, 6)), order=4, box=50.0),
    small_zoom(32, ((24, 8),), order=6, box=80.0),
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


def to_dev(arrs):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in arrs]


@pytest.mark.parametrize("mixed", [False, True], ids=["fp64", "mixed"])
@pytest.mark.parametrize("geom", GEOMS, ids=lambda g: "o%d_L%d" % (g.order, g.n_levels))
def test_lla_matches_oracle(lib, geom, mixed):
    deltas = make_delta(geom, 41)
    ref = lpt_pipeline(geom, deltas, tol=1e-9)
    # scale so that the Hessian reaches O(0.3): a visibly non-linear density
    a1 = 0.3 / max(np.abs(d).max() for d in deltas)
    a2 = 0.5 * a1 * a1
    kw = dict(tol=1e-9)
    if mixed:
        kw.update(precision=lib.MG_MIXED, inner_cycles=2)
    h = lib.Hierarchy(lib.config_from_geometry(geom, **kw))
    for two in (False, True):
        phi2 = ref["phi2"] if two else None
        want = lla_density(OracleHierarchy(geom), ref["phi1"], phi2, a1, a2 if two else 0.0)
        got = h.lla_density(to_dev(ref["phi1"]), to_dev(phi2) if two else None, a1,
                            a2 if two else 0.0)
        for g, w in zip(got, want):
            g = g.cpu().numpy()
            assert np.std(w) > 1e-2
            err = np.sqrt(np.sum((g - w) ** 2) / np.sum((w - 1.0) ** 2))
            assert err < TOL, err
    h.close()
