"""GPU failure detection without a fault: the bounded device wait of the TMA-staged
smoother runs out on purpose (an mbarrier whose expected byte count is raised so
its phase never completes, while every copy lands), the kernel returns with its
error flag set, the library reports MG_ETIMEOUT, and the CUDA context stays usable:
a solve right after it still matches the oracle."""

import numpy as np
import pytest

from oracle.lpt import lpt_pipeline
from synthetic import make_delta, small_zoom

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


def test_wait_limit_reports_timeout_and_context_survives(lib):
    import time
    import torch
    from paper_1103_6031_gb300 import mg
    t0 = time.perf_counter()
    assert mg.selftest_wait_limit() == "MG_ETIMEOUT"
    assert time.perf_counter() - t0 < 60.0
    geom = small_zoom(16, ((16, 4),), order=4, box=50.0)
    deltas = make_delta(geom, 5)
    ref = lpt_pipeline(geom, deltas, tol=0.0, cycles=3)
    h = lib.Hierarchy(lib.config_from_geometry(geom, tol=0.0, max_cycles=3, tma="all"))
    out, i1, i2 = h.pipeline([torch.from_numpy(np.ascontiguousarray(d)).cuda() for d in deltas])
    for l in range(geom.n_levels):
        a = out["phi2"][l].cpu().numpy()
        b = ref["phi2"][l]
        assert np.sqrt(np.sum((a - b) ** 2) / np.sum(b * b)) < 1e-10
