"""The allocation-free 2LPT source entry point against the hierarchy entry point.

mg_lpt2_source_periodic_static exists for callers that cannot allocate device
memory at the time they need tau: its working memory is a static device array
inside the library.  Through the C ABI it must give the same tau as
mg_lpt2_source on a one-level periodic hierarchy, on consecutive calls with
different inputs (nothing may carry over between calls), the oracle's tau,
and it must refuse grids larger than its static array with a clear message."""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_6031_gb300 as pkg
    lib = pkg.load_library()
    fn = lib.mg_lpt2_source_periodic_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                   ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_char_p, ctypes.c_size_t]
    return torch, pkg, fn


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b * b)))


@pytest.mark.parametrize("order,shape,box", [(6, (48, 40, 36), 75.0), (2, (16, 16, 16), 1.0),
                                             (4, (64, 64, 64), 100.0)])
def test_static_tau_matches_hierarchy_entry_point(env, order, shape, box):
    torch, pkg, fn = env
    h = pkg.Hierarchy(pkg.make_config(shape, box, order))
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(17)
    for call in range(2):
        phi = torch.from_numpy(rng.standard_normal(shape)).cuda()
        expect = h.lpt2_source([phi])[0]
        tau = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
        msg = ctypes.create_string_buffer(256)
        st = fn(phi.data_ptr(), tau.data_ptr(), shape[0], shape[1], shape[2], box, order,
                stream, msg, 256)
        torch.cuda.synchronize()
        assert st == 0, msg.value
        assert _rel(tau, expect) <= TOL, call
    h.close()


@pytest.mark.parametrize("order,shape,box", [(6, (24, 20, 18), 30.0), (4, (32, 32, 32), 1.0)])
def test_static_tau_matches_oracle_and_allocates_nothing(env, order, shape, box):
    """Against the CPU oracle's 2LPT source of the same periodic grid (Sec. 3.1.2),
    on two calls in a row; around the second call neither torch's allocator nor the
    device's free memory changes."""
    from oracle.hierarchy import Hierarchy as OracleHierarchy
    from oracle.lpt import lpt2_source
    from synthetic import Geometry
    torch, pkg, fn = env
    geom = Geometry(shape, box, order, ())
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(23)
    for call in range(2):
        x = rng.standard_normal(shape)
        expect = lpt2_source(OracleHierarchy(geom), [x])[0]
        phi = torch.from_numpy(x).cuda()
        tau = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
        msg = ctypes.create_string_buffer(256)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        held0 = torch.cuda.memory_allocated()
        st = fn(phi.data_ptr(), tau.data_ptr(), shape[0], shape[1], shape[2], box, order,
                stream, msg, 256)
        torch.cuda.synchronize()
        assert st == 0, msg.value
        got = tau.cpu().numpy()
        assert np.sqrt(np.sum((got - expect) ** 2) / np.sum(expect ** 2)) <= TOL, call
        if call == 1:   # the first call may load the library's module; the second may not grow
            free1, _ = torch.cuda.mem_get_info()
            assert torch.cuda.memory_allocated() == held0
            assert free1 == free0


def test_static_tau_rejects_oversize_grid(env):
    torch, pkg, fn = env
    shape = (96, 96, 96)
    phi = torch.zeros(shape, dtype=torch.float64, device="cuda")
    tau = torch.zeros(shape, dtype=torch.float64, device="cuda")
    msg = ctypes.create_string_buffer(256)
    st = fn(phi.data_ptr(), tau.data_ptr(), 96, 96, 96, 1.0, 6, None, msg, 256)
    assert st == 1
    assert b"static array" in msg.value
