"""The FP64 issue-rate probe (mg_fp64_fma_rate), the measured denominator of the
float64 stencils' roofline: a plausible rate, stable over repeated calls, and its
arguments checked before any launch."""

import ctypes

import pytest

pytestmark = pytest.mark.gpu


def test_fp64_fma_rate_is_plausible_and_stable():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1103_6031_gb300 import mg
    rates = [mg.fp64_fma_rate(4096) for _ in range(3)]
    # GB300: about 2 FP64 FMAs per clock per SM (152 SMs, <= 2.07 GHz) = <= 0.63 T/s
    for r in rates:
        assert 1e11 < r < 1.5e12, rates
    assert max(rates) / min(rates) < 1.2, rates
    out = ctypes.c_double(-1.0)
    assert mg.load_library().mg_fp64_fma_rate(4, None, ctypes.byref(out)) == 1   # iters too small
    assert mg.load_library().mg_fp64_fma_rate(4096, None, None) == 1
