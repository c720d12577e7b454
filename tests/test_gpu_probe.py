"""The FP64 issue-rate probe (mg_fp64_fma_rate), the measured denominator of the
float64 stencils' roofline: a plausible rate, stable over repeated calls, and its
arguments checked before any launch; and the event-pair floor probe
(mg_event_pair_floor)."""

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


def test_event_pair_floor_is_small_and_positive():
    """The event-pair floor: a few microseconds at most on a GB300, positive, stable
    over calls; invalid arguments rejected before any launch."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1103_6031_gb300 import mg
    floors = [mg.event_pair_floor(200) for _ in range(3)]
    for f in floors:
        assert 0.0 < f < 20.0, floors
    assert max(floors) - min(floors) < 2.0, floors
    out = ctypes.c_double(-1.0)
    assert mg.load_library().mg_event_pair_floor(0, None, ctypes.byref(out)) == 1
    assert mg.load_library().mg_event_pair_floor(2000, None, ctypes.byref(out)) == 1
    assert mg.load_library().mg_event_pair_floor(10, None, None) == 1
