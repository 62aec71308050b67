"""The FP64 rate probe behind the FP64 form's roofline: fused multiply-add
chains on every SM, timed with CUDA events.  Its rate must be positive and
within a factor of four of the nominal GB300 FP64 rate (1.25 TFLOP/s, i.e.
0.625 T fused multiply-adds per second), and stable between two calls."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def hl():
    import __graft_entry__ as g
    g.build()
    from paper_2002_03644_gb300 import hlbm
    return hlbm


@pytest.mark.parametrize("iters", [0, -5, 1 << 25])
def test_probe_refuses_bad_arguments(hl, iters):
    out = ctypes.c_double(0.0)
    assert hl._lib().hlbm_selftest_fp64_rate(None, iters, ctypes.addressof(out)) == hl.HLBM_ERR_ARG
    assert hl._lib().hlbm_selftest_fp64_rate(None, 1000, None) == hl.HLBM_ERR_ARG


@pytest.mark.gpu
def test_probe_measures_a_plausible_stable_rate(hl):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    r1 = hl.hlbm_selftest_fp64_rate()
    r2 = hl.hlbm_selftest_fp64_rate()
    nominal = 1.25e12 / 2.0
    assert nominal / 4.0 < r1 < 4.0 * nominal, r1
    assert abs(r1 - r2) < 0.1 * r1, (r1, r2)
