"""Failure detection without a device fault.  The bounded device-side wait
(the one the TMA and tensor-core kernels use) runs out on an mbarrier that
nothing arrives on; the host reads HLBM_ERR_TIMEOUT; the device keeps
working: the same wait with its arrival made completes, and a time step
afterwards still matches the oracle."""
import time

import pytest

from paper_2002_03644_gb300 import inputs
from test_gpu_parity import TOL, compare, run_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2002_03644_gb300 import hlbm
    torch.cuda.set_device(0)
    return hlbm


def test_wait_that_runs_out_reports_timeout_and_the_device_stays_usable(hl):
    t0 = time.perf_counter()
    assert hl.hlbm_selftest_wait(2_000_000, False) == hl.HLBM_ERR_TIMEOUT  # about 1 ms of SM clock
    assert time.perf_counter() - t0 < 5.0
    assert hl.hlbm_selftest_wait(2_000_000, True) == hl.HLBM_OK
    case = inputs.random_smooth(37, 23, seed=5, amp=0.04, mu=2e-3, sigma=0.3)
    _, _, got, ref = run_pair(hl, case, 1, 5)
    compare(got, ref, case.gamma, TOL[1])
