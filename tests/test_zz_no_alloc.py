"""hlbm_diagnostics_noalloc: the diagnostics for callers that may not allocate
device memory (for example code living inside another component's memory
budget, or running while that component builds a CUDA graph).  Its scratch
is a fixed static device array instead of memory owned by a handle.

Checked through the C ABI against hlbm_diagnostics on the same state, on two
calls in a row (a large grid, then a smaller one, so that the second call
runs over partials the first call left behind in the shared array).  This
file sorts last so that a run stopping at the first failure has already run
every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

from paper_2002_03644_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2002_03644_gb300 import hlbm
    torch.cuda.set_device(0)
    return torch, hlbm


def _state_on_device(torch, hl, s, nx, ny, precision):
    """Copy a handle's state (after the blob header) into a caller-owned CUDA
    tensor; returns (tensor, pitch)."""
    esize = 8 if precision == hl.HLBM_FP64 else 4
    pitch = (nx + 31) // 32 * 32
    payload = 13 * pitch * ny * esize
    blob = s.state()
    assert blob.size > payload
    dev = torch.from_numpy(blob[blob.size - payload:].copy()).cuda()
    return dev, pitch


def _compare(d_new, d_ref):
    assert d_new[7] == d_ref[7] == 0
    for k in range(4):  # sums: FP64 accumulation in a different block order
        assert abs(d_new[k] - d_ref[k]) <= 1e-12 * max(1.0, abs(d_ref[0])), k
    for k in (4, 5, 6):  # min / max are order-independent
        assert d_new[k] == d_ref[k], k


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_diagnostics_match_handle_diagnostics_twice(env, precision):
    torch, hl = env
    stream = torch.cuda.Stream()
    for n, steps in ((640, 7), (200, 4)):  # 409600 then 40000 cells
        case = inputs.random_smooth(n, n // 2 + 3, seed=n, amp=0.05, mu=2e-3, sigma=0.5)
        s = hl.Solver(case.nx, case.ny, precision=precision, **case.params())
        s.init(*case.fields())
        s.step(steps)
        d_ref = s.diagnostics()
        dev, pitch = _state_on_device(torch, hl, s, case.nx, case.ny, precision)
        torch.cuda.synchronize()
        d_new = hl.hlbm_diagnostics_noalloc(dev.data_ptr(), precision, case.nx, case.ny, pitch,
                                            case.gamma, stream=stream.cuda_stream)
        _compare(d_new, d_ref)
        s.close()


def test_noalloc_rejects_grids_beyond_the_static_scratch(env):
    _, hl = env
    n = hl.HLBM_NOALLOC_MAX_CELLS
    with pytest.raises(hl.HlbmError) as e:
        # rejected on the size alone, before the pointer is looked at
        hl.hlbm_diagnostics_noalloc(0, 1, 4097, 4096, 4097 + 31, 1.4)
    assert e.value.code == hl.HLBM_ERR_ARG
    assert "exceed" in str(e.value) and str(n) in str(e.value)
