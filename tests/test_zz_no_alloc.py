"""hlbm_diagnostics_noalloc: the diagnostics for callers that may not allocate
device memory (for example code living inside another component's memory
budget, which hands out buffers but forbids new allocations).  Its scratch
is a fixed static device array instead of memory owned by a handle.

Checked through the C ABI against hlbm_diagnostics on the same state, on two
calls in a row (a large grid, then a smaller one, so that the second call
runs over partials the first call left behind in the shared array).  The
refusals (precisions without a static-scratch kernel, NULL pointers, the
legacy default stream) need no GPU: the call returns before it touches
CUDA.  On the GPU, a call on a stream that is being captured is refused,
and a call on another stream while a capture is open leaves that capture
valid.  This file sorts last so that a run stopping at the first failure
has already run every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_2002_03644_gb300 import inputs


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


@pytest.mark.gpu
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


@pytest.mark.gpu
def test_noalloc_rejects_grids_beyond_the_static_scratch(env):
    _, hl = env
    n = hl.HLBM_NOALLOC_MAX_CELLS
    with pytest.raises(hl.HlbmError) as e:
        # rejected on the size alone, before the pointer is looked at
        hl.hlbm_diagnostics_noalloc(0, 1, 4097, 4096, 4097 + 31, 1.4)
    assert e.value.code == hl.HLBM_ERR_ARG
    assert "exceed" in str(e.value) and str(n) in str(e.value)


@pytest.fixture(scope="module")
def cabi():
    """The library through ctypes, without a GPU."""
    import __graft_entry__ as g
    g.build()
    from paper_2002_03644_gb300 import hlbm
    return hlbm


# an address that is never dereferenced: every case below is refused on its
# arguments before the call touches CUDA
_FAKE = 0x10000


@pytest.mark.parametrize("precision", [2, 3, 4])
def test_noalloc_refuses_precisions_without_a_static_scratch_kernel(cabi, precision):
    hl = cabi
    out = np.zeros(8)
    code = hl._lib().hlbm_diagnostics_noalloc(_FAKE, precision, 32, 16, 32, 1.4, out.ctypes.data, _FAKE)
    assert code == hl.HLBM_ERR_ARG


@pytest.mark.parametrize("what", ["state", "out", "stream"])
def test_noalloc_refuses_null_pointers_and_the_legacy_stream(cabi, what):
    hl = cabi
    out = np.zeros(8)
    state = 0 if what == "state" else _FAKE
    outp = None if what == "out" else out.ctypes.data
    stream = None if what == "stream" else _FAKE
    code = hl._lib().hlbm_diagnostics_noalloc(state, 1, 32, 16, 32, 1.4, outp, stream)
    assert code == hl.HLBM_ERR_ARG


@pytest.mark.gpu
def test_noalloc_refuses_a_capturing_stream_and_leaves_other_captures_valid(env):
    """A relaxed-mode capture is open on one stream.  The call on that very
    stream is refused (HLBM_ERR_ARG, nothing enqueued); the call on a second,
    non-capturing stream runs.  The capture still ends in a valid graph whose
    replay does the captured work."""
    torch, hl = env
    case = inputs.random_smooth(96, 64, seed=3, amp=0.05, mu=2e-3, sigma=0.5)
    s = hl.Solver(case.nx, case.ny, precision=1, **case.params())
    s.init(*case.fields())
    s.step(3)
    d_ref = s.diagnostics()
    dev, pitch = _state_on_device(torch, hl, s, case.nx, case.ny, 1)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    # the first call on the device loads the module, before any capture
    _compare(hl.hlbm_diagnostics_noalloc(dev.data_ptr(), 1, case.nx, case.ny, pitch, case.gamma,
                                         stream=side.cuda_stream), d_ref)
    x = torch.zeros(1024, device="cuda")
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=cap, capture_error_mode="relaxed"):
        x.add_(1.0)
        with pytest.raises(hl.HlbmError) as e:
            hl.hlbm_diagnostics_noalloc(dev.data_ptr(), 1, case.nx, case.ny, pitch, case.gamma,
                                        stream=cap.cuda_stream)
        assert e.value.code == hl.HLBM_ERR_ARG
        d_side = hl.hlbm_diagnostics_noalloc(dev.data_ptr(), 1, case.nx, case.ny, pitch, case.gamma,
                                             stream=side.cuda_stream)
        x.add_(2.0)
    _compare(d_side, d_ref)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 6.0 and float(x.min()) == 6.0
    s.close()
