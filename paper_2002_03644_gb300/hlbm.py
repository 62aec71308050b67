"""Python binding of libhlbm (include/hlbm.h): the same entry points, argument
marshalling only.  Every step of the method runs in the CUDA library; there
is no fallback: if libhlbm.so is missing or a call fails, an exception is
raised.

Arrays may be numpy arrays (host memory) or torch tensors (a CUDA tensor is
passed as device memory, a CPU tensor as host memory).  Field arrays are
float64, contiguous, shape [ny, nx]; a1 arrays are [3, ny, nx].
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

HLBM_FP64, HLBM_FP32, HLBM_FP32_F16POP, HLBM_FP32_BF16POP, HLBM_FP32_MOMENTS = 0, 1, 2, 3, 4
HLBM_BC_PERIODIC, HLBM_BC_ZEROGRAD, HLBM_BC_DIRICHLET, HLBM_BC_WALL = 0, 1, 2, 3
HLBM_MEM_HOST, HLBM_MEM_DEVICE = 0, 1
HLBM_OK, HLBM_ERR_ARG, HLBM_ERR_CFL, HLBM_ERR_NONFINITE = 0, -1, -2, -3
HLBM_ERR_CUDA, HLBM_ERR_STATE, HLBM_ERR_NOMEM, HLBM_ERR_UNSUPPORTED = -4, -5, -6, -7
HLBM_ERR_TIMEOUT = -8
HLBM_ABL_CENTRED_E1, HLBM_ABL_NO_E2 = 1, 2

ENTRY_POINTS = (
    "hlbm_create", "hlbm_init_fields", "hlbm_step", "hlbm_get_macros", "hlbm_get_populations",
    "hlbm_diagnostics", "hlbm_state_bytes", "hlbm_get_state", "hlbm_set_state", "hlbm_step_count",
    "hlbm_synchronize", "hlbm_destroy", "hlbm_strerror", "hlbm_last_error", "hlbm_abi_version",
    "hlbm_diagnostics_noalloc", "hlbm_selftest_wait", "hlbm_selftest_fp64_rate", "hlbm_debug_check",
    "hlbm_batch_create", "hlbm_batch_case", "hlbm_batch_step", "hlbm_batch_autotune", "hlbm_batch_tile",
    "hlbm_batch_destroy",
    "hlbm_sur_create", "hlbm_sur_param_count", "hlbm_sur_set_params", "hlbm_sur_get_params", "hlbm_sur_forward",
    "hlbm_sur_predict",
    "hlbm_sur_backward", "hlbm_sur_backward_ex", "hlbm_sur_adam", "hlbm_sur_synchronize", "hlbm_sur_destroy",
)
HLBM_NOALLOC_MAX_CELLS = 16777216


class hlbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("phi_mode", ctypes.c_int32),
        ("gamma", ctypes.c_double), ("Pr", ctypes.c_double), ("mu", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("bc", ctypes.c_int32 * 4), ("bc_state", (ctypes.c_double * 4) * 4),
        ("diag_every", ctypes.c_int32), ("check_cfl", ctypes.c_int32),
        ("ablation", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5),
    ]


def make_params(nx, ny, precision=HLBM_FP64, gamma=1.4, Pr=0.71, mu=1e-4, sigma=0.0,
                bc=(HLBM_BC_PERIODIC,) * 4, bc_state=None, phi_mode=0, diag_every=0, check_cfl=0, ablation=0):
    p = hlbm_params()
    p.nx, p.ny, p.precision, p.phi_mode = int(nx), int(ny), int(precision), int(phi_mode)
    p.gamma, p.Pr, p.mu, p.sigma = float(gamma), float(Pr), float(mu), float(sigma)
    for k in range(4):
        p.bc[k] = int(bc[k])
    if bc_state is not None:
        bs = np.asarray(bc_state, dtype=np.float64).reshape(4, 4)
        for k in range(4):
            for q in range(4):
                p.bc_state[k][q] = float(bs[k, q])
    p.diag_every, p.check_cfl, p.ablation = int(diag_every), int(check_cfl), int(ablation)
    return p


class HlbmError(RuntimeError):
    def __init__(self, code, detail=""):
        self.code = code
        super().__init__(f"hlbm error {code}: {_strerror(code)}" + (f" ({detail})" if detail else ""))


_lock = threading.Lock()
_libh = None
_P = ctypes.c_void_p
_PD = ctypes.c_void_p  # pointers are passed as raw addresses


def library_path() -> str:
    """libhlbm.so, or the index-checking debug build libhlbm_debug.so when
    the environment sets HLBM_LIBRARY=debug (build it with
    build.build_library(debug=True))."""
    return _build.LIB_DEBUG if os.environ.get("HLBM_LIBRARY") == "debug" else _build.LIB


def _lib():
    global _libh
    with _lock:
        if _libh is not None:
            return _libh
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        lib.hlbm_create.restype = ctypes.c_int
        lib.hlbm_create.argtypes = [ctypes.POINTER(hlbm_params), _P, ctypes.POINTER(_P)]
        lib.hlbm_init_fields.restype = ctypes.c_int
        lib.hlbm_init_fields.argtypes = [_P, _PD, _PD, _PD, _PD, _PD, ctypes.c_int]
        lib.hlbm_step.restype = ctypes.c_int
        lib.hlbm_step.argtypes = [_P, ctypes.c_int64]
        lib.hlbm_get_macros.restype = ctypes.c_int
        lib.hlbm_get_macros.argtypes = [_P, _PD, _PD, _PD, _PD, _PD, _PD, ctypes.c_int]
        lib.hlbm_get_populations.restype = ctypes.c_int
        lib.hlbm_get_populations.argtypes = [_P, _PD, ctypes.c_int]
        lib.hlbm_diagnostics.restype = ctypes.c_int
        lib.hlbm_diagnostics.argtypes = [_P, _PD]
        lib.hlbm_state_bytes.restype = ctypes.c_int
        lib.hlbm_state_bytes.argtypes = [_P, ctypes.POINTER(ctypes.c_size_t)]
        lib.hlbm_get_state.restype = ctypes.c_int
        lib.hlbm_get_state.argtypes = [_P, _PD, ctypes.c_size_t]
        lib.hlbm_set_state.restype = ctypes.c_int
        lib.hlbm_set_state.argtypes = [_P, _PD, ctypes.c_size_t]
        lib.hlbm_step_count.restype = ctypes.c_int64
        lib.hlbm_step_count.argtypes = [_P]
        lib.hlbm_synchronize.restype = ctypes.c_int
        lib.hlbm_synchronize.argtypes = [_P]
        lib.hlbm_destroy.restype = None
        lib.hlbm_destroy.argtypes = [_P]
        lib.hlbm_strerror.restype = ctypes.c_char_p
        lib.hlbm_strerror.argtypes = [ctypes.c_int]
        lib.hlbm_last_error.restype = ctypes.c_char_p
        lib.hlbm_last_error.argtypes = [_P]
        lib.hlbm_abi_version.restype = ctypes.c_int
        lib.hlbm_abi_version.argtypes = []
        lib.hlbm_batch_create.restype = ctypes.c_int
        lib.hlbm_batch_create.argtypes = [ctypes.POINTER(hlbm_params), ctypes.c_int, _P, ctypes.POINTER(_P)]
        lib.hlbm_batch_case.restype = ctypes.c_int
        lib.hlbm_batch_case.argtypes = [_P, ctypes.c_int, ctypes.POINTER(_P)]
        lib.hlbm_batch_step.restype = ctypes.c_int
        lib.hlbm_batch_step.argtypes = [_P, ctypes.c_int64]
        lib.hlbm_batch_autotune.restype = ctypes.c_int
        lib.hlbm_batch_autotune.argtypes = [_P, ctypes.POINTER(ctypes.c_int)]
        lib.hlbm_batch_tile.restype = ctypes.c_int
        lib.hlbm_batch_tile.argtypes = [_P] + [ctypes.POINTER(ctypes.c_int)] * 4
        lib.hlbm_batch_destroy.restype = None
        lib.hlbm_batch_destroy.argtypes = [_P]
        lib.hlbm_sur_create.restype = ctypes.c_int
        lib.hlbm_sur_create.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, _P, ctypes.POINTER(_P)]
        lib.hlbm_sur_param_count.restype = ctypes.c_int64
        lib.hlbm_sur_param_count.argtypes = [_P]
        lib.hlbm_sur_set_params.restype = ctypes.c_int
        lib.hlbm_sur_set_params.argtypes = [_P, _PD, ctypes.c_int]
        lib.hlbm_sur_get_params.restype = ctypes.c_int
        lib.hlbm_sur_get_params.argtypes = [_P, _PD, _PD, ctypes.c_int]
        lib.hlbm_sur_forward.restype = ctypes.c_int
        lib.hlbm_sur_forward.argtypes = [_P, _PD, _PD, ctypes.c_int]
        lib.hlbm_sur_predict.restype = ctypes.c_int
        lib.hlbm_sur_predict.argtypes = [_P, _PD, _PD, ctypes.c_int]
        lib.hlbm_sur_backward.restype = ctypes.c_int
        lib.hlbm_sur_backward.argtypes = [_P, _PD, ctypes.POINTER(ctypes.c_double)]
        lib.hlbm_sur_backward_ex.restype = ctypes.c_int
        lib.hlbm_sur_backward_ex.argtypes = [_P, _PD, _PD, ctypes.c_int, _PD, ctypes.POINTER(ctypes.c_double)]
        lib.hlbm_sur_adam.restype = ctypes.c_int
        lib.hlbm_sur_adam.argtypes = [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]
        lib.hlbm_sur_synchronize.restype = ctypes.c_int
        lib.hlbm_sur_synchronize.argtypes = [_P]
        lib.hlbm_sur_destroy.restype = None
        lib.hlbm_sur_destroy.argtypes = [_P]
        lib.hlbm_diagnostics_noalloc.restype = ctypes.c_int
        lib.hlbm_diagnostics_noalloc.argtypes = [_PD, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 ctypes.c_double, _PD, _P]
        lib.hlbm_selftest_wait.restype = ctypes.c_int
        lib.hlbm_selftest_wait.argtypes = [_P, ctypes.c_longlong, ctypes.c_int]
        lib.hlbm_selftest_fp64_rate.restype = ctypes.c_int
        lib.hlbm_selftest_fp64_rate.argtypes = [_P, ctypes.c_int, _PD]
        lib.hlbm_debug_check.restype = ctypes.c_int
        lib.hlbm_debug_check.argtypes = [_P, _P, _P]
        _libh = lib
        return lib


def _strerror(code):
    try:
        return _lib().hlbm_strerror(int(code)).decode()
    except Exception:
        return "?"


def _check(code, h=None):
    if code != HLBM_OK:
        detail = ""
        if h:
            try:
                detail = _lib().hlbm_last_error(h).decode()
            except Exception:
                pass
        raise HlbmError(code, detail)


def _addr(a, n, keep):
    """(address, mem_kind) of an FP64 contiguous array with n elements."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != n:
            raise ValueError("torch tensors must be float64, contiguous, with the field's size")
        keep.append(a)
        return a.data_ptr(), (HLBM_MEM_DEVICE if a.is_cuda else HLBM_MEM_HOST)
    arr = np.asarray(a)
    if arr.dtype != np.float64 or not arr.flags["C_CONTIGUOUS"] or arr.size != n:
        raise ValueError("numpy arrays must be float64, C-contiguous, with the field's size")
    keep.append(arr)
    return arr.ctypes.data, HLBM_MEM_HOST


def _one_kind(kinds):
    ks = {k for k in kinds if k is not None}
    if len(ks) > 1:
        raise ValueError("all arrays of one call must live in the same memory (host or device)")
    return ks.pop() if ks else HLBM_MEM_HOST


# ---- the C entry points ---------------------------------------------------------

def hlbm_abi_version():
    return _lib().hlbm_abi_version()


def hlbm_strerror(code):
    return _strerror(code)


def hlbm_last_error(h):
    return _lib().hlbm_last_error(h).decode()


def hlbm_create(params: hlbm_params, stream=None):
    """Returns an opaque handle.  stream: a cudaStream_t as int (e.g.
    torch.cuda.current_stream().cuda_stream) or None."""
    h = _P()
    _check(_lib().hlbm_create(ctypes.byref(params), stream or None, ctypes.byref(h)))
    return h.value


def hlbm_init_fields(h, rho, ux, uy, theta, a1=None, n=None):
    keep = []
    if n is None:
        n = int(np.prod(np.shape(rho)))
    ptrs, kinds = [], []
    for a, m in ((rho, n), (ux, n), (uy, n), (theta, n), (a1, 3 * n)):
        p, k = _addr(a, m, keep)
        ptrs.append(p); kinds.append(k)
    _check(_lib().hlbm_init_fields(h, *ptrs, _one_kind(kinds)), h)


def hlbm_step(h, n):
    _check(_lib().hlbm_step(h, int(n)), h)


def hlbm_get_macros(h, rho=None, ux=None, uy=None, theta=None, s=None, a1=None, n=None):
    keep = []
    ref = next(a for a in (rho, ux, uy, theta, s, a1) if a is not None)
    if n is None:
        n = int(np.prod(np.shape(ref))) // (3 if ref is a1 else 1)
    ptrs, kinds = [], []
    for a, m in ((rho, n), (ux, n), (uy, n), (theta, n), (s, n), (a1, 3 * n)):
        p, k = _addr(a, m, keep)
        ptrs.append(p); kinds.append(k)
    _check(_lib().hlbm_get_macros(h, *ptrs, _one_kind(kinds)), h)


def hlbm_get_populations(h, F):
    keep = []
    p, k = _addr(F, int(np.prod(np.shape(F))), keep)
    _check(_lib().hlbm_get_populations(h, p, k), h)


def hlbm_diagnostics(h):
    out = np.zeros(8)
    _check(_lib().hlbm_diagnostics(h, out.ctypes.data), h)
    return out


def hlbm_state_bytes(h):
    n = ctypes.c_size_t()
    _check(_lib().hlbm_state_bytes(h, ctypes.byref(n)), h)
    return n.value


def hlbm_get_state(h):
    buf = np.zeros(hlbm_state_bytes(h), dtype=np.uint8)
    _check(_lib().hlbm_get_state(h, buf.ctypes.data, buf.size), h)
    return buf


def hlbm_set_state(h, buf):
    b = np.ascontiguousarray(np.asarray(buf, dtype=np.uint8))
    _check(_lib().hlbm_set_state(h, b.ctypes.data, b.size), h)


def hlbm_step_count(h):
    return _lib().hlbm_step_count(h)


def hlbm_synchronize(h):
    _check(_lib().hlbm_synchronize(h), h)


def hlbm_destroy(h):
    if h:
        _lib().hlbm_destroy(h)


def hlbm_diagnostics_noalloc(state_ptr, precision, nx, ny, pitch, gamma, stream=None):
    """Diagnostics of a caller-held device state without any allocation by
    the library (for callers that may not allocate device memory).
    state_ptr: device address of 13 planes [ny][pitch].  stream: an explicit
    cudaStream_t (int) that is not being captured; None (the legacy default
    stream) and a capturing stream are refused, as are grids above
    HLBM_NOALLOC_MAX_CELLS cells."""
    out = np.zeros(8)
    code = _lib().hlbm_diagnostics_noalloc(state_ptr, int(precision), int(nx), int(ny), int(pitch),
                                           float(gamma), out.ctypes.data, stream or None)
    if code != HLBM_OK and int(nx) * int(ny) > HLBM_NOALLOC_MAX_CELLS:
        raise HlbmError(code, f"{int(nx) * int(ny)} cells exceed the static scratch capacity of "
                              f"{HLBM_NOALLOC_MAX_CELLS} cells")
    _check(code)
    return out


def hlbm_selftest_wait(budget_cycles, arrive, stream=None):
    """Run the library's bounded device-side wait on its own: an mbarrier
    armed for one arrival, which the device thread makes (arrive=True) or
    never makes, polled for at most budget_cycles SM clock cycles.  Returns
    the status code (HLBM_ERR_TIMEOUT when the wait ran out, HLBM_OK when it
    completed) instead of raising."""
    return _lib().hlbm_selftest_wait(stream or None, int(budget_cycles), 1 if arrive else 0)


def hlbm_selftest_fp64_rate(iters=1 << 15, stream=None):
    """Measured FP64 fused multiply-adds per second of this GPU (eight
    independent chains per thread, all SMs busy); 2 flops each."""
    out = ctypes.c_double(0.0)
    _check(_lib().hlbm_selftest_fp64_rate(stream or None, int(iters), ctypes.addressof(out)))
    return out.value


def hlbm_debug_check():
    """(site, a, b) of the first failed index check since the last call (site
    0: none), read and cleared; HlbmError(HLBM_ERR_UNSUPPORTED) from the
    release build."""
    v = [ctypes.c_longlong(0) for _ in range(3)]
    _check(_lib().hlbm_debug_check(*[ctypes.addressof(x) for x in v]))
    return tuple(x.value for x in v)


def hlbm_batch_create(params_list, stream=None):
    """A batch of FP32 cases advanced together (one persistent launch per
    step, replayed from a CUDA graph).  Returns the opaque batch pointer."""
    arr = (hlbm_params * len(params_list))(*params_list)
    b = _P()
    _check(_lib().hlbm_batch_create(arr, len(params_list), stream or None, ctypes.byref(b)))
    return b.value


def hlbm_batch_case(b, index):
    h = _P()
    _check(_lib().hlbm_batch_case(b, int(index), ctypes.byref(h)))
    return h.value


def hlbm_batch_step(b, n):
    _check(_lib().hlbm_batch_step(b, int(n)))


def hlbm_batch_autotune(b):
    t = ctypes.c_int()
    _check(_lib().hlbm_batch_autotune(b, ctypes.byref(t)))
    return t.value


def hlbm_batch_tile(b):
    v = [ctypes.c_int() for _ in range(4)]
    _check(_lib().hlbm_batch_tile(b, *[ctypes.byref(x) for x in v]))
    return tuple(x.value for x in v)


def hlbm_batch_destroy(b):
    if b:
        _lib().hlbm_batch_destroy(b)


def torch_stream_handle(stream=None):
    """Stream handle for the C ABI: `stream` itself (an int handle or a
    torch.cuda.Stream), else torch's current stream.  torch's legacy default
    stream (handle 0) is passed as cudaStreamLegacy (1): a NULL stream asks
    the library for a stream of its own, which is not ordered with torch's
    work."""
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    import torch
    h = int(torch.cuda.current_stream().cuda_stream)
    return h if h != 0 else 1


def hlbm_sur_create(widths, H, W, batch_max, stream=None):
    arr = (ctypes.c_int * len(widths))(*[int(w) for w in widths])
    s = _P()
    _check(_lib().hlbm_sur_create(len(widths) - 1, arr, int(H), int(W), int(batch_max), stream or None,
                                  ctypes.byref(s)))
    return s.value


def hlbm_sur_param_count(s):
    return _lib().hlbm_sur_param_count(s)


def _f32_ptr(a):
    """(address, mem_kind) of a contiguous float32 torch tensor or numpy array."""
    if hasattr(a, "data_ptr"):
        import torch
        assert a.dtype == torch.float32 and a.is_contiguous()
        return a.data_ptr(), (HLBM_MEM_DEVICE if a.is_cuda else HLBM_MEM_HOST)
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data, HLBM_MEM_HOST


def hlbm_sur_set_params(s, params):
    p, k = _f32_ptr(params)
    _check(_lib().hlbm_sur_set_params(s, p, k))


def hlbm_sur_get_params(s, params=None, grads=None):
    kinds = set()
    pp = gg = None
    if params is not None:
        pp, k = _f32_ptr(params); kinds.add(k)
    if grads is not None:
        gg, k = _f32_ptr(grads); kinds.add(k)
    _check(_lib().hlbm_sur_get_params(s, pp, gg, kinds.pop() if kinds else HLBM_MEM_HOST))


def hlbm_sur_forward(s, x, y, batch):
    """x, y: CUDA float32 tensors [B, H, W, C] (y may be None)."""
    _check(_lib().hlbm_sur_forward(s, x.data_ptr(), None if y is None else y.data_ptr(), int(batch)))


def hlbm_sur_predict(s, x, y, batch):
    """Inference (no pre-activations kept): x, y CUDA float32 tensors [B, H, W, C]."""
    _check(_lib().hlbm_sur_predict(s, x.data_ptr(), None if y is None else y.data_ptr(), int(batch)))


def hlbm_sur_backward(s, target):
    loss = ctypes.c_double()
    _check(_lib().hlbm_sur_backward(s, target.data_ptr(), ctypes.byref(loss)))
    return loss.value


def hlbm_sur_backward_ex(s, target, dy=None, accumulate=False, dx=None):
    """Backward pass for a rollout through the network: dL/dy = 2 (y -
    target) / n + dy; parameter gradients added to the held ones when
    accumulate; dL/dx written to dx.  Tensors: contiguous float32 on the
    surrogate's device.  Returns the mean squared error against target."""
    for t in (target, dy, dx):
        if t is not None and not t.is_contiguous():
            raise ValueError("hlbm_sur_backward_ex: tensors must be contiguous")
    loss = ctypes.c_double()
    _check(_lib().hlbm_sur_backward_ex(s, target.data_ptr(), None if dy is None else dy.data_ptr(),
                                       int(bool(accumulate)), None if dx is None else dx.data_ptr(),
                                       ctypes.byref(loss)))
    return loss.value


def hlbm_sur_adam(s, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(_lib().hlbm_sur_adam(s, lr, beta1, beta2, eps))


def hlbm_sur_synchronize(s):
    _check(_lib().hlbm_sur_synchronize(s))


def hlbm_sur_destroy(s):
    if s:
        _lib().hlbm_sur_destroy(s)


# ---- convenience wrapper ----------------------------------------------------------

class Solver:
    """Owns one handle (or borrows one, see Batch).  Example:
        s = Solver(nx, ny, precision=HLBM_FP32, mu=1e-4)
        s.init(rho, ux, uy, theta); s.step(100); m = s.macros()
    """

    def __init__(self, nx, ny, stream=None, _borrowed=None, **params):
        self.nx, self.ny = int(nx), int(ny)
        self.params = make_params(nx, ny, **params)
        self._owned = _borrowed is None
        self.h = hlbm_create(self.params, stream) if self._owned else _borrowed

    def close(self):
        if self.h and self._owned:
            hlbm_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, rho, ux, uy, theta, a1=None):
        hlbm_init_fields(self.h, rho, ux, uy, theta, a1, n=self.nx * self.ny)

    def step(self, n=1):
        hlbm_step(self.h, n)

    def macros(self):
        shp = (self.ny, self.nx)
        out = {k: np.zeros(shp) for k in ("rho", "ux", "uy", "theta", "s")}
        a1 = np.zeros((3,) + shp)
        hlbm_get_macros(self.h, out["rho"], out["ux"], out["uy"], out["theta"], out["s"], a1,
                        n=self.nx * self.ny)
        out["a1"] = a1
        return out

    def populations(self):
        F = np.zeros((9, self.ny, self.nx))
        hlbm_get_populations(self.h, F)
        return F

    def diagnostics(self):
        return hlbm_diagnostics(self.h)

    def state(self):
        return hlbm_get_state(self.h)

    def set_state(self, buf):
        hlbm_set_state(self.h, buf)

    @property
    def step_count(self):
        return hlbm_step_count(self.h)

    def synchronize(self):
        hlbm_synchronize(self.h)


class Batch:
    """Many FP32 cases advanced together.  cases: list of dicts with nx, ny and
    the keyword parameters of make_params.  batch.cases[i] is a Solver view of
    case i (init / macros / diagnostics); batch.step(n) advances all."""

    def __init__(self, cases, stream=None):
        plist = [make_params(c["nx"], c["ny"], **{k: v for k, v in c.items() if k not in ("nx", "ny")})
                 for c in cases]
        self.b = hlbm_batch_create(plist, stream)
        self.cases = [Solver(c["nx"], c["ny"], _borrowed=hlbm_batch_case(self.b, i),
                             **{k: v for k, v in c.items() if k not in ("nx", "ny")})
                      for i, c in enumerate(cases)]

    def step(self, n=1):
        hlbm_batch_step(self.b, n)

    def autotune(self):
        return hlbm_batch_autotune(self.b)

    def tile(self):
        return hlbm_batch_tile(self.b)

    def close(self):
        if self.b:
            for c in self.cases:
                c.h = None
            hlbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
