"""Python access to the FP64 CPU oracle (``hlbm_oracle.c``).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The product library
(``paper_2002_03644_gb300``) never imports it.

The oracle restates the equations of the time step of Renard et al. (arXiv
2002.03644) -- collision and streaming, moments, the entropy update, the
closure correction, the equilibrium and a1 (Sec. 2-3) -- in plain C with FP64
arithmetic; this module only marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hlbm_oracle.c")
LIB = os.path.join(HERE, "libhlbm_oracle.so")

BC_PERIODIC, BC_ZEROGRAD, BC_DIRICHLET, BC_WALL = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None

_D = ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)


def build_oracle(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no FMA contraction so that x86
    and Arm hosts round the same way)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, SRC, "-lm"]
    # OpenMP only splits the rows of per-cell passes over threads (results
    # are the same); without it the library runs every pass on one thread.
    if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], stderr=subprocess.DEVNULL).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build_oracle()
        lib = ctypes.CDLL(LIB)
        lib.hlbmo_create.restype = ctypes.c_void_p
        lib.hlbmo_create.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D, _D,
                                     ctypes.POINTER(ctypes.c_int), _PD, ctypes.c_int, ctypes.c_int]
        lib.hlbmo_destroy.argtypes = [ctypes.c_void_p]
        lib.hlbmo_init.restype = ctypes.c_int
        lib.hlbmo_init.argtypes = [ctypes.c_void_p, _PD, _PD, _PD, _PD, _PD]
        lib.hlbmo_step.restype = ctypes.c_int
        lib.hlbmo_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
        lib.hlbmo_get.argtypes = [ctypes.c_void_p, _PD, _PD, _PD, _PD, _PD, _PD]
        lib.hlbmo_get_psi.argtypes = [ctypes.c_void_p, _PD]
        lib.hlbmo_get_feq.argtypes = [ctypes.c_void_p, _PD]
        lib.hlbmo_get_post_collision.argtypes = [ctypes.c_void_p, _PD]
        lib.hlbmo_entropy_rhs.argtypes = [ctypes.c_void_p, _PD]
        lib.hlbmo_step_count.restype = ctypes.c_long
        lib.hlbmo_step_count.argtypes = [ctypes.c_void_p]
        lib.hlbmo_set_threads.argtypes = [ctypes.c_void_p, ctypes.c_int]
        lib.hlbmo_max_threads.restype = ctypes.c_int
        lib.hlbmo_feq_cell.argtypes = [_D, _D, _D, _D, _PD]
        lib.hlbmo_f1_cell.argtypes = [_D, _D, _D, _D, _D, _D, _PD]
        lib.hlbmo_a1_high.argtypes = [_D, _D, _D, _D, _D, _D, _PD]
        lib.hlbmo_psi_cell.argtypes = [_D, _D, _D, _PD]
        lib.hlbmo_gamma_closure.restype = _D
        lib.hlbmo_gamma_closure.argtypes = [_D, _D, _D]
        lib.hlbmo_hermite.restype = _D
        lib.hlbmo_hermite.argtypes = [ctypes.c_int] * 6
        lib.hlbmo_lattice.argtypes = [_PD, _PD, _PD]
        lib.hlbmo_muscl_term.restype = _D
        lib.hlbmo_muscl_term.argtypes = [_D] * 6
        _lib = lib
        return lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_PD)


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None:
        assert a.size == n, (a.size, n)
    return a


# ---- per-cell functions (pins) ------------------------------------------------

def lattice():
    lib = _load()
    cx, cy, w = np.zeros(9), np.zeros(9), np.zeros(9)
    lib.hlbmo_lattice(_ptr(cx), _ptr(cy), _ptr(w))
    return cx, cy, w


def hermite(i, order, a=0, b=0, g=0, e=0):
    return _load().hlbmo_hermite(i, order, a, b, g, e)


def feq_cell(rho, ux, uy, theta):
    out = np.zeros(9)
    _load().hlbmo_feq_cell(rho, ux, uy, theta, _ptr(out))
    return out


def f1_cell(axx, axy, ayy, ux, uy, theta):
    out = np.zeros(9)
    _load().hlbmo_f1_cell(axx, axy, ayy, ux, uy, theta, _ptr(out))
    return out


def a1_high(axx, axy, ayy, ux, uy, theta):
    out = np.zeros(3)
    _load().hlbmo_a1_high(axx, axy, ayy, ux, uy, theta, _ptr(out))
    return out


def psi_cell(exx, exy, eyy):
    out = np.zeros(9)
    _load().hlbmo_psi_cell(exx, exy, eyy, _ptr(out))
    return out


def gamma_closure(rho, ua, theta):
    return _load().hlbmo_gamma_closure(rho, ua, theta)


def muscl_term(u, smm, sm, s0, sp, spp):
    return _load().hlbmo_muscl_term(u, smm, sm, s0, sp, spp)


# ---- whole-grid solver ---------------------------------------------------------

class Oracle:
    """FP64 CPU solver of the paper's time step (Sec. 3).  Arrays are row-major [ny][nx]."""

    def __init__(self, nx, ny, gamma=1.4, Pr=0.71, mu=1e-3, sigma=0.0,
                 bc=(BC_PERIODIC,) * 4, bc_state=None, phi_mode=0, ablation=0):
        self.lib = _load()
        self.nx, self.ny = int(nx), int(ny)
        bcs = np.zeros(16) if bc_state is None else _f64(bc_state, 16)
        bca = (ctypes.c_int * 4)(*[int(b) for b in bc])
        self._h = self.lib.hlbmo_create(self.nx, self.ny, gamma, Pr, mu, sigma, bca,
                                        _ptr(bcs), int(phi_mode), int(ablation))
        if not self._h:
            raise ValueError("oracle: invalid arguments or out of memory")
        self.params = dict(gamma=gamma, Pr=Pr, mu=mu, sigma=sigma, bc=tuple(bc),
                           bc_state=bcs.copy(), phi_mode=phi_mode, ablation=ablation)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self.lib.hlbmo_destroy(h)
            self._h = None

    @property
    def n(self):
        return self.nx * self.ny

    def init(self, rho, ux, uy, theta, a1=None):
        n = self.n
        self._keep = [_f64(rho, n), _f64(ux, n), _f64(uy, n), _f64(theta, n),
                      None if a1 is None else _f64(a1, 3 * n)]
        self.lib.hlbmo_init(self._h, *[_ptr(a) for a in self._keep])

    def step(self, nsteps=1):
        self.lib.hlbmo_step(self._h, int(nsteps))

    @property
    def step_count(self):
        return self.lib.hlbmo_step_count(self._h)

    def set_threads(self, n):
        """Split the rows of each per-cell pass over n threads (the results
        do not change); 1, the default, runs them in order."""
        self.lib.hlbmo_set_threads(self._h, int(n))

    def macros(self):
        """dict of rho, ux, uy, theta, s (each [ny, nx]) and a1 ([3, ny, nx])."""
        n, shp = self.n, (self.ny, self.nx)
        out = {k: np.zeros(n) for k in ("rho", "ux", "uy", "theta", "s")}
        a1 = np.zeros(3 * n)
        self.lib.hlbmo_get(self._h, _ptr(out["rho"]), _ptr(out["ux"]), _ptr(out["uy"]),
                           _ptr(out["theta"]), _ptr(out["s"]), _ptr(a1))
        res = {k: v.reshape(shp) for k, v in out.items()}
        res["a1"] = a1.reshape((3,) + shp)
        return res

    def psi(self):
        out = np.zeros(9 * self.n)
        self.lib.hlbmo_get_psi(self._h, _ptr(out))
        return out.reshape(9, self.ny, self.nx)

    def feq(self):
        out = np.zeros(9 * self.n)
        self.lib.hlbmo_get_feq(self._h, _ptr(out))
        return out.reshape(9, self.ny, self.nx)

    def post_collision(self):
        out = np.zeros(9 * self.n)
        self.lib.hlbmo_get_post_collision(self._h, _ptr(out))
        return out.reshape(9, self.ny, self.nx)

    def entropy_rhs(self):
        out = np.zeros(self.n)
        self.lib.hlbmo_entropy_rhs(self._h, _ptr(out))
        return out.reshape(self.ny, self.nx)


def max_threads():
    """Processors the oracle can split its rows over (1 without OpenMP)."""
    return _load().hlbmo_max_threads()
