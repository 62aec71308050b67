"""Argument checks of the C ABI that need no GPU: every entry point refuses
empty grids, grids above the size limit and parameters outside their
ranges before it touches CUDA, with the documented error code."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def hl():
    import __graft_entry__ as g
    g.build()
    from paper_2002_03644_gb300 import hlbm
    return hlbm


def _create(hl, **kw):
    base = dict(nx=16, ny=16, precision=hl.HLBM_FP32)
    base.update(kw)
    h = ctypes.c_void_p()
    return hl._lib().hlbm_create(ctypes.byref(hl.make_params(**base)), None, ctypes.byref(h))


BAD = [
    ("empty x", dict(nx=0), "ARG"),
    ("empty y", dict(ny=0), "ARG"),
    ("negative size", dict(nx=-4), "ARG"),
    ("above 2^28 cells", dict(nx=1 << 15, ny=(1 << 13) + 1), "ARG"),
    ("unknown precision", dict(precision=9), "UNSUPPORTED"),
    ("gamma <= 1", dict(gamma=1.0), "ARG"),
    ("Pr <= 0", dict(Pr=0.0), "ARG"),
    ("negative mu", dict(mu=-1e-3), "ARG"),
    ("sigma > 1", dict(sigma=1.5), "ARG"),
    ("sigma < 0", dict(sigma=-0.1), "ARG"),
    ("phi_mode 2", dict(phi_mode=2), "ARG"),
    ("periodic x- without x+", dict(bc=(0, 1, 0, 0)), "ARG"),
    ("unknown side kind", dict(bc=(7, 7, 0, 0)), "UNSUPPORTED"),
    ("Dirichlet side with rho = 0", dict(bc=(2, 1, 0, 0), bc_state=np.zeros((4, 4))), "ARG"),
    ("wall on a one-cell-wide grid", dict(nx=1, bc=(3, 3, 0, 0), bc_state=np.full((4, 4), 0.2)), "ARG"),
    ("walls with the moment state", dict(precision=4, bc=(0, 0, 3, 3), bc_state=np.full((4, 4), 0.2)), "UNSUPPORTED"),
    ("negative diag_every", dict(diag_every=-1), "ARG"),
    ("unknown ablation bit", dict(ablation=4), "ARG"),
]


@pytest.mark.parametrize("name,kw,code", BAD, ids=[b[0] for b in BAD])
def test_create_refuses_bad_parameters(hl, name, kw, code):
    assert _create(hl, **kw) == getattr(hl, f"HLBM_ERR_{code}")


def test_create_refuses_null_arguments(hl):
    h = ctypes.c_void_p()
    assert hl._lib().hlbm_create(None, None, ctypes.byref(h)) == hl.HLBM_ERR_ARG
    p = hl.make_params(16, 16)
    assert hl._lib().hlbm_create(ctypes.byref(p), None, None) == hl.HLBM_ERR_ARG


def test_batch_refuses_empty_lists_and_other_precisions(hl):
    b = ctypes.c_void_p()
    p = (hl.hlbm_params * 1)(hl.make_params(16, 16, precision=hl.HLBM_FP32))
    assert hl._lib().hlbm_batch_create(p, 0, None, ctypes.byref(b)) == hl.HLBM_ERR_ARG
    q = (hl.hlbm_params * 1)(hl.make_params(16, 16, precision=hl.HLBM_FP64))
    assert hl._lib().hlbm_batch_create(q, 1, None, ctypes.byref(b)) == hl.HLBM_ERR_UNSUPPORTED


@pytest.mark.parametrize("widths,H,W,B", [
    ((4,), 8, 8, 1),            # no layer
    ((4, 16, 5), 8, 8, 1),      # output width differs from the input (residual)
    ((4, 0, 4), 8, 8, 1),       # an empty layer
    ((4, 16, 4), 0, 8, 1),      # empty image
    ((4, 16, 4), 8, 8, 0),      # empty batch
])
def test_surrogate_refuses_bad_shapes(hl, widths, H, W, B):
    arr = (ctypes.c_int * len(widths))(*widths)
    s = ctypes.c_void_p()
    assert hl._lib().hlbm_sur_create(len(widths) - 1, arr, H, W, B, None, ctypes.byref(s)) == hl.HLBM_ERR_ARG
