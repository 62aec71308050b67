"""CPU checks of the C ABI: the library builds and loads, exports every entry
point that include/hlbm.h declares, and its parameter struct has the layout
the header gives (checked against gcc's view of the header)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(hlbm_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2002_03644_gb300 import hlbm
    return ctypes.CDLL(hlbm.library_path())


def test_every_declared_entry_point_is_exported(lib):
    names = header_functions()
    assert "hlbm_step" in names and "hlbm_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2002_03644_gb300 import hlbm
    for n in header_functions():
        assert n in hlbm.ENTRY_POINTS and hasattr(hlbm, n), n


def test_params_layout_matches_header():
    from paper_2002_03644_gb300 import hlbm
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "hlbm.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(hlbm_params), offsetof(hlbm_params, gamma),
         offsetof(hlbm_params, bc), offsetof(hlbm_params, bc_state), offsetof(hlbm_params, diag_every),
         offsetof(hlbm_params, check_cfl), offsetof(hlbm_params, reserved));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, c], check=True)
        out = list(map(int, subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()))
    P = hlbm.hlbm_params
    want = [ctypes.sizeof(P), P.gamma.offset, P.bc.offset, P.bc_state.offset, P.diag_every.offset,
            P.check_cfl.offset, P.reserved.offset]
    assert out == want


def test_status_strings_and_version(lib):
    from paper_2002_03644_gb300 import hlbm
    assert hlbm.hlbm_abi_version() == 1
    for code in range(0, -9, -1):
        assert hlbm.hlbm_strerror(code) not in ("", "unknown status")


def test_invalid_params_rejected_without_touching_the_gpu(lib):
    from paper_2002_03644_gb300 import hlbm
    bad = [dict(nx=0), dict(gamma=1.0), dict(sigma=1.5), dict(mu=-1.0), dict(Pr=0.0),
           dict(bc=(0, 1, 0, 0)), dict(precision=7), dict(phi_mode=2)]
    for kw in bad:
        args = dict(nx=8, ny=8)
        args.update(kw)
        p = hlbm.make_params(**args)
        h = ctypes.c_void_p()
        code = lib.hlbm_create(ctypes.byref(p), None, ctypes.byref(h))
        assert code in (hlbm.HLBM_ERR_ARG, hlbm.HLBM_ERR_UNSUPPORTED), (kw, code)
        assert not h.value


def test_wall_sides_validated_without_touching_the_gpu(lib):
    """Walls: two cells across the wall, a positive wall temperature, no
    moment state and no batches; each is refused before any CUDA call."""
    from paper_2002_03644_gb300 import hlbm
    W, P = hlbm.HLBM_BC_WALL, hlbm.HLBM_BC_PERIODIC
    bs = [[1.0, 0.0, 0.0, 0.2]] * 4
    cases = [(dict(bc=(W, W, P, P), nx=1), hlbm.HLBM_ERR_ARG),
             (dict(bc=(P, P, W, W), ny=1), hlbm.HLBM_ERR_ARG),
             (dict(bc=(P, P, W, W), bc_state=[[1.0, 0.0, 0.0, 0.2]] * 3 + [[1.0, 0.0, 0.0, 0.0]]), hlbm.HLBM_ERR_ARG),
             (dict(bc=(P, P, W, W), precision=hlbm.HLBM_FP32_MOMENTS), hlbm.HLBM_ERR_UNSUPPORTED)]
    for kw, want in cases:
        args = dict(nx=8, ny=8, bc_state=bs)
        args.update(kw)
        p = hlbm.make_params(**args)
        h = ctypes.c_void_p()
        assert lib.hlbm_create(ctypes.byref(p), None, ctypes.byref(h)) == want, kw
        assert not h.value
    arr = (hlbm.hlbm_params * 1)(hlbm.make_params(8, 8, precision=hlbm.HLBM_FP32, bc=(P, P, W, W), bc_state=bs))
    b = ctypes.c_void_p()
    assert lib.hlbm_batch_create(arr, 1, None, ctypes.byref(b)) == hlbm.HLBM_ERR_UNSUPPORTED
    assert not b.value


def test_product_path_has_no_oracle_dependency():
    """The package never imports, links or runs anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_2002_03644_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                for pat in (r"^\s*(from|import)\s+oracle", r"hlbm_oracle", r"libhlbm_oracle", r"hlbmo_"):
                    assert not re.search(pat, txt, flags=re.M), (os.path.join(dirpath, f), pat)


def test_stream_handles_passed_through():
    """An explicit stream (int handle or an object with .cuda_stream) reaches
    the C ABI unchanged; torch's legacy default stream is never passed as
    NULL, which would ask the library for an unordered stream of its own."""
    from paper_2002_03644_gb300 import hlbm

    class FakeStream:
        cuda_stream = 0x5eed

    assert hlbm.torch_stream_handle(7) == 7
    assert hlbm.torch_stream_handle(FakeStream()) == 0x5eed


def test_selftest_wait_budget_checked_without_touching_the_gpu(lib):
    """A wait budget outside 1 .. 2^31 cycles is refused before any CUDA
    call."""
    from paper_2002_03644_gb300 import hlbm
    for budget in (0, -5, (1 << 31) + 1):
        assert hlbm.hlbm_selftest_wait(budget, False) == hlbm.HLBM_ERR_ARG
