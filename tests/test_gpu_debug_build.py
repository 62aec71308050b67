"""The index-checking debug build (HLBM_DEBUG, libhlbm_debug.so).  Its step
kernels check the cell of every global access and the marching kernel's
ring slots; a failed check is recorded and the access skipped, never
trapped.  Run in a child process (a process loads one build of the
library): every step kernel family -- the marching kernel on an all-periodic
grid and with every boundary kind (FP32, FP16 storage, and FP64 with its
cache planes of the level macros), the tiled kernel, the moment state and a
batch -- runs clean (no failed check) and still meets its parity bound
against the oracle (FP64 1e-10, FP32 1e-4).  The release build answers HLBM_ERR_UNSUPPORTED."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, os, sys
sys.path.insert(0, os.environ["HLBM_ROOT"]); sys.path.insert(0, os.path.join(os.environ["HLBM_ROOT"], "tests"))
import numpy as np
import torch
torch.cuda.set_device(0)
from paper_2002_03644_gb300 import hlbm, inputs
from test_gpu_parity import run_pair, compare, TOL, _env
out = {"library": hlbm.library_path(), "checks": []}
bs = np.array([[1.02, 0.08, 0.01, 0.21], [0.98, 0.05, -0.02, 0.19], [1.01, 0.06, 0.03, 0.2], [0.99, 0.07, 0.0, 0.205]])
runs = [("march periodic", dict(HLBM_MARCH=0), 1, (0, 0, 0, 0)),
        ("march boundaries", dict(HLBM_MARCH=0, HLBM_MARCH_ROWS=5), 1, (1, 2, 2, 1)),
        ("tiled boundaries", dict(HLBM_MARCH=-1), 1, (1, 1, 2, 2)),
        ("moments periodic", dict(), 4, (0, 0, 0, 0)),
        ("moments boundaries", dict(HLBM_MARCH_ROWS=3), 4, (2, 1, 1, 1)),
        ("fp16 march", dict(HLBM_MARCH=0), 2, (0, 0, 0, 0)),
        ("fp64 march boundaries", dict(HLBM_MARCH=0, HLBM_MARCH_ROWS=5), 0, (1, 2, 2, 1)),
        ("fp64 march periodic", dict(HLBM_MARCH=0), 0, (0, 0, 0, 0))]
for name, env, prec, bc in runs:
    case = inputs.random_smooth(101, 67, seed=3, amp=0.04, u0=(0.06, 0.01), theta0=0.2, mu=3e-3, sigma=0.5,
                                bc=bc, bc_state=bs)
    with _env(**env):
        _, _, got, ref = run_pair(hlbm, case, prec, 9)
    site = hlbm.hlbm_debug_check()
    if prec != 2:
        compare(got, ref, case.gamma, TOL[prec if prec in (0, 1) else 1])
    out["checks"].append([name, list(site)])
cases = [inputs.vortex(n=n, R=n / 12.0) for n in (48, 96)] + [inputs.sod(nx=160, ny=4, C0=3.875, mu=3e-6, sigma=0.0)]
b = hlbm.Batch([dict(nx=c.nx, ny=c.ny, precision=1, **c.params()) for c in cases])
for v, c in zip(b.cases, cases):
    v.init(*c.fields())
b.autotune()
b.step(20)
out["checks"].append(["batch", list(hlbm.hlbm_debug_check())])
b.close()
print(json.dumps(out))
"""


@pytest.fixture(scope="module")
def builds():
    import __graft_entry__ as g
    g.build()
    from paper_2002_03644_gb300 import build, hlbm
    return build, hlbm


def test_release_build_has_no_index_checks(builds):
    _, hl = builds
    with pytest.raises(hl.HlbmError) as e:
        hl.hlbm_debug_check()
    assert e.value.code == hl.HLBM_ERR_UNSUPPORTED


@pytest.mark.gpu
def test_debug_build_runs_every_step_kernel_clean(builds):
    build, _ = builds
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = build.build_library(debug=True)
    env = dict(os.environ, HLBM_LIBRARY="debug", HLBM_ROOT=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["library"] == lib
    for name, (site, a, b) in out["checks"]:
        assert site == 0, (name, site, a, b)
