"""The row-marching fused kernel (two columns per thread) against the FP64
oracle in all its variants: HLBM_MARCH=0 (64 threads, <= 128 registers, the
FP32 default), 1 (96 threads), 2 (128 threads), 3 (64 threads, no register
cap), each instantiated for sigma = 0 / > 0 and both Phi forms.  The same
tolerances as the tiled kernel (1e-10 FP64, 1e-4 FP32), every boundary set,
grids that leave a ragged last strip (odd widths included, so that a pair
straddles the edge), and row segments of 1, 3 and all rows (each segment
refills its row rings from four rows above its first row).  The 16-bit
storage forms are checked on both the marching and the tiled kernel."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2002_03644_gb300 import inputs
from test_gpu_parity import BCS, TOL, _env, a1_bound, compare, run_pair
from test_gpu_precision import BOUND, errors

pytestmark = pytest.mark.gpu

BS = np.array([[1.02, 0.08, 0.01, 0.21], [0.98, 0.05, -0.02, 0.19],
               [1.01, 0.06, 0.03, 0.2], [0.99, 0.07, 0.0, 0.205]])


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


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("variant", range(4))
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 2, 2, 1)])
def test_march_variants(hl, precision, variant, bc):
    case = inputs.random_smooth(173, 141, seed=31, amp=0.04, u0=(0.06, 0.01), theta0=0.2, mu=3e-3,
                                sigma=0.5, bc=bc, bc_state=BS)
    with _env(HLBM_MARCH=variant):
        _, _, got, ref = run_pair(hl, case, precision, 9)
    compare(got, ref, case.gamma, TOL[precision], a1_own=a1_bound(precision, case.sigma, 9))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("variant", [0, 2])
@pytest.mark.parametrize("bc", BCS)
def test_march_boundaries(hl, precision, variant, bc):
    case = inputs.random_smooth(53, 41, seed=21, amp=0.04, u0=(0.06, 0.01), theta0=0.2, mu=3e-3,
                                sigma=0.5, bc=bc, bc_state=BS)
    with _env(HLBM_MARCH=variant, HLBM_MARCH_ROWS=5):
        _, _, got, ref = run_pair(hl, case, precision, 20)
    compare(got, ref, case.gamma, TOL[precision], a1_own=a1_bound(precision, case.sigma, 20))


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("rows", [1, 3, 100000])
@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 5), (37, 23), (130, 67), (185, 9)])
@pytest.mark.parametrize("sigma", [0.0, 0.7])
def test_march_segments(hl, precision, variant, rows, nx, ny, sigma):
    case = inputs.random_smooth(nx, ny, seed=100 + nx, amp=0.05, mu=2e-3, sigma=sigma)
    with _env(HLBM_MARCH=variant, HLBM_MARCH_ROWS=rows):
        _, _, got, ref = run_pair(hl, case, precision, 12)
    compare(got, ref, case.gamma, TOL[precision], a1_own=a1_bound(precision, sigma, 12))


@pytest.mark.parametrize("precision", [0, 1])
def test_march_phi_fd_and_ablations(hl, precision):
    for phi_mode, ablation in ((1, 0), (0, 1), (0, 2), (0, 3)):
        case = inputs.random_smooth(70, 44, seed=8, amp=0.05, mu=2e-3, sigma=0.3)
        case.phi_mode = phi_mode
        case.ablation = ablation
        for variant in (0, 3):
            with _env(HLBM_MARCH=variant):
                _, _, got, ref = run_pair(hl, case, precision, 10)
            compare(got, ref, case.gamma, TOL[precision], a1_own=a1_bound(precision, case.sigma, 10))


def test_march_16bit_forms_within_their_bounds(hl):
    case = inputs.vortex(n=256, R=8.0)
    ora = Oracle(case.nx, case.ny, **case.params())
    ora.init(*case.fields())
    ora.step(200)
    ref = ora.macros()
    for prec, variant in ((2, 0), (3, 0), (2, -1), (3, -1)):
        with _env(HLBM_MARCH=variant):
            s = hl.Solver(case.nx, case.ny, precision=prec, **case.params())
        s.init(*case.fields())
        s.step(200)
        got = s.macros()
        s.close()
        e = errors(got, ref, case.gamma)
        for k in ("rho", "ux", "uy", "theta", "s"):
            assert e[k]["linf"] <= BOUND[prec], (prec, k, e[k])


@pytest.mark.parametrize("precision", [1, 2, 3])
@pytest.mark.parametrize("sigma", [0.0, 0.5])
def test_periodic_instantiation_equals_general_kernel(hl, sigma, precision):
    """On an all-periodic grid the default FP32-arithmetic kernel (FP32 and
    the 16-bit storage forms) compiles the boundary selections out; every
    value must equal the general kernel's bitwise."""
    case = inputs.random_smooth(173, 141, seed=41, amp=0.05, u0=(0.06, -0.02), theta0=0.2, mu=3e-3, sigma=sigma)
    out = []
    for general in ("0", "1"):
        with _env(HLBM_MARCH=0, HLBM_MARCH_GENERAL=general):
            s = hl.Solver(case.nx, case.ny, precision=precision, **case.params())
        s.init(*case.fields())
        s.step(25)
        out.append(s.macros())
        s.close()
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k
