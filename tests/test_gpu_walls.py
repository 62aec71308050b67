"""Wall sides (no-slip, fixed temperature) on the GPU against the FP64
oracle, with the tolerances of the other parity tests (1e-10 FP64, 1e-4
FP32): moving and resting walls at temperatures above and below the gas, on
the y sides, the x sides and all four, with periodic, zero-gradient and
Dirichlet partner sides (corners), sigma = 0 and > 0, both Phi forms, grids
from two cells across to several tiles with ragged tails.  Walls always take the tiled kernel, whatever the kernel-choice
variables say; the 16-bit storage forms stay within their error bounds;
and the thermal Couette flow (Sec. 4.4) matches the analytic profile."""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2002_03644_gb300 import inputs
from test_gpu_parity import TOL, _env, compare, run_pair
from test_gpu_precision import BOUND, errors

pytestmark = pytest.mark.gpu

W = inputs.BC_WALL
BS = np.array([[1.02, 0.08, 0.01, 0.21], [0.98, 0.05, -0.02, 0.19],
               [1.0, 0.03, 0.0, 0.19], [1.0, -0.05, 0.0, 0.215]])


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


def wall_case(nx, ny, xbc=(0, 0), sigma=0.5, seed=21, phi_mode=0):
    case = inputs.random_smooth(nx, ny, seed=seed, amp=0.04, u0=(0.06, 0.01), theta0=0.2, mu=3e-3,
                                sigma=sigma, bc=tuple(xbc) + (W, W), bc_state=BS)
    case.phi_mode = phi_mode
    return case


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nx,ny", [(1, 2), (5, 3), (37, 23), (70, 44), (101, 67)])
@pytest.mark.parametrize("xbc", [(0, 0), (1, 1), (2, 1)])
def test_walls_against_oracle(hl, precision, nx, ny, xbc):
    case = wall_case(nx, ny, xbc, seed=100 + nx)
    _, _, got, ref = run_pair(hl, case, precision, 15)
    compare(got, ref, case.gamma, TOL[precision])


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("nx,ny", [(2, 1), (3, 5), (41, 37), (67, 101)])
@pytest.mark.parametrize("bc", [(W, W, 0, 0), (W, W, 1, 1), (W, W, 2, 1), (W, W, W, W), (1, W, W, 1)],
                         ids=["xwall-per", "xwall-zg", "xwall-dir", "all-walls", "mixed"])
def test_x_walls_against_oracle(hl, precision, nx, ny, bc):
    """Walls on the x sides (and on all four), every kind of partner side,
    corners included."""
    if (bc[2] == W or bc[3] == W) and ny < 2:
        pytest.skip("a y wall needs two rows")
    bs = BS[[2, 3, 0, 1]][:, [0, 2, 1, 3]].copy()  # x walls: wall velocity along y
    bs[2:] = BS[2:]
    if bc[2] == 2:
        bs[2] = BS[0]
    case = inputs.random_smooth(nx, ny, seed=300 + nx, amp=0.04, u0=(0.01, 0.06), theta0=0.2, mu=3e-3,
                                sigma=0.5, bc=bc, bc_state=bs)
    _, _, got, ref = run_pair(hl, case, precision, 15)
    compare(got, ref, case.gamma, TOL[precision])


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("sigma,phi_mode", [(0.0, 0), (1.0, 0), (0.4, 1)])
def test_walls_sigma_and_phi_forms(hl, precision, sigma, phi_mode):
    case = wall_case(53, 41, (1, 2), sigma=sigma, seed=5, phi_mode=phi_mode)
    _, _, got, ref = run_pair(hl, case, precision, 20)
    compare(got, ref, case.gamma, TOL[precision])


def test_walls_keep_the_tiled_kernel(hl):
    """The marching and TMA variables cannot move a case with walls off the
    tiled kernel (which alone reads the wall ghost rows)."""
    case = wall_case(130, 67, (0, 0), seed=7)
    for env in (dict(HLBM_MARCH=0), dict(HLBM_MARCH=2), dict(HLBM_FP32_TMA=0)):
        with _env(**env):
            _, _, got, ref = run_pair(hl, case, 1, 12)
        compare(got, ref, case.gamma, TOL[1])


def test_walls_16bit_forms_within_their_bounds(hl):
    case = wall_case(96, 64, (0, 0), seed=11)
    ora = Oracle(case.nx, case.ny, **case.params())
    ora.init(*case.fields())
    ora.step(100)
    ref = ora.macros()
    for prec in (2, 3):
        s = hl.Solver(case.nx, case.ny, precision=prec, **case.params())
        s.init(*case.fields())
        s.step(100)
        got = s.macros()
        s.close()
        e = errors(got, ref, case.gamma)
        for k in ("rho", "ux", "uy", "theta", "s"):
            assert e[k]["linf"] <= BOUND[prec], (prec, k, e[k])


def test_walls_state_roundtrip(hl):
    case = wall_case(40, 30, (0, 0), seed=3)
    a = hl.Solver(case.nx, case.ny, precision=1, **case.params())
    a.init(*case.fields())
    a.step(4)
    blob = a.state()
    a.step(6)
    b = hl.Solver(case.nx, case.ny, precision=1, **case.params())
    b.set_state(blob)
    b.step(6)
    ma, mb = a.macros(), b.macros()
    for k in ma:
        assert np.array_equal(ma[k], mb[k]), k


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kw", [dict(), dict(Ma=1.2), dict(Pr=2.0), dict(gamma=1.67)],
                         ids=["Ma0.8", "Ma1.2", "Pr2", "gamma1.67"])
def test_gpu_thermal_couette_between_walls(hl, precision, kw):
    """Thermal Couette flow (Sec. 4.4) between wall sides after 150,000
    steps: the velocity within 1e-3 of U, the temperature rise within 1e-3
    of the analytic peak in FP64 (the FP64 oracle reaches 1e-4 and 3e-7) and
    1e-2 in FP32, whose rounding of theta (about 1e-8 per step on a rise of
    5e-3) shifts the slow thermal balance (6e-3 at Pr 2)."""
    from test_oracle_physics import couette_errors
    case = inputs.couette(**kw, steps=150000)
    s = hl.Solver(case.nx, case.ny, precision=precision, **case.params())
    s.init(*case.fields())
    s.step(case.steps)
    eT, eu = couette_errors(case, s.macros())
    assert eT < (1e-3 if precision == 0 else 1e-2), eT
    assert eu < 1e-3, eu
