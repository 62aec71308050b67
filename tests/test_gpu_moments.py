"""The moment-state form (HLBM_FP32_MOMENTS: rho, u, s and a1 stored, the
populations rebuilt every step) against the FP64 oracle, with the FP32
tolerance of the population form (1e-4 of each field's scale): sizes that
leave ragged strips and segments, sigma = 0 and > 0, every boundary set,
both Phi forms and the original-model ablations, row segments of 1, 3 and
all rows; plus the checkpoint round trip, diagnostics and the one call it
does not support (the populations)."""
import numpy as np
import pytest

from paper_2002_03644_gb300 import inputs
from test_gpu_parity import BCS, TOL, _env, a1_bound, compare, run_pair

pytestmark = pytest.mark.gpu

MOM = 4  # HLBM_FP32_MOMENTS
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


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 5), (37, 23), (117, 67), (233, 41)])
@pytest.mark.parametrize("sigma", [0.0, 0.6])
def test_moments_periodic_random_fields(hl, nx, ny, sigma):
    case = inputs.random_smooth(nx, ny, seed=100 + nx, amp=0.05, mu=2e-3, sigma=sigma)
    _, _, got, ref = run_pair(hl, case, MOM, 12)
    compare(got, ref, case.gamma, TOL[1], a1_own=a1_bound(1, sigma, 12))


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("sigma", [0.0, 0.5])
def test_moments_boundaries(hl, bc, sigma):
    case = inputs.random_smooth(53, 41, seed=21, amp=0.04, u0=(0.06, 0.01), theta0=0.2, mu=3e-3,
                                sigma=sigma, bc=bc, bc_state=BS)
    with _env(HLBM_MARCH_ROWS=5):
        _, _, got, ref = run_pair(hl, case, MOM, 20)
    compare(got, ref, case.gamma, TOL[1], a1_own=a1_bound(1, sigma, 20))


@pytest.mark.parametrize("rows", [1, 3, 100000])
@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 2, 2, 1), (1, 1, 1, 1)])
def test_moments_segments(hl, rows, bc):
    case = inputs.random_smooth(130, 67, seed=7, amp=0.04, u0=(0.05, -0.02), theta0=0.2, mu=3e-3,
                                sigma=0.3, bc=bc, bc_state=BS)
    with _env(HLBM_MARCH_ROWS=rows):
        _, _, got, ref = run_pair(hl, case, MOM, 12)
    compare(got, ref, case.gamma, TOL[1], a1_own=a1_bound(1, case.sigma, 12))


def test_moments_phi_fd_ablations_and_given_a1(hl):
    for phi_mode, ablation in ((1, 0), (0, 1), (0, 2), (0, 3)):
        case = inputs.random_smooth(70, 44, seed=8, amp=0.05, mu=2e-3, sigma=0.3)
        case.phi_mode = phi_mode
        case.ablation = ablation
        _, _, got, ref = run_pair(hl, case, MOM, 10)
        compare(got, ref, case.gamma, TOL[1], a1_own=a1_bound(1, case.sigma, 10))
    case = inputs.random_smooth(30, 26, seed=4, amp=0.04, mu=3e-3, sigma=0.4)
    a1 = np.random.default_rng(3).normal(size=(3, case.ny, case.nx)) * 1e-4
    _, _, got, ref = run_pair(hl, case, MOM, 6, a1=a1)
    compare(got, ref, case.gamma, TOL[1])


def test_moments_vortex_and_sod(hl):
    case = inputs.vortex(n=256, R=8.0)
    _, _, got, ref = run_pair(hl, case, MOM, 40)
    compare(got, ref, case.gamma, TOL[1], a1_own=a1_bound(1, case.sigma, 40))
    # a shock: L2 over the fields (rounding differences grow at the discontinuities)
    case = inputs.sod(C0=3.875, mu=3e-6, sigma=0.0)
    _, _, got, ref = run_pair(hl, case, MOM, 100)
    for k in ("rho", "ux", "theta"):
        d = (got[k] - ref[k]) / np.abs(ref[k]).max()
        assert np.sqrt(np.mean(d * d)) < 1e-4, k


def test_moments_state_roundtrip_diagnostics_and_populations(hl):
    case = inputs.vortex(n=96, R=6.0)
    a = hl.Solver(case.nx, case.ny, precision=MOM, **case.params())
    a.init(*case.fields())
    a.step(5)
    blob = a.state()
    a.step(5)
    b = hl.Solver(case.nx, case.ny, precision=MOM, **case.params())
    b.set_state(blob)
    b.step(5)
    ma, mb = a.macros(), b.macros()
    for k in ma:
        assert np.array_equal(ma[k], mb[k]), k
    # diagnostics: mass and momentum of the stored moments
    d = a.diagnostics()
    assert abs(d[0] - ma["rho"].sum()) < 1e-6 * d[0]
    assert abs(d[1] - (ma["rho"] * ma["ux"]).sum()) < 1e-6 * d[0]
    assert d[7] == 0
    # mass is conserved to FP32 rounding
    c = hl.Solver(case.nx, case.ny, precision=MOM, **case.params())
    c.init(*case.fields())
    m0 = c.diagnostics()[0]
    c.step(50)
    assert abs(c.diagnostics()[0] - m0) < 1e-5 * m0
    with pytest.raises(hl.HlbmError) as e:
        a.populations()
    assert e.value.code == hl.HLBM_ERR_UNSUPPORTED


@pytest.mark.parametrize("sigma", [0.0, 0.6])
def test_moments_periodic_instantiation_equals_general_kernel(hl, sigma):
    """All-periodic grids take the moment kernel with the boundary
    selections compiled out; it must equal the general kernel bitwise."""
    from test_gpu_parity import _env
    case = inputs.random_smooth(130, 67, seed=9, amp=0.05, u0=(0.05, -0.02), theta0=0.2, mu=3e-3, sigma=sigma)
    out = []
    for general in ("0", "1"):
        with _env(HLBM_MARCH_GENERAL=general):
            s = hl.Solver(case.nx, case.ny, precision=MOM, **case.params())
        s.init(*case.fields())
        s.step(25)
        out.append(s.macros())
        s.close()
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k
