"""The CUDA path against the paper's own numbers and closed forms, without
the oracle in between: shear-wave viscosity errors of Table 1 (present
model, and the original model's divergence at Ma >= 1 with centred E1), the
acoustic decay rate and sound speed of Sec. 4.3 / 5.1, and the Sod tube
against the exact Riemann solution."""
import math
import os

import numpy as np
import pytest

from oracle import exact_riemann as er
from paper_2002_03644_gb300 import inputs

pytestmark = pytest.mark.gpu
R_GAS = 287.15


@pytest.fixture(scope="module")
def hl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2002_03644_gb300 import hlbm
    return hlbm


def _rows(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


def _shear(hl, nu_phys, Ma, precision, ablation=0, span=30000, every=250):
    Tr = 800.0
    C0 = math.sqrt(R_GAS * Tr) * math.sqrt(3.0)
    th = 300.0 / Tr
    c = math.sqrt(1.4 * th / 3.0)
    nu = nu_phys / ((1.0 / 200.0) * C0)
    case = inputs.shear_wave(ny=200, Ma=Ma, mu=nu, a0_over_c=(20.0 / C0) / c, theta0=th)
    case.ablation = ablation
    s = hl.Solver(case.nx, case.ny, precision=precision, **case.params())
    s.init(*case.fields())
    ts, mx = [], []
    while True:
        m = s.macros()
        ux = m["ux"]
        if not np.isfinite(ux).all() or np.abs(ux).max() > 1.0:
            return None, s.step_count
        ts.append(s.step_count)
        mx.append(ux.max())
        if s.step_count >= span:
            break
        s.step(every)
    slope = np.polyfit(np.array(ts, float), np.log(mx), 1)[0]
    return (-slope / case.meta["k"] ** 2 - nu) / nu, s.step_count


@pytest.mark.parametrize("row", range(6))
def test_gpu_shear_wave_matches_table1(hl, golden_dir, row):
    """FP64: the viscosity error of Table 1 within 11 %, the bound the
    oracle's own pin holds (its worst row is 10.1 % off)."""
    nu_phys, Ma, eps_paper = map(float, _rows(golden_dir, "shear_wave_table1.txt")[row])
    eps, _ = _shear(hl, nu_phys, Ma, 0)
    assert eps is not None
    assert abs(eps - eps_paper) <= 0.11 * eps_paper, (eps, eps_paper)


@pytest.mark.parametrize("row", range(6))
def test_gpu_shear_wave_fp32_viscosity(hl, golden_dir, row):
    """FP32 cannot resolve Table 1's errors themselves (a few 1e-4 to 1e-3):
    rounding in a state of order 1 perturbs u by about 1e-7 per step, and
    over the 30,000 steps of the fit this shifts the fitted decay rate by
    about 1e-3 relative, the size of epsilon.  FP32 is held to the
    viscosity itself: |epsilon| < 3e-3 at every Mach number of the table."""
    nu_phys, Ma, _ = map(float, _rows(golden_dir, "shear_wave_table1.txt")[row])
    eps, _ = _shear(hl, nu_phys, Ma, 1)
    assert eps is not None
    assert abs(eps) < 3e-3, eps


@pytest.mark.parametrize("row", range(3))
def test_gpu_original_model_upwinding_matches_table1(hl, golden_dir, row):
    nu_s, ma_s, want = _rows(golden_dir, "shear_wave_table1_original.txt")[row]
    eps, n = _shear(hl, float(nu_s), float(ma_s), 0, ablation=hl.HLBM_ABL_CENTRED_E1)
    if want == "diverged":
        assert eps is None, (eps, n)
    else:
        assert eps is not None and abs(eps - float(want)) <= 0.15 * float(want)


def _acoustic(hl, precision, gamma, dp_rel):
    Tr = 1478.75
    C0 = math.sqrt(R_GAS * Tr) * math.sqrt(3.0)
    nu = 0.01 / (101325.0 / (R_GAS * 300.0)) / ((0.1 / 200.0) * C0)
    case = inputs.acoustic_wave(nx=200, ny=2, mu=nu, gamma=gamma, sigma=0.95, Pr=0.71, dp_rel=dp_rel)
    s = hl.Solver(case.nx, case.ny, precision=precision, **case.params())
    s.init(*case.fields())
    k = case.meta["k"]
    xx = np.arange(case.nx) + 0.5
    ts, amp, ph = [], [], []
    for _ in range(41):
        m = s.macros()
        pp = (m["rho"] * m["theta"] / 3.0)[0]
        pp = pp - pp.mean()
        a, b = 2 * np.mean(pp * np.sin(k * xx)), 2 * np.mean(pp * np.cos(k * xx))
        ts.append(s.step_count); amp.append(math.hypot(a, b)); ph.append(math.atan2(b, a))
        s.step(250)
    ts = np.array(ts, float)
    alpha = -np.polyfit(ts, np.log(amp), 1)[0] / k ** 2
    speed = -np.polyfit(ts, np.unwrap(ph), 1)[0] / k
    alpha_th = 0.5 * nu + 0.5 * (gamma - 1.0) * nu / 0.71
    c_th = math.sqrt(gamma * case.theta.mean() / 3.0)
    return alpha, alpha_th, speed, c_th


@pytest.mark.parametrize("gamma", [1.4, 2.0])
def test_gpu_acoustic_decay_and_sound_speed(hl, gamma):
    """FP64, the 5 Pa wave of Sec. 4.3: decay rate within 2 % of the
    linear-acoustics value, sound speed within 1e-4."""
    alpha, alpha_th, speed, c_th = _acoustic(hl, 0, gamma, 5.0 / 101325.0)
    assert abs(alpha - alpha_th) < 0.02 * alpha_th
    assert abs(speed - c_th) < 1e-4 * c_th


@pytest.mark.parametrize("gamma", [1.4, 2.0])
def test_gpu_fp32_sound_speed(hl, gamma):
    """FP32 checks the sound speed only, on a 2e-3 wave (still linear).  It
    cannot resolve the wave's damping: the thermal part needs the Laplacian
    of theta across one cell, k^2 theta' = 3e-8 for the 5 Pa wave, about two
    FP32 ulps of theta, and rounding of that size also dominates the
    viscous decay of a wave this weak over 10^4 steps."""
    _, _, speed, c_th = _acoustic(hl, 1, gamma, 2e-3)
    assert abs(speed - c_th) < 1e-4 * c_th


@pytest.mark.parametrize("precision", [0, 1])
def test_gpu_sod_against_exact_solution(hl, precision):
    case = inputs.sod(C0=3.875, mu=3e-6, sigma=0.0)
    s = hl.Solver(case.nx, case.ny, precision=precision, **case.params())
    s.init(*case.fields())
    s.step(case.steps)
    m = s.macros()
    t = case.steps * case.meta["dx"] / case.meta["C0"]
    x = (np.arange(case.nx) + 0.5) / case.nx
    r, u, p = er.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (x - 0.5) / t)
    assert np.isfinite(m["rho"]).all()
    assert np.mean(np.abs(m["rho"][0] - r)) < 1.5e-2
    assert np.mean(np.abs(m["ux"][0] * case.meta["C0"] - u)) < 2.5e-2


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kw", [dict(), dict(Ma=0.4), dict(Ma=1.2), dict(Pr=2.0), dict(Pr=0.3), dict(gamma=1.67)],
                         ids=["Ma0.8", "Ma0.4", "Ma1.2", "Pr2", "Pr0.3", "gamma1.67"])
def test_gpu_thermal_couette(hl, precision, kw):
    """Thermal Couette flow (Sec. 4.4) between Dirichlet sides for the Mach,
    Prandtl and gamma variations of the paper's figure: the steady
    temperature rise matches the analytic parabola within 5 % of its peak and
    the velocity is linear within 2 % of U (these walls leave 3.6 % and
    0.9 %, as in the oracle; wall sides are tested in test_gpu_walls)."""
    from test_oracle_physics import couette_errors
    case = inputs.couette(**kw, steps=150000, walls="dirichlet")
    s = hl.Solver(case.nx, case.ny, precision=precision, **case.params())
    s.init(*case.fields())
    s.step(case.steps)
    eT, eu = couette_errors(case, s.macros())
    assert eT < 0.05, eT
    assert eu < 0.02, eu
