"""Physics pins of the whole oracle against closed forms and the paper's
printed numbers: exact Riemann solution (Sod), shear-wave viscosity
(Table 1 of Sec. 4.1), acoustic decay rate (Sec. 4.3), isentropic sound
speed (eq. speed of sound), second-order convergence of the convected
vortex (Sec. 4.2)."""
import math
import os

import numpy as np
import pytest

from oracle import exact_riemann as er
from oracle.oracle import Oracle
from paper_2002_03644_gb300 import inputs

R_GAS = 287.15  # J/(kg K), Sec. 2.1


def run(case, steps):
    o = Oracle(case.nx, case.ny, **case.params())
    o.init(*case.fields())
    o.step(steps)
    return o


# ---- exact Riemann solver: self-consistency against jump conditions ----------

def test_exact_riemann_solver_satisfies_jump_conditions():
    g = 1.4
    L, Rr = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    ps, us, rl, rr = er.star_state(L, Rr, g)
    # right-moving shock: Rankine-Hugoniot mass and momentum flux balance
    S = (rr * us - Rr[0] * Rr[1]) / (rr - Rr[0])
    mflux_l, mflux_r = rr * (us - S), Rr[0] * (Rr[1] - S)
    assert abs(mflux_l - mflux_r) < 1e-12
    mom_l = rr * us * (us - S) + ps
    mom_r = Rr[0] * Rr[1] * (Rr[1] - S) + Rr[2]
    assert abs(mom_l - mom_r) < 1e-12
    # energy flux balance across the shock: (E + p) u - S E on both sides
    E = lambda r, u, p: p / (g - 1) + 0.5 * r * u * u
    flux = lambda r, u, p: (E(r, u, p) + p) * u - S * E(r, u, p)
    assert abs(flux(rr, us, ps) - flux(*Rr)) < 1e-12
    # left rarefaction: isentropic and the left Riemann invariant is constant
    assert abs(ps / rl ** g - L[2] / L[0] ** g) < 1e-12
    cl, cs = math.sqrt(g * L[2] / L[0]), math.sqrt(g * ps / rl)
    assert abs((L[1] + 2 * cl / (g - 1)) - (us + 2 * cs / (g - 1))) < 1e-12
    # inside the fan the solution is sonic along its characteristic
    xi = np.linspace(-cl + 1e-6, us - cs - 1e-6, 7)
    r, u, p = er.sample(L, Rr, xi, g)
    c = np.sqrt(g * p / r)
    assert np.allclose(u - c, xi, atol=1e-12)


def test_sod_matches_exact_solution():
    c = inputs.sod(C0=3.875, mu=3e-6, sigma=0.0)
    o = run(c, c.steps)
    m = o.macros()
    t = c.steps * c.meta["dx"] / c.meta["C0"]
    assert abs(t - 0.2) < 1e-3
    x = (np.arange(c.nx) + 0.5) / c.nx
    r, u, p = er.sample((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), (x - 0.5) / t)
    rho = m["rho"]
    assert np.isfinite(rho).all()
    # quasi-1D: every row equal
    assert np.abs(rho - rho[0]).max() < 1e-12
    assert np.mean(np.abs(rho[0] - r)) < 1.5e-2
    uphys = m["ux"][0] * c.meta["C0"]
    assert np.mean(np.abs(uphys - u)) < 2.5e-2
    pphys = (m["rho"][0] * m["theta"][0]) * c.meta["T_r"]
    assert np.mean(np.abs(pphys - p)) < 1.5e-2


def _shear_case(nu_phys, Ma, ablation=0):
    Tr = 800.0
    C0 = math.sqrt(R_GAS * Tr) * math.sqrt(3.0)
    dx = 1.0 / 200.0
    th = 300.0 / Tr
    c = math.sqrt(1.4 * th / 3.0)
    nu = nu_phys / (dx * C0)
    case = inputs.shear_wave(ny=200, Ma=Ma, mu=nu, a0_over_c=(20.0 / C0) / c, theta0=th)
    case.ablation = ablation
    return case, nu


def _shear_eps(nu_phys, Ma, span=30000, every=250, ablation=0):
    case, nu = _shear_case(nu_phys, Ma, ablation)
    o = Oracle(case.nx, case.ny, **case.params())
    o.init(*case.fields())
    ts, mx = [], []
    while True:
        ts.append(o.step_count)
        mx.append(o.macros()["ux"].max())
        if o.step_count >= span:
            break
        o.step(every)
    slope = np.polyfit(np.array(ts, float), np.log(mx), 1)[0]
    return (-slope / case.meta["k"] ** 2 - nu) / nu


def _table1(golden_dir):
    with open(os.path.join(golden_dir, "shear_wave_table1.txt")) as f:
        return [tuple(map(float, l.split())) for l in f if l.strip() and not l.startswith("#")]


@pytest.mark.slow
@pytest.mark.parametrize("row", range(6))
def test_shear_wave_viscosity_matches_table1(row, golden_dir):
    """Sec. 4.1: nu measured from the fitted decay of max(u_x) reproduces
    the printed relative errors of the present model within 11 % (measured:
    10.1 % at nu = 0.1 m^2/s, Ma 0.5, and 0.3 % to 3.3 % on the other five
    rows)."""
    nu_phys, Ma, eps_paper = _table1(golden_dir)[row]
    eps = _shear_eps(nu_phys, Ma)
    assert abs(eps - eps_paper) <= 0.11 * eps_paper, (nu_phys, Ma, eps, eps_paper)


def _original_rows(golden_dir):
    with open(os.path.join(golden_dir, "shear_wave_table1_original.txt")) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


@pytest.mark.slow
@pytest.mark.parametrize("row", range(3))
def test_original_model_upwinding_reproduces_table1(row, golden_dir):
    """Improvement (1) of the paper (Sec. 3.2): with E1 by centred
    differences, as in the original model, the shear wave diverges at
    Ma >= 1 and gives the printed error at Ma = 0.5 (Table 1, column O)."""
    nu_s, ma_s, want = _original_rows(golden_dir)[row]
    nu_phys, Ma = float(nu_s), float(ma_s)
    if want == "diverged":
        case, _ = _shear_case(nu_phys, Ma, ablation=1)
        o = Oracle(case.nx, case.ny, **case.params())
        o.init(*case.fields())
        blew = False
        for _ in range(60):
            o.step(500)
            ux = o.macros()["ux"]
            if not np.isfinite(ux).all() or np.abs(ux).max() > 1.0:
                blew = True
                break
        assert blew, (nu_phys, Ma)
        # and the paper's upwind E1 stays stable over the same span
        case0, _ = _shear_case(nu_phys, Ma, ablation=0)
        o0 = Oracle(case0.nx, case0.ny, **case0.params())
        o0.init(*case0.fields())
        o0.step(o.step_count)
        assert np.isfinite(o0.macros()["ux"]).all()
    else:
        eps = _shear_eps(nu_phys, Ma, ablation=1)
        assert abs(eps - float(want)) <= 0.15 * float(want), (eps, want)


def _acoustic(gamma, ablation=0):
    Tr = 1478.75
    C0 = math.sqrt(R_GAS * Tr) * math.sqrt(3.0)
    dx = 0.1 / 200.0
    rho_inf = 101325.0 / (R_GAS * 300.0)
    nu = 0.01 / rho_inf / (dx * C0)
    c = inputs.acoustic_wave(nx=200, ny=2, mu=nu, gamma=gamma, sigma=0.95, Pr=0.71)
    c.ablation = ablation
    o = Oracle(c.nx, c.ny, **c.params())
    o.init(*c.fields())
    k = c.meta["k"]
    xx = np.arange(c.nx) + 0.5
    ts, amp, ph = [], [], []
    for _ in range(41):
        m = o.macros()
        pp = (m["rho"] * m["theta"] / 3.0)[0]
        pp = pp - pp.mean()
        a, b = 2 * np.mean(pp * np.sin(k * xx)), 2 * np.mean(pp * np.cos(k * xx))
        ts.append(o.step_count); amp.append(math.hypot(a, b)); ph.append(math.atan2(b, a))
        o.step(250)
    ts = np.array(ts, float)
    alpha = -np.polyfit(ts, np.log(amp), 1)[0] / k ** 2
    speed = -np.polyfit(ts, np.unwrap(ph), 1)[0] / k
    return nu, alpha, speed, c


@pytest.mark.parametrize("gamma", [1.4, 2.0, 1.1])
def test_acoustic_decay_rate_and_sound_speed(gamma):
    """Sec. 4.3: alpha = (D-1)/D nu + (gamma-1)/2 nu/Pr, including the
    polyatomic case where E2 removes the spurious bulk viscosity; and the
    isentropic speed of sound c^2 = gamma c_s^2 theta (eq. speed of sound)."""
    nu, alpha, speed, c = _acoustic(gamma)
    alpha_th = 0.5 * nu + 0.5 * (gamma - 1.0) * nu / 0.71
    assert abs(alpha - alpha_th) < 0.02 * alpha_th
    c_th = math.sqrt(gamma * c.theta.mean() / 3.0)
    assert abs(speed - c_th) < 1e-4 * c_th


def test_without_e2_a_polyatomic_gas_is_overdamped():
    """Improvement (2), Sec. 4.3: without E2 the trace of the viscous stress
    is wrong for gamma != (D+2)/D, adding bulk viscosity (the measured decay
    rate is 40 % too high at gamma = 1.4); at gamma = 2 = (D+2)/D, E2 is zero
    and nothing changes."""
    nu, a_on, _, _ = _acoustic(1.4)
    _, a_off, _, _ = _acoustic(1.4, ablation=2)
    th = 0.5 * nu + 0.2 * nu / 0.71
    assert abs(a_on - th) < 0.02 * th
    assert a_off > 1.25 * th
    _, b_on, _, _ = _acoustic(2.0)
    _, b_off, _, _ = _acoustic(2.0, ablation=2)
    assert abs(b_on - b_off) < 1e-9 * b_on


def _vortex_error(n, R):
    c = inputs.vortex(n=n, R=R, noise=0.0)
    u0 = c.meta["c_inf"] * c.meta["Ma"]
    steps = int(round(n / u0))
    m = run(c, steps).macros()
    shift = u0 * steps - n
    # analytic solution: the initial vortex advected by u0 * steps (periodic
    # box of n cells, so the displacement modulo n is `shift`)
    X, Y = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
    g, Mv, th = 1.4, c.meta["beta"] * c.meta["Ma"], c.meta["theta_inf"]
    r2 = ((X - 0.5 * n - shift) / R) ** 2 + ((Y - 0.5 * n) / R) ** 2
    Tr = 1.0 - 0.5 * (g - 1.0) * Mv * Mv * np.exp(1.0 - r2)
    pa = Tr ** (1.0 / (g - 1.0)) * th * Tr / 3.0
    p = m["rho"] * m["theta"] / 3.0
    return np.sqrt(np.mean((p - pa) ** 2)) / np.sqrt(np.mean((pa - th / 3.0) ** 2))


def test_supersonic_vortex_converges_at_second_order():
    """Sec. 4.2 at Ma = 1.2, beta = 0.2: after one pass through the periodic
    box the pressure error against the translated initial vortex falls by
    about 4x when the grid and radius are doubled."""
    e1 = _vortex_error(64, 4.0)
    e2 = _vortex_error(128, 8.0)
    assert e2 < 0.12
    assert e1 / e2 > 3.0


def couette_analytic(case):
    """Steady temperature between plates at the same temperature T_w (Sec. 4.4,
    eq. couette analy): (T - T_w)/T_w = (y/H) Pr Ma^2 (gamma - 1)/2 (1 - y/H);
    the velocity is linear, u = U y / H.  Cell j lies at y = j + y0: y0 = 1/2
    between wall sides, 1 between Dirichlet sides (their ghost-row centres
    are the plates)."""
    H, U, th = case.meta["H"], case.meta["U"], case.meta["theta_w"]
    y = np.arange(case.ny) + case.meta["y0"]
    T = th * (1.0 + (y / H) * case.Pr * case.meta["Ma"] ** 2 * (case.gamma - 1.0) / 2.0 * (1.0 - y / H))
    return T, U * y / H


def couette_errors(case, m):
    """Profile errors: temperature over the analytic peak rise, velocity over U."""
    T_an, u_an = couette_analytic(case)
    rise = (T_an - case.meta["theta_w"]).max()
    return (float(np.abs(m["theta"][:, 0] - T_an).max() / rise),
            float(np.abs(m["ux"][:, 0] - u_an).max() / case.meta["U"]))


@pytest.mark.slow
def test_thermal_couette_profile():
    """Viscous heating balanced by conduction (Sec. 4.4, Ma 0.8, Pr 0.71,
    gamma 1.4, sigma 0.9) between wall sides: after 100,000 steps the
    temperature rise matches the analytic parabola within 1e-3 of its peak
    and the velocity is linear within 1e-3 of U (measured: 1.4e-4 and
    3.4e-5); the mass drifts by less than 1e-3.  A dropped viscous-heating
    term (no rise), a wrong conductivity (rise off by its ratio), a wall at
    the wrong place (profile shifted by half a cell) or a wrong wall velocity
    fails it."""
    case = inputs.couette()
    o = Oracle(case.nx, case.ny, **case.params())
    o.init(*case.fields())
    o.step(100000)
    m = o.macros()
    eT, eu = couette_errors(case, m)
    assert eT < 1e-3, eT
    assert eu < 1e-3, eu
    assert abs(m["rho"].mean() - 1.0) < 1e-3


@pytest.mark.slow
def test_thermal_couette_dirichlet_sides():
    """The same flow between Dirichlet sides (equilibrium ghost rows whose
    centres are the plates): within 5 % of the peak rise and 2 % of U.  These
    walls leave a 3.6 % shortfall of the rise and a 0.9 % slip."""
    case = inputs.couette(walls="dirichlet")
    o = Oracle(case.nx, case.ny, **case.params())
    o.init(*case.fields())
    o.step(case.steps)
    eT, eu = couette_errors(case, o.macros())
    assert eT < 0.05, eT
    assert eu < 0.02, eu
