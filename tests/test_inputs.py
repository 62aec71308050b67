"""The seeded input recipes against what they state (CPU).  The vortex is a
steady solution of the Euler equations in its own frame, which pins the
reading of its printed profile independently of the formula.  Its far
field has the stated sound speed and Mach number, and its density noise
keeps the pressure.  The four-quadrant states and the batched sweep's
draws are checked as stated."""
import numpy as np
import pytest

from paper_2002_03644_gb300 import inputs

CS2 = 1.0 / 3.0


def test_vortex_far_field():
    """theta_inf = 300 / 1478.75 at gamma = 1.4 gives c_inf = sqrt(gamma
    c_s^2 theta_inf) = 4/13 exactly, so the far field moves at 1.2 x 4/13
    along x with rho = 1 (Sec. 4.2)."""
    c = inputs.vortex(n=1024, noise=0.0)
    assert c.meta["c_inf"] == pytest.approx(4.0 / 13.0, rel=1e-14)
    assert c.ux[0, 0] == pytest.approx(1.2 * 4.0 / 13.0, rel=1e-14)
    assert abs(c.uy[0, 0]) < 1e-15
    assert c.rho[0, 0] == pytest.approx(1.0, rel=1e-14)
    assert c.theta[0, 0] == pytest.approx(300.0 / 1478.75, rel=1e-14)


def test_vortex_is_a_steady_euler_solution_in_its_frame():
    """With v = u - (U_inf, 0), the steady momentum balance
    rho (v . grad) v + grad p = 0, where p = rho c_s^2 theta, holds to the
    accuracy of centred differences over the vortex.  This holds only for
    the profile that satisfies radial equilibrium.  The printed density
    formula, with its extra factor r, fails it."""
    n, R = 384, 40.0
    c = inputs.vortex(n=n, R=R, noise=0.0)
    U = 1.2 * c.meta["c_inf"]
    vx, vy = c.ux - U, c.uy
    p = c.rho * CS2 * c.theta

    def ddx(a):
        return 0.5 * (np.roll(a, -1, axis=1) - np.roll(a, 1, axis=1))

    def ddy(a):
        return 0.5 * (np.roll(a, -1, axis=0) - np.roll(a, 1, axis=0))

    rx = c.rho * (vx * ddx(vx) + vy * ddy(vx)) + ddx(p)
    ry = c.rho * (vx * ddx(vy) + vy * ddy(vy)) + ddy(p)
    scale = max(np.abs(ddx(p)).max(), np.abs(ddy(p)).max())
    assert max(np.abs(rx).max(), np.abs(ry).max()) < 2e-3 * scale
    # the printed density (an extra factor r in the exponent's prefactor)
    # leaves a residual of the size of the gradient itself
    X, Y = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
    r2 = ((X - 0.5 * n) ** 2 + (Y - 0.5 * n) ** 2) / R ** 2
    g = 1.4
    mav = 0.2 * 1.2
    t_wrong = 1.0 - 0.5 * (g - 1.0) * mav ** 2 * np.sqrt(r2) * np.exp(1.0 - r2)
    p_wrong = t_wrong ** (g / (g - 1.0)) * CS2 * c.meta["theta_inf"]
    rx_wrong = c.rho * (vx * ddx(vx) + vy * ddy(vx)) + ddx(p_wrong)
    assert np.abs(rx_wrong).max() > 0.1 * scale


def test_vortex_noise_keeps_the_pressure():
    """The seeded +-1e-6 density noise (O-19) holds p = rho theta fixed, is
    bounded, takes both signs and repeats with the seed."""
    a = inputs.vortex(n=128, R=4.0, noise=0.0)
    b = inputs.vortex(n=128, R=4.0)
    b2 = inputs.vortex(n=128, R=4.0)
    d = b.rho - a.rho
    assert np.abs(d).max() <= 1e-6 * (1.0 + 1e-12)
    assert (d > 0).any() and (d < 0).any()
    assert np.allclose(b.rho * b.theta, a.rho * a.theta, rtol=1e-14, atol=0.0)
    assert np.array_equal(b.rho, b2.rho)


def test_four_quadrant_states():
    """The four quadrant states (rho, u, v, p), counter-clockwise from the
    upper right, in lattice units: u / C_0 and theta = (p / rho) / T_r
    with T_r = C_0^2 c_s^2."""
    n = 64
    c = inputs.four_quadrant(n=n)
    C0 = c.meta["C0"]
    Tr = C0 * C0 * CS2
    want = {(48, 48): (1.5, 0.0, 0.0, 1.5), (48, 16): (0.532, 1.206, 0.0, 0.3),
            (16, 16): (0.138, 1.206, 1.206, 0.029), (16, 48): (0.532, 0.0, 1.206, 0.3)}
    for (j, i), (r, u, v, p) in want.items():
        assert c.rho[j, i] == pytest.approx(r)
        assert c.ux[j, i] * C0 == pytest.approx(u)
        assert c.uy[j, i] * C0 == pytest.approx(v)
        assert c.rho[j, i] * c.theta[j, i] * Tr == pytest.approx(p)
    assert c.bc == (inputs.BC_ZEROGRAD,) * 4


def test_batch_sweep_draws():
    """64 cases from seed 2002: sizes from {128, 256, 512, 1024}^2, Ma in
    [0.1, 1.5], gamma from {1.4, 1.3, 1.67}, each far field at CFL
    (Ma + 1) sqrt(gamma theta / 3) = 0.7; 29 900 800 cells in all."""
    cases = inputs.batch_sweep()
    assert len(cases) == 64
    assert sum(c.nx * c.ny for c in cases) == 29_900_800
    for c in cases:
        assert c.nx == c.ny and c.nx in (128, 256, 512, 1024)
        assert 0.1 <= c.meta["Ma"] <= 1.5
        assert c.gamma in (1.4, 1.3, 1.67)
        cfl = (c.meta["Ma"] + 1.0) * np.sqrt(c.gamma * c.meta["theta_inf"] * CS2)
        assert cfl == pytest.approx(0.7, rel=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_surrogate_fields_hold_the_lowest_modes_around_a_mean_flow(seed):
    """Surrogate training fields: only the 8 lowest Fourier modes per axis
    on rho, u and theta, around a mean flow whose Mach number is drawn in
    [0.3, 1.2]."""
    n = 64
    c = inputs.random_fourier(n=n, seed=seed)
    theta0 = 300.0 / 1478.75
    c0 = np.sqrt(1.4 * theta0 * CS2)
    mx, my = c.ux.mean(), c.uy.mean()
    ma = np.hypot(mx, my) / c0
    assert 0.3 <= ma <= 1.2 and ma == pytest.approx(c.meta["Ma"], rel=1e-12)
    k = np.fft.fftfreq(n) * n
    KY, KX = np.meshgrid(k, k, indexing="ij")
    outside = (np.abs(KX) >= 8) | (np.abs(KY) >= 8)
    for f in (c.rho - 1.0, c.ux - mx, c.uy - my, c.theta / theta0 - 1.0):
        F = np.abs(np.fft.fft2(f))
        assert F.max() > 0.0
        assert F[outside].max() < 1e-10 * F.max()
        assert F[0, 0] < 1e-10 * F.max()  # no mean in the perturbation
