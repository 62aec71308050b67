"""Seeded synthetic inputs for the hybrid LBM step.

This module is shared by the tests, the oracle runs and the benchmark.  It
holds only input recipes -- initial fields (rho, u_x, u_y, theta) in lattice
units and the case parameters -- and a counter-based random generator.  It
contains none of the method's arithmetic.

Lattice units follow Sec. 2.1 of Renard et al. (arXiv 2002.03644): dx = dt = 1,
c_s^2 = 1/3, theta = T / T_r, and the lattice speed C_0 = sqrt(r T_r) / c_s
maps physical velocities to lattice ones (u_lat = u / C_0).  With the gas
constant r = 1 and a reference density of 1, a physical state (rho, u, p)
becomes rho_lat = rho, u_lat = u / C_0, theta = (p / rho) / T_r with
T_r = C_0^2 c_s^2.

Arrays are float64 numpy arrays of shape [ny, nx] (row-major, x fastest).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

BC_PERIODIC, BC_ZEROGRAD, BC_DIRICHLET, BC_WALL = 0, 1, 2, 3
CS2 = 1.0 / 3.0

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Counter-based SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): the i-th
    output is the finaliser applied to seed + (i + 1) * golden gamma."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (counters.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of SplitMix64(seed, offset + i)."""
    z = splitmix64(seed, np.arange(offset, offset + n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclasses.dataclass
class Case:
    """One initial-value problem in lattice units."""
    name: str
    nx: int
    ny: int
    rho: np.ndarray
    ux: np.ndarray
    uy: np.ndarray
    theta: np.ndarray
    gamma: float = 1.4
    Pr: float = 0.71
    mu: float = 1e-4
    sigma: float = 0.0
    bc: tuple = (BC_PERIODIC,) * 4
    bc_state: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((4, 4)))
    phi_mode: int = 0
    ablation: int = 0  # bit 1: centred E1, bit 2: no E2 (original-model parts)
    steps: int = 100
    meta: dict = dataclasses.field(default_factory=dict)

    def params(self) -> dict:
        return dict(gamma=self.gamma, Pr=self.Pr, mu=self.mu, sigma=self.sigma,
                    bc=tuple(self.bc), bc_state=np.asarray(self.bc_state, dtype=np.float64).reshape(16),
                    phi_mode=self.phi_mode, ablation=self.ablation)

    def fields(self):
        return self.rho, self.ux, self.uy, self.theta


def _grid(nx, ny):
    """Cell centres x_i = i + 1/2, y_j = j + 1/2 (cell units)."""
    x = np.arange(nx, dtype=np.float64) + 0.5
    y = np.arange(ny, dtype=np.float64) + 0.5
    return np.meshgrid(x, y)  # X[j, i], Y[j, i]


def sod(nx=400, ny=4, C0=12.5, mu=3.0e-6, sigma=0.4, gamma=1.4, Pr=0.71, t_end=0.2):
    """Sod shock tube on a unit-length tube: left (rho, u, p) = (1, 0, 1),
    right (0.125, 0, 0.1), interface at x = 0.5; zero-gradient ends in x,
    periodic in y.  With dx = 1/nx and dt = dx / C0, t_end takes
    t_end * C0 * nx steps (1000 for the defaults)."""
    X, _ = _grid(nx, ny)
    T_r = C0 * C0 * CS2
    left = X < 0.5 * nx
    rho = np.where(left, 1.0, 0.125)
    p = np.where(left, 1.0, 0.1)
    theta = (p / rho) / T_r
    z = np.zeros_like(rho)
    steps = int(round(t_end * C0 * nx))
    return Case("sod", nx, ny, rho, z.copy(), z.copy(), theta, gamma=gamma, Pr=Pr, mu=mu,
                sigma=sigma, bc=(BC_ZEROGRAD, BC_ZEROGRAD, BC_PERIODIC, BC_PERIODIC), steps=steps,
                meta=dict(C0=C0, T_r=T_r, t_end=t_end, dx=1.0 / nx))


def vortex(n=1024, Ma=1.2, beta=0.2, R=32.0, gamma=1.4, Pr=0.71, mu=1.5e-6, sigma=0.0,
           theta_inf=300.0 / 1478.75, noise=1e-6, seed=2002, steps=10000, ny=None):
    """Isentropic vortex convected along x in a periodic box (Sec. 4.2).

    u_theta = c_inf Ma_v r exp((1 - r^2) / 2) with r = |x - x_c| / R and
    Ma_v = beta * Ma; the isentropic temperature from radial equilibrium is
    T / T_inf = 1 - (gamma - 1) / 2 Ma_v^2 exp(1 - r^2) (the printed density
    formula carries a stray factor r; this is the profile that satisfies
    dp/dr = rho u_theta^2 / r), rho = rho_inf (T / T_inf)^(1 / (gamma - 1)).
    theta_inf = 300 / 1478.75 gives c_inf = sqrt(gamma theta / 3) = 4/13 at
    gamma = 1.4.  A seeded uniform perturbation of +-noise is added to rho
    with the pressure held fixed."""
    nx = int(n)
    ny = nx if ny is None else int(ny)
    X, Y = _grid(nx, ny)
    xc, yc = 0.5 * nx, 0.5 * ny
    c_inf = math.sqrt(gamma * theta_inf * CS2)
    Ma_v = beta * Ma
    dx, dy = (X - xc) / R, (Y - yc) / R
    r2 = dx * dx + dy * dy
    amp = c_inf * Ma_v * np.exp(0.5 * (1.0 - r2))
    ux = Ma * c_inf - amp * dy
    uy = amp * dx
    Tr = 1.0 - 0.5 * (gamma - 1.0) * Ma_v * Ma_v * np.exp(1.0 - r2)
    rho = Tr ** (1.0 / (gamma - 1.0))
    theta = theta_inf * Tr
    if noise:
        p = rho * theta  # held fixed (times c_s^2)
        rho = rho + noise * (2.0 * uniform01(seed, nx * ny).reshape(ny, nx) - 1.0)
        theta = p / rho
    return Case("vortex", nx, ny, rho, ux, uy, theta, gamma=gamma, Pr=Pr, mu=mu, sigma=sigma,
                bc=(BC_PERIODIC,) * 4, steps=steps,
                meta=dict(Ma=Ma, beta=beta, R=R, theta_inf=theta_inf, c_inf=c_inf, noise=noise,
                          seed=seed))


def four_quadrant(n=4096, C0=4.5, mu=1e-4, sigma=0.0, gamma=1.4, Pr=0.71, t_end=0.3):
    """Two-dimensional four-quadrant Riemann problem on a unit square with
    zero-gradient sides.  States (rho, u, v, p), counter-clockwise from the
    upper-right quadrant: (1.5, 0, 0, 1.5), (0.532, 1.206, 0, 0.3),
    (0.138, 1.206, 1.206, 0.029), (0.532, 0, 1.206, 0.3)."""
    X, Y = _grid(n, n)
    T_r = C0 * C0 * CS2
    right, top = X >= 0.5 * n, Y >= 0.5 * n
    states = {
        (True, True): (1.5, 0.0, 0.0, 1.5),
        (False, True): (0.532, 1.206, 0.0, 0.3),
        (False, False): (0.138, 1.206, 1.206, 0.029),
        (True, False): (0.532, 0.0, 1.206, 0.3),
    }
    rho = np.zeros((n, n)); u = np.zeros((n, n)); v = np.zeros((n, n)); p = np.zeros((n, n))
    for (r, t), (rr, uu, vv, pp) in states.items():
        m = (right == r) & (top == t)
        rho[m], u[m], v[m], p[m] = rr, uu, vv, pp
    theta = (p / rho) / T_r
    steps = int(round(t_end * C0 * n))
    return Case("four_quadrant", n, n, rho, u / C0, v / C0, theta, gamma=gamma, Pr=Pr, mu=mu,
                sigma=sigma, bc=(BC_ZEROGRAD,) * 4, steps=steps, meta=dict(C0=C0, T_r=T_r))


def shear_wave(ny=200, nx=2, Ma=0.5, a0_over_c=0.05, theta0=300.0 / 800.0, gamma=1.4, Pr=0.71,
               mu=1e-3, sigma=0.0, steps=2000):
    """Quasi-1D shear wave (Sec. 4.1): p, T uniform, u_x = a0 sin(2 pi y / L_y),
    u_y = Ma c; the amplitude of u_x decays as exp(-nu k^2 t) with
    nu = mu / rho.  Periodic box nx x ny with one wavelength along y."""
    X, Y = _grid(nx, ny)
    c = math.sqrt(gamma * theta0 * CS2)
    ux = a0_over_c * c * np.sin(2.0 * math.pi * Y / ny)
    uy = np.full_like(ux, Ma * c)
    rho = np.ones_like(ux)
    theta = np.full_like(ux, theta0)
    return Case("shear_wave", nx, ny, rho, ux, uy, theta, gamma=gamma, Pr=Pr, mu=mu, sigma=sigma,
                steps=steps, meta=dict(a0=a0_over_c * c, k=2.0 * math.pi / ny, c=c))


def acoustic_wave(nx=200, ny=2, dp_rel=5.0 / 101325.0, theta0=300.0 / 1478.75, gamma=1.4,
                  Pr=0.71, mu=1e-3, sigma=0.95, steps=2000):
    """Isentropic sinusoidal acoustic wave along x (Sec. 4.3):
    p' = dp sin(2 pi x / L), T / T_inf = (p / p_inf)^((gamma-1)/gamma),
    u_x = p' / (rho c); rho follows from p = rho T."""
    X, Y = _grid(nx, ny)
    p_inf = CS2 * theta0  # rho_inf = 1
    c = math.sqrt(gamma * theta0 * CS2)
    pp = dp_rel * p_inf * np.sin(2.0 * math.pi * X / nx)
    p = p_inf + pp
    theta = theta0 * (p / p_inf) ** ((gamma - 1.0) / gamma)
    rho = p / (CS2 * theta)
    ux = pp / (rho * c)
    uy = np.zeros_like(ux)
    return Case("acoustic_wave", nx, ny, rho, ux, uy, theta, gamma=gamma, Pr=Pr, mu=mu,
                sigma=sigma, steps=steps, meta=dict(k=2.0 * math.pi / nx, c=c, dp=dp_rel * p_inf))


def couette(ny=100, nx=2, Ma=0.8, gamma=1.4, Pr=0.71, mu=0.1, sigma=0.9, theta_w=300.0 / 1500.0, steps=70000,
            walls="wall"):
    """Thermal Couette flow (Sec. 4.4): gas at rest and at the wall
    temperature between a wall at rest (the y- side) and a wall moving along
    x at U = Ma c (the y+ side), both at theta_w; periodic in x.  T_r = 1500 K
    and T_w = 300 K give theta_w = 0.2; sigma = 0.9 as in the paper.

    walls="wall": wall sides, half-way between the ghost and the first
    interior row, so the plates are H = ny apart and cell j lies at
    y = j + 1/2.  walls="dirichlet": Dirichlet sides whose ghost-row centres
    are the plates, H = ny + 1 and cell j at y = j + 1."""
    c = math.sqrt(gamma * theta_w * CS2)
    U = Ma * c
    shape = (ny, nx)
    bc_state = np.array([[1.0, 0.0, 0.0, theta_w], [1.0, 0.0, 0.0, theta_w],
                         [1.0, 0.0, 0.0, theta_w], [1.0, U, 0.0, theta_w]])
    if walls == "wall":
        side, H, y0 = BC_WALL, float(ny), 0.5
    elif walls == "dirichlet":
        side, H, y0 = BC_DIRICHLET, ny + 1.0, 1.0
    else:
        raise ValueError(walls)
    return Case("couette", nx, ny, np.ones(shape), np.zeros(shape), np.zeros(shape), np.full(shape, theta_w),
                gamma=gamma, Pr=Pr, mu=mu, sigma=sigma, bc=(BC_PERIODIC, BC_PERIODIC, side, side),
                bc_state=bc_state, steps=steps, meta=dict(U=U, H=H, y0=y0, Ma=Ma, theta_w=theta_w))


def gaussian_pulse_1d(nx=200, ny=2, width=20.0, dp_rel=1e-4, theta0=300.0 / 1478.75, gamma=1.4,
                      Pr=0.71, mu=1e-4, sigma=0.95, steps=200):
    """Gaussian isentropic pressure pulse at rest in a periodic tube (Sec. 5.1,
    sound-speed measurement): p' = dp exp(-x^2 / (2 R^2)), T by the isentropic
    law, u = 0 (the pulse splits into two waves moving at +-c)."""
    X, _ = _grid(nx, ny)
    p_inf = CS2 * theta0
    xc = 0.5 * nx
    pp = dp_rel * p_inf * np.exp(-((X - xc) ** 2) / (2.0 * width * width))
    p = p_inf + pp
    theta = theta0 * (p / p_inf) ** ((gamma - 1.0) / gamma)
    rho = p / (CS2 * theta)
    z = np.zeros_like(rho)
    return Case("gaussian_pulse", nx, ny, rho, z.copy(), z.copy(), theta, gamma=gamma, Pr=Pr,
                mu=mu, sigma=sigma, steps=steps,
                meta=dict(c=math.sqrt(gamma * theta0 * CS2), xc=xc, width=width))


def random_smooth(nx, ny, seed=7, amp=0.05, modes=4, rho0=1.0, theta0=0.2, u0=(0.1, 0.05),
                  gamma=1.4, Pr=0.71, mu=1e-3, sigma=0.5, bc=(BC_PERIODIC,) * 4, bc_state=None,
                  steps=20):
    """Sum of seeded random Fourier modes (the lowest `modes` wavenumbers per
    axis) on rho, u_x, u_y and theta around a mean state.  Periodic in both
    directions by construction."""
    out = []
    r = uniform01(seed, 4 * modes * modes * 3).reshape(4, modes, modes, 3)
    # sum over (kx, ky) of a cos(2 pi (kx x / nx + ky y / ny) + ph) at the cell
    # centres, evaluated as Re(E_y C E_x) with C[ky, kx] = a exp(i ph)
    k = np.arange(modes)
    ex = np.exp(2j * math.pi * np.outer(k, np.arange(nx) + 0.5) / nx)  # [kx, x]
    ey = np.exp(2j * math.pi * np.outer(np.arange(ny) + 0.5, k) / ny)  # [y, ky]
    KX, KY = np.meshgrid(k, k, indexing="ij")
    for f in range(4):
        a = (2.0 * r[f, :, :, 0] - 1.0) / (1.0 + KX * KX + KY * KY)  # [kx, ky]
        a[0, 0] = 0.0
        c = (a * np.exp(2j * math.pi * r[f, :, :, 1])).T  # [ky, kx]
        out.append(amp * np.real(ey @ c @ ex))
    rho = rho0 * (1.0 + out[0])
    ux = u0[0] + out[1]
    uy = u0[1] + out[2]
    theta = theta0 * (1.0 + out[3])
    bs = np.zeros((4, 4)) if bc_state is None else np.asarray(bc_state, dtype=np.float64)
    return Case("random_smooth", nx, ny, rho, ux, uy, theta, gamma=gamma, Pr=Pr, mu=mu,
                sigma=sigma, bc=tuple(bc), bc_state=bs, steps=steps, meta=dict(seed=seed))


def uniform(nx, ny, rho=1.0, ux=0.1, uy=-0.05, theta=0.25, **kw):
    """A uniform state (a fixed point of the scheme on a periodic grid)."""
    f = lambda v: np.full((ny, nx), float(v))
    return Case("uniform", nx, ny, f(rho), f(ux), f(uy), f(theta), **kw)


def batch_sweep(ncase=64, seed=2002, steps=2000, mu=1.5e-6, beta=0.2, cfl=0.7):
    """Vortex-convection cases of uneven size and physics for the batched
    form: N drawn uniformly from {128, 256, 512, 1024}, Ma uniform in
    [0.1, 1.5], gamma from {1.4, 1.3, 1.67}, all from counter-based draws of
    `seed`; theta_inf of each case sets CFL = (Ma + 1) sqrt(gamma theta / 3)
    to `cfl`; vortex radius N / 32, strength beta."""
    r = uniform01(seed, 3 * ncase).reshape(ncase, 3)
    sizes = (128, 256, 512, 1024)
    gammas = (1.4, 1.3, 1.67)
    out = []
    for k in range(ncase):
        n = sizes[min(3, int(r[k, 0] * 4))]
        ma = 0.1 + 1.4 * r[k, 1]
        gamma = gammas[min(2, int(r[k, 2] * 3))]
        theta_inf = 3.0 * (cfl / (ma + 1.0)) ** 2 / gamma
        c = vortex(n=n, Ma=ma, beta=beta, R=n / 32.0, gamma=gamma, mu=mu, theta_inf=theta_inf, noise=1e-6,
                   seed=seed + k + 1, steps=steps)
        c.name = f"vortex{n}_Ma{ma:.2f}_g{gamma}"
        out.append(c)
    return out


def random_fourier(n=256, seed=0, modes=8, amp=0.05, ma_range=(0.3, 1.2), theta0=300.0 / 1478.75,
                   gamma=1.4, Pr=0.71, mu=1e-4, sigma=0.0):
    """Seeded smooth periodic field for the surrogate's training data: the
    `modes` lowest Fourier modes per axis with random amplitudes (overall
    relative amplitude `amp`) on rho, u_x, u_y and theta, around a mean flow
    of Mach uniform in ma_range in a random direction."""
    r = uniform01(seed, 2)
    ma = ma_range[0] + (ma_range[1] - ma_range[0]) * r[0]
    ang = 2.0 * math.pi * r[1]
    c0 = math.sqrt(gamma * theta0 * CS2)
    u0 = (ma * c0 * math.cos(ang), ma * c0 * math.sin(ang))
    case = random_smooth(n, n, seed=seed + 1, amp=amp, modes=modes, rho0=1.0, theta0=theta0, u0=u0,
                         gamma=gamma, Pr=Pr, mu=mu, sigma=sigma)
    case.name = "random_fourier"
    case.meta.update(Ma=ma, angle=ang)
    return case
