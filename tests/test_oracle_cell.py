"""Pins of the oracle's per-cell building blocks against mathematics the paper
fixes: lattice isotropy, Hermite polynomials and their D2Q9 orthogonality,
the equilibrium (against the Maxwellian's moments and a product closed form),
the off-equilibrium reconstruction and its recurrence (against an
anisotropic Gaussian), the correction force and the closure defect.

Independent references are built here from numpy's probabilists' Hermite
polynomials and Gauss-Hermite quadrature of continuous Gaussians."""
import itertools
import math

import numpy as np
import pytest
from numpy.polynomial import hermite_e as He

from oracle import oracle as O

CS2 = 1.0 / 3.0
CS = math.sqrt(CS2)


def he(n, z):
    c = np.zeros(n + 1)
    c[n] = 1.0
    return He.hermeval(z, c)


def tensor_hermite(cx, cy, nxn, nyn):
    """Component of the order-(nxn+nyn) Hermite tensor with nxn x-indices and
    nyn y-indices: c_s^n He_nx(c_x / c_s) He_ny(c_y / c_s)."""
    return CS ** (nxn + nyn) * he(nxn, cx / CS) * he(nyn, cy / CS)


def gauss2d(mean, cov, npts=12):
    """Nodes and weights of a 2-D Gaussian N(mean, cov) by tensor Gauss-Hermite."""
    z, w = He.hermegauss(npts)
    w = w / math.sqrt(2.0 * math.pi)
    L = np.linalg.cholesky(np.asarray(cov, dtype=np.float64))
    Z1, Z2 = np.meshgrid(z, z, indexing="ij")
    W2 = np.outer(w, w)
    pts = np.stack([Z1.ravel(), Z2.ravel()])
    xs = (L @ pts) + np.asarray(mean).reshape(2, 1)
    return xs[0], xs[1], W2.ravel()


SUPPORTED = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2), (2, 1), (1, 2), (2, 2)]


@pytest.fixture(scope="module")
def lat():
    return O.lattice()


def test_lattice_isotropy(lat):
    cx, cy, w = lat
    assert np.isclose(w.sum(), 1.0, atol=1e-15)
    for a in range(1, 6):
        for b in range(0, 6 - a + 1):
            m = np.sum(w * cx ** a * cy ** b)
            # Gaussian moments of N(0, c_s^2 I) up to order 5 per direction
            ex = (0 if a % 2 else CS2 ** (a // 2) * math.prod(range(a - 1, 0, -2)))
            ey = (0 if b % 2 else CS2 ** (b // 2) * math.prod(range(b - 1, 0, -2)))
            if a <= 4 and b <= 4 and a + b <= 5:
                assert np.isclose(m, ex * ey, atol=1e-15), (a, b, m, ex * ey)
    # closure relation of the standard lattice: c^3 = c (Sec. 2.3)
    assert np.allclose(cx ** 3, cx) and np.allclose(cy ** 3, cy)


def test_hermite_polynomials_match_tensor_hermite(lat):
    cx, cy, _ = lat
    for order in range(5):
        for idx in itertools.product((0, 1), repeat=order):
            nxn = idx.count(0)
            nyn = order - nxn
            args = list(idx) + [0] * (4 - order)
            for i in range(9):
                got = O.hermite(i, order, *args)
                ref = tensor_hermite(cx[i], cy[i], nxn, nyn)
                assert abs(got - ref) < 1e-14, (order, idx, i, got, ref)


def test_supported_basis_orthogonal_on_d2q9(lat):
    cx, cy, w = lat
    H = np.array([[tensor_hermite(cx[i], cy[i], a, b) for i in range(9)] for a, b in SUPPORTED])
    gram = (H * w) @ H.T
    norms = np.array([CS2 ** (a + b) * math.factorial(a) * math.factorial(b) for a, b in SUPPORTED])
    assert np.allclose(gram, np.diag(norms), atol=1e-15)


RNG = np.random.default_rng(2002)
STATES = [(1.0, 0.0, 0.0, 1.0)] + [
    (RNG.uniform(0.3, 2.0), RNG.uniform(-0.5, 0.5), RNG.uniform(-0.5, 0.5), RNG.uniform(0.1, 1.2))
    for _ in range(12)
]


@pytest.mark.parametrize("state", STATES)
def test_equilibrium_matches_maxwellian_moments(state, lat):
    cx, cy, w = lat
    rho, ux, uy, th = state
    f = O.feq_cell(rho, ux, uy, th)
    X, Y, Wq = gauss2d((ux, uy), np.eye(2) * th * CS2)
    for a in range(3):
        for b in range(3):
            disc = np.sum(f * cx ** a * cy ** b)
            cont = rho * np.sum(Wq * X ** a * Y ** b)
            assert abs(disc - cont) < 1e-13 * max(1.0, abs(cont)), (a, b, disc, cont)
    if state == (1.0, 0.0, 0.0, 1.0):
        assert np.allclose(f, w, atol=1e-16)


@pytest.mark.parametrize("state", STATES)
def test_equilibrium_product_form(state, lat):
    cx, cy, _ = lat
    rho, ux, uy, th = state

    def g(c, u):  # D1Q3 factor with moments 1, u, u^2 + theta/3
        return 1.0 - u * u - th / 3.0 if c == 0 else 0.5 * (u * u + c * u + th / 3.0)

    ref = np.array([rho * g(cx[i], ux) * g(cy[i], uy) for i in range(9)])
    assert np.allclose(O.feq_cell(rho, ux, uy, th), ref, atol=1e-15, rtol=1e-14)


@pytest.mark.parametrize("state", STATES[1:6])
def test_offequilibrium_reconstruction_recovers_moments(state, lat):
    cx, cy, _ = lat
    _, ux, uy, th = state
    axx, axy, ayy = RNG.normal(size=3) * 1e-2
    f1 = O.f1_cell(axx, axy, ayy, ux, uy, th)
    hi = O.a1_high(axx, axy, ayy, ux, uy, th)
    want = {(0, 0): 0.0, (1, 0): 0.0, (0, 1): 0.0, (2, 0): axx, (1, 1): axy, (0, 2): ayy,
            (2, 1): hi[0], (1, 2): hi[1], (2, 2): hi[2]}
    for (a, b), v in want.items():
        proj = np.sum(f1 * np.array([tensor_hermite(cx[i], cy[i], a, b) for i in range(9)]))
        assert abs(proj - v) < 1e-15, ((a, b), proj, v)


def _gauss_hermite_coeff(rho, u, cov, a, b):
    X, Y, Wq = gauss2d(u, cov, npts=14)
    return rho * np.sum(Wq * tensor_hermite(X, Y, a, b))


@pytest.mark.parametrize("state", STATES[1:7])
def test_recurrence_exact_for_anisotropic_gaussian(state):
    """The recurrence for a1_xxy, a1_yyx, a1_xxyy (Sec. 3.3) reproduces the
    first-order change of the Hermite coefficients of a Gaussian whose
    covariance is perturbed away from theta c_s^2 I at fixed rho and u."""
    rho, ux, uy, th = state
    D = RNG.normal(size=(2, 2)) * 0.3
    D = 0.5 * (D + D.T)
    eps = 1e-4
    base = np.eye(2) * th * CS2

    def coeffs(e):
        cov = base + e * CS2 * D
        return {k: _gauss_hermite_coeff(rho, (ux, uy), cov, *k) for k in [(2, 0), (1, 1), (0, 2), (2, 1), (1, 2), (2, 2)]}

    cp, cm = coeffs(eps), coeffs(-eps)
    d = {k: (cp[k] - cm[k]) / (2 * eps) for k in cp}
    hi = O.a1_high(d[(2, 0)], d[(1, 1)], d[(0, 2)], ux, uy, th)
    scale = max(abs(v) for v in d.values())
    assert abs(hi[0] - d[(2, 1)]) < 1e-7 * scale
    assert abs(hi[1] - d[(1, 2)]) < 1e-7 * scale
    assert abs(hi[2] - d[(2, 2)]) < 1e-7 * scale


def test_correction_force_moments(lat):
    cx, cy, _ = lat
    for _ in range(10):
        exx, exy, eyy = RNG.normal(size=3)
        psi = O.psi_cell(exx, exy, eyy)
        assert abs(psi.sum()) < 1e-15
        assert abs(np.sum(cx * psi)) < 1e-15 and abs(np.sum(cy * psi)) < 1e-15
        for (a, b), v in {(2, 0): exx, (1, 1): exy, (0, 2): eyy}.items():
            h = np.array([tensor_hermite(cx[i], cy[i], a, b) for i in range(9)])
            assert abs(np.sum(h * psi) - v) < 1e-14


@pytest.mark.parametrize("state", STATES[1:8])
def test_closure_defect_is_minus_third_order_maxwellian_moment(state):
    rho, ux, uy, th = state
    a_xxx = _gauss_hermite_coeff(rho, (ux, uy), np.eye(2) * th * CS2, 3, 0)
    a_yyy = _gauss_hermite_coeff(rho, (ux, uy), np.eye(2) * th * CS2, 0, 3)
    assert abs(O.gamma_closure(rho, ux, th) + a_xxx) < 1e-13
    assert abs(O.gamma_closure(rho, uy, th) + a_yyy) < 1e-13


def test_muscl_linear_data_is_exact():
    for u in (0.7, 0.3, -0.2, -0.9):
        for k in (0.5, -1.3, 2e-3):
            s = 3.0 + k * np.arange(-2, 3)
            assert abs(O.muscl_term(u, *s) - u * k) < 1e-14 * max(1, abs(u * k)) * 10
    assert O.muscl_term(0.0, 0, 1, 5, 2, 7) == 0.0


def test_muscl_update_is_monotone():
    """s_i - nu (...) stays within the range of s_{i-1}, s_i, s_{i+1} for a
    Courant number |u| <= 1/2 (TVD bound of a limited MUSCL update)."""
    rng = np.random.default_rng(5)
    for _ in range(4000):
        s = rng.normal(size=5) * rng.choice([1e-3, 1.0, 10.0])
        if rng.random() < 0.3:
            s = np.cumsum(np.abs(s))  # monotone data
        u = rng.uniform(-0.5, 0.5)
        new = s[2] - O.muscl_term(u, *s)
        lo, hi = min(s[1:4]), max(s[1:4])
        tol = 1e-12 * max(1.0, np.abs(s).max())
        assert lo - tol <= new <= hi + tol, (u, s, new)
