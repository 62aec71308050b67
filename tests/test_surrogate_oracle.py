"""Pins of the surrogate reference (oracle/surrogate_oracle.py) against
independent routes: circular convolution by FFT, finite differences of its
own forward pass, and the standard normal CDF for GELU."""
import math

import numpy as np
import pytest

from oracle import surrogate_oracle as S

RNG = np.random.default_rng(11)


def test_periodic_conv_matches_fft_circular_correlation():
    x = RNG.normal(size=(2, 3, 7, 9))
    W = RNG.normal(size=(4, 3, 3, 3))
    b = RNG.normal(size=4)
    got = S.conv3x3_periodic(x, W, b)
    H, Wd = 7, 9
    ref = np.zeros((2, 4, H, Wd))
    Fx = np.fft.fft2(x)
    for o in range(4):
        for c in range(3):
            k = np.zeros((H, Wd))
            for p in (-1, 0, 1):
                for q in (-1, 0, 1):
                    # correlation: out(i) = sum_p w(p) x(i + p) -> kernel at -p
                    k[(-p) % H, (-q) % Wd] += W[o, c, p + 1, q + 1]
            ref[:, o] += np.real(np.fft.ifft2(Fx[:, c] * np.fft.fft2(k)))
        ref[:, o] += b[o]
    assert np.allclose(got, ref, atol=1e-12)


def test_gelu_is_x_times_normal_cdf():
    xs = np.linspace(-6, 6, 101)
    cdf = np.array([0.5 * math.erfc(-v / math.sqrt(2.0)) for v in xs])
    assert np.allclose(S.gelu(xs), xs * cdf, atol=1e-15)
    h = 1e-6
    fd = (S.gelu(xs + h) - S.gelu(xs - h)) / (2 * h)
    assert np.allclose(S.gelu_grad(xs), fd, atol=1e-8)


def _net(widths, seed=0):
    r = np.random.default_rng(seed)
    return [(r.normal(size=(o, c, 3, 3)) * (1.0 / math.sqrt(9 * c)), r.normal(size=o) * 0.1)
            for c, o in zip(widths[:-1], widths[1:])]


@pytest.mark.parametrize("widths", [(2, 3, 2), (4, 5, 5, 4)])
def test_backward_matches_finite_differences(widths):
    params = _net(widths)
    x = RNG.normal(size=(2, widths[0], 5, 6))
    t = RNG.normal(size=x.shape)
    y, cache = S.forward(params, x)
    grads, dx = S.backward(params, cache, y, t)

    def L(ps, xx):
        return S.loss(S.forward(ps, xx)[0], t)

    h = 1e-6
    for l, (W, b) in enumerate(params):
        for idx in [(0, 0, 0, 0), (widths[l + 1] - 1, widths[l] - 1, 2, 1), (0, widths[l] - 1, 1, 2)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h; Wm[idx] -= h
            pp = list(params); pp[l] = (Wp, b)
            pm = list(params); pm[l] = (Wm, b)
            fd = (L(pp, x) - L(pm, x)) / (2 * h)
            assert abs(grads[l][0][idx] - fd) < 1e-7 * max(1.0, abs(fd)), (l, idx)
        bp, bm = b.copy(), b.copy()
        bp[0] += h; bm[0] -= h
        pp = list(params); pp[l] = (W, bp)
        pm = list(params); pm[l] = (W, bm)
        fd = (L(pp, x) - L(pm, x)) / (2 * h)
        assert abs(grads[l][1][0] - fd) < 1e-7 * max(1.0, abs(fd))
    for idx in [(0, 0, 0, 0), (1, widths[0] - 1, 4, 5)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h; xm[idx] -= h
        fd = (L(params, xp) - L(params, xm)) / (2 * h)
        assert abs(dx[idx] - fd) < 1e-7 * max(1.0, abs(fd))


def test_adam_first_step_moves_by_lr_times_sign():
    p = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    p1, m, v = S.adam_update(p, g, np.zeros(3), np.zeros(3), 1, lr=1e-2)
    # bias-corrected first step: m_hat / sqrt(v_hat) = sign(g) (eps aside)
    assert np.allclose(p1, p - 1e-2 * np.sign(g), atol=1e-7)
