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


def test_two_call_chain_rule_matches_finite_differences():
    """Two calls chained, y1 = f(x), y2 = f(y1), with the loss of both:
    L = loss(y2, t2) + loss(y1, t1).  The gradient by backward_dy (the second
    call's dL/dy1 added to the first call's own dL/dy1) against central
    differences of L, for weights, biases and the input."""
    widths = (3, 4, 3)
    params = _net(widths, seed=7)
    x = RNG.normal(size=(2, widths[0], 5, 6))
    t1, t2 = RNG.normal(size=x.shape), RNG.normal(size=x.shape)

    def L(ps, xx):
        y1 = S.forward(ps, xx)[0]
        return S.loss(S.forward(ps, y1)[0], t2) + S.loss(y1, t1)

    y1, c1 = S.forward(params, x)
    y2, c2 = S.forward(params, y1)
    g2, dy1 = S.backward(params, c2, y2, t2)
    g1, dx = S.backward_dy(params, c1, dy1 + 2.0 * (y1 - t1) / y1.size)
    grads = [(a[0] + b[0], a[1] + b[1]) for a, b in zip(g1, g2)]
    h = 1e-6
    for l, (W, b) in enumerate(params):
        for idx in [(0, 0, 0, 0), (widths[l + 1] - 1, widths[l] - 1, 2, 1)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h; Wm[idx] -= h
            pp = list(params); pp[l] = (Wp, b)
            pm = list(params); pm[l] = (Wm, b)
            fd = (L(pp, x) - L(pm, x)) / (2 * h)
            assert abs(grads[l][0][idx] - fd) < 1e-7 * max(1.0, abs(fd)), (l, idx)
        bp, bm = b.copy(), b.copy()
        bp[-1] += h; bm[-1] -= h
        pp = list(params); pp[l] = (W, bp)
        pm = list(params); pm[l] = (W, bm)
        fd = (L(pp, x) - L(pm, x)) / (2 * h)
        assert abs(grads[l][1][-1] - fd) < 1e-7 * max(1.0, abs(fd))
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


# ---- the BF16-storage form ------------------------------------------------

def _bf16_bits(x32):
    """Float32 -> nearest BF16 (ties to even) by the usual bit-level route:
    add 0x7FFF plus the lowest kept bit, then clear the low 16 bits."""
    u = np.asarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_round_matches_bit_level_float32_rounding():
    r = np.random.default_rng(21)
    x = (r.normal(size=20000) * 10.0 ** r.uniform(-6, 6, size=20000)).astype(np.float32)
    assert np.array_equal(S.bf16_round(x.astype(np.float64)), _bf16_bits(x))


def test_bf16_round_keeps_bf16_values_and_ties_to_even():
    k = np.arange(128, 256)
    exact = np.concatenate([k * 2.0 ** -7, -k * 2.0 ** 3])
    assert np.array_equal(S.bf16_round(exact), exact)
    # midpoints between neighbours 1 + j 2^-7 and 1 + (j + 1) 2^-7 go to even j
    assert S.bf16_round(1.0 + 2.0 ** -8) == 1.0
    assert S.bf16_round(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    x = np.random.default_rng(2).normal(size=1000)
    # unit roundoff of 8 significant bits: 2^-8
    assert np.max(np.abs(S.bf16_round(x) - x) / np.abs(x)) <= 2.0 ** -8


def test_bf16_network_without_rounding_to_do_is_the_exact_network():
    """With one layer (no hidden activation to round), BF16 inputs and BF16
    weights the BF16 form is the exact network bitwise; with hidden layers it
    stays within BF16 rounding of it."""
    r = np.random.default_rng(8)
    W = S.bf16_round(r.normal(size=(3, 3, 3, 3)) * 0.3)
    b = r.normal(size=3)
    x = S.bf16_round(r.normal(size=(2, 3, 5, 7)))
    y, _ = S.forward([(W, b)], x)
    yb, _ = S.forward_bf16([(W, b)], x)
    assert np.array_equal(y, yb)
    params = _net((4, 8, 8, 4), seed=3)
    x = r.normal(size=(2, 4, 6, 8))
    t = r.normal(size=x.shape)
    y, cache = S.forward(params, x)
    yb, cb = S.forward_bf16(params, x)
    assert np.linalg.norm(yb - y) <= 2.0 ** -6 * np.linalg.norm(y - x)
    g, _ = S.backward(params, cache, y, t)
    gb = S.backward_bf16(cb, yb, t)
    for (dw, db), (dwb, dbb) in zip(g, gb):
        assert np.linalg.norm(dwb - dw) <= 2.0 ** -5 * np.linalg.norm(dw)
        assert np.linalg.norm(dbb - db) <= 2.0 ** -5 * np.linalg.norm(db)
