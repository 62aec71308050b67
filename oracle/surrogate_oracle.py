"""FP64 CPU reference of the learned K-step surrogate -- TEST INFRASTRUCTURE.

Only tests/ may import this module.  It states, in plain numpy, the network
the GPU kernels implement, so that their forward outputs and gradients can
be checked element by element.

Network: a stack of 3x3 convolutions with periodic padding on a [B, C, H, W]
field; GELU (the exact form 0.5 x (1 + erf(x / sqrt 2))) after every layer
but the last; the output is added to the input (the network predicts the
change of the normalised state over K time steps).  Loss: mean squared
error over all elements.

Definitions (written out, no library convolution):
  conv(x, W, b)[n, o, i, j] = b[o] + sum_c sum_{p,q in -1..1}
                              W[o, c, p+1, q+1] x[n, c, (i+p) mod H, (j+q) mod W]
The backward pass applies the chain rule to these sums.
"""
from __future__ import annotations

import math

import numpy as np

try:
    from scipy.special import erf as _erf
except Exception:  # pragma: no cover - scipy is present in the test image
    _erf = np.vectorize(math.erf)

SQRT2 = math.sqrt(2.0)
INV_SQRT_2PI = 1.0 / math.sqrt(2.0 * math.pi)


def conv3x3_periodic(x, W, b):
    """x [N, C, H, W], W [O, C, 3, 3], b [O] -> [N, O, H, W]."""
    N, C, H, Wd = x.shape
    O = W.shape[0]
    out = np.zeros((N, O, H, Wd))
    for p in (-1, 0, 1):
        for q in (-1, 0, 1):
            # xs[n, c, i, j] = x[n, c, (i+p) mod H, (j+q) mod W]
            xs = np.roll(x, shift=(-p, -q), axis=(2, 3))
            out += np.einsum("oc,ncij->noij", W[:, :, p + 1, q + 1], xs)
    return out + b[None, :, None, None]


def conv3x3_periodic_backward(x, W, dout):
    """Gradients of sum(dout * conv(x, W, b)) with respect to x, W and b."""
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for p in (-1, 0, 1):
        for q in (-1, 0, 1):
            xs = np.roll(x, shift=(-p, -q), axis=(2, 3))
            dW[:, :, p + 1, q + 1] = np.einsum("noij,ncij->oc", dout, xs)
            # d/dxs = W^T dout, and xs is x shifted by (-p, -q): shift back
            dxs = np.einsum("oc,noij->ncij", W[:, :, p + 1, q + 1], dout)
            dx += np.roll(dxs, shift=(p, q), axis=(2, 3))
    db = dout.sum(axis=(0, 2, 3))
    return dx, dW, db


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / SQRT2))


def gelu_grad(x):
    """d/dx of 0.5 x (1 + erf(x / sqrt 2)) = Phi(x) + x phi(x)."""
    return 0.5 * (1.0 + _erf(x / SQRT2)) + x * INV_SQRT_2PI * np.exp(-0.5 * x * x)


def forward(params, x):
    """params: list of (W, b); returns (y, cache)."""
    acts = [x]
    pre = []
    h = x
    L = len(params)
    for l, (W, b) in enumerate(params):
        z = conv3x3_periodic(h, W, b)
        pre.append(z)
        h = gelu(z) if l < L - 1 else z
        acts.append(h)
    y = x + h
    return y, (acts, pre)


def loss(y, target):
    return float(np.mean((y - target) ** 2))


def backward(params, cache, y, target):
    """Gradients of loss(y, target) with respect to every (W, b) and x."""
    return backward_dy(params, cache, 2.0 * (y - target) / y.size)


def backward_dy(params, cache, dy):
    """Chain rule through y = x + net(x) from a given dL/dy: the gradients
    with respect to every (W, b) and dL/dx (the residual path included).
    Chaining two calls, y1 = f(x) and y2 = f(y1), the dL/dx of the second
    call is the upstream gradient of the first."""
    acts, pre = cache
    L = len(params)
    dh = dy.copy()
    grads = [None] * L
    for l in range(L - 1, -1, -1):
        dz = dh * gelu_grad(pre[l]) if l < L - 1 else dh
        W, _ = params[l]
        dx, dW, db = conv3x3_periodic_backward(acts[l], W, dz)
        grads[l] = (dW, db)
        dh = dx
    dx_total = dy + dh  # residual path
    return grads, dx_total


# ---- the same network with BF16 storage -----------------------------------
# The configuration trains the network "in BF16 with FP32 accumulation":
# inputs, weights, hidden activations and the back-propagated gradients that
# enter the tensor-core products are held in BF16 (8 significant bits);
# every sum is exact here (FP64) instead of FP32.  What remains between this
# and the GPU is FP32 accumulation order and the rare BF16 rounding that an
# FP32 sum puts on the other side of a rounding boundary.

def bf16_round(a):
    """Round to the nearest BF16 value (8 significant bits), ties to even:
    a = m 2^e with 0.5 <= |m| < 1, and m 2^8 is rounded to an integer."""
    m, e = np.frexp(np.asarray(a, dtype=np.float64))
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def forward_bf16(params, x):
    """forward() with BF16 storage: the input, the weights and every hidden
    activation rounded to BF16; biases, sums and the residual stay exact (the
    residual adds the unrounded input)."""
    pb = [(bf16_round(W), b) for W, b in params]
    h = bf16_round(x)
    acts, pre = [h], []
    L = len(pb)
    for l, (W, b) in enumerate(pb):
        z = conv3x3_periodic(h, W, b)
        pre.append(z)
        if l < L - 1:
            h = bf16_round(gelu(z))
        acts.append(h)
    return x + pre[-1], (acts, pre, pb)


def backward_bf16(cache, y, target):
    """backward() with BF16 storage: each layer's pre-activation gradient dz
    enters the weight-gradient and input-gradient products rounded to BF16,
    with the layer's BF16 weights and activations; the bias gradient sums
    the unrounded dz."""
    acts, pre, pb = cache
    L = len(pb)
    dz = 2.0 * (y - target) / y.size
    grads = [None] * L
    for l in range(L - 1, -1, -1):
        dzb = bf16_round(dz)
        dx, dW, _ = conv3x3_periodic_backward(acts[l], pb[l][0], dzb)
        grads[l] = (dW, dz.sum(axis=(0, 2, 3)))
        if l > 0:
            dz = dx * gelu_grad(pre[l - 1])
    return grads


def adam_update(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) on arrays, returning new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
