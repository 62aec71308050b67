"""Learned K-step surrogate of the hybrid LBM step.

A stack of periodic 3x3 convolutions maps the normalised state
(rho, u_x, u_y, theta) on a periodic grid to the state K time steps later
(y = x + net(x)).  Forward, backward and Adam run in the library's own CUDA
kernels (include/hlbm.h, hlbm_sur_*); this module only prepares data and
drives them.  Training data are rollouts of the HLBM solver itself.
The HLBM stays the judge and the fallback: `hybrid_rollout` re-runs the
solver every `judge_every` surrogate calls and continues from the solver's
state when the surrogate's error exceeds a tolerance.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import hlbm, inputs

FIELDS = ("rho", "ux", "uy", "theta")


def init_params(widths, seed=0, last_scale=1e-2):
    """He-normal weights, zero biases; the last layer starts small so that
    the untrained network is close to y = x."""
    rng = np.random.default_rng(seed)
    out = []
    L = len(widths) - 1
    for l in range(L):
        ci, co = widths[l], widths[l + 1]
        w = rng.normal(size=(co, ci, 9)) * math.sqrt(2.0 / (9 * ci))
        if l == L - 1:
            w *= last_scale
        out.append(w.ravel())
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32)


def solver_state(solver):
    m = solver.macros()
    return np.stack([m[k] for k in FIELDS], axis=-1)  # [ny, nx, 4]


def make_dataset(nsamples, n=256, K=16, pairs_per_run=4, seed=0, mu=1e-4, stream=None):
    """(x, y) pairs [nsamples, n, n, 4] (float64): the HLBM state and the
    state K steps later, from seeded random-Fourier initial fields (several
    consecutive pairs per run)."""
    xs, ys = [], []
    run = 0
    while len(xs) < nsamples:
        case = inputs.random_fourier(n=n, seed=seed * 100003 + run, mu=mu)
        s = hlbm.Solver(n, n, stream=stream, precision=hlbm.HLBM_FP32, **case.params())
        s.init(*case.fields())
        cur = solver_state(s)
        for _ in range(pairs_per_run):
            s.step(K)
            nxt = solver_state(s)
            xs.append(cur)
            ys.append(nxt)
            cur = nxt
            if len(xs) >= nsamples:
                break
        s.close()
        run += 1
    return np.stack(xs), np.stack(ys)


def make_dataset_device(nsamples, n=256, K=16, pairs_per_run=4, seed=0, mu=1e-4, stream=None):
    """Like make_dataset, but the pairs stay on the GPU as float32 tensors
    [nsamples, n, n, 4] (the solver writes its fields straight into device
    memory)."""
    import torch
    X = torch.empty((nsamples, n, n, 4), dtype=torch.float32, device="cuda")
    Y = torch.empty_like(X)
    f64 = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in range(4)]
    filled, run = 0, 0

    def grab(s, dst):
        hlbm.hlbm_get_macros(s.h, rho=f64[0], ux=f64[1], uy=f64[2], theta=f64[3], n=n * n)
        for q in range(4):
            dst[..., q] = f64[q]

    s = None
    while filled < nsamples:
        case = inputs.random_fourier(n=n, seed=seed * 100003 + run, mu=mu)
        if s is None:  # every run shares the parameters: one handle, re-initialised per run
            s = hlbm.Solver(n, n, stream=stream, precision=hlbm.HLBM_FP32, **case.params())
        s.init(*case.fields())
        grab(s, X[filled])
        for k in range(pairs_per_run):
            s.step(K)
            grab(s, Y[filled])
            filled += 1
            if filled >= nsamples:
                break
            if k + 1 < pairs_per_run:
                X[filled].copy_(Y[filled - 1])
        run += 1
    if s is not None:
        s.close()
    return X, Y


class DeviceNormaliser:
    """Per-channel affine map fitted on training inputs held on the GPU."""

    def __init__(self, X):
        flat = X.reshape(-1, X.shape[-1]).double()
        self.mean = flat.mean(dim=0).float()
        self.std = (flat.std(dim=0) + 1e-12).float()

    def fwd(self, a):
        return (a - self.mean) / self.std

    def inv(self, a):
        return a * self.std + self.mean


class Normaliser:
    """Per-channel affine map fitted on training inputs."""

    def __init__(self, x):
        self.mean = x.reshape(-1, x.shape[-1]).mean(axis=0)
        self.std = x.reshape(-1, x.shape[-1]).std(axis=0) + 1e-12

    def fwd(self, a):
        return (a - self.mean) / self.std

    def inv(self, a):
        return a * self.std + self.mean


class Surrogate:
    """Owns one hlbm_sur handle.  Tensors are CUDA float32 [B, H, W, C].
    Its work runs on `stream` (default: torch's current stream at creation),
    so that tensors passed in and out are ordered with torch's own work on
    that stream."""

    def __init__(self, widths=(4, 64, 64, 64, 64, 64, 4), H=256, W=256, batch_max=16, seed=0, stream=None):
        self.widths = tuple(int(w) for w in widths)
        self.H, self.W, self.batch_max = int(H), int(W), int(batch_max)
        self.s = hlbm.hlbm_sur_create(self.widths, H, W, batch_max, hlbm.torch_stream_handle(stream))
        self.nparam = hlbm.hlbm_sur_param_count(self.s)
        self.set_params(init_params(self.widths, seed))

    def close(self):
        if self.s:
            hlbm.hlbm_sur_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparam
        hlbm.hlbm_sur_set_params(self.s, p)

    def params(self):
        p = np.zeros(self.nparam, dtype=np.float32)
        hlbm.hlbm_sur_get_params(self.s, params=p)
        return p

    def grads(self):
        g = np.zeros(self.nparam, dtype=np.float32)
        hlbm.hlbm_sur_get_params(self.s, grads=g)
        return g

    def forward(self, x, y=None):
        import torch
        if y is None:
            y = torch.empty_like(x)
        hlbm.hlbm_sur_forward(self.s, x, y, x.shape[0])
        return y

    def predict(self, x, y=None):
        """Inference only: like forward, without keeping the pre-activations
        a backward pass needs."""
        import torch
        if y is None:
            y = torch.empty_like(x)
        hlbm.hlbm_sur_predict(self.s, x, y, x.shape[0])
        return y

    def synchronize(self):
        """Wait for the surrogate's work; raises HlbmError if a tensor-core
        kernel reported a timeout."""
        hlbm.hlbm_sur_synchronize(self.s)

    def train_step(self, x, target, lr):
        hlbm.hlbm_sur_forward(self.s, x, None, x.shape[0])
        loss = hlbm.hlbm_sur_backward(self.s, target)
        hlbm.hlbm_sur_adam(self.s, lr)
        return loss

    def rollout_grads(self, x, targets):
        """Gradients of the loss of a rollout through the network, y_1 =
        f(x), y_j = f(y_(j-1)), L = sum_j mean((y_j - targets[j-1])^2), left
        in the parameter gradients.  The inputs of the calls come from a
        first pass without stored activations; the backward passes then run
        from the last call to the first, each after a forward pass that
        restores its activations, the dL/dx of a call being the upstream
        gradient of the one before.  Returns the mean of the calls' losses."""
        import torch
        k = len(targets)
        ins = [x]
        for _ in range(k - 1):
            ins.append(self.predict(ins[-1]))
        g, total = None, 0.0
        for j in range(k - 1, -1, -1):
            hlbm.hlbm_sur_forward(self.s, ins[j], None, x.shape[0])
            dx = torch.empty_like(x) if j > 0 else None
            total += hlbm.hlbm_sur_backward_ex(self.s, targets[j], g, accumulate=j < k - 1, dx=dx)
            g = dx
        return total / k

    def train_step_rollout(self, x, targets, lr):
        """One Adam step on the loss of a rollout of len(targets) calls."""
        loss = self.rollout_grads(x, targets)
        hlbm.hlbm_sur_adam(self.s, lr)
        return loss

    def fit(self, X, Y, epochs=10, batch=8, lr=1e-3, seed=0, log=None, lr_final=None, noise=0.0,
            pushforward=0.0, pairs_per_run=None, rollout=1, rollout_from=0.5):
        """X, Y: CUDA float32 [N, H, W, C] (normalised).  The learning rate
        goes from `lr` to `lr_final` (default: stays at lr) along a cosine
        over the epochs.  With noise > 0 every input batch gets seeded
        Gaussian noise of that standard deviation (the target stays the
        solver's result), so that the network learns to advance states that
        carry its own earlier errors, as in a rollout.  With pushforward > 0
        (and X, Y holding runs of `pairs_per_run` consecutive pairs, X[i] =
        Y[i - 1] inside a run), in the second half of the epochs that
        fraction of the samples that have a predecessor take as input the
        network's own prediction from the predecessor instead of the solver's
        state, with the solver's next state as the target: the network is
        trained on the states its rollouts reach.  With rollout = k > 1 (and
        runs of `pairs_per_run` pairs), from the epoch `rollout_from` x epochs
        on, every step trains on the loss of k calls chained through the
        network, from the samples whose run holds k - 1 more pairs (targets:
        the solver's states 1 .. k calls later), back-propagated through
        the chain.  Returns the mean loss of every epoch."""
        import torch
        rng = np.random.default_rng(seed)
        gen = torch.Generator(device=X.device)
        gen.manual_seed(int(seed) + 1)
        hist = []
        N = X.shape[0]
        self.fit_calls = 0  # forward and backward passes of one sample each, summed
        for ep in range(epochs):
            unroll = rollout > 1 and pairs_per_run and ep >= rollout_from * epochs
            if unroll:
                starts = np.flatnonzero(np.arange(N) % pairs_per_run <= pairs_per_run - rollout)
                order = starts[rng.permutation(starts.size)]
            else:
                order = rng.permutation(N)
            tot, cnt = 0.0, 0
            lr_ep = lr
            if lr_final is not None and epochs > 1:
                lr_ep = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * ep / (epochs - 1)))
            for b0 in range(0, order.size - batch + 1, batch):
                sel = order[b0:b0 + batch]
                idx = torch.as_tensor(sel, device=X.device)
                xb = X[idx].contiguous()
                if unroll:
                    if noise > 0.0:
                        xb = xb + noise * torch.randn(xb.shape, device=X.device, generator=gen)
                    targets = [Y[idx + j].contiguous() for j in range(rollout)]
                    tot += self.train_step_rollout(xb, targets, lr_ep)
                    cnt += 1
                    self.fit_calls += rollout * batch
                    continue
                if pushforward > 0.0 and pairs_per_run and 2 * ep >= epochs:
                    pick = np.flatnonzero((sel % pairs_per_run != 0) & (rng.random(len(sel)) < pushforward))
                    if pick.size:
                        prev = torch.as_tensor(sel[pick] - 1, device=X.device)
                        xb[torch.as_tensor(pick, device=X.device)] = self.predict(X[prev].contiguous())
                if noise > 0.0:
                    xb = xb + noise * torch.randn(xb.shape, device=X.device, generator=gen)
                tot += self.train_step(xb, Y[idx].contiguous(), lr_ep)
                cnt += 1
                self.fit_calls += batch
            self.synchronize()
            hist.append(tot / max(cnt, 1))
            if log:
                log(ep, hist[-1])
        return hist


def hybrid_rollout(sur, norm, case, calls, K=16, judge_every=8, tol=None, stream=None):
    """Advance `case` by calls * K steps with the surrogate, re-running the
    HLBM over the same K steps every `judge_every` calls.  The judged error
    (max-abs over the normalised fields) is recorded; above `tol` the
    rollout continues from the solver's state (fallback).  Returns the final
    state [H, W, 4] and a list of (call, error, fell_back)."""
    import torch
    n = case.nx
    state = np.stack(case.fields(), axis=-1)
    log = []
    for k in range(calls):
        x = torch.from_numpy(norm.fwd(state)[None].astype(np.float32)).cuda()
        y = norm.inv(sur.predict(x)[0].double().cpu().numpy())
        if (k + 1) % judge_every == 0:
            s = hlbm.Solver(n, n, stream=stream, precision=hlbm.HLBM_FP32, **case.params())
            s.init(*[np.ascontiguousarray(state[..., q]) for q in range(4)])
            s.step(K)
            ref = solver_state(s)
            s.close()
            err = float(np.abs(norm.fwd(y) - norm.fwd(ref)).max())
            back = tol is not None and err > tol
            log.append((k, err, back))
            state = ref if back else y
        else:
            state = y
    return state, log


class FieldJudge:
    """The HLBM as the surrogate's judge: one FP32 solver handle (the cases
    of a rollout share their parameters) that advances a device state
    [H, W, 4] (rho, u_x, u_y, theta, float32) by K time steps, with device
    buffers only (no host copies)."""

    def __init__(self, n, params, stream=None):
        import torch
        self.n = n
        self.solver = hlbm.Solver(n, n, stream=stream, precision=hlbm.HLBM_FP32, **params)
        self.f64 = [torch.empty((n, n), dtype=torch.float64, device="cuda") for _ in range(4)]

    def advance(self, state, K, out):
        """out[...] = the state K steps after `state` (both [H, W, 4] float32
        CUDA tensors); a1 starts from its finite-difference form, the
        initialisation of Sec. 3.5."""
        for q in range(4):
            self.f64[q].copy_(state[..., q])
        self.solver.init(*self.f64)
        self.solver.step(K)
        n2 = self.n * self.n
        hlbm.hlbm_get_macros(self.solver.h, rho=self.f64[0], ux=self.f64[1], uy=self.f64[2],
                             theta=self.f64[3], n=n2)
        for q in range(4):
            out[..., q] = self.f64[q]
        return out

    def close(self):
        self.solver.close()


def hybrid_rollout_device(sur, norm, judge, state, calls, K=16, judge_every=8, tol=None):
    """Advance a batch of states [B, H, W, 4] (float32, CUDA, physical
    fields) by calls * K time steps with the surrogate, the HLBM judging every
    `judge_every`-th call.  The judge re-runs that call's K steps from the
    same states; the judged error of a state is the max-abs difference of the
    normalised fields.  A state whose error is finite and within `tol` (any
    finite error when tol is None) continues from the surrogate's result.
    Any other state -- drifted, or broken by the unjudged calls before it --
    is advanced again by the HLBM over the whole window since the previous
    judged call, from its state there (the fallback), so that no rejected
    window carries on.  `norm` is a DeviceNormaliser.  Returns (state, log)
    with log entries (call, sample, error, fell_back)."""
    import torch
    B = state.shape[0]
    log = []
    ckpt, ckpt_call = state.clone(), 0
    ref = torch.empty_like(state[0])
    for k in range(calls):
        prev = state
        state = norm.inv(sur.predict(norm.fwd(state).contiguous()))
        if (k + 1) % judge_every == 0:
            for b in range(B):
                judge.advance(prev[b], K, ref)
                err = float((norm.fwd(state[b]) - norm.fwd(ref)).abs().max())
                ok = math.isfinite(err) and (tol is None or err <= tol)
                if not ok:
                    judge.advance(ckpt[b], (k + 1 - ckpt_call) * K, state[b])
                log.append((k, b, err, not ok))
            ckpt, ckpt_call = state.clone(), k + 1
    return state, log


def _predict_workload(calls):
    """A fixed inference workload for timing and profiling the convolution
    kernels: the K = 16 network (4-64x5-4) with seeded random weights, one
    predict call on a seeded normal 16 x 256 x 256 x 4 input three times for
    warm-up, then `calls` more."""
    import torch
    torch.cuda.set_device(0)
    sur = Surrogate((4, 64, 64, 64, 64, 64, 4), 256, 256, batch_max=16, seed=0)
    x = torch.from_numpy(np.random.default_rng(1).normal(size=(16, 256, 256, 4)).astype(np.float32)).cuda()
    y = torch.empty_like(x)
    for _ in range(3 + calls):
        sur.predict(x, y)
    sur.synchronize()
    print("mean |y|", float(y.abs().mean()))
    sur.close()


if __name__ == "__main__":
    import sys
    _predict_workload(int(sys.argv[1]) if len(sys.argv) > 1 else 2)
