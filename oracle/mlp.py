"""Plain FP64 oracle of the learned coarse-derivative surrogate (the "learned part":
a multilayer perceptron that maps the coarse state c to the least-squares slope of the
coarse coefficients that a resolved burst would measure, Section 3.3, Eq.
(leastsquares)).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Written with numpy in FP64; it
shares no code with the CUDA kernels.

Network: x -> z_1 = W_1 x + b_1 -> a_1 = GELU(z_1) -> ... -> y = W_L a_{L-1} + b_L, GELU
in its erf form GELU(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2. Inputs and targets are
z-scored per component: x = (c - mu_in) / sigma_in, t = (s - mu_out) / sigma_out, and the
prediction is s = y sigma_out + mu_out. Loss: mean squared error over the batch and the
outputs, L = sum (y - t)^2 / (B D_out). Optimiser: Adam (Kingma & Ba 2015) with bias
correction. Weights are stored as W[d_out][d_in].
"""
from __future__ import annotations

import math

import numpy as np
import scipy.special

from . import splitmix64

GAMMA = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1


def bf16_round(x):
    """Round FP32 values to the nearest bfloat16 (8 significant bits), ties to even;
    returned as float64. Inputs are first rounded to FP32."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    nan = np.isnan(f)
    out = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def gelu(z):
    return 0.5 * z * (1.0 + scipy.special.erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + scipy.special.erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def param_sizes(dims):
    """Flat parameter vector: W_1 [d1][d0], b_1 [d1], W_2, b_2, ... (FP32 in the library)."""
    out = []
    for l in range(len(dims) - 1):
        out.append(("W", l, dims[l + 1] * dims[l]))
        out.append(("b", l, dims[l + 1]))
    return out


def unflatten(flat, dims):
    Ws, bs, o = [], [], 0
    for kind, l, n in param_sizes(dims):
        seg = np.asarray(flat[o:o + n], dtype=np.float64)
        if kind == "W":
            Ws.append(seg.reshape(dims[l + 1], dims[l]))
        else:
            bs.append(seg)
        o += n
    return Ws, bs


def flatten(Ws, bs):
    parts = []
    for W, b in zip(Ws, bs):
        parts += [np.ravel(W), np.ravel(b)]
    return np.concatenate(parts)


def splitmix64_vec(seed, start, n):
    """Outputs start .. start+n-1 of the splitmix64 sequence of `seed` (numpy uint64
    arithmetic, which wraps modulo 2^64): output i is the splitmix64 mix of seed + (i+1) gamma,
    the same value as splitmix64(seed + i gamma) of the C oracle."""
    with np.errstate(over="ignore"):
        z = (np.uint64(seed & MASK) + (np.arange(start, start + n, dtype=np.uint64) + np.uint64(1)) * np.uint64(GAMMA))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def init_params(dims, seed):
    """Initial weights from the splitmix64 sequence: u_i = (s_i >> 40) 2^-24 with s_i the
    i-th output for the flat index i of W_l entries; W = (2u - 1) a_l in FP32 with
    a_l = sqrt(6 / d_in) for hidden layers (He uniform) and sqrt(3 / d_in) for the last
    layer; biases 0. Returned as the flat FP32 vector."""
    flat = []
    idx = 0
    for kind, l, n in param_sizes(dims):
        if kind == "b":
            flat.append(np.zeros(n, np.float32))
            idx += n
            continue
        last = l == len(dims) - 2
        a = np.float32(math.sqrt((3.0 if last else 6.0) / dims[l]))
        u = (splitmix64_vec(seed, idx, n) >> np.uint64(40)).astype(np.float64)
        u = (u * 2.0 ** -24).astype(np.float32)
        flat.append((np.float32(2.0) * u - np.float32(1.0)) * a)
        idx += n
    return np.concatenate(flat).astype(np.float32)


def forward(Ws, bs, x):
    """Returns (y, zs, acts): pre-activations z_l of the hidden layers, their GELU
    outputs, and the output y; x is [B][d0]."""
    a = np.asarray(x, np.float64)
    zs, acts = [], [a]
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = a @ W.T + b
        if l == len(Ws) - 1:
            return z, zs, acts
        zs.append(z)
        a = gelu(z)
        acts.append(a)
    raise ValueError("empty network")


def loss_and_grads(Ws, bs, x, t):
    """MSE loss and its gradients (dW_l, db_l) by the chain rule, layer by layer."""
    y, zs, acts = forward(Ws, bs, x)
    B, D = y.shape
    loss = float(np.sum((y - t) ** 2) / (B * D))
    g = 2.0 * (y - t) / (B * D)  # dL/dy
    dWs, dbs = [None] * len(Ws), [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        dWs[l] = g.T @ acts[l]
        dbs[l] = g.sum(axis=0)
        if l > 0:
            g = (g @ Ws[l]) * gelu_grad(zs[l - 1])
    return loss, dWs, dbs


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1) of flat FP64 arrays; returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def zscore_stats(X, period=0):
    """Per-component mean and standard deviation (population) of the rows of X; components
    whose deviation is below 1e-6 of the largest one get that floor instead. With period
    P > 0 both are pooled over each block of P consecutive components."""
    X = np.asarray(X, np.float64)
    if period:
        N, D = X.shape
        Xb = X.reshape(N, D // period, period)
        mu = np.repeat(Xb.mean(axis=(0, 2)), period)
        sd = np.repeat(np.sqrt(((Xb - Xb.mean(axis=(0, 2))[None, :, None]) ** 2).mean(axis=(0, 2))), period)
    else:
        mu = X.mean(axis=0)
        sd = np.sqrt(((X - mu) ** 2).mean(axis=0))
    floor = 1e-6 * max(sd.max(), 1e-30)
    return mu, np.maximum(sd, floor)


def ls_slope_with_sigma(samples, dt):
    """Least-squares line fit of samples [(K+1)][n] at t_p = p dt (Section 3.3, Eq.
    (leastsquares)), with the standard error of each slope from the fit residuals:
    sigma^2 = sum_p r_p^2 / (K - 1) / sum_p (t_p - tbar)^2 (needs K >= 2)."""
    y = np.asarray(samples, np.float64)
    K = y.shape[0] - 1
    tp = np.arange(K + 1) * dt
    tbar = tp.mean()
    sxx = np.sum((tp - tbar) ** 2)
    ybar = y.mean(axis=0)
    slope = ((tp - tbar)[:, None] * (y - ybar)).sum(axis=0) / sxx
    resid = y - (ybar + slope * (tp - tbar)[:, None])
    sigma = np.sqrt(np.sum(resid ** 2, axis=0) / (K - 1) / sxx)
    return slope, sigma


def gate(s_mlp, s_probe, sigma_probe, c_last, leap, tol, nsig):
    """A-posteriori check of a predicted slope against a short probe burst. The estimated
    error is the relative change the slope difference makes to the projected coarse state,
    e = leap ||s_mlp - s_probe|| / ||c_last|| (c_last the probe's last sample, leap =
    Delta t - K_probe delta t); the probe's own noise gives the floor
    nsig leap ||sigma_probe|| / ||c_last||. Accept when e <= max(tol, floor).
    Returns (accept, e, max(tol, floor), ||s_probe||)."""
    cn = float(np.linalg.norm(c_last))
    err = leap * float(np.linalg.norm(np.asarray(s_mlp) - np.asarray(s_probe))) / cn
    floor = max(tol, nsig * leap * float(np.linalg.norm(sigma_probe)) / cn)
    return err <= floor, err, floor, float(np.linalg.norm(s_probe))
