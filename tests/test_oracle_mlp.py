"""Pins of the FP64 oracle of the learned coarse-derivative MLP: rounding, GELU,
brute-force forward, finite-difference gradients, closed-form Adam steps, the
least-squares slope and its standard error. No GPU needed."""
import math

import numpy as np
import pytest
import scipy.stats

import oracle as orc
from oracle import mlp


def test_bf16_round_known_values():
    x = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-9, 1.0 + 2**-7, -2.5, 3.0e38, 1e-40, 0.0, 65504.0])
    want = np.array([1.0, 1.0, 1.0 + 2**-7, 1.0 + 2**-7, -2.5, 2.9975e38, 0.0, 0.0, 65536.0])
    got = mlp.bf16_round(x)
    assert got[0] == 1.0 and got[1] == 1.0            # tie to even
    assert got[2] == 1.0 + 2**-7 and got[3] == 1.0 + 2**-7
    assert got[4] == -2.5 and got[7] == 0.0 and got[8] == 65536.0
    assert abs(got[5] - want[5]) / want[5] < 2**-8
    assert abs(got[6]) < 1e-39
    # 8 significant bits: every result is an integer times a power of two with |m| < 256
    r = mlp.bf16_round(np.random.default_rng(0).standard_normal(1000))
    m, e = np.frexp(r)
    assert np.all(np.abs(m * 256) == np.round(np.abs(m * 256)))


def test_gelu_identities_and_derivative():
    x = np.linspace(-6, 6, 241)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert np.allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-15)   # z Phi(z) + z Phi(-z) = z
    assert mlp.gelu(np.array([12.0]))[0] == pytest.approx(12.0, rel=1e-15)
    assert abs(mlp.gelu(np.array([-12.0]))[0]) < 1e-30
    h = 1e-5
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(x), fd, atol=1e-9)
    # GELU(1) = Phi(1) with the normal CDF of the library
    assert mlp.gelu(np.array([1.0]))[0] == pytest.approx(scipy.stats.norm.cdf(1.0), rel=1e-14)


def _net(dims, seed):
    rng = np.random.default_rng(seed)
    Ws = [rng.standard_normal((dims[l + 1], dims[l])) / math.sqrt(dims[l]) for l in range(len(dims) - 1)]
    bs = [0.1 * rng.standard_normal(dims[l + 1]) for l in range(len(dims) - 1)]
    return Ws, bs


def test_forward_brute_force():
    dims = [3, 4, 2]
    Ws, bs = _net(dims, 1)
    x = np.random.default_rng(2).standard_normal((5, 3))
    y, zs, acts = mlp.forward(Ws, bs, x)
    for b in range(5):
        h = []
        for i in range(4):
            z = bs[0][i]
            for k in range(3):
                z += Ws[0][i][k] * x[b][k]
            h.append(0.5 * z * (1.0 + math.erf(z / math.sqrt(2.0))))
        for j in range(2):
            o = bs[1][j]
            for i in range(4):
                o += Ws[1][j][i] * h[i]
            assert y[b][j] == pytest.approx(o, rel=1e-13, abs=1e-15)


def test_gradients_match_central_differences():
    dims = [6, 5, 4, 3]
    Ws, bs = _net(dims, 3)
    rng = np.random.default_rng(4)
    x, t = rng.standard_normal((7, 6)), rng.standard_normal((7, 3))
    loss, dWs, dbs = mlp.loss_and_grads(Ws, bs, x, t)
    flat = mlp.flatten(Ws, bs)
    grad = mlp.flatten(dWs, dbs)
    h = 1e-6
    fd = np.zeros_like(flat)
    for i in range(flat.size):
        p, m = flat.copy(), flat.copy()
        p[i] += h
        m[i] -= h
        lp = mlp.loss_and_grads(*mlp.unflatten(p, dims), x, t)[0]
        lm = mlp.loss_and_grads(*mlp.unflatten(m, dims), x, t)[0]
        fd[i] = (lp - lm) / (2 * h)
    assert np.abs(grad - fd).max() <= 1e-6 * np.abs(fd).max()
    assert loss == pytest.approx(np.mean((mlp.forward(Ws, bs, x)[0] - t) ** 2), rel=1e-15)


def test_adam_closed_form_steps():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    theta, m, v = np.ones(4), np.zeros(4), np.zeros(4)
    lr, eps = 1e-2, 1e-8
    for t in range(1, 6):
        # a constant gradient keeps m_hat = g and v_hat = g^2 at every step
        new, m, v = mlp.adam_step(theta, g, m, v, t, lr, eps=eps)
        assert np.allclose(new - theta, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)
        theta = new


def test_init_params_distribution_and_sequence():
    dims = [64, 32, 16]
    p = mlp.init_params(dims, 11)
    assert p.dtype == np.float32 and p.size == 64 * 32 + 32 + 32 * 16 + 16
    Ws, bs = mlp.unflatten(p, dims)
    for l, W in enumerate(Ws):
        a = math.sqrt((3.0 if l == 1 else 6.0) / dims[l])
        assert np.abs(W).max() <= a
        assert abs(W.mean()) < 0.1 * a
        assert np.var(W) == pytest.approx(a * a / 3, rel=0.15)
    assert all(np.all(b == 0) for b in bs)
    # the vectorised sequence equals the C oracle's splitmix64 of the counter
    seq = mlp.splitmix64_vec(11, 5, 3)
    for i in range(3):
        assert int(seq[i]) == orc.splitmix64((11 + (5 + i) * mlp.GAMMA) & mlp.MASK)


def test_ls_slope_with_sigma():
    dt, K = 0.1, 5
    tp = np.arange(K + 1) * dt
    exact = 2.0 + 3.0 * tp[:, None] * np.array([1.0, -0.5])[None, :]
    s, sig = mlp.ls_slope_with_sigma(exact, dt)
    assert np.allclose(s, [3.0, -1.5], rtol=1e-12) and np.all(sig < 1e-12)
    y = np.random.default_rng(5).standard_normal((K + 1, 3))
    s, sig = mlp.ls_slope_with_sigma(y, dt)
    for i in range(3):
        r = scipy.stats.linregress(tp, y[:, i])
        assert s[i] == pytest.approx(r.slope, rel=1e-12)
        assert sig[i] == pytest.approx(r.stderr, rel=1e-12)
        # the C oracle's normal-equation slope
        assert s[i] == pytest.approx(orc.ls_slope(y[:, i], dt), rel=1e-12)


def test_gate_rule():
    s = np.array([1.0, 0.0])
    c = np.array([3.0, 4.0])  # |c| = 5
    assert mlp.gate(s, s, np.zeros(2), c, 10.0, 1e-2, 3.0)[0]
    # e = 10 * 0.004 / 5 = 0.008 <= 1e-2; 0.006 -> 0.012 > 1e-2
    acc, e, fl, nrm = mlp.gate(s + [0.004, 0], s, np.zeros(2), c, 10.0, 1e-2, 3.0)
    assert acc and e == pytest.approx(0.008) and fl == 1e-2 and nrm == 1.0
    assert not mlp.gate(s + [0.006, 0], s, np.zeros(2), c, 10.0, 1e-2, 3.0)[0]
    # a noisy probe widens the acceptance floor: 3 * 10 * 0.001 / 5 = 0.006 -> still 1e-2;
    # sigma 0.0025 -> 0.015 >= 0.012
    assert not mlp.gate(s + [0.006, 0], s, np.array([0.001, 0.0]), c, 10.0, 1e-2, 3.0)[0]
    acc, e, fl, _ = mlp.gate(s + [0.006, 0], s, np.array([0.0025, 0.0]), c, 10.0, 1e-2, 3.0)
    assert acc and fl == pytest.approx(0.015)
