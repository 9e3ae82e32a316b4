"""GPU parity of the learned-surrogate kernels (BF16 tcgen05 tensor-core MLP) and of the gate
against the FP64 CPU oracle (oracle/mlp.py), through the C ABI.

Tolerances (BF16 operands, FP32 accumulation):
  initial weights .... bit-exact (same splitmix64 sequence and FP32 arithmetic)
  z-score statistics . 1e-6 relative (FP64 sums in another order, stored as FP32)
  forward ............ relative L2 <= 2e-2 against the FP64 network with the same
                       BF16-rounded weights
  gradients .......... cosine >= 0.999 and relative L2 <= 2e-2 per layer
  Adam ............... 1e-6 relative (FP32 against FP64 on the same gradient)
  gate ............... decision exact; statistics 1e-10 relative (FP64 both)
"""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
import paper_1610_01071_gb300 as pe
from paper_1610_01071_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def cos(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))


FULL = [512, 512, 512, 512, 512]


@pytest.mark.parametrize("dims", [[64, 128, 64], FULL])
def test_init_matches_oracle(dims):
    net = pe.MLP(dims, max_batch=64, device=DEV)
    net.init(7)
    got = net.params().cpu().numpy()
    want = omlp.init_params(dims, 7)
    assert np.array_equal(got, want)
    mirror = net.params_bf16().float().cpu().numpy().astype(np.float64)
    assert np.array_equal(mirror, omlp.bf16_round(want))
    _check_transposed_mirror(net, dims)


@pytest.mark.parametrize("period", [0, 32])
def test_fit_norm_matches_oracle(period):
    X, Y = inputs.regression_set(3000, 128, 64, 1)
    net = pe.MLP([128, 64, 64], device=DEV)
    net.init(0)
    net.fit_norm(dev(X), dev(Y), period)
    nm = net.norm().cpu().numpy().astype(np.float64)
    mu, sd = omlp.zscore_stats(X, period)
    mo, so = omlp.zscore_stats(Y, period)
    for got, want in ((nm[0, :128], mu), (nm[1, :128], sd), (nm[2, :64], mo), (nm[3, :64], so)):
        assert np.allclose(got, want, rtol=1e-6, atol=1e-7)


def _reference(dims, p, X, Y, rows):
    mu, sd = omlp.zscore_stats(X)
    mo, so = omlp.zscore_stats(Y)
    Ws, bs = omlp.unflatten(p, dims)
    Ws = [omlp.bf16_round(W) for W in Ws]  # the GPU's BF16 weights
    return Ws, bs, (X[rows] - mu) / sd, (Y[rows] - mo) / so, mo, so


@pytest.mark.parametrize("dims,B", [(FULL, 1), (FULL, 256), ([128, 64, 192], 7), ([128, 64, 192], 100),
                                    ([64, 64], 65)])
def test_forward_matches_oracle(dims, B):
    p = inputs.random_mlp_params(dims, 3)
    X, Y = inputs.regression_set(512, dims[0], dims[-1], 2)
    net = pe.MLP(dims, max_batch=256, device=DEV)
    net.init(0)
    net.set_params(dev(p))
    net.fit_norm(dev(X), dev(Y))
    y = net.forward(dev(X[:B])).cpu().numpy().astype(np.float64)
    Ws, bs, x, _, mo, so = _reference(dims, p, X, Y, np.arange(B))
    yz = omlp.forward(Ws, bs, x)[0]
    assert rel((y - mo) / so, yz) <= 2e-2
    # the FP64 entry (the context's coarse state) gives the same network output
    y64 = net.forward(dev(X[:B].astype(np.float64))).cpu().numpy()
    assert np.array_equal(y64.astype(np.float32), y.astype(np.float32))


@pytest.mark.parametrize("dims,B", [(FULL, 64), ([128, 64, 192], 96), ([64, 64], 32)])
def test_gradients_match_oracle(dims, B):
    p = inputs.random_mlp_params(dims, 4)
    X, Y = inputs.regression_set(1000, dims[0], dims[-1], 5)
    rows = np.random.default_rng(6).integers(0, 1000, B).astype(np.int32)
    net = pe.MLP(dims, max_batch=128, device=DEV)
    net.init(0)
    net.set_params(dev(p))
    net.fit_norm(dev(X), dev(Y))
    loss = net.grad(dev(X), dev(Y), rows=dev(rows))
    Ws, bs, x, t, _, _ = _reference(dims, p, X, Y, rows)
    L, dWs, dbs = omlp.loss_and_grads(Ws, bs, x, t)
    assert loss == pytest.approx(L, rel=2e-2)
    gW, gb = omlp.unflatten(net.grads().cpu().numpy(), dims)
    for l in range(len(dims) - 1):
        for got, want in ((gW[l], dWs[l]), (gb[l], dbs[l])):
            assert cos(got, want) >= 0.999, l
            assert rel(got, want) <= 2e-2, l


def _check_transposed_mirror(net, dims):
    # the data-gradient GEMMs read W_l^T: the transposed mirror must hold the mirror's weights
    m = net.params_bf16().float().cpu().numpy()
    t = net.params_bf16_transposed().float().cpu().numpy()
    off = 0
    for l in range(len(dims) - 1):
        n = dims[l + 1] * dims[l]
        W = m[off:off + n].reshape(dims[l + 1], dims[l])
        assert np.array_equal(t[off:off + n].reshape(dims[l], dims[l + 1]), W.T)
        off += n + dims[l + 1]


def test_adam_matches_oracle():
    dims = [128, 64, 192]
    p = inputs.random_mlp_params(dims, 8)
    g = inputs.random_mlp_params(dims, 9, scale=0.01)
    net = pe.MLP(dims, max_batch=64, device=DEV)
    net.init(0)
    net.set_params(dev(p))
    net.grads().copy_(dev(g))
    lr = 1e-3
    theta, m, v = p.astype(np.float64), np.zeros(p.size), np.zeros(p.size)
    for t in range(1, 4):
        net.adam(lr)
        theta, m, v = omlp.adam_step(theta, g.astype(np.float64), m, v, t, lr)
    got = net.params().cpu().numpy().astype(np.float64)
    assert np.abs(got - theta).max() <= 1e-6 * np.abs(theta).max() + 1e-4 * lr
    gm, gv = (a.cpu().numpy().astype(np.float64) for a in net.adam_state())
    assert np.allclose(gm, m, rtol=1e-5, atol=1e-12) and np.allclose(gv, v, rtol=1e-5, atol=1e-16)
    assert np.array_equal(net.params_bf16().float().cpu().numpy().astype(np.float64), omlp.bf16_round(got))
    _check_transposed_mirror(net, dims)


def test_training_reduces_loss_and_graph_replay_is_deterministic():
    dims = [128, 256, 256, 128]
    X, Y = inputs.regression_set(4096, 128, 128, 10)
    dX, dY = dev(X), dev(Y)
    rows = dev(np.arange(128, dtype=np.int32))
    s = torch.cuda.Stream(DEV)
    torch.cuda.synchronize(DEV)
    net = pe.MLP(dims, max_batch=128, device=DEV, stream=s)
    net.init(1)
    net.fit_norm(dX, dY)
    l0 = net.grad(dX, dY, rows=rows)
    net.train(dX, dY, 128, 400, 1e-3, seed=5)
    l1 = net.grad(dX, dY, rows=rows)
    assert l1 < 0.2 * l0
    # one captured step replayed k times == k eager steps, bit for bit
    a = pe.MLP(dims, max_batch=128, device=DEV, stream=s)
    b = pe.MLP(dims, max_batch=128, device=DEV, stream=s)
    for n in (a, b):
        n.init(2)
        n.fit_norm(dX, dY, 32)
    a.train(dX, dY, 64, 6, 1e-3, seed=9, shift_period=32)
    for _ in range(6):
        b.train(dX, dY, 64, 1, 1e-3, seed=9, shift_period=32)
    s.synchronize()
    assert torch.equal(a.params(), b.params())
    assert a.sync_status() == 0 and b.sync_status() == 0 and net.sync_status() == 0


@pytest.mark.parametrize("Ks,n", [(5, 512), (2, 64), (19, 1000)])
def test_gate_matches_oracle(Ks, n):
    rng = np.random.default_rng(Ks + n)
    dt, dT = 0.1, 20.0
    leap = dT - Ks * dt
    tp = np.arange(Ks + 1) * dt
    samples = rng.standard_normal(n) + rng.standard_normal(n) * tp[:, None] + 1e-6 * rng.standard_normal((Ks + 1, n))
    s_probe, sig = omlp.ls_slope_with_sigma(samples, dt)
    d = rng.standard_normal(n)
    d /= np.linalg.norm(d)
    cn = np.linalg.norm(samples[Ks])
    tol = 1e-2
    for e_target in (0.5 * tol, 2.0 * tol):  # one accepted, one rejected (noise floor below tol)
        s_mlp = s_probe + e_target * cn / leap * d
        coarse, slope = torch.zeros(n, dtype=torch.float64, device=DEV), torch.zeros(n, dtype=torch.float64, device=DEV)
        r = pe._binding.gate(dev(samples), dt, dT, dev(s_mlp), coarse, slope, tol=tol, noise_sigmas=3.0)
        acc, err, floor, norm = omlp.gate(s_mlp, s_probe, sig, samples[Ks], leap, tol, 3.0)
        assert acc == (e_target < tol)
        assert bool(r["accepted"]) == acc
        assert r["err"] == pytest.approx(err, rel=1e-10)
        assert r["floor"] == pytest.approx(floor, rel=1e-10)
        assert r["norm"] == pytest.approx(norm, rel=1e-10)
        assert r["sigma"] == pytest.approx(np.linalg.norm(sig), rel=1e-10)
        if acc:
            assert np.allclose(coarse.cpu().numpy(), samples[Ks] + leap * s_mlp, rtol=1e-14, atol=1e-14)
            assert np.array_equal(slope.cpu().numpy(), s_mlp)
        else:
            assert not coarse.any() and not slope.any()
    # a noisy probe raises the floor above tol
    noisy = samples + 0.05 * rng.standard_normal(samples.shape)
    s_n, sig_n = omlp.ls_slope_with_sigma(noisy, dt)
    r = pe._binding.gate(dev(noisy), dt, dT, dev(s_n), torch.zeros(n, dtype=torch.float64, device=DEV),
                         torch.zeros(n, dtype=torch.float64, device=DEV), tol=tol, noise_sigmas=3.0)
    want = omlp.gate(s_n, s_n, sig_n, noisy[Ks], leap, tol, 3.0)
    assert r["floor"] == pytest.approx(want[2], rel=1e-10) and r["floor"] > tol and r["accepted"] == 1


def test_surrogate_step_rejected_equals_projective_step():
    """With a zero tolerance every prediction is rejected and the gated step must reproduce
    pe_step bit for bit (the probe is the first K_probe steps of the same burst)."""
    cfg = pe.make_config(512, 64, 20, 512 * 256, 256.0, 0.1, 20.0, seed=3)
    a, b = pe.Context(cfg, device=DEV), pe.Context(cfg, device=DEV)
    a.load_initial(0.3)
    b.load_initial(0.3)
    net = pe.MLP([128, 128, 128], max_batch=1, device=DEV)
    net.init(1)
    for _ in range(3):
        a.step()
        st = b.step_surrogate(net, K_probe=5, tol=0.0, noise_sigmas=0.0)
        assert st["accepted"] == 0 and st["fine_steps"] == 20
        assert torch.equal(a.get_coarse(), b.get_coarse())
        assert torch.equal(a.get_slope(), b.get_slope())
    assert a.diagnostics().fine_steps == b.diagnostics().fine_steps
    assert a.sync_status() == 0 and b.sync_status() == 0


def test_surrogate_step_accepted_leaps_from_the_probe():
    cfg = pe.make_config(512, 64, 20, 512 * 256, 256.0, 0.1, 20.0, seed=4)
    ctx = pe.Context(cfg, device=DEV)
    ctx.load_initial(0.3)
    net = pe.MLP([128, 128, 128], max_batch=1, device=DEV)
    net.init(2)
    c0 = ctx.get_coarse().reshape(1, -1).clone()
    s_mlp = net.forward(c0).reshape(-1)
    st = ctx.step_surrogate(net, K_probe=4, tol=1e30, noise_sigmas=0.0)
    assert st["accepted"] == 1 and st["fine_steps"] == 4
    cs = ctx.view("coarse_samples", torch.float64, 5 * 128).view(5, 128)
    want = cs[4] + (20.0 - 4 * 0.1) * s_mlp
    assert torch.allclose(ctx.get_coarse().reshape(-1), want, rtol=1e-14, atol=1e-14)
    assert torch.equal(ctx.get_slope().reshape(-1), s_mlp)
    d = ctx.diagnostics()
    assert d.fine_steps == 4 and d.macro_steps == 1


def _pairs(ncell, nc, ppc, amps, steps, seed0):
    """(c at the start of a macro step, least-squares slope of that step) along projective runs."""
    n = 2 * nc
    X, Y = [], []
    for ai, a in enumerate(amps):
        ctx = pe.Context(pe.make_config(ncell, nc, 20, ncell * ppc, ncell * 0.5, 0.1, 20.0, seed=seed0 + ai),
                         device=DEV)
        ctx.load_initial(float(a))
        for _ in range(steps):
            x = torch.empty(n, dtype=torch.float32, device=DEV)
            ctx.export_f32(0, x)
            ctx.step()
            y = torch.empty(n, dtype=torch.float32, device=DEV)
            ctx.export_f32(1, y)
            X.append(x)
            Y.append(y)
    return torch.stack(X).contiguous(), torch.stack(Y).contiguous()


def test_trained_surrogate_saves_fine_steps_at_unchanged_accuracy():
    """Trained on the bursts' own (c, slope) pairs of the ion-wave workload (4096 cells, 256
    coefficients per moment), the gated surrogate runs the wave with far fewer fine steps
    than the projective method without it, and stays within 0.5 % (coarse density, Section
    4.1.1 measure) of that method's state."""
    ncell, nc, steps = 4096, 256, 30
    X, Y = _pairs(ncell, nc, 1024, np.linspace(0.05, 0.6, 12), 40, 200)
    s = torch.cuda.Stream(DEV)
    torch.cuda.synchronize(DEV)
    net = pe.MLP([2 * nc, 512, 512, 512, 2 * nc], max_batch=256, device=DEV, stream=s)
    net.init(3)
    net.fit_norm(X, Y, nc)
    rows = torch.arange(256, dtype=torch.int32, device=DEV)
    l0 = net.grad(X, Y, rows=rows)
    net.train(X, Y, 256, 4000, 1e-3, seed=1, shift_period=nc)
    net.train(X, Y, 256, 2000, 2e-4, seed=2, shift_period=nc)
    l1 = net.grad(X, Y, rows=rows)
    assert l1 < 0.5 * l0
    cfg = pe.make_config(ncell, nc, 20, ncell * 4096, ncell * 0.5, 0.1, 20.0, seed=999)
    ref, sur = pe.Context(cfg, device=DEV), pe.Context(cfg, device=DEV)
    ref.load_initial(0.5)
    sur.load_initial(0.5)
    accepted, fine, errs = 0, 0, []
    for _ in range(steps):
        ref.step()
        st = sur.step_surrogate(net, K_probe=5, tol=3e-3, noise_sigmas=3.0)
        accepted += st["accepted"]
        fine += st["fine_steps"]
        errs.append(round(st["err"], 5))
    a, b = ref.measure()[0].cpu().numpy(), sur.measure()[0].cpu().numpy()
    eps = float(np.sqrt(((a - b) ** 2).sum() / (a * a + b * b).sum()))
    print(f"surrogate: loss {l0:.3g} -> {l1:.3g}, accepted {accepted}/{steps}, fine steps {fine} vs {20 * steps}, "
          f"eps vs projective {eps:.4f}, estimated errors {errs}")
    assert ref.sync_status() == 0 and sur.sync_status() == 0
    assert accepted >= steps // 2
    assert fine <= 0.6 * 20 * steps
    assert eps <= 5e-3
