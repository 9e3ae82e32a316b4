"""GPU parity of the ion-pressure variable (Section 3.2, EFREE's n, V, P active) against the
oracle, through the C ABI: the second-moment restriction sample, its coarsening, the lifting
profiles (n, u, T), the loader at a local temperature, and whole macro steps of the context
with coarse_kind = PE_COARSE_MOMENTS_PRESSURE."""
import numpy as np
import pytest
import torch

import oracle as orc
import paper_1610_01071_gb300 as pe
from paper_1610_01071_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def to_dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in arrs]


@pytest.mark.parametrize("tau,ncell,N", [(0.0, 256, 1 << 16), (3.7, 256, (1 << 16) + 3), (20.0, 2048, 1 << 18)])
def test_second_moment_sample_matches_oracle(tau, ncell, N):
    dx, dt, qm = 0.5, 0.1, 1.0
    c, t, v, w = inputs.random_particles(N, ncell, seed=31)
    s_w = orc.fx_shift(2.0 * ncell / N)
    s_p = orc.fx_shift(2.0 * ncell / N * 32.0)
    s_e = pe.second_moment_shift(N, ncell, 2.0 * ncell / N, 32.0)
    E = inputs.random_field(ncell, seed=6, amp=0.05)
    E0 = inputs.random_field(ncell, seed=7, amp=0.05)
    dc, dt_, dv, dw = to_dev(c, t, v, w)
    Ef, E0f = to_dev(E.astype(np.float32), E0.astype(np.float32))
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    out = torch.empty(3 * ncell, dtype=torch.int64, device=DEV)
    args = pe.make_sample_args(E0f, tau, qm, 1 / dx, s_w, s_p, out, s_e=s_e)
    pe.sample(dc, dt_, dv, dw, Ef, ncell, qm * dt, 1.0, args, status=st)
    so = orc.State(c, t, v, w)
    Eo = E.astype(np.float32).astype(np.float64)
    vbar = so.v + 0.5 * qm * dt * orc.gather(Eo, c, t)
    E0o = E0.astype(np.float32).astype(np.float64)
    dens, mom = orc.restrict_sample(so, vbar, E0o, ncell, dx, tau, qm)
    sec = orc.restrict_second_moment(so, vbar, E0o, ncell, dx, tau, qm)
    g = out.cpu().numpy()
    assert int(st.item()) == 0
    for row, s, want in ((0, s_w, dens), (1, s_p, mom), (2, s_e, sec)):
        got = g[row * ncell:(row + 1) * ncell] * 2.0 ** -(s + 24)
        assert np.max(np.abs(got - want)) < 1e-4 * np.max(np.abs(want))
    # the density and momentum rows are those of the two-moment sample, bit for bit
    out2 = torch.empty(2 * ncell, dtype=torch.int64, device=DEV)
    pe.sample(dc, dt_, dv, dw, Ef, ncell, qm * dt, 1.0, pe.make_sample_args(E0f, tau, qm, 1 / dx, s_w, s_p, out2))
    assert np.array_equal(g[:2 * ncell], out2.cpu().numpy())
    # Haar bins: exact bin sums of the nodal fixed-point rows, all three moments
    for bsh in (1, 4):
        outb = torch.empty(3 * (ncell >> bsh), dtype=torch.int64, device=DEV)
        pe.sample(dc, dt_, dv, dw, Ef, ncell, qm * dt, 1.0,
                  pe.make_sample_args(E0f, tau, qm, 1 / dx, s_w, s_p, outb, bin_shift=bsh, s_e=s_e), status=st)
        want_b = g.reshape(3, ncell >> bsh, 1 << bsh).sum(axis=-1).reshape(-1)
        assert np.array_equal(outb.cpu().numpy(), want_b)
    assert int(st.item()) == 0


@pytest.mark.parametrize("bin_shift", [0, 3])
def test_fused_push_second_moment_equals_sample_pass(bin_shift):
    # the fused pass samples the current particles before moving them: its rows equal those of
    # the sample-only pass on the same state (nodal and Haar-binned)
    ncell, N, dx, dt, qm = 512, (1 << 17) + 1, 0.5, 0.1, 1.0
    c, t, v, w = inputs.random_particles(N, ncell, seed=2)
    s_w = orc.fx_shift(2.0 * ncell / N)
    s_p = orc.fx_shift(2.0 * ncell / N * 32.0)
    s_e = pe.second_moment_shift(N, ncell, 2.0 * ncell / N, 32.0)
    E = inputs.random_field(ncell, seed=8, amp=0.05)
    Ef, = to_dev(E.astype(np.float32))
    a = to_dev(c, t, v, w)
    b = [x.clone() for x in a]
    out_s = torch.empty(3 * (ncell >> bin_shift), dtype=torch.int64, device=DEV)
    out_p = torch.empty_like(out_s)
    pe.sample(*a, Ef, ncell, qm * dt, 0.5,
              pe.make_sample_args(Ef, 5.0, qm, 1 / dx, s_w, s_p, out_s, bin_shift=bin_shift, s_e=s_e))
    pe.push(*b, Ef, ncell, dt / dx, qm * dt, 0.5, s_w,
            sample=pe.make_sample_args(Ef, 5.0, qm, 1 / dx, s_w, s_p, out_p, bin_shift=bin_shift, s_e=s_e))
    assert torch.equal(out_s, out_p)
    # the pushed particles are those of the plain push
    c2 = to_dev(c, t, v, w)
    pe.push(*c2, Ef, ncell, dt / dx, qm * dt, 0.5, s_w)
    for x, y in zip(b, c2):
        assert torch.equal(x, y)


@pytest.mark.parametrize("wav,ncell,nc,bsh", [("haar", 128, 16, 0), ("haar", 4096, 256, 0), ("coif4", 512, 32, 0),
                                              ("haar", 4096, 256, 4), ("haar", 128, 16, 2)])
def test_coarsen_pressure_matches_oracle(wav, ncell, nc, bsh):
    rng = np.random.default_rng(ncell + 1)
    nsamp, s_w, s_p, s_e = 4, 30, 25, 21
    fx = rng.integers(-(1 << 50), 1 << 50, size=(nsamp, 3, ncell), dtype=np.int64)
    rows = fx.reshape(nsamp, 3, ncell >> bsh, 1 << bsh).sum(axis=-1)  # bin sums when bsh > 0
    out = pe.coarsen_pressure(*to_dev(rows), nsamp, ncell, s_w, s_p, s_e, nc, wavelet=wav,
                              bin_shift=bsh).cpu().numpy()
    for p in range(nsamp):
        for m, s in ((0, s_w), (1, s_p), (2, s_e)):
            want = orc.coarsen(fx[p, m] * 2.0 ** -(s + 24), nc, wav)
            assert np.allclose(out[p, m], want, rtol=1e-12, atol=1e-12 * np.max(np.abs(want)))


@pytest.mark.parametrize("wav,ncell,nc", [("haar", 256, 32), ("coif4", 4096, 256)])
def test_refine_pressure_matches_oracle(wav, ncell, nc):
    x = np.arange(ncell) / ncell
    n = 1.0 + 0.6 * np.cos(2 * np.pi * x) + 0.45 * np.cos(6 * np.pi * x)  # dips below 0: clamped
    u = 0.3 * np.sin(2 * np.pi * x)
    T = 0.9 + 0.4 * np.cos(4 * np.pi * x)
    coarse = np.stack([orc.coarsen(f, nc, wav) for f in (n, n * u, n * (u * u + T))])
    coarse[2, ::7] *= 0.5  # some second moments below n u^2: T clamps to 0 there
    pn, pu, pT = pe.refine_pressure(*to_dev(coarse), ncell, wavelet=wav)
    nf, uf, Tf = orc.lift_profile_pressure(*(orc.refine(coarse[k], ncell, wav) for k in range(3)))
    assert np.allclose(pn.cpu().numpy(), nf, rtol=1e-6, atol=1e-6 * nf.max())
    assert np.allclose(pu.cpu().numpy(), uf, rtol=1e-5, atol=1e-5 * np.abs(uf).max())
    assert np.allclose(pT.cpu().numpy(), Tf, rtol=1e-5, atol=1e-5 * Tf.max())
    assert np.all(pT.cpu().numpy() >= 0.0)


@pytest.mark.parametrize("ncell,ppc", [(128, 1024), (64, 3), (4096, 256)])
def test_quiet_start_thermal_matches_oracle(ncell, ppc):
    N = ncell * ppc
    nprof, uprof = orc.sine_profile(ncell, ncell * 0.5, 0.3)
    tprof = 1.0 + 0.5 * np.sin(2 * np.pi * np.arange(ncell) / ncell)
    seed = 777
    f32 = [a.astype(np.float32) for a in (nprof, uprof, tprof)]
    s_w = orc.fx_shift(8.0 / ppc)
    cell, theta, v, w, rho = pe.quiet_start_thermal(N, ncell, *to_dev(*f32), seed, s_w)
    st = orc.quiet_start_thermal(N, ncell, *f32, seed)
    assert np.array_equal(cell.cpu().numpy(), st.cell)
    assert np.max(np.abs(theta.cpu().numpy() - st.theta)) < 1e-7
    assert np.allclose(w.cpu().numpy(), st.w, rtol=2e-6)
    assert np.max(np.abs(v.cpu().numpy() - st.v)) < 3e-5
    assert torch.equal(rho, pe.deposit(cell, theta, w, ncell, s_w))


def test_quiet_start_thermal_at_uniform_temperature_is_the_plain_loader():
    ncell, N = 512, 512 * 128
    nprof, uprof = orc.sine_profile(ncell, 256.0, 0.2)
    pn, pu = to_dev(nprof.astype(np.float32), uprof.astype(np.float32))
    pT = torch.full((ncell,), 4.0, dtype=torch.float32, device=DEV)
    s_w = orc.fx_shift(8.0 / 128)
    a = pe.quiet_start_thermal(N, ncell, pn, pu, pT, 5, s_w)
    b = pe.quiet_start(N, ncell, pn, pu, 2.0, 5, s_w)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


SMALL = dict(ncell=128, L=64.0, N=128 * 256, dt=0.1, K=6, M=3, n_coarse=16, v_th=1.0, qm=1.0, amp=0.1)


def make_ctx(cfg, seed, **kw):
    dT = cfg["M"] * cfg["K"] * cfg["dt"]
    c = pe.make_config(cfg["ncell"], cfg["n_coarse"], cfg["K"], cfg["N"], cfg["L"], cfg["dt"], dT, qm=cfg["qm"],
                       v_th=cfg["v_th"], seed=seed, newton_tol=1e-11, coarse="moments_pressure", **kw)
    return pe.Context(c, device=DEV)


def oracle_state(cfg, seed):
    nprof, uprof = orc.sine_profile(cfg["ncell"], cfg["L"], cfg["amp"])
    return orc.quiet_start(cfg["N"], cfg["ncell"], nprof.astype(np.float32), uprof.astype(np.float32), cfg["v_th"],
                           seed)


def test_initial_coarse_state_has_the_three_moments():
    ctx = make_ctx(SMALL, seed=3)
    ctx.load_initial(SMALL["amp"])
    got = ctx.get_coarse().cpu().numpy()
    assert got.shape == (3, SMALL["n_coarse"])
    st = oracle_state(SMALL, 3)
    dens, mom = orc.restrict_sample(st, st.v, np.zeros(SMALL["ncell"]), SMALL["ncell"], 0.5, 0.0, 1.0)
    sec = orc.restrict_second_moment(st, st.v, np.zeros(SMALL["ncell"]), SMALL["ncell"], 0.5, 0.0, 1.0)
    want = np.stack([orc.coarsen(f, SMALL["n_coarse"]) for f in (dens, mom, sec)])
    assert np.allclose(got[:2], want[:2], rtol=1e-5, atol=1e-5 * np.abs(want).max())
    # the second moment's fixed point resolves 2^-s_e per particle (v_cap^2 = 1024 of headroom):
    # here s_e = 17, i.e. 2e-3 of a typical w V^2, random over the ~256 ions of a node
    assert np.max(np.abs(got[2] - want[2])) < 1e-4 * np.abs(want[2]).max()
    assert ctx.sync_status() == 0


@pytest.mark.parametrize("wavelet", ["haar", "coif4"])
def test_two_macro_steps_with_lift_match_oracle(wavelet):
    cfg = SMALL
    ctx = make_ctx(cfg, seed=17, wavelet=wavelet)
    ctx.load_initial(cfg["amp"])
    ctx.step()
    got1 = ctx.get_coarse().cpu().numpy()
    ctx.step()  # lifts at the local temperature of the projected state
    got2 = ctx.get_coarse().cpu().numpy()
    assert ctx.sync_status() == 0
    d = ctx.diagnostics()
    assert d.macro_steps == 2
    ocfg = dict(cfg, s_w=d.s_w, dT=cfg["M"] * cfg["K"] * cfg["dt"], wavelet=wavelet)
    c1, _, phi = orc.efpi_macro_step_pressure(oracle_state(cfg, 17), ocfg, np.zeros(cfg["ncell"]))
    assert np.max(np.abs(got1 - c1)) < 1e-4 * np.max(np.abs(c1))
    # lifting seed of macro step m: seed + 0x632BE59BD9B4E019 (m + 1)
    seed2 = (17 + 0x632BE59BD9B4E019 * 2) % 2**64
    st = orc.lift_pressure(c1, ocfg, seed2)
    c2, _, _ = orc.efpi_macro_step_pressure(st, ocfg, phi)
    assert np.max(np.abs(got2 - c2)) < 2e-4 * np.max(np.abs(c2))


def test_projection_conserves_charge_and_checkpoint_restores():
    cfg = SMALL
    ctx = make_ctx(cfg, seed=4)
    ctx.load_initial(cfg["amp"])
    c0 = ctx.get_coarse().cpu().numpy()
    ctx.step()
    c1 = ctx.get_coarse().cpu().numpy()
    # Haar: the density's coefficient sum is the charge; the least-squares weights sum to zero
    assert abs(c1[0].sum() - c0[0].sum()) < 1e-6 * abs(c0[0].sum())
    img = ctx.checkpoint()
    ctx.step()
    c2 = ctx.get_coarse().cpu().numpy()
    ctx.restore(img)
    ctx.step()
    assert np.array_equal(ctx.get_coarse().cpu().numpy(), c2)
    assert ctx.sync_status() == 0
