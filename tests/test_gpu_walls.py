"""GPU parity of the bounded-grid path (Section 4.2's slab expansion: absorbing walls at
nodes 0 and ncell-1, phi' = 0 there) against the FP64 CPU oracle, through the C ABI.

Tolerances (stated per result):
  field solve (FP64 linear solve) ... phi within 1e-9 absolute, E within 1e-8 of max|E|
  push ............................... positions within 1e-5 cell, velocities 1e-5 relative;
                                       the absorbed set equal except for ions whose FP64 end
                                       point lies within 1e-4 cell of a wall
  restriction sample ................. within 1e-4 of the sample's max
  equal-weight loading ............... positions within 2e-6 cell (FP32 offset), weights 1e-7
                                       relative, velocities 2e-5 absolute; deposit bit-exact
                                       against pe_deposit of the loaded particles
  charge accounting .................. exact (integers)
"""
import numpy as np
import pytest
import torch

import oracle as orc
import paper_1610_01071_gb300 as pe
from paper_1610_01071_gb300 import _binding as pb
from paper_1610_01071_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def to_dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in arrs]


def status_word():
    return torch.zeros(1, dtype=torch.int32, device=DEV)


def _slab_dep(ncell, s_w, N=None, seed=0):
    n, u = orc.slab_profile(ncell)
    st = orc.quiet_start_equal(N or 64 * ncell, ncell, n, u, 1.0, seed)
    return orc.deposit_fx(st.cell, st.theta, st.w, ncell, s_w), st


@pytest.mark.parametrize("ncell,mode", [(64, "boltzmann"), (512, "boltzmann"), (2048, "linearized"),
                                        (8192, "boltzmann")])
def test_field_walls_matches_oracle(ncell, mode):
    dx, s_w = 0.5, 24
    rho, _ = _slab_dep(ncell, s_w, N=16 * ncell)
    m = 1 if mode == "linearized" else 0
    dep = rho * 2.0 ** -(s_w + 24)
    phi_o, _, fail = orc.newton_pb_walls(dep, dx, phi0=np.zeros(ncell), mode=m, tol=1e-12, maxit=80)
    assert fail == 0
    E_o = orc.efield_walls(phi_o, dx)
    phi = torch.zeros(ncell, dtype=torch.float64, device=DEV)
    st = status_word()
    E, Ef, diag = pe.field(*to_dev(rho), ncell, dx, s_w, phi, mode=mode, tol=1e-12, maxit=80, status=st,
                           boundary="absorbing")
    assert int(st.item()) == 0 and int(diag[1]) == 1
    assert np.max(np.abs(phi.cpu().numpy() - phi_o)) < 1e-9
    assert np.max(np.abs(E.cpu().numpy() - E_o)) < 1e-8 * np.max(np.abs(E_o))
    e = E.cpu().numpy()
    assert e[0] == 0.0 and e[-1] == 0.0
    if ncell >= 2048 and m == 0:
        # the vacuum potential is far below the plasma's: the ill-conditioned solve (FP64 needed)
        assert phi_o[0] < -10.0


def test_field_walls_manufactured_cosine_on_gpu():
    ncell, dx = 4096, 0.5
    j = np.arange(ncell)
    a1, a2 = np.pi * 3 / (ncell - 1), np.pi * 11 / (ncell - 1)
    phi_star = 0.6 * np.cos(a1 * j) + 0.25 * np.cos(a2 * j)
    K1, K2 = (2 / dx * np.sin(a1 / 2)) ** 2, (2 / dx * np.sin(a2 / 2)) ** 2
    dens = K1 * 0.6 * np.cos(a1 * j) + K2 * 0.25 * np.cos(a2 * j) + np.exp(phi_star)
    dep = dens.copy()
    dep[[0, -1]] *= 0.5
    s_w = 20
    rho = np.rint(dep * 2.0 ** (s_w + 24)).astype(np.int64)
    phi = torch.zeros(ncell, dtype=torch.float64, device=DEV)
    pe.field(*to_dev(rho), ncell, dx, s_w, phi, tol=1e-13, boundary="absorbing")
    assert np.max(np.abs(phi.cpu().numpy() - phi_star)) < 1e-10


def _bounded_particles(N, ncell, seed, v_scale=1.0):
    c, t, v, w = inputs.random_particles(N, ncell - 1, seed=seed)  # cells 0 .. ncell-2
    return c, t, (v * v_scale).astype(np.float32), w


@pytest.mark.parametrize("ncell,N,kick", [(64, 4099, 0.5), (512, (1 << 16) + 2, 1.0), (8192, 1 << 20, 1.0)])
def test_push_walls_matches_oracle(ncell, N, kick):
    dx, dt, qm = 0.5, 0.1, 1.0
    c, t, v, w = _bounded_particles(N, ncell, seed=ncell + 1, v_scale=min(2.0 * ncell / 64, 16.0))
    w[::13] = 0.0  # already absorbed: frozen
    s_w = orc.fx_shift(4.0 * ncell / N)
    E = inputs.random_field(ncell, seed=3, amp=0.1)
    E[[0, -1]] = 0.0
    Ef = E.astype(np.float32)
    dc, dt_, dv, dw, dEf = to_dev(c, t, v, w, Ef)
    st = status_word()
    rho = pe.push(dc, dt_, dv, dw, dEf, ncell, dt / dx, qm * dt, kick, s_w, status=st, boundary="absorbing")
    so = orc.State(c, t, v, w)
    orc.push_walls(so, Ef.astype(np.float64), ncell, dx, dt, qm, kick=kick)
    gc, gt, gv, gw = (x.cpu().numpy() for x in (dc, dt_, dv, dw))
    assert int(st.item()) == 0
    Xo = so.cell + so.theta
    # FP64 end points of the live ions, to find the borderline ones near the walls
    vo = v.astype(np.float64) + kick * qm * dt * orc.gather(Ef.astype(np.float64), c, t)
    Xend = c + t.astype(np.float64) + vo * dt / dx
    border = (np.abs(Xend) < 1e-4) | (np.abs(Xend - (ncell - 1)) < 1e-4)
    ok = ~border
    assert np.array_equal((gw == 0)[ok], (so.w == 0)[ok])
    absorbed = (so.w == 0) & (w > 0)
    assert absorbed.sum() > 10
    live = (so.w > 0) & ok
    assert np.max(np.abs((gc + gt)[live] - Xo[live])) < 1e-5
    assert np.max(np.abs(gv[live] - so.v[live]) / np.maximum(1.0, np.abs(so.v[live]))) < 1e-5
    dead = (gw == 0)
    assert np.all(gv[dead & (w > 0)] == 0) and np.all(gt[dead & (w > 0)] == 0)
    assert np.all(np.isin(gc[dead & (w > 0)], [0, ncell - 1]))
    frozen = w == 0
    assert np.array_equal(gc[frozen], c[frozen]) and np.array_equal(gt[frozen], t[frozen])
    assert np.all((gc[gw > 0] >= 0) & (gc[gw > 0] < ncell - 1))
    # fused deposit = deposit of the pushed state, charge = the live ions' fixed-point weights
    assert torch.equal(rho, pe.deposit(dc, dt_, dw, ncell, s_w))
    wq = np.rint(gw.astype(np.float64) * 2.0**s_w).astype(np.int64)
    total = int(np.sum(rho.cpu().numpy().astype(object)))  # exact: the int64 sum can exceed 2^63
    assert total == int(wq.sum()) << 24


@pytest.mark.parametrize("tau", [0.0, 5.0, 24.0])
def test_sample_walls_matches_oracle(tau):
    ncell, N, dx, dt, qm = 256, 1 << 16, 0.5, 0.1, 1.0
    c, t, v, w = _bounded_particles(N, ncell, seed=31, v_scale=3.0)
    w[::11] = 0.0
    s_w = orc.fx_shift(4.0 * ncell / N)
    s_p = orc.fx_shift(4.0 * ncell / N * 32.0)
    E = inputs.random_field(ncell, seed=4, amp=0.05)
    E0 = inputs.random_field(ncell, seed=5, amp=0.05)
    dc, dt_, dv, dw = to_dev(c, t, v, w)
    Ef, E0f = to_dev(E.astype(np.float32), E0.astype(np.float32))
    out = torch.empty(2 * ncell, dtype=torch.int64, device=DEV)
    args = pe.make_sample_args(E0f, tau, qm, 1 / dx, s_w, s_p, out, boundary="absorbing")
    pe.sample(dc, dt_, dv, dw, Ef, ncell, qm * dt, 1.0, args)
    so = orc.State(c, t, v, w)
    Eo = E.astype(np.float32).astype(np.float64)
    vbar = so.v + 0.5 * qm * dt * orc.gather(Eo, c, t)
    dens, mom = orc.restrict_sample_walls(so, vbar, E0.astype(np.float32).astype(np.float64), ncell, dx, tau, qm)
    g = out.cpu().numpy()
    gd, gm = g[:ncell] * 2.0 ** -(s_w + 24), g[ncell:] * 2.0 ** -(s_p + 24)
    assert np.max(np.abs(gd - dens)) < 1e-4 * np.max(np.abs(dens))
    assert np.max(np.abs(gm - mom)) < 1e-4 * np.max(np.abs(mom))
    if tau > 0:
        assert dens.sum() < 0.95 * (w.astype(np.float64).sum())  # the walls removed a part
    for b in (2, 5):  # binned Haar form: exact bin sums of the nodal sample
        outb = torch.empty(2 * (ncell >> b), dtype=torch.int64, device=DEV)
        argb = pe.make_sample_args(E0f, tau, qm, 1 / dx, s_w, s_p, outb, bin_shift=b, boundary="absorbing")
        pe.sample(dc, dt_, dv, dw, Ef, ncell, qm * dt, 1.0, argb)
        assert np.array_equal(outb.cpu().numpy(), g.reshape(2, ncell >> b, 1 << b).sum(axis=-1).reshape(-1))


@pytest.mark.parametrize("ncell,N,profile", [(64, 6400, "slab"), (512, (1 << 16) + 3, "slab"),
                                             (256, 1 << 15, "cos"), (8192, 1 << 22, "slab")])
def test_quiet_start_equal_matches_oracle(ncell, N, profile):
    if profile == "slab":
        n, u = orc.slab_profile(ncell)
    else:
        j = np.arange(ncell)
        n = 1.0 + 0.5 * np.cos(np.pi * 2 * j / (ncell - 1))
        u = 0.2 * np.sin(np.pi * 2 * j / (ncell - 1))
    n32, u32 = n.astype(np.float32), u.astype(np.float32)
    seed = 77
    s_w = orc.fx_shift(4.0 * ncell / N)
    st = status_word()
    cell, theta, v, w, rho = pe.quiet_start_equal(N, ncell, *to_dev(n32, u32), 1.0, seed, s_w, status=st)
    so = orc.quiet_start_equal(N, ncell, n32.astype(np.float64), u32.astype(np.float64), 1.0, seed)
    gc, gt, gv, gw = (x.cpu().numpy() for x in (cell, theta, v, w))
    assert int(st.item()) == 0
    assert np.max(np.abs((gc + gt.astype(np.float64)) - (so.cell + so.theta))) < 2e-6 * max(1.0, ncell / 1024)
    assert np.all((gt >= 0) & (gt < 1)) and np.all((gc >= 0) & (gc < ncell - 1))
    blocks = gc[: (N // 4096) * 4096].reshape(-1, 4096)  # cells non-decreasing from block to block
    assert np.all(blocks.max(axis=1)[:-1] <= blocks.min(axis=1)[1:])
    assert np.allclose(gw, so.w, rtol=1e-7)
    assert np.max(np.abs(gv - so.v)) < 2e-5
    assert torch.equal(rho, pe.deposit(cell, theta, w, ncell, s_w))
    if profile == "slab":
        counts = np.bincount(gc, minlength=ncell)
        assert counts[: 7 * ncell // 16 - 1].sum() == 0 and counts[9 * ncell // 16 + 1:].sum() == 0


def test_quiet_start_equal_wall_factor_and_empty_profile():
    ncell, N = 128, 12800
    n = np.ones(ncell, np.float32)
    n[[0, -1]] = 0.5  # deposits at the walls: with wall factor 2 the profile is uniform
    cell, theta, _, w, _ = pe.quiet_start_equal(N, ncell, *to_dev(n, np.zeros(ncell, np.float32)), 0.0, 1, 20,
                                                wall_factor=2.0)
    X = cell.cpu().numpy() + theta.cpu().numpy().astype(np.float64)
    s = np.arange(N)
    full = (s | 4095) < N
    point = np.where(full, (s & ~4095) | sum(((s >> b) & 1) << (11 - b) for b in range(12)), s)
    assert np.allclose(X, (point + 0.5) / N * (ncell - 1), atol=2e-5)
    st = status_word()
    z = np.zeros(ncell, np.float32)
    cell, theta, _, w, rho = pe.quiet_start_equal(N, ncell, *to_dev(z, z), 1.0, 1, 20, status=st)
    assert int(st.item()) & 4  # no mass: flagged, weight-0 particles, no fault
    assert float(w.abs().sum()) == 0.0 and int(rho.abs().sum()) == 0


def _small_slab_cfg(**kw):
    c = dict(ncell=256, n_coarse=32, K=10, nparticles=256 * 128, L=128.0, dt=0.1, dT=4.0, v_th=1.0, seed=5,
             boundary="absorbing", newton_tol=1e-12, newton_maxit=80)
    c.update(kw)
    return pe.make_config(c.pop("ncell"), c.pop("n_coarse"), c.pop("K"), c.pop("nparticles"), c.pop("L"),
                          c.pop("dt"), c.pop("dT"), **c)


def _ctx_state(ctx):
    return [x.cpu().numpy() for x in ctx.particles()]


def test_context_slab_load_burst_matches_oracle():
    cfg = _small_slab_cfg()
    ctx = pe.Context(cfg, device=DEV)
    ctx.load_initial(profile="slab")
    c, t, v, w = _ctx_state(ctx)
    ncell, dx = 256, 0.5
    n, u = orc.slab_profile(ncell)
    so = orc.quiet_start_equal(256 * 128, ncell, n, u, 1.0, 5)
    assert np.max(np.abs((c + t.astype(np.float64)) - (so.cell + so.theta))) < 2e-6
    s_w = ctx.diagnostics().s_w
    st = orc.State(c, t, v, w)
    samples, phi, fails = orc.burst_walls(st, ncell, dx, 0.1, 1.0, 10, 4.0, s_w, np.zeros(ncell), tol=1e-12)
    assert fails == 0
    ctx.burst()
    assert ctx.sync_status() == 0
    b = 3  # Haar bins of 256 / 32 nodes: samples hold exact bin sums
    nb = ncell >> b
    gs = ctx.view("samples_fx", torch.int64, 11 * 2 * nb).cpu().numpy().reshape(11, 2, nb)
    for p in (0, 5, 10):
        want = samples[p, 0].reshape(-1, 1 << b).sum(axis=-1)
        got = gs[p, 0] * 2.0 ** -(s_w + 24)
        assert np.max(np.abs(got - want)) < 1e-4 * np.max(np.abs(want)), p
    c2, t2, v2, w2 = _ctx_state(ctx)
    live = st.w > 0
    assert np.max(np.abs((c2 + t2.astype(np.float64))[live] - (st.cell + st.theta)[live])) < 1e-4


def test_context_plain_pic_charge_accounting_and_absorption():
    cfg = _small_slab_cfg(v_th=4.0, sort_every=10)
    ctx = pe.Context(cfg, device=DEV)
    ctx.load_initial(profile="slab")
    m0 = ctx.moments()
    ctx.pic_steps(300)
    assert ctx.sync_status() == 0
    m1 = ctx.moments()
    c, t, v, w = _ctx_state(ctx)
    s_w = ctx.diagnostics().s_w
    dead = w == 0
    assert dead.sum() > 1000  # fast ions reached the walls
    # exact: initial charge = live charge + the absorbed ions' fixed-point weights
    wq_live = np.rint(w[~dead].astype(np.float64) * 2.0**s_w).astype(np.int64)
    assert m1["charge_fx"] == int(wq_live.sum()) << 24
    n_abs = int(dead.sum())
    wq_each = int(np.rint(np.float64(np.float32(w[~dead][0])) * 2.0**s_w))  # equal weights
    assert m0["charge_fx"] == m1["charge_fx"] + (n_abs * wq_each << 24)
    assert np.all(np.isin(c[dead], [0, 255])) and np.all(v[dead] == 0)
    assert np.all((c[~dead] >= 0) & (c[~dead] < 255))


def test_context_slab_projective_steps_follow_plain_pic():
    # projective steps on the bounded grid against the resolved run to the same time. The
    # moment closure lifts a Maxwellian of the fixed v_th at every macro step, which heats the
    # cold expanding front and drives ions to the walls early: the projective run loses charge
    # faster than the resolved one (measured: 26 % against 9 % by T = 20 here). The bounds
    # below only fence that known closure error; they are not an accuracy claim.
    cfg = _small_slab_cfg()
    ef, ref = pe.Context(cfg, device=DEV), pe.Context(cfg, device=DEV)
    ef.load_initial(profile="slab")
    ref.load_initial(profile="slab")
    q0 = ef.moments()["charge"]
    for _ in range(5):
        ef.step()
    ref.pic_steps(5 * 40)
    assert ef.sync_status() == 0 and ref.sync_status() == 0
    a = ef.get_coarse().cpu().numpy()[0]
    b = ref.measure().cpu().numpy()[0]
    eps = float(np.sqrt(np.sum((a - b) ** 2) / np.sum(a * a + b * b)))
    ef.lift()
    q_ef, q_ref = ef.moments()["charge"], ref.moments()["charge"]
    print(f"slab T=20: eps {eps:.4f}, charge left projective {q_ef / q0:.4f}, resolved {q_ref / q0:.4f}")
    assert np.all(np.isfinite(a))
    assert q_ref < q0 and q_ef < q0
    assert abs(q_ef - q_ref) < 0.3 * q0
    assert eps < 0.3


# ----------------------------------------------------------------- phase space on the bounded grid


@pytest.mark.parametrize("filt", [0, 1, 2, 3, 6, 7])
def test_ps_project_filters_match_oracle(filt):
    rng = np.random.default_rng(10 + filt)
    K, nxc, nv = 10, 32, 24
    y = rng.standard_normal((K + 1, nxc, nv))
    out, sl = pb.ps_project(*to_dev(y), 0.1, 4.0, filt)
    want, wsl = orc.ps_project(y, 0.1, 4.0, filt)
    assert np.allclose(sl.cpu().numpy(), wsl, rtol=1e-12, atol=1e-12)
    assert np.allclose(out.cpu().numpy(), want, rtol=1e-12, atol=1e-11)


def _ps_tables(nxc, nv, vmin, dv, seed):
    rng = np.random.default_rng(seed)
    x = (np.arange(nxc) + 0.5) / nxc
    vc = vmin + dv * (np.arange(nv) + 0.5)
    n = 8.0 * (1.0 + 0.6 * np.cos(np.pi * x)) * (x > 0.2)  # vacuum on the left
    H = n[:, None] * np.exp(-0.5 * ((vc[None, :] - 0.5 * np.sin(np.pi * x)[:, None]) / 0.8) ** 2) * dv
    H *= 1.0 + 0.05 * rng.standard_normal(H.shape)
    return H


@pytest.mark.parametrize("ncell,b,nv,N", [(64, 2, 16, 3 * 4096 + 6), (512, 4, 32, 1 << 16), (8192, 4, 64, 1 << 21)])
def test_ps_quiet_start_equal_matches_oracle(ncell, b, nv, N):
    nxc = ncell >> b
    vmin, dv = -6.0, 12.0 / nv
    H = _ps_tables(nxc, nv, vmin, dv, ncell)
    mass, cdf, table, _ = pb.ps_lift_tables(*to_dev(H))
    s_w = orc.fx_shift(4.0 * float(mass.sum()) / N)
    st = status_word()
    cell, theta, v, w, rho = pb.ps_quiet_start_equal(N, ncell, b, mass, table, vmin, dv, 99, s_w, status=st)
    so = orc.ps_quiet_start_equal(N, ncell, b, mass.cpu().numpy(), cdf.cpu().numpy(), vmin, dv, 99)
    gc, gt, gv, gw = (x.cpu().numpy() for x in (cell, theta, v, w))
    assert int(st.item()) == 0
    assert np.max(np.abs((gc + gt.astype(np.float64)) - (so.cell + so.theta))) < 2e-6 * max(1.0, ncell / 1024)
    assert np.all((gc >= 0) & (gc < ncell - 1)) and np.all((gt >= 0) & (gt < 1))
    assert np.allclose(gw, so.w, rtol=1e-7)
    # FP32 inversion inside a cell whose density vanishes at an edge (t ~ sqrt(r) there) moves
    # a few velocities by a fraction of a cell; typical differences are at the FP32 level
    dv_ = np.abs(gv - so.v)
    assert dv_.max() <= 0.2 * dv and dv_.mean() <= 2e-6 * 12.0
    assert np.sum(dv_ > 5e-5) <= max(3, 1e-4 * N)
    assert torch.equal(rho, pe.deposit(cell, theta, w, ncell, s_w))
    # equal weights, placed by mass: the vacuum bins receive no ions
    assert np.all(gc[gw > 0] >= int(0.2 * ncell) - (1 << b))


def _small_ps_slab_cfg(**kw):
    c = dict(ncell=256, n_coarse=32, K=10, nparticles=256 * 128, L=128.0, dt=0.1, dT=4.0, v_th=1.0, seed=5,
             boundary="absorbing", newton_tol=1e-12, newton_maxit=80, coarse="phase_space", n_v=32, v_max=8.0,
             ps_filter=3)
    c.update(kw)
    return pe.make_config(c.pop("ncell"), c.pop("n_coarse"), c.pop("K"), c.pop("nparticles"), c.pop("L"),
                          c.pop("dt"), c.pop("dT"), **c)


def test_context_ps_slab_burst_matches_oracle():
    cfg = _small_ps_slab_cfg()
    ctx = pe.Context(cfg, device=DEV)
    ctx.load_initial(profile="slab")
    c, t, v, w = _ctx_state(ctx)
    s_w = ctx.diagnostics().s_w
    st = orc.State(c, t, v, w)
    samples, phi, fails = orc.ps_burst_walls(st, 256, 0.5, 0.1, 1.0, 10, 4.0, s_w, np.zeros(256), 3, -8.0, 0.5, 32,
                                             tol=1e-12)
    assert fails == 0
    ctx.burst()
    assert ctx.sync_status() == 0
    got = ctx.view("samples_fx", torch.int64, 11 * 32 * 32).cpu().numpy().reshape(11, 32, 32)
    for p in (0, 5, 10):
        g, h = got[p].astype(np.float64), samples[p].astype(np.float64)
        assert int(got[p].astype(object).sum()) == pytest.approx(int(samples[p].astype(object).sum()), rel=1e-4)
        assert np.abs(g - h).sum() <= 2e-3 * h.sum(), p


def test_context_ps_slab_projective_steps_follow_plain_pic():
    # the phase-space variable on the bounded grid, against the resolved run at T = 20. The
    # co-moving restriction (Appendix B) carries each ion over tau = Delta t - p delta t <= 4
    # with the burst-start field at its position; at the expansion front that field is a spike,
    # so the projected velocities overshoot and the front reaches the walls early: with these
    # steps the oracle and the GPU keep 77 % of the charge against 91 % resolved (92 % without
    # a leap, Delta t = K delta t). The bounds fence that known error of the method here.
    cfg = _small_ps_slab_cfg()
    ef = pe.Context(cfg, device=DEV)
    ref = pe.Context(_small_slab_cfg(), device=DEV)
    ef.load_initial(profile="slab")
    ref.load_initial(profile="slab")
    q0 = ref.moments()["charge"]
    for _ in range(5):
        ef.step()
    ref.pic_steps(5 * 40)
    assert ef.sync_status() == 0 and ref.sync_status() == 0
    H = ef.get_coarse().cpu().numpy()  # [nxc, n_v] masses
    nb = 256 // 32
    dens = H.sum(axis=1) * 2.0 ** (-(np.log2(256) + 3) / 2)  # Haar density coefficient of each bin
    want = ref.measure().cpu().numpy()[0]
    eps = float(np.sqrt(np.sum((dens - want) ** 2) / np.sum(dens**2 + want**2)))
    ef.lift()
    q_ef, q_ref = ef.moments()["charge"], ref.moments()["charge"]
    print(f"slab phase space T=20: eps {eps:.4f}, charge left projective {q_ef / q0:.4f}, resolved {q_ref / q0:.4f}")
    assert np.all(np.isfinite(H)) and nb == 8
    assert q_ref < q0 and q_ef < q0
    assert abs(q_ef - q_ref) < 0.25 * q0
    assert eps < 0.3


def test_slab_full_size_properties():
    # the slab workload at its full size and in the benchmark's launch configuration (2^25 ions,
    # 8192 cells): properties that hold at any size, checked exactly
    w = inputs.workload("slab")
    cfg = pe.make_config(w["ncell"], w["n_coarse"], w["K"], w["N"], w["L"], w["dt"], w["dT"], v_th=w["v_th"], seed=21,
                         sort_every=20, newton_tol=1e-10, newton_maxit=80, boundary="absorbing")
    ctx = pe.Context(cfg, device=DEV)
    ctx.load_initial(profile="slab")
    ncell, N = w["ncell"], w["N"]
    cell, theta, v, wt = ctx.particles()
    # per-cell counts: particle i sits in cell c iff C_c <= (i + 1/2) M / N < C_{c+1} (FP64 profile)
    n, _ = orc.slab_profile(ncell)
    n = n.astype(np.float32).astype(np.float64)
    C = np.concatenate([[0.0], np.cumsum(0.5 * (n[:-1] + n[1:]))])
    M = C[-1]
    want = (np.ceil(C[1:] * N / M - 0.5) - np.ceil(C[:-1] * N / M - 0.5)).astype(np.int64)
    counts = torch.bincount(cell.long(), minlength=ncell).cpu().numpy()
    assert np.abs(counts[:-1] - want).max() <= 1 and counts.sum() == N and counts[-1] == 0
    ww = wt.cpu().numpy()
    assert np.all(ww == ww[0]) and ww[0] == np.float32(M / N)
    vv = v.cpu().numpy().astype(np.float64)
    assert abs(vv.mean()) < 1e-4 and vv.var() == pytest.approx(1.0, rel=1e-3)
    # plain steps with absorption: the live ions' fixed-point charge is the deposit, exactly
    m0 = ctx.moments()
    ctx.pic_steps(400)
    assert ctx.sync_status() == 0
    m1 = ctx.moments()
    wq = np.rint(ctx.particles()[3].cpu().numpy().astype(np.float64) * 2.0 ** ctx.diagnostics().s_w)
    # in weight units (the deposit units' total, sum w_q 2^24, exceeds 2^63 at this size)
    assert m1["charge_wq"] == int(wq.astype(np.int64).sum())
    assert m1["charge_wq"] <= m0["charge_wq"] and m1["invalid"] == 0
    wrapped = (((m0["charge_wq"] << 24) + (1 << 63)) % (1 << 64)) - (1 << 63)  # int64 two's complement
    assert m0["charge_fx"] == wrapped
