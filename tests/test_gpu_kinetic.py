"""GPU parity of the kinetic-electron path (Section 4.1: both species are particles in the
PIC bursts, q_e/m_e = -1800; the field is the periodic Poisson equation for the net charge)
against the oracle: the Poisson kernel, the Boltzmann electrons of a load, plain two-species
PIC with and without the periodic electron reset, and a projective macro step.

Tolerances: the Poisson solve agrees to FP64 summation-order rounding (1e-10 of max |E|);
particle states after a few FP32 steps to 1e-4 of a cell and of the thermal speed; coarse
states to 1e-4 of their largest entry (the fixed-point samples against the FP64 oracle)."""
import numpy as np
import pytest
import torch

import oracle as orc
import paper_1610_01071_gb300 as pe

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
QM_E = -1800.0
V_TH_E = float(np.float32(np.sqrt(-QM_E)))
MASK64 = 0xFFFFFFFFFFFFFFFF

KIN = dict(ncell=64, L=18.0, N=64 * 64, dt=0.25 / np.sqrt(-QM_E), K=6, M=5, n_coarse=16, v_th=0.22, amp=0.2)


def electron_seed(s):
    return (s & MASK64) ^ 0xD1B54A32D192ED03


@pytest.mark.parametrize("ncell", [8, 64, 1024, 8192])
@pytest.mark.parametrize("neutral", [True, False])
def test_field_kinetic_matches_oracle(ncell, neutral):
    rng = np.random.default_rng(ncell + neutral)
    s_w = 30
    base = (1.0 + 0.3 * np.cos(2 * np.pi * np.arange(ncell) / ncell)) * 2.0 ** (s_w + 24 - 6)
    rho_i = np.round(base * (1 + 0.05 * rng.normal(size=ncell))).astype(np.int64)
    rho_e = np.round(base * (1 + 0.05 * rng.normal(size=ncell))).astype(np.int64) if neutral else np.zeros(
        ncell, np.int64)
    dx = 0.37
    phi, E, Ef = pe.field_kinetic(torch.from_numpy(rho_i).to(DEV), torch.from_numpy(rho_e).to(DEV), ncell, dx, s_w)
    torch.cuda.synchronize()
    r = (rho_i - rho_e).astype(np.float64) * 2.0 ** -(s_w + 24)
    phi_o, E_o = orc.poisson_periodic(r, dx)
    E, phi = E.cpu().numpy(), phi.cpu().numpy()
    assert np.abs(E - E_o).max() <= 1e-10 * np.abs(E_o).max()
    assert np.abs(phi - phi_o).max() <= 1e-10 * np.abs(phi_o).max()
    assert np.array_equal(Ef.cpu().numpy(), E.astype(np.float32))


def test_field_kinetic_rejects_bad_sizes():
    z = torch.zeros(12, dtype=torch.int64, device=DEV)
    with pytest.raises(pe.PepicError):
        pe.field_kinetic(z, z, 12, 0.5, 30)
    z = torch.zeros(16384, dtype=torch.int64, device=DEV)
    with pytest.raises(pe.PepicError):
        pe.field_kinetic(z, z, 16384, 0.5, 30)


def test_boltzmann_profile_is_exp_phi_with_the_ions_drift():
    phi = torch.linspace(-3.0, 2.0, 512, dtype=torch.float64, device=DEV)
    prof = pe.boltzmann_profile(phi, 512).cpu().numpy()
    want = np.exp(phi.cpu().numpy())
    assert np.allclose(prof[0], want, rtol=2e-7, atol=0)
    assert not prof[1].any()  # no ion moments: no drift
    # V_e = V_i = m 2^-s_p / (n 2^-s_w) where the ion density is positive, 0 elsewhere
    rng = np.random.default_rng(2)
    s_w, s_p = 30, 27
    n = rng.integers(0, 2**40, 512)
    n[::7] = 0
    u = rng.normal(size=512) * 0.3
    m = np.round(u * n * 2.0 ** (s_p - s_w)).astype(np.int64)
    mom = torch.from_numpy(np.concatenate([n, m]).astype(np.int64)).to(DEV)
    prof = pe.boltzmann_profile(phi, 512, mom, s_w, s_p).cpu().numpy()
    want_u = np.where(n > 0, m / np.where(n > 0, n, 1) * 2.0 ** (s_w - s_p), 0.0)
    assert np.allclose(prof[1], want_u.astype(np.float32), rtol=1e-6, atol=0)
    assert not prof[1][::7].any()


def make_kinetic(cfg, seed, **kw):
    dT = cfg["M"] * cfg["K"] * cfg["dt"]
    c = pe.make_config(cfg["ncell"], cfg["n_coarse"], cfg["K"], cfg["N"], cfg["L"], cfg["dt"], dT, qm=1.0,
                       v_th=cfg["v_th"], seed=seed, newton_tol=1e-11, electrons="kinetic", **kw)
    return pe.Context(c, device=DEV)


def oracle_ions(cfg, seed):
    nprof, uprof = orc.sine_profile(cfg["ncell"], cfg["L"], cfg["amp"])
    return orc.quiet_start(cfg["N"], cfg["ncell"], nprof.astype(np.float32), uprof.astype(np.float32),
                           float(np.float32(cfg["v_th"])), seed)


def oracle_electrons(cfg, ions, s_w, seed, u=None):
    # the loading of the library: Poisson-Boltzmann potential of the ion deposit, then the
    # quiet start on the FP32 profiles exp(phi) and the ions' mean velocity (V_e = V_i): the
    # given lifting profile u, else the ion particles' nodal mean velocity (a plain-PIC reset)
    ncell = cfg["ncell"]
    dx = cfg["L"] / ncell
    dens = orc.deposit_fx(ions.cell, ions.theta, ions.w, ncell, s_w) * 2.0 ** -(s_w + 24)
    phi = orc.newton_pb(dens, dx, phi0=np.zeros(ncell), tol=1e-11)[0]
    prof = np.exp(phi).astype(np.float32)
    if u is None:
        u = orc.ion_mean_velocity(ions, ncell)
    return orc.quiet_start(cfg["N"], ncell, prof, np.asarray(u).astype(np.float32), V_TH_E, seed)


def sine_u(cfg):
    return orc.sine_profile(cfg["ncell"], cfg["L"], cfg["amp"])[1]


def state_of(ctx, species):
    c, t, v, w = (a.cpu().numpy() for a in ctx.particles(species=species))
    return orc.State(c, t, v, w)


def assert_states_close(got, want, ncell, v_scale, what):
    d = (got.cell + got.theta.astype(np.float64)) - (want.cell + want.theta)
    d = (d + ncell / 2) % ncell - ncell / 2  # periodic distance in cells
    assert np.abs(d).max() < 1e-4, f"{what}: position {np.abs(d).max()} cells"
    assert np.abs(got.v - want.v).max() < 1e-4 * v_scale, f"{what}: velocity {np.abs(got.v - want.v).max()}"
    assert np.allclose(got.w, want.w, rtol=1e-6, atol=0), what


def test_load_places_boltzmann_electrons_like_the_oracle():
    cfg = KIN
    ctx = make_kinetic(cfg, seed=3)
    ctx.load_initial(cfg["amp"])
    assert ctx.sync_status() == 0
    d = ctx.diagnostics()
    ions = oracle_ions(cfg, 3)
    elec = oracle_electrons(cfg, ions, d.s_w, electron_seed(3), u=sine_u(cfg))
    gi, ge = state_of(ctx, "ions"), state_of(ctx, "electrons")
    assert np.array_equal(gi.cell, ions.cell) and np.array_equal(ge.cell, elec.cell)
    assert np.array_equal(ge.theta, elec.theta.astype(np.float32))
    assert_states_close(ge, elec, cfg["ncell"], V_TH_E, "electrons")
    assert d.e_v_at_integer == 1
    # the loaded electrons balance the ions' charge (fixed point: to the rounding of each weight)
    rho_i = ctx.view("rho", torch.int64, cfg["ncell"]).cpu().numpy()
    rho_e = ctx.view("rho_e", torch.int64, cfg["ncell"]).cpu().numpy()
    total = float(rho_i.sum(dtype=object))
    assert abs(float(rho_e.sum(dtype=object)) - total) <= 1e-6 * total


@pytest.mark.parametrize("reset_every", [0, 4])
def test_plain_two_species_pic_matches_oracle(reset_every):
    cfg = KIN
    nsteps = 9
    seed = 5
    ctx = make_kinetic(cfg, seed=seed, reset_every=reset_every)
    ctx.load_initial(cfg["amp"])
    ctx.pic_steps(nsteps)
    assert ctx.sync_status() == 0
    d = ctx.diagnostics()
    s_w = d.s_w
    ncell, dx = cfg["ncell"], cfg["L"] / cfg["ncell"]
    ions = oracle_ions(cfg, seed)
    elec = oracle_electrons(cfg, ions, s_w, electron_seed(seed), u=sine_u(cfg))
    done, v_int, e_int = 0, True, True
    while done < nsteps:
        if reset_every and done > 0 and done % reset_every == 0:
            # Section 4.1's reset: electrons reloaded in equilibrium with the current ions
            elec = oracle_electrons(cfg, ions, s_w, electron_seed(seed + 0x9E3779B97F4A7C15 * done))
            e_int = True
        n = min(nsteps - done, reset_every - done % reset_every if reset_every else nsteps)
        orc.pic_steps_kinetic(ions, elec, ncell, dx, cfg["dt"], 1.0, QM_E, n, s_w, vel_at_integer=v_int,
                              e_vel_at_integer=e_int)
        done += n
        v_int = e_int = False
    assert_states_close(state_of(ctx, "ions"), ions, ncell, cfg["v_th"], "ions")
    assert_states_close(state_of(ctx, "electrons"), elec, ncell, V_TH_E, "electrons")


def test_kinetic_macro_step_matches_oracle():
    cfg = KIN
    seed = 7
    ctx = make_kinetic(cfg, seed=seed)
    ctx.load_initial(cfg["amp"])
    ctx.step()
    assert ctx.sync_status() == 0
    got = ctx.get_coarse().cpu().numpy()
    d = ctx.diagnostics()
    ncell, nc, K = cfg["ncell"], cfg["n_coarse"], cfg["K"]
    dx = cfg["L"] / ncell
    dT = cfg["M"] * K * cfg["dt"]
    ions = oracle_ions(cfg, seed)
    elec = oracle_electrons(cfg, ions, d.s_w, electron_seed(seed), u=sine_u(cfg))
    samples, _ = orc.burst_kinetic(ions, elec, ncell, dx, cfg["dt"], 1.0, QM_E, K, dT, d.s_w)
    cs = np.stack([np.concatenate([orc.coarsen(samples[p, 0], nc), orc.coarsen(samples[p, 1], nc)])
                   for p in range(K + 1)])
    coarse, _ = orc.ls_project(cs, cfg["dt"], dT)
    want = coarse.reshape(2, nc)
    assert np.max(np.abs(got - want)) < 1e-4 * np.max(np.abs(want))
    # after the burst both species moved K steps: compare the particle states too
    assert_states_close(state_of(ctx, "ions"), ions, ncell, cfg["v_th"], "ions")
    assert_states_close(state_of(ctx, "electrons"), elec, ncell, V_TH_E, "electrons")


def test_kinetic_lift_reloads_boltzmann_electrons():
    cfg = KIN
    ctx = make_kinetic(cfg, seed=11)
    ctx.load_initial(cfg["amp"])
    ctx.step()
    coarse = ctx.get_coarse().cpu().numpy()
    ctx.lift()
    assert ctx.sync_status() == 0
    d = ctx.diagnostics()
    assert d.e_v_at_integer == 1 and d.v_at_integer == 1
    gi = state_of(ctx, "ions")
    # electrons in equilibrium with the lifted ions (the GPU's own lifted ions as input), drifting
    # with the lifting profile's velocity u = m / n of the refined coarse state
    ncell = cfg["ncell"]
    _, u = orc.lift_profile(orc.refine(coarse[0], ncell), orc.refine(coarse[1], ncell))
    lift_seed = (11 + 0x632BE59BD9B4E019 * (d.macro_steps + 1)) & MASK64
    elec = oracle_electrons(cfg, gi, d.s_w, electron_seed(lift_seed), u=u)
    assert_states_close(state_of(ctx, "electrons"), elec, ncell, V_TH_E, "electrons")


def test_ps_mean_velocity_matches_oracle():
    rng = np.random.default_rng(4)
    nxc, nv, b = 64, 32, 2
    p = rng.uniform(0.0, 1.0, (nxc, nv))
    cdf = np.concatenate([np.zeros((nxc, 1)), np.cumsum(p, axis=1) / p.sum(axis=1, keepdims=True)], axis=1)
    got = pe._binding.ps_mean_velocity(torch.from_numpy(cdf).to(DEV), -3.0, 6.0 / nv, b, nxc << b).cpu().numpy()
    want = orc.ps_mean_velocity(cdf, -3.0, 6.0 / nv, b, nxc << b)
    assert np.allclose(got, want.astype(np.float32), rtol=2e-6, atol=1e-7)
    # a symmetric distribution has no drift; all mass in one cell drifts at its centre
    sym = np.linspace(0, 1, nv + 1)[None, :].repeat(nxc, 0)
    assert np.abs(pe._binding.ps_mean_velocity(torch.from_numpy(sym).to(DEV), -3.0, 6.0 / nv, b,
                                               nxc << b).cpu().numpy()).max() < 1e-6
    one = np.zeros((nxc, nv + 1))
    one[:, 10:] = 1.0
    u1 = pe._binding.ps_mean_velocity(torch.from_numpy(one).to(DEV), -3.0, 6.0 / nv, b, nxc << b).cpu().numpy()
    assert np.allclose(u1, -3.0 + 9.5 * 6.0 / nv, atol=1e-6)


def test_phase_space_lift_gives_the_electrons_the_ions_drift():
    cfg = KIN
    dT = cfg["M"] * cfg["K"] * cfg["dt"]
    c = pe.make_config(cfg["ncell"], cfg["n_coarse"], cfg["K"], cfg["N"], cfg["L"], cfg["dt"], dT, qm=1.0,
                       v_th=cfg["v_th"], seed=12, newton_tol=1e-11, electrons="kinetic", coarse="phase_space",
                       n_v=32, v_max=2.0, ps_filter=3)
    ctx = pe.Context(c, device=DEV)
    ctx.load_initial(cfg["amp"])
    ctx.step()
    ctx.lift()
    assert ctx.sync_status() == 0
    d = ctx.diagnostics()
    gi = state_of(ctx, "ions")
    ncell, nc, nv = cfg["ncell"], cfg["n_coarse"], 32
    # V_e = V_i from the lifted phase-space tables: the library's reconstructed CDF rows (in the
    # phase buffer after the bin masses) through the oracle's mean velocity
    off = ((8 * nc + 255) // 256) * 256 // 8
    cdf = ctx.view("phase", torch.float64)[off:off + nc * (nv + 1)].cpu().numpy().reshape(nc, nv + 1)
    u = orc.ps_mean_velocity(cdf, -2.0, 4.0 / nv, 2, ncell)
    lift_seed = (12 + 0x632BE59BD9B4E019 * (d.macro_steps + 1)) & MASK64
    elec = oracle_electrons(cfg, gi, d.s_w, electron_seed(lift_seed), u=u)
    assert_states_close(state_of(ctx, "electrons"), elec, ncell, V_TH_E, "electrons")
    assert np.abs(u).max() > 0.05  # the ion wave's drift is there to be carried


def test_kinetic_contexts_are_not_batched():
    c = pe.make_config(64, 16, 4, 64 * 16, 32.0, 0.005, 0.1, electrons="kinetic")
    ctx = pe.Context(c, device=DEV)
    with pytest.raises(pe.PepicError):  # the batched ensemble runs Boltzmann electrons only
        pe.Batch([ctx])


def test_kinetic_diagnostics_cover_both_species_and_conserve_energy():
    cfg = KIN
    ctx = make_kinetic(cfg, seed=13)
    ctx.load_initial(cfg["amp"])
    m0 = ctx.moments()
    dx = cfg["L"] / cfg["ncell"]
    ge = state_of(ctx, "electrons")  # velocities at integer time after the load
    ke = 0.5 * np.sum(ge.w * ge.v**2) * dx / -QM_E
    assert m0["electron_energy"] == pytest.approx(ke, rel=1e-5)
    assert m0["total_energy"] == pytest.approx(m0["kinetic"] + m0["field_energy"] + m0["electron_energy"], rel=1e-12)
    assert m0["cfl"] >= np.abs(ge.v).max() * cfg["dt"] / dx * (1 - 1e-6)  # the electrons set it
    assert m0["invalid"] == 0
    ctx.pic_steps(40)
    m1 = ctx.moments()
    assert ctx.sync_status() == 0
    # the two-species system conserves energy up to the slow heating of explicit PIC, and its
    # momentum (ions plus electrons of mass w / |q_e/m_e|) up to the fixed-point deposit
    assert abs(m1["total_energy"] - m0["total_energy"]) < 1e-3 * m0["total_energy"]
    assert abs(m1["momentum"] - m0["momentum"]) < 1e-4 * cfg["L"] * cfg["amp"]


def test_kinetic_full_size_properties():
    # the bench's iaw_kinetic workload at full size (2^23 ions + 2^23 electrons, 1024 cells):
    # both species' fixed-point charge is conserved exactly through pushes and sorts, the field
    # of the actual deposits matches the oracle's Poisson solve, and macro steps run clean
    from paper_1610_01071_gb300 import inputs

    w = inputs.workload("iaw_kinetic")
    c = pe.make_config(w["ncell"], w["n_coarse"], w["K"], w["N"], w["L"], w["dt"], w["dT"], qm=w["qm"],
                       v_th=w["v_th"], seed=11, sort_every=20, newton_tol=1e-10, coarse="phase_space", n_v=w["n_v"],
                       v_max=w["v_max"], ps_filter=3, electrons="kinetic", qm_e=w["qm_e"])
    ctx = pe.Context(c, device=DEV)
    ctx.load_initial(w["amplitude"])
    ncell = w["ncell"]

    def charge(name):
        return int(ctx.view(name, torch.int64, ncell).cpu().numpy().sum(dtype=object))

    qi0, qe0 = charge("rho"), charge("rho_e")
    assert abs(qe0 - qi0) <= 1e-6 * qi0  # the Boltzmann electrons balance the ions
    m0 = ctx.moments()
    ctx.pic_steps(45)  # crosses two sorts
    assert ctx.sync_status() == 0
    assert (charge("rho"), charge("rho_e")) == (qi0, qe0)
    m1 = ctx.moments()
    assert abs(m1["total_energy"] - m0["total_energy"]) < 1e-3 * m0["total_energy"]
    s_w = ctx.diagnostics().s_w
    rho_i = ctx.view("rho", torch.int64, ncell).cpu().numpy()
    rho_e = ctx.view("rho_e", torch.int64, ncell).cpu().numpy()
    _, E_o = orc.poisson_periodic((rho_i - rho_e).astype(np.float64) * 2.0 ** -(s_w + 24), w["L"] / ncell)
    E = ctx.view("E", torch.float64, ncell).cpu().numpy()
    assert np.abs(E - E_o).max() <= 1e-10 * np.abs(E_o).max()
    ctx.step()
    ctx.step()
    assert ctx.sync_status() == 0
    assert np.all(np.isfinite(ctx.get_coarse().cpu().numpy()))


def test_electron_energy_is_sampled_projected_and_lifted():
    """The electrons' kinetic energy as a global active variable (Section 4.2; te_active): the
    burst samples it at every step (the oracle's energy of the same two-species trajectory,
    1e-5), the leap projects it by the least-squares rule (1e-12 on the sampled values), and
    the lift loads the electrons at T_e = projected / initial energy: their potential solves
    -T_e psi'' + e^psi = n_i and their energy is the projected one to the quiet start's
    quadrature (2e-3). A checkpoint keeps the temperature state."""
    cfg = KIN
    seed = 13
    ncell, K = cfg["ncell"], cfg["K"]
    dx, dt = cfg["L"] / ncell, cfg["dt"]
    dT = cfg["M"] * K * dt
    ctx = make_kinetic(cfg, seed=seed, te_active=True)
    ctx.load_initial(cfg["amp"])
    d0 = ctx.diagnostics()
    assert d0.T_e == 1.0
    ions = oracle_ions(cfg, seed)
    elec = oracle_electrons(cfg, ions, d0.s_w, electron_seed(seed), u=sine_u(cfg))
    W0 = orc.electron_kinetic_energy(elec, np.zeros(ncell), ncell, dx, dt, QM_E, 0.5)
    assert d0.W_e == pytest.approx(W0, rel=1e-5)
    ctx.step()
    assert ctx.sync_status() == 0
    we = ctx.view("rho_e", torch.float64).cpu().numpy()[3 * ncell:3 * ncell + K + 4]
    want = []
    for p in range(K + 1):
        _, E = orc.field_kinetic(ions, elec, ncell, dx, d0.s_w)
        want.append(orc.electron_kinetic_energy(elec, E, ncell, dx, dt, QM_E, 0.5 if p == 0 else 1.0))
        if p < K:
            orc.pic_steps_kinetic(ions, elec, ncell, dx, dt, 1.0, QM_E, 1, d0.s_w, vel_at_integer=(p == 0))
    np.testing.assert_allclose(we[:K + 1], want, rtol=1e-5)
    proj, _ = orc.ls_project(we[:K + 1].reshape(K + 1, 1), dt, dT)
    assert we[K + 2] == pytest.approx(proj[0], rel=1e-12)
    ctx.lift()
    assert ctx.sync_status() == 0
    d = ctx.diagnostics()
    assert d.T_e == pytest.approx(we[K + 2] / d0.W_e, rel=1e-12) and d.W_e == we[K + 2]
    psi = ctx.view("phi", torch.float64, ncell).cpu().numpy()
    gi = state_of(ctx, "ions")
    n_i = orc.deposit_fx(gi.cell, gi.theta.astype(np.float64), gi.w.astype(np.float64), ncell, d.s_w) * 2.0 ** -(
        d.s_w + 24)
    lap = (np.roll(psi, -1) - 2 * psi + np.roll(psi, 1)) / dx ** 2
    assert np.max(np.abs(-d.T_e * lap + np.exp(psi) - n_i)) < 1e-6 * np.max(n_i)
    We = orc.electron_kinetic_energy(state_of(ctx, "electrons"), np.zeros(ncell), ncell, dx, dt, QM_E, 0.5)
    assert We == pytest.approx(we[K + 2], rel=2e-3)
    ctx.step()  # a checkpoint holds a coarse state: the one after a projection
    img = ctx.checkpoint()
    ctx2 = make_kinetic(cfg, seed=seed, te_active=True)
    ctx2.restore(img)
    ctx.lift()
    ctx2.lift()
    assert ctx.diagnostics().T_e == ctx2.diagnostics().T_e
    assert ctx.sync_status() == 0 and ctx2.sync_status() == 0
