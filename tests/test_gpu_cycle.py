"""GPU parity of whole bursts, projective macro steps and plain PIC against the oracle
(context API of the C ABI).

Burst-level coarse moments must agree with the oracle within 3 sigma of the ensemble
sampling noise; sigma is estimated from oracle runs that differ only in the
quiet-start shift (seed). In practice the GPU and the oracle, started from the same
seed, agree far more closely (FP32 against FP64 trajectories); that tighter bound is
checked too.
"""
import numpy as np
import pytest
import torch

import oracle as orc
import paper_1610_01071_gb300 as pe

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")

SMALL = dict(ncell=128, L=64.0, N=128 * 256, dt=0.1, K=10, M=4, n_coarse=16, v_th=1.0, qm=1.0, amp=0.1)


def make_ctx(cfg, seed, **kw):
    dT = cfg["M"] * cfg["K"] * cfg["dt"]
    c = pe.make_config(cfg["ncell"], cfg["n_coarse"], cfg["K"], cfg["N"], cfg["L"], cfg["dt"], dT,
                       qm=cfg["qm"], v_th=cfg["v_th"], seed=seed, newton_tol=1e-11, **kw)
    return pe.Context(c, device=DEV)


def oracle_cfg(cfg, s_w, **kw):
    o = dict(cfg, s_w=s_w, dT=cfg["M"] * cfg["K"] * cfg["dt"])
    o.update(kw)
    return o


def oracle_state(cfg, seed):
    nprof, uprof = orc.sine_profile(cfg["ncell"], cfg["L"], cfg["amp"])
    return orc.quiet_start(cfg["N"], cfg["ncell"], nprof.astype(np.float32), uprof.astype(np.float32),
                           cfg["v_th"], seed)


def coarse_samples_oracle(cfg, seed, s_w):
    st = oracle_state(cfg, seed)
    _, cs, _ = orc.efpi_macro_step(st, oracle_cfg(cfg, s_w), np.zeros(cfg["ncell"]))
    return cs


def test_initial_coarse_state_matches_oracle():
    ctx = make_ctx(SMALL, seed=3)
    ctx.load_initial(SMALL["amp"])
    got = ctx.get_coarse().cpu().numpy()
    st = oracle_state(SMALL, 3)
    d, m = orc.deposit_f64(st.cell, st.theta, st.w, SMALL["ncell"], vel=st.v)
    want = np.stack([orc.coarsen(d, SMALL["n_coarse"]), orc.coarsen(m, SMALL["n_coarse"])])
    assert np.allclose(got, want, rtol=1e-5, atol=1e-5 * np.abs(want).max())
    assert ctx.sync_status() == 0


def test_burst_samples_within_three_sigma_of_oracle():
    cfg = SMALL
    ctx = make_ctx(cfg, seed=1)
    ctx.load_initial(cfg["amp"])
    ctx.burst()
    ctx.restrict()
    K, nc = cfg["K"], cfg["n_coarse"]
    got = ctx.view("coarse_samples", torch.float64)[: (K + 1) * 2 * nc].reshape(K + 1, 2, nc).cpu().numpy()
    assert ctx.sync_status() == 0
    s_w = ctx.diagnostics().s_w
    ens = np.stack([coarse_samples_oracle(cfg, seed, s_w) for seed in (1, 2, 3, 4, 5, 6, 7, 8)])
    sigma = ens.std(axis=0, ddof=1)
    same_seed = ens[0]
    diff = np.abs(got - same_seed)
    assert np.all(diff <= 3 * sigma + 1e-12)
    # tighter: FP32 particles against FP64 particles from the same quiet start
    assert np.max(diff) < 1e-4 * np.max(np.abs(same_seed))


def test_macro_step_matches_oracle():
    cfg = SMALL
    ctx = make_ctx(cfg, seed=9)
    ctx.load_initial(cfg["amp"])
    ctx.step()
    got = ctx.get_coarse().cpu().numpy()
    assert ctx.sync_status() == 0
    s_w = ctx.diagnostics().s_w
    want, _, _ = orc.efpi_macro_step(oracle_state(cfg, 9), oracle_cfg(cfg, s_w), np.zeros(cfg["ncell"]))
    assert np.max(np.abs(got - want)) < 1e-4 * np.max(np.abs(want))


@pytest.mark.parametrize("wavelet", ["haar", "coif4"])
def test_two_macro_steps_with_lift_match_oracle(wavelet):
    cfg = dict(SMALL, K=6, M=3)
    ctx = make_ctx(cfg, seed=17, wavelet=wavelet)
    ctx.load_initial(cfg["amp"])
    ctx.step()
    ctx.step()  # lifts from the projected coarse state
    got = ctx.get_coarse().cpu().numpy()
    assert ctx.sync_status() == 0
    d = ctx.diagnostics()
    assert d.macro_steps == 2
    ocfg = oracle_cfg(cfg, d.s_w, wavelet=wavelet)
    c1, _, phi = orc.efpi_macro_step(oracle_state(cfg, 17), ocfg, np.zeros(cfg["ncell"]))
    # lifting seed of macro step m: seed + 0x632BE59BD9B4E019 (m + 1), its splitmix64 shift
    seed2 = (17 + 0x632BE59BD9B4E019 * 2) % 2**64
    st = orc.lift(c1, dict(ocfg, N=cfg["N"]), seed2)
    c2, _, _ = orc.efpi_macro_step(st, ocfg, phi)
    assert np.max(np.abs(got - c2)) < 2e-4 * np.max(np.abs(c2))


def test_plain_pic_matches_oracle_and_conserves_charge():
    cfg = dict(SMALL, N=128 * 64)
    ctx = make_ctx(cfg, seed=2, sort_every=4)
    ctx.load_initial(cfg["amp"])
    q0 = int(ctx.view("rho", torch.int64, cfg["ncell"]).sum())
    ctx.pic_steps(13)
    got = ctx.measure().cpu().numpy()
    q1 = int(ctx.view("rho", torch.int64, cfg["ncell"]).sum())
    assert ctx.sync_status() == 0
    assert q0 == q1  # the fixed-point charge is exactly conserved through push, deposit and sort
    s_w = ctx.diagnostics().s_w
    st = oracle_state(cfg, 2)
    dx = cfg["L"] / cfg["ncell"]
    phi, _ = orc.pic_steps(st, cfg["ncell"], dx, cfg["dt"], cfg["qm"], 13, s_w, np.zeros(cfg["ncell"]), tol=1e-11)
    rho = orc.deposit_fx(st.cell, st.theta, st.w, cfg["ncell"], s_w) * 2.0 ** -(s_w + 24)
    phi, _, _ = orc.newton_pb(rho, dx, phi0=phi, tol=1e-11)
    E = orc.efield(phi, dx)
    vbar = st.v + 0.5 * cfg["qm"] * cfg["dt"] * orc.gather(E, st.cell, st.theta)
    d, m = orc.deposit_f64(st.cell, st.theta, st.w, cfg["ncell"], vel=vbar)
    want = np.stack([orc.coarsen(d, cfg["n_coarse"]), orc.coarsen(m, cfg["n_coarse"])])
    assert np.max(np.abs(got - want)) < 1e-4 * np.max(np.abs(want))


def test_projection_conserves_total_charge():
    cfg = SMALL
    ctx = make_ctx(cfg, seed=4)
    ctx.load_initial(cfg["amp"])
    c0 = ctx.get_coarse().cpu().numpy()
    ctx.step()
    c1 = ctx.get_coarse().cpu().numpy()
    # Remark (charge conservation): the least-squares weights sum to zero
    assert c1[0].sum() == pytest.approx(c0[0].sum(), rel=1e-9)


def test_cold_drifting_plasma_is_a_fixed_point_on_gpu():
    cfg = dict(SMALL, v_th=0.0, amp=0.0)
    ctx = make_ctx(cfg, seed=0)
    ctx.load_initial(0.0)
    c0 = ctx.get_coarse().cpu().numpy()
    for _ in range(2):
        ctx.step()
    c2 = ctx.get_coarse().cpu().numpy()
    assert ctx.sync_status() == 0
    assert np.max(np.abs(c2 - c0)) < 1e-9
