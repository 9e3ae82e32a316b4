"""FP64 particles (the small ion-wave workload, 128 cells, 2^17 ions, run with double-precision
particles as well as FP32): the FP64 kernels against the FP64 oracle. Positions follow the
oracle to 1e-12 of a cell through plain PIC steps and through a burst; the deposit is bit-exact.
The error of a projective macro step then separates: the FP64 particles' run differs from the
oracle only by the fixed-point restriction rule (the oracle sums its samples in FP64); the FP32
particles' run adds its precision error to that."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1610_01071_gb300 import _binding as pb
from paper_1610_01071_gb300 import inputs
from paper_1610_01071_gb300.fp64 import FP64Realisation

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")

W = inputs.workload("iaw_small")  # 128 cells, L = 64, 2^17 ions, K = 20, dT = 20, 16 Haar coefficients


def fp64_run(**kw):
    cfg = dict(W, **kw)
    r = FP64Realisation(cfg["ncell"], cfg["n_coarse"], cfg["K"], cfg["N"], cfg["L"], cfg["dt"], cfg["dT"],
                        qm=cfg["qm"], v_th=cfg["v_th"], seed=5, newton_tol=1e-12, device=DEV)
    nprof, uprof = orc.sine_profile(cfg["ncell"], cfg["L"], cfg["amplitude"])  # closed-form input
    r.load(torch.from_numpy(nprof).to(DEV), torch.from_numpy(uprof).to(DEV))
    return r, cfg


def state(r):
    return orc.State(r.cell.cpu().numpy(), r.theta.cpu().numpy(), r.v.cpu().numpy(), r.w.cpu().numpy())


def test_fp64_quiet_start_matches_oracle_and_deposits_exactly():
    r, cfg = fp64_run()
    st = state(r)
    nprof, uprof = orc.sine_profile(cfg["ncell"], cfg["L"], cfg["amplitude"])
    so = orc.quiet_start(cfg["N"], cfg["ncell"], nprof, uprof, cfg["v_th"], 5)
    assert np.array_equal(st.cell, so.cell)
    assert np.max(np.abs(st.theta - so.theta)) <= 1e-15
    assert np.max(np.abs(st.w - so.w) / so.w) <= 1e-14
    assert np.max(np.abs(st.v - so.v)) <= 1e-12  # Phi^-1 in double on both sides
    assert np.array_equal(r.rho.cpu().numpy(), orc.deposit_fx(st.cell, st.theta, st.w, cfg["ncell"], r.s_w))
    assert r.sync_status() == 0


def test_fp64_plain_pic_positions_follow_the_oracle_to_1e12():
    r, cfg = fp64_run()
    st = state(r)
    r.pic_steps(12)
    got = state(r)
    assert r.sync_status() == 0
    dx = cfg["L"] / cfg["ncell"]
    orc.pic_steps(st, cfg["ncell"], dx, cfg["dt"], cfg["qm"], 12, r.s_w, np.zeros(cfg["ncell"]), tol=1e-12)
    d = (got.cell + got.theta) - (st.cell + st.theta)
    d = (d + cfg["ncell"] / 2) % cfg["ncell"] - cfg["ncell"] / 2
    assert np.max(np.abs(d)) < 1e-12
    assert np.max(np.abs(got.v - st.v)) < 1e-12 * np.max(np.abs(st.v))
    # the deposit of the pushed particles is the oracle rule applied to them, bit for bit
    assert np.array_equal(r.rho.cpu().numpy(), orc.deposit_fx(got.cell, got.theta, got.w, cfg["ncell"], r.s_w))


def test_macro_step_error_separates_into_precision_and_method():
    r, cfg = fp64_run()
    st64 = state(r)
    r.burst()
    pos64 = state(r)
    r.restrict_project()
    c64 = r.coarse.cpu().numpy()
    assert r.sync_status() == 0
    ocfg = dict(cfg, s_w=r.s_w)
    want64, _, _ = orc.efpi_macro_step(st64, ocfg, np.zeros(cfg["ncell"]))  # advances st64 through the burst
    err64 = np.max(np.abs(c64 - want64)) / np.max(np.abs(want64))
    d = (pos64.cell + pos64.theta) - (st64.cell + st64.theta)
    pos_err64 = np.max(np.abs((d + cfg["ncell"] / 2) % cfg["ncell"] - cfg["ncell"] / 2))
    # the same workload with FP32 particles through the context API
    c = pb.make_config(cfg["ncell"], cfg["n_coarse"], cfg["K"], cfg["N"], cfg["L"], cfg["dt"], cfg["dT"],
                       qm=cfg["qm"], v_th=cfg["v_th"], seed=5, newton_tol=1e-12)
    ctx = pb.Context(c, device=DEV)
    ctx.load_initial(cfg["amplitude"])
    st32 = orc.State(*[x.cpu().numpy() for x in ctx.particles()])
    ctx.burst()
    pos32 = orc.State(*[x.cpu().numpy() for x in ctx.particles()])
    ctx.restrict()
    ctx.project()
    c32 = ctx.get_coarse().cpu().numpy()
    want32, _, _ = orc.efpi_macro_step(st32, dict(ocfg, s_w=ctx.diagnostics().s_w), np.zeros(cfg["ncell"]))
    err32 = np.max(np.abs(c32 - want32)) / np.max(np.abs(want32))
    d = (pos32.cell + pos32.theta.astype(np.float64)) - (st32.cell + st32.theta)
    pos_err32 = np.max(np.abs((d + cfg["ncell"] / 2) % cfg["ncell"] - cfg["ncell"] / 2))
    print(f"burst vs the FP64 oracle: positions FP64 {pos_err64:.1e} / FP32 {pos_err32:.1e} cells; "
          f"macro step coarse FP64 {err64:.2e} / FP32 {err32:.2e}")
    assert pos_err64 < 1e-12  # the same method as the oracle, in the same precision
    assert pos_err32 > 1e3 * pos_err64  # FP32 particles: their precision error
    assert err64 < 1e-5  # the fixed-point restriction rule against the oracle's FP64 sums
    assert err32 < 1e-4
