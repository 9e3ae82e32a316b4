"""GPU parity of the wavelet form of the phase-space variable (Section 3.3 as stated: hat rows
of the repeated 1-2-1 rule in x, periodized DWT in v, Eq. interpolation and the Appendix C
loading of the lifted histograms) against the FP64 CPU oracle, through the C ABI.

Tolerances: the hat-row sample on dyadic data within 1e-12 of the oracle's FP64 fine histogram
restricted by Eq. (restriction) (every FP32 step exact; the oracle sums in FP64), its charge
exact on any data; the DWT in v and its inverse within 1e-12; the loader's positions exact,
weights within 1e-6 relative and velocities within the FP32 evaluation of FP64 tables.
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


def dev(*arrs):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in arrs]


def _tent_sample(c, t, v, w, E0, ncell, b, nvf, vmin, dv, tau, s_w, dx=0.5):
    dc, dt_, dv_, dw, dE = dev(c, t, v, w, E0.astype(np.float32))
    out = torch.zeros(((ncell >> b), nvf), dtype=torch.int64, device=DEV)
    a = pb.make_sample_args(dE, tau, 1.0, 1.0 / dx, s_w, s_w - 6, out, bin_shift=b, n_v=nvf, v_min=vmin, dv=dv,
                            x_tent=True)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    pe.sample(dc, dt_, dv_, dw, dE, ncell, 0.1, 0.5, a, status=st)
    return out.cpu().numpy(), int(st.item())


@pytest.mark.parametrize("ncell,N,b,nvf,tau", [(64, 1, 2, 16, 2.5), (64, 4099, 2, 16, 2.5), (512, 1 << 16, 3, 64, 6.0),
                                               (4096, (1 << 20) + 3, 4, 256, 20.0), (4096, 1 << 18, 4, 128, 180.0)])
def test_tent_rows_match_the_restricted_fine_histogram_on_dyadic_data(ncell, N, b, nvf, tau):
    rng = np.random.default_rng(N + ncell)
    c = np.sort(rng.integers(0, ncell, N)).astype(np.int32)
    t = (rng.integers(0, 1 << 10, N) / 1024.0).astype(np.float32)
    v = (rng.integers(-6 * 64, 6 * 64, N) / 64.0).astype(np.float32)
    w = ((1 + rng.integers(0, 64, N)) / 64.0 * ncell / max(N, 1)).astype(np.float32)
    w = np.ldexp(np.round(np.ldexp(w, 20)), -20).astype(np.float32)
    E0 = rng.integers(-128, 128, ncell) / 1024.0
    vmin, dv = -8.0, 16.0 / nvf
    s_w = orc.fx_shift(float(w.max()) * 2)
    got, st = _tent_sample(c, t, v, w, E0, ncell, b, nvf, vmin, dv, tau, s_w)
    assert st == 0
    wq = np.rint(w.astype(np.float64) * 2.0 ** s_w).astype(np.int64)
    assert int(got.astype(object).sum()) == int(wq.astype(object).sum()) << 24  # every hat splits w_q 2^24
    st_o = orc.State(c, t.astype(np.float64), v.astype(np.float64), w.astype(np.float64))
    H = orc.ps_hist_fine(st_o, v.astype(np.float64), E0, ncell, 0.5, tau, 1.0, vmin, dv, nvf)
    want = orc.restrict_121(H, b)
    g = got.astype(np.float64) * 2.0 ** -(s_w + 24 + b)
    assert np.max(np.abs(g - want)) <= 1e-12 * np.abs(want).max()


def test_tent_rows_on_general_data():
    ncell, N, b, nvf = 4096, 1 << 20, 4, 256
    c, t, v, w = inputs.random_particles(N, ncell, seed=31)
    E0 = inputs.random_field(ncell, 32, 0.05)
    s_w = orc.fx_shift(3.0 * ncell / N)
    got, st = _tent_sample(c, t, v, w, E0, ncell, b, nvf, -8.0, 16.0 / nvf, 17.3, s_w)
    assert st == 0
    wq = np.rint(w.astype(np.float64) * 2.0 ** s_w).astype(np.int64)
    assert int(got.astype(object).sum()) == int(wq.astype(object).sum()) << 24
    st_o = orc.State(c, t.astype(np.float64), v.astype(np.float64), w.astype(np.float64))
    H = orc.ps_hist_fine(st_o, v.astype(np.float64), E0.astype(np.float32).astype(np.float64), ncell, 0.5, 17.3, 1.0,
                         -8.0, 16.0 / nvf, nvf)
    want = orc.restrict_121(H, b)
    g = got.astype(np.float64) * 2.0 ** -(s_w + 24 + b)
    # FP32 targets near a cell edge move a weight to the neighbouring cell: a small L1 share
    assert np.abs(g - want).sum() <= 1e-4 * np.abs(want).sum()


@pytest.mark.parametrize("wav", ["haar", "d4", "coif4"])
@pytest.mark.parametrize("nvf,nvc,b", [(16, 16, 0), (64, 16, 2), (256, 64, 4), (1024, 32, 3)])
def test_coarsen_and_refine_in_v_match_the_oracle(wav, nvf, nvc, b):
    rng = np.random.default_rng(nvf + nvc)
    rows = rng.integers(-(1 << 40), 1 << 44, size=(3, 5, nvf)).astype(np.int64)
    s_w = 14
    got = pb.ps_coarsen_v(dev(rows)[0], s_w, b, nvc, wav).cpu().numpy()
    want = orc.ps_coarsen_v(rows.astype(np.float64) * 2.0 ** -(s_w + 24 + b), nvc, wav)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.abs(want).max()
    C = rng.normal(size=(7, nvc))
    got = pb.ps_refine_v(dev(C)[0], nvf, wav).cpu().numpy()
    want = orc.ps_refine_v(C, nvf, wav)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.abs(want).max()


def _smooth_hist(nxc, nvf, seed, noise=0.02):
    rng = np.random.default_rng(seed)
    x = np.arange(nxc) / nxc
    vc = -8.0 + 16.0 / nvf * (np.arange(nvf) + 0.5)
    n = 1.0 + 0.4 * np.cos(2 * np.pi * x)
    u = 0.5 * np.sin(2 * np.pi * x)
    H = n[:, None] * np.exp(-0.5 * (vc[None, :] - u[:, None]) ** 2) * (16.0 / nvf) / np.sqrt(2 * np.pi)
    return np.abs(H + noise * H.max() * rng.standard_normal(H.shape)) + 1e-6 * H.max()


@pytest.mark.parametrize("ncell,ppc,b,nvf", [(64, 64, 2, 16), (4096, 256, 4, 256), (512, 1000, 3, 64)])
def test_node_tables_and_loader_match_the_oracle(ncell, ppc, b, nvf):
    nxc = ncell >> b
    H = _smooth_hist(nxc, nvf, ncell + nvf)
    mass, cdf, _ = orc.ps_lift_tables(H)
    dm, dcdf, _, _ = pb.ps_lift_tables(dev(H)[0])
    assert np.array_equal(dm.cpu().numpy(), mass) and np.array_equal(dcdf.cpu().numpy(), cdf)
    table, dens = pb.ps_node_tables(dm, dcdf, ncell)
    nfine = orc.interpolate_x(mass, b)
    assert np.allclose(dens.cpu().numpy(), nfine, rtol=1e-7, atol=0)
    N = ncell * ppc
    vmin, dv = -8.0, 16.0 / nvf
    s_w = orc.fx_shift(8.0 * float(mass.max()) / ppc)
    cell, theta, v, w, rho = pb.ps_quiet_start_nodes(N, ncell, table, dens, vmin, dv, 777, s_w)
    st = orc.ps_quiet_start_nodes(N, ncell, b, mass, cdf, vmin, dv, 777)
    assert np.array_equal(cell.cpu().numpy(), st.cell)
    assert np.array_equal(theta.cpu().numpy(), st.theta.astype(np.float32))
    assert np.allclose(w.cpu().numpy(), st.w, rtol=2e-6, atol=0)
    dv_ = np.abs(v.cpu().numpy() - st.v)
    # FP32 CDF rows: a rounding of F moves r by ~6e-8 / p_k inside a cell of mass p_k
    assert dv_.max() <= 2e-3 and dv_.mean() <= 1e-5 * 16.0
    th, ww = theta.cpu().numpy(), w.cpu().numpy()
    assert np.array_equal(rho.cpu().numpy(), orc.deposit_fx(st.cell, th, ww, ncell, s_w))


WCFG = dict(ncell=128, L=64.0, N=128 * 256, dt=0.1, K=6, M=3, n_coarse=16, v_th=1.0, qm=1.0, amp=0.1, n_v=64,
            n_v_coarse=16, v_max=8.0)


def _wctx(cfg, seed, wavelet):
    dT = cfg["M"] * cfg["K"] * cfg["dt"]
    c = pe.make_config(cfg["ncell"], cfg["n_coarse"], cfg["K"], cfg["N"], cfg["L"], cfg["dt"], dT, qm=cfg["qm"],
                       v_th=cfg["v_th"], seed=seed, newton_tol=1e-11, wavelet=wavelet, coarse="phase_space",
                       n_v=cfg["n_v"], v_max=cfg["v_max"], n_v_coarse=cfg["n_v_coarse"])
    return pe.Context(c, device=DEV)


@pytest.mark.parametrize("wavelet", ["coif4", "haar"])
def test_wavelet_form_cycle_matches_the_oracle(wavelet):
    """The context cycle of the wavelet form: initial restriction (1e-5 of its maximum), one
    macro step from the loaded particles (1e-4) and a second after the lifting (2e-4 in L1), against
    the oracle's literal steps (fine histogram, Eq. restriction, DWT in v, LS leap; synthesis,
    reconstruction per coarse node, Eq. interpolation, loading)."""
    cfg = WCFG
    ncell, nc, nvf, nvc = cfg["ncell"], cfg["n_coarse"], cfg["n_v"], cfg["n_v_coarse"]
    ctx = _wctx(cfg, 17, wavelet)
    ctx.load_initial(cfg["amp"])
    c0 = ctx.get_coarse().cpu().numpy()
    assert c0.shape == (nc, nvc)
    s_w = ctx.diagnostics().s_w
    nprof, uprof = orc.sine_profile(ncell, cfg["L"], cfg["amp"])
    st = orc.quiet_start(cfg["N"], ncell, nprof.astype(np.float32), uprof.astype(np.float32), cfg["v_th"], 17)
    b = int(np.log2(ncell // nc))
    dx = cfg["L"] / ncell
    H = orc.ps_hist_fine(st, st.v, np.zeros(ncell), ncell, dx, 0.0, cfg["qm"], -cfg["v_max"], 2 * cfg["v_max"] / nvf, nvf)
    want0 = orc.ps_wavelet_restrict(H, b, nvc, wavelet)
    assert np.max(np.abs(c0 - want0)) < 1e-5 * np.max(np.abs(want0))
    ocfg = dict(cfg, s_w=s_w, dT=cfg["M"] * cfg["K"] * cfg["dt"], wavelet=wavelet)
    ctx.step()
    c1g = ctx.get_coarse().cpu().numpy()
    c1, _, phi = orc.efpi_ps_wavelet_macro_step(st, ocfg, np.zeros(ncell))
    assert np.max(np.abs(c1g - c1)) < 1e-4 * np.max(np.abs(c1))
    assert abs(c1g.sum() - c0.sum()) < 1e-9 * c0.sum()  # Remark on charge conservation
    ctx.step()  # lifts from the projected coarse state
    c2g = ctx.get_coarse().cpu().numpy()
    assert ctx.sync_status() == 0
    seed2 = (17 + 0x632BE59BD9B4E019 * 2) % 2**64
    st2, _ = orc.ps_wavelet_lift(c1, dict(ocfg, N=cfg["N"]), seed2)
    c2, _, _ = orc.efpi_ps_wavelet_macro_step(st2, ocfg, phi)
    # after the lift, FP32 against FP64 inverse CDFs now and then put a particle in the next
    # velocity cell: one particle moves w / 2^b (5e-4 here, 1.3e-3 of the maximum) between
    # neighbouring rows of a coefficient set, so the bound is on the L1 norm, with a looser maximum
    assert np.abs(c2g - c2).sum() < 2e-4 * np.abs(c2).sum()
    assert np.max(np.abs(c2g - c2)) < 2e-3 * np.max(np.abs(c2))
    assert abs(c2g.sum() - c0.sum()) < 1e-5 * c0.sum()
