"""GPU parity of each hot-path kernel against the FP64 CPU oracle, through the C ABI.

Tolerances (stated per result):
  deposit ............ bit-exact (same fixed-point rule, same FP32 inputs)
  field solve ........ phi within 1e-9 absolute, E within 1e-8 of max|E| (both FP64 Newton)
  push ............... positions within 1e-5 cell, velocities within 1e-5 relative (FP32 vs FP64)
  restriction sample . within 1e-4 of the sample's max (FP32 co-moving positions)
  coarsen / project .. 1e-12 relative (FP64 on both sides)
  lifting ............ profiles 1e-6 relative (FP32 output), velocities 2e-5 absolute
"""
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


def status_word():
    return torch.zeros(1, dtype=torch.int32, device=DEV)


# ----------------------------------------------------------------- deposit


@pytest.mark.parametrize("ncell,N,sort", [(8, 1, True), (8, 5, True), (128, (1 << 14) + 3, True),
                                          (128, 4099, False), (4096, (1 << 20) + 1, True),
                                          (16384, 1 << 18, True), (16384, 1 << 16, False)])
def test_deposit_bit_exact(ncell, N, sort):
    c, t, v, w = inputs.random_particles(N, ncell, seed=N + ncell, sort=sort)
    s_w = orc.fx_shift(2.0 * ncell / N)
    st = status_word()
    rho = pe.deposit(*to_dev(c, t, w), ncell, s_w, status=st)
    assert np.array_equal(rho.cpu().numpy(), orc.deposit_fx(c, t, w, ncell, s_w))
    assert int(st.item()) == 0


def test_deposit_empty_and_range_flag():
    c, t, v, w = inputs.random_particles(100, 64, seed=3)
    rho = pe.deposit(*to_dev(c[:0], t[:0], w[:0]), 64, 20)
    assert int(rho.abs().sum()) == 0
    c = c.copy()
    c[7] = 64  # out of range: skipped and flagged, never a fault
    st = status_word()
    rho = pe.deposit(*to_dev(c, t, w), 64, 20, status=st)
    assert int(st.item()) & 4
    keep = np.ones(100, bool)
    keep[7] = False
    assert np.array_equal(rho.cpu().numpy(), orc.deposit_fx(c[keep], t[keep], w[keep], 64, 20))
    # a weight beyond the fixed-point range is reported, not trapped
    c[7] = 3
    w = w.copy()
    w[9] = 100.0
    st = status_word()
    pe.deposit(*to_dev(c, t, w), 64, 20, status=st)
    assert int(st.item()) & 2


def test_deposit_full_size_iaw_large():
    cfg = inputs.workload("iaw_large")
    ncell, N = cfg["ncell"], cfg["N"]
    c, t, v, w = inputs.random_particles(N, ncell, seed=11)
    s_w = orc.fx_shift(8.0 * ncell / N)
    rho = pe.deposit(*to_dev(c, t, w), ncell, s_w)
    assert np.array_equal(rho.cpu().numpy(), orc.deposit_fx(c, t, w, ncell, s_w))


# ----------------------------------------------------------------- field solve


@pytest.mark.parametrize("ncell,mode", [(8, "boltzmann"), (128, "boltzmann"), (1024, "boltzmann"),
                                        (2048, "linearized"), (4096, "boltzmann"), (8192, "boltzmann"),
                                        (256, "linearized")])
def test_field_matches_oracle_newton(ncell, mode):
    L = ncell * 0.5
    n = inputs.random_density(ncell, seed=ncell, amp=0.4)
    s_w = 20
    rho = np.rint(n * 2.0 ** (s_w + 24)).astype(np.int64)
    n_q = rho * 2.0 ** -(s_w + 24)
    phi_o, _, fail = orc.newton_pb(n_q, L / ncell, phi0=np.zeros(ncell), mode=1 if mode == "linearized" else 0,
                                   tol=1e-12)
    assert fail == 0
    E_o = orc.efield(phi_o, L / ncell)
    phi = torch.zeros(ncell, dtype=torch.float64, device=DEV)
    st = status_word()
    E, Ef, diag = pe.field(*to_dev(rho), ncell, L / ncell, s_w, phi, mode=mode, tol=1e-12, status=st)
    assert int(st.item()) == 0 and int(diag[1]) == 1
    assert np.max(np.abs(phi.cpu().numpy() - phi_o)) < 1e-9
    assert np.max(np.abs(E.cpu().numpy() - E_o)) < 1e-8 * np.max(np.abs(E_o))
    assert np.max(np.abs(Ef.cpu().numpy() - E_o)) < 1e-6 * np.max(np.abs(E_o))


def test_field_manufactured_solution_on_gpu():
    ncell, L = 4096, 2048.0
    dx = L / ncell
    x = np.arange(ncell) * dx
    phi_star = 0.7 * np.cos(2 * np.pi * x / L) + 0.2 * np.sin(2 * np.pi * 9 * x / L)
    n = -(np.roll(phi_star, 1) - 2 * phi_star + np.roll(phi_star, -1)) / dx**2 + np.exp(phi_star)
    s_w = 20
    rho = np.rint(n * 2.0 ** (s_w + 24)).astype(np.int64)
    phi = torch.zeros(ncell, dtype=torch.float64, device=DEV)
    pe.field(*to_dev(rho), ncell, dx, s_w, phi, tol=1e-13)
    # the only error left is the 2^-45 quantisation of n
    assert np.max(np.abs(phi.cpu().numpy() - phi_star)) < 1e-10


@pytest.mark.parametrize("ncell", [256, 4096])
def test_field_reports_non_convergence_without_fault(ncell):
    n = inputs.random_density(ncell, seed=1, amp=0.4)
    rho = np.rint(n * 2.0**44).astype(np.int64)
    phi = torch.full((ncell,), -30.0, dtype=torch.float64, device=DEV)
    st = status_word()
    _, _, diag = pe.field(*to_dev(rho), ncell, 0.5, 20, phi, maxit=2, status=st)
    assert int(st.item()) & 1 and int(diag[1]) == 0 and int(diag[0]) == 2


# ----------------------------------------------------------------- push


def _oracle_field(c, t, w, ncell, dx, s_w):
    rho = orc.deposit_fx(c, t, w, ncell, s_w)
    phi, _, fail = orc.newton_pb(rho * 2.0 ** -(s_w + 24), dx, phi0=np.zeros(ncell), tol=1e-12)
    assert fail == 0
    return orc.efield(phi, dx), phi


def _cell_dist(c1, t1, c2, t2, ncell):
    d = (c1.astype(np.float64) + t1) - (c2.astype(np.float64) + t2)
    return np.abs((d + ncell / 2) % ncell - ncell / 2)


@pytest.mark.parametrize("ncell,N,kick", [(128, (1 << 15) + 2, 0.5), (4096, 1 << 20, 1.0), (64, 4099, 1.0)])
def test_single_step_matches_oracle(ncell, N, kick):
    dx, dt, qm = 0.5, 0.1, 1.0
    c, t, v, w = inputs.random_particles(N, ncell, seed=7 + ncell, sort=True)
    s_w = orc.fx_shift(2.0 * ncell / N)
    E_o, phi_o = _oracle_field(c, t, w, ncell, dx, s_w)
    dc, dt_, dv, dw = to_dev(c, t, v, w)
    rho = pe.deposit(dc, dt_, dw, ncell, s_w)
    phi = torch.zeros(ncell, dtype=torch.float64, device=DEV)
    E, Ef, _ = pe.field(rho, ncell, dx, s_w, phi, tol=1e-12)
    assert np.max(np.abs(E.cpu().numpy() - E_o)) < 1e-5 * np.max(np.abs(E_o))
    st = status_word()
    rho2 = pe.push(dc, dt_, dv, dw, Ef, ncell, dt / dx, qm * dt, kick, s_w, status=st)
    so = orc.State(c, t, v, w)
    orc.push(so, E_o, ncell, dx, dt, qm, kick=kick)
    gc, gt, gv = dc.cpu().numpy(), dt_.cpu().numpy(), dv.cpu().numpy()
    assert int(st.item()) == 0
    assert np.max(_cell_dist(gc, gt, so.cell, so.theta, ncell)) < 1e-5
    assert np.max(np.abs(gv - so.v) / np.maximum(1.0, np.abs(so.v))) < 1e-5
    assert np.all((gt >= 0) & (gt < 1)) and np.all((gc >= 0) & (gc < ncell))
    # deposit of the pushed state: exact charge, values within the position tolerance
    rho_o = orc.deposit_fx(so.cell, so.theta, so.w, ncell, s_w)
    r = rho2.cpu().numpy()
    assert int(r.sum()) == int(rho_o.sum())
    assert np.max(np.abs(r - rho_o)) < 1e-5 * np.max(np.abs(rho_o))


def test_fused_deposit_bit_exact_on_exact_arithmetic():
    # E = 0 and velocities / offsets on a dyadic lattice make FP32 and FP64 drift identical,
    # so the fused deposit of the pushed particles must equal the oracle's bit for bit
    ncell, N = 256, (1 << 16) + 1
    rng = np.random.default_rng(5)
    c = np.sort(rng.integers(0, ncell, N)).astype(np.int32)
    t = (rng.integers(0, 1024, N) / 1024).astype(np.float32)
    v = (rng.integers(-256, 256, N) / 64).astype(np.float32)
    w = (rng.integers(1, 64, N) / 64 * ncell / N).astype(np.float32)
    s_w = orc.fx_shift(ncell / N)
    dc, dt_, dv, dw = to_dev(c, t, v, w)
    Ef = torch.zeros(ncell, dtype=torch.float32, device=DEV)
    rho = pe.push(dc, dt_, dv, dw, Ef, ncell, 0.25, 0.1, 1.0, s_w)
    so = orc.State(c, t, v, w)
    orc.push(so, np.zeros(ncell), ncell, 1.0, 0.25, 1.0)
    assert np.array_equal(rho.cpu().numpy(), orc.deposit_fx(so.cell, so.theta, so.w, ncell, s_w))
    assert np.array_equal(dc.cpu().numpy(), so.cell)
    assert np.array_equal(dt_.cpu().numpy().astype(np.float64), so.theta)


# ----------------------------------------------------------------- restriction sample


@pytest.mark.parametrize("tau", [0.0, 3.7, 20.0])
def test_sample_matches_oracle(tau):
    ncell, N, dx, dt, qm = 256, 1 << 16, 0.5, 0.1, 1.0
    c, t, v, w = inputs.random_particles(N, ncell, seed=21)
    s_w = orc.fx_shift(2.0 * ncell / N)
    s_p = orc.fx_shift(2.0 * ncell / N * 32.0)
    E = inputs.random_field(ncell, seed=4, amp=0.05)
    E0 = inputs.random_field(ncell, seed=5, amp=0.05)
    dc, dt_, dv, dw = to_dev(c, t, v, w)
    Ef, E0f = to_dev(E.astype(np.float32), E0.astype(np.float32))
    out = torch.empty(2 * ncell, dtype=torch.int64, device=DEV)
    args = pe.make_sample_args(E0f, tau, qm, 1 / dx, s_w, s_p, out)
    pe.sample(dc, dt_, dv, dw, Ef, ncell, qm * dt, 1.0, args)
    so = orc.State(c, t, v, w)
    Eo = E.astype(np.float32).astype(np.float64)
    vbar = so.v + 0.5 * qm * dt * orc.gather(Eo, c, t)
    dens, mom = orc.restrict_sample(so, vbar, E0.astype(np.float32).astype(np.float64), ncell, dx, tau, qm)
    g = out.cpu().numpy()
    gd, gm = g[:ncell] * 2.0 ** -(s_w + 24), g[ncell:] * 2.0 ** -(s_p + 24)
    assert np.max(np.abs(gd - dens)) < 1e-4 * np.max(np.abs(dens))
    assert np.max(np.abs(gm - mom)) < 1e-4 * np.max(np.abs(mom))
    assert gd.sum() == pytest.approx(dens.sum(), rel=1e-7)
    # binned form (Haar restriction): exact bin sums of the nodal fixed-point sample
    for b in (1, 3, 5):
        outb = torch.empty(2 * (ncell >> b), dtype=torch.int64, device=DEV)
        argb = pe.make_sample_args(E0f, tau, qm, 1 / dx, s_w, s_p, outb, bin_shift=b)
        pe.sample(dc, dt_, dv, dw, Ef, ncell, qm * dt, 1.0, argb)
        want = g.reshape(2, ncell >> b, 1 << b).sum(axis=-1).reshape(-1)
        assert np.array_equal(outb.cpu().numpy(), want)


# ----------------------------------------------------------------- coarse variables


@pytest.mark.parametrize("wav,ncell,nc", [("haar", 128, 16), ("haar", 4096, 256), ("d4", 512, 32), ("haar", 64, 64),
                                          ("coif4", 512, 32), ("coif4", 4096, 256), ("coif4", 64, 8)])
def test_coarsen_matches_oracle(wav, ncell, nc):
    rng = np.random.default_rng(ncell)
    nsamp, s_w, s_p = 5, 30, 25
    fx = rng.integers(-(1 << 50), 1 << 50, size=(nsamp, 2, ncell), dtype=np.int64)
    out = pe.coarsen(*to_dev(fx), nsamp, ncell, s_w, s_p, nc, wavelet=wav).cpu().numpy()
    for p in range(nsamp):
        for m, s in ((0, s_w), (1, s_p)):
            want = orc.coarsen(fx[p, m] * 2.0 ** -(s + 24), nc, wav)
            assert np.allclose(out[p, m], want, rtol=1e-12, atol=1e-12 * np.max(np.abs(want)))


@pytest.mark.parametrize("ncell,nc,b", [(128, 16, 3), (4096, 256, 4), (256, 32, 2)])
def test_coarsen_binned_haar_matches_oracle(ncell, nc, b):
    rng = np.random.default_rng(b)
    nsamp, s_w, s_p = 3, 30, 25
    fx = rng.integers(-(1 << 50), 1 << 50, size=(nsamp, 2, ncell), dtype=np.int64)
    binned = fx.reshape(nsamp, 2, ncell >> b, 1 << b).sum(axis=-1)
    out = pe.coarsen(*to_dev(binned), nsamp, ncell, s_w, s_p, nc, bin_shift=b).cpu().numpy()
    for p in range(nsamp):
        for m, s in ((0, s_w), (1, s_p)):
            want = orc.coarsen(fx[p, m] * 2.0 ** -(s + 24), nc, "haar")
            assert np.allclose(out[p, m], want, rtol=1e-12, atol=1e-12 * np.max(np.abs(want)))


@pytest.mark.parametrize("K", [1, 6, 20, 31])
def test_ls_project_matches_oracle(K):
    rng = np.random.default_rng(K)
    samples = rng.standard_normal((K + 1, 512))
    out, slope = pe.ls_project(*to_dev(samples), 0.1, 20.0)
    want, wslope = orc.ls_project(samples, 0.1, 20.0)
    assert np.allclose(slope.cpu().numpy(), wslope, rtol=1e-11, atol=1e-11)
    assert np.allclose(out.cpu().numpy(), want, rtol=1e-11, atol=1e-10)


@pytest.mark.parametrize("wav,ncell,nc", [("haar", 128, 16), ("haar", 4096, 256), ("d4", 256, 32),
                                          ("coif4", 256, 32), ("coif4", 4096, 256)])
def test_refine_matches_oracle(wav, ncell, nc):
    rng = np.random.default_rng(nc)
    coarse = np.stack([1.0 + 0.6 * rng.standard_normal(nc), 0.3 * rng.standard_normal(nc)]) * 2.0 ** (
        -np.log2(nc) / 2)
    coarse[0, 3] = -0.5  # a negative density to exercise the clamp
    pn, pu = pe.refine(*to_dev(coarse), ncell, wavelet=wav)
    nf = orc.refine(coarse[0], ncell, wav)
    mf = orc.refine(coarse[1], ncell, wav)
    nf, uf = orc.lift_profile(nf, mf)
    assert np.allclose(pn.cpu().numpy(), nf, rtol=1e-6, atol=1e-6 * nf.max())
    assert np.allclose(pu.cpu().numpy(), uf, rtol=1e-5, atol=1e-5 * np.abs(uf).max())


# ----------------------------------------------------------------- lifting / quiet start


@pytest.mark.parametrize("ncell,ppc", [(128, 1024), (64, 3), (4096, 256)])
def test_quiet_start_matches_oracle(ncell, ppc):
    N = ncell * ppc
    nprof, uprof = orc.sine_profile(ncell, ncell * 0.5, 0.3)
    seed = 12345
    pn, pu = to_dev(nprof.astype(np.float32), uprof.astype(np.float32))
    s_w = orc.fx_shift(8.0 / ppc)
    cell, theta, v, w, rho = pe.quiet_start(N, ncell, pn, pu, 1.0, seed, s_w)
    st = orc.quiet_start(N, ncell, nprof.astype(np.float32), uprof.astype(np.float32), 1.0, seed)
    assert np.array_equal(cell.cpu().numpy(), st.cell)
    assert np.max(np.abs(theta.cpu().numpy() - st.theta)) < 1e-7
    assert np.allclose(w.cpu().numpy(), st.w, rtol=2e-6)
    assert np.max(np.abs(v.cpu().numpy() - st.v)) < 2e-5
    # the fused deposit equals the plain deposit kernel on the generated particles
    assert torch.equal(rho, pe.deposit(cell, theta, w, ncell, s_w))


# ----------------------------------------------------------------- sort


@pytest.mark.parametrize("ncell,N", [(64, 1000), (4096, (1 << 20) + 3)])
def test_sort_is_a_sorted_permutation(ncell, N):
    c, t, v, w = inputs.random_particles(N, ncell, seed=9, sort=False)
    oc, ot, ov, ow = [x.cpu().numpy() for x in pe.sort(*to_dev(c, t, v, w), ncell)]
    assert np.all(np.diff(oc) >= 0)
    key_in = np.lexsort((w, v, t, c))
    key_out = np.lexsort((ow, ov, ot, oc))
    for a, b in ((c, oc), (t, ot), (v, ov), (w, ow)):
        assert np.array_equal(a[key_in], b[key_out])
