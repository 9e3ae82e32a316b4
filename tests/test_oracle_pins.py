"""Pins of the FP64 CPU oracle against closed forms, invariants, brute force,
library routines and the paper's own numbers. No GPU needed.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
swapped theta / 1-theta, a wrong sign or index, a transposed operand) fails it.
"""
import numpy as np
import pytest
import scipy.special

import oracle as orc
from paper_1610_01071_gb300 import inputs
from conftest import read_golden

# ----------------------------------------------------------------- generator


def test_splitmix64_reference_outputs():
    g = 0x9E3779B97F4A7C15
    for k, hexval in read_golden("splitmix64_seed0.txt"):
        assert orc.splitmix64((int(k) * g) % 2**64) == int(hexval, 16)


def test_fx_shift_rule():
    assert orc.fx_shift(1.0) == 22
    assert orc.fx_shift(2.0 ** -9) == 31
    assert orc.fx_shift(0.3) == 23  # ceil(log2 0.3) = -1
    assert orc.fx_shift(3.0) == 20


# ----------------------------------------------------------------- deposit (Section 2.2)


def _state(N, ncell, seed, **kw):
    c, t, v, w = inputs.random_particles(N, ncell, seed, **kw)
    return c, t.astype(np.float64), v.astype(np.float64), w.astype(np.float64)


def test_deposit_fx_charge_conservation_exact():
    ncell = 64
    c, t, v, w = _state(5000, ncell, 1)
    s_w = orc.fx_shift(2 * 1.5 * ncell / 5000)
    rho = orc.deposit_fx(c, t, w, ncell, s_w)
    wq = np.rint(w * 2.0**s_w).astype(np.int64)
    assert int(rho.sum()) == int((wq * (1 << 24)).sum())


def test_deposit_fx_first_moment_is_particle_position():
    # CIC puts the charge's centre at the particle: sum_j j q_j = w_q (cell + theta_q/2^24),
    # exactly, away from the periodic seam. A swapped theta/(1-theta) fails this.
    ncell = 64
    rng = np.random.default_rng(3)
    c = rng.integers(2, ncell - 3, 300).astype(np.int32)
    t = rng.random(300, dtype=np.float32).astype(np.float64)
    w = (rng.random(300) + 0.5).astype(np.float32).astype(np.float64)
    s_w = 20
    for i in range(50):
        rho = orc.deposit_fx(c[i:i + 1], t[i:i + 1], w[i:i + 1], ncell, s_w)
        tq = int(np.rint(t[i] * 2**24))
        wq = int(np.rint(w[i] * 2.0**s_w))
        assert int((np.arange(ncell) * rho).sum()) == wq * (int(c[i]) * 2**24 + tq)
        assert int(rho.sum()) == wq * 2**24


def test_deposit_uniform_lattice_gives_uniform_density():
    ncell, ppc = 32, 16
    c = np.repeat(np.arange(ncell), ppc).astype(np.int32)
    t = np.tile((np.arange(ppc) + 0.5) / ppc, ncell)
    w = np.full(ncell * ppc, 1.0 / ppc)
    rho = orc.deposit_fx(c, t, w, ncell, 22)
    assert np.all(rho == rho[0])
    assert rho[0] * 2.0 ** -(22 + 24) == pytest.approx(1.0, rel=0, abs=1e-12)


def test_deposit_fx_matches_f64_within_quantisation():
    ncell, N = 128, 20000
    c, t, v, w = _state(N, ncell, 5)
    s_w = orc.fx_shift(1.5 * ncell / N)
    n_fx = orc.deposit_fx(c, t, w, ncell, s_w) * 2.0 ** -(s_w + 24)
    n_64 = orc.deposit_f64(c, t, w, ncell)
    # per particle: |w - w_q 2^-s| <= 2^-(s+1), |theta - theta_q 2^-24| <= 2^-25
    per = 2.0 ** -(s_w + 1) + w.max() * 2.0**-25
    counts = np.bincount(c, minlength=ncell) + np.bincount((c + 1) % ncell, minlength=ncell)
    assert np.all(np.abs(n_fx - n_64) <= counts * per * 1.01 + 1e-15)


# ----------------------------------------------------------------- field (Section 3.3)


def test_cyclic_tridiag_matches_dense_solve():
    rng = np.random.default_rng(0)
    n = 37
    a, c = -0.7, -1.3
    b = 2.5 + rng.random(n)
    d = rng.standard_normal(n)
    A = np.diag(b) + np.diag(np.full(n - 1, a), -1) + np.diag(np.full(n - 1, c), 1)
    A[0, n - 1] = a
    A[n - 1, 0] = c
    x = orc.cyclic_tridiag(a, b, c, d)
    assert np.allclose(x, np.linalg.solve(A, d), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("mode", [0, 1])
def test_newton_manufactured_solution(mode):
    # phi* = a cos(2 pi m x / L) + b sin(...); n := -D2 phi* + g(phi*). Newton must return phi*.
    ncell, L = 256, 128.0
    dx = L / ncell
    x = np.arange(ncell) * dx
    phi_star = 0.8 * np.cos(2 * np.pi * 3 * x / L) - 0.4 * np.sin(2 * np.pi * 7 * x / L)
    lap = (np.roll(phi_star, 1) - 2 * phi_star + np.roll(phi_star, -1)) / dx**2
    g = np.exp(phi_star) if mode == 0 else 1.0 + phi_star
    n = -lap + g
    phi, iters, fail = orc.newton_pb(n, dx, phi0=np.zeros(ncell), mode=mode, tol=1e-13)
    assert fail == 0
    assert np.max(np.abs(phi - phi_star)) < 1e-12
    if mode == 1:
        assert iters <= 2  # linear problem: one update, one confirming update


def test_newton_linear_limit_fourier_multiplier():
    # small perturbation: phi_hat = n_hat / (1 + K^2), K = (2/dx) sin(k dx / 2)
    ncell, L = 128, 64.0
    dx = L / ncell
    x = np.arange(ncell) * dx
    m = 5
    k = 2 * np.pi * m / L
    eps = 1e-7
    n = 1.0 + eps * np.cos(k * x)
    phi, _, fail = orc.newton_pb(n, dx, tol=1e-15)
    assert fail == 0
    K2 = (2.0 / dx * np.sin(k * dx / 2)) ** 2
    amp = 2.0 / ncell * np.sum(phi * np.cos(k * x))
    assert amp == pytest.approx(eps / (1 + K2), rel=1e-5)


def test_efield_of_sinusoid_is_exact_centred_difference():
    ncell, L = 64, 32.0
    dx = L / ncell
    x = np.arange(ncell) * dx
    k = 2 * np.pi * 3 / L
    E = orc.efield(np.sin(k * x), dx)
    assert np.allclose(E, -np.cos(k * x) * np.sin(k * dx) / dx, atol=1e-14)


# ----------------------------------------------------------------- push (Section 2.2)


def _single(cell, theta, v, w=1.0):
    return orc.State(np.array([cell]), np.array([theta]), np.array([v]), np.array([w]))


def test_push_uniform_field_is_exact_parabola():
    # leapfrog started with a half kick is exact for a constant force
    ncell, L, dt, qm, E0 = 64, 32.0, 0.1, 1.0, 0.37
    dx = L / ncell
    E = np.full(ncell, E0)
    x0, v0 = 10.3, -0.8
    st = _single(int(x0 // dx), (x0 % dx) / dx, v0)
    nsteps = 37
    orc.push(st, E, ncell, dx, dt, qm, kick=0.5)
    for _ in range(nsteps - 1):
        orc.push(st, E, ncell, dx, dt, qm, kick=1.0)
    T = nsteps * dt
    x_exact = (x0 + v0 * T + 0.5 * qm * E0 * T * T) % L
    x = (st.cell[0] + st.theta[0]) * dx
    assert x == pytest.approx(x_exact, abs=1e-11)
    assert st.v[0] == pytest.approx(v0 + qm * E0 * (T - 0.5 * dt), abs=1e-12)


def test_push_harmonic_orbit_matches_discrete_leapfrog_solution():
    # E = -w0^2 (x - xc) on the nodes; CIC interpolation of a linear function is exact,
    # and leapfrog's orbit is x_n - xc = A cos(W n dt) with sin(W dt / 2) = w0 dt / 2.
    ncell, L, dt, qm, w0 = 128, 64.0, 0.2, 1.0, 0.9
    dx = L / ncell
    xc = 32.0
    E = -w0**2 * (np.arange(ncell) * dx - xc)
    A = 5.0
    st = _single(int((xc + A) // dx), ((xc + A) % dx) / dx, 0.0)
    W = 2 * np.arcsin(w0 * dt / 2) / dt
    orc.push(st, E, ncell, dx, dt, qm, kick=0.5)
    errs = []
    for n in range(1, 200):
        x = (st.cell[0] + st.theta[0]) * dx
        errs.append(abs(x - (xc + A * np.cos(W * n * dt))))
        orc.push(st, E, ncell, dx, dt, qm, kick=1.0)
    assert max(errs) < 1e-10


def test_push_free_streaming_wraps():
    ncell, L, dt = 32, 16.0, 0.25
    dx = L / ncell
    st = _single(30, 0.25, 3.3)
    for _ in range(100):
        orc.push(st, np.zeros(ncell), ncell, dx, dt, 1.0)
    x = (st.cell[0] + st.theta[0]) * dx
    assert x == pytest.approx((30.25 * dx + 3.3 * 100 * dt) % L, abs=1e-11)


# ----------------------------------------------------------------- restriction (App. B)


def test_restrict_sample_tau_zero_is_plain_deposit():
    ncell = 64
    c, t, v, w = _state(3000, ncell, 7)
    st = orc.State(c, t, v, w)
    E0 = inputs.random_field(ncell, 2)
    d, m = orc.restrict_sample(st, v, E0, ncell, 0.5, 0.0, 1.0)
    d2, m2 = orc.deposit_f64(c, t, w, ncell, vel=v)
    assert np.allclose(d, d2, atol=1e-14) and np.allclose(m, m2, atol=1e-14)


def test_restrict_sample_follows_characteristics():
    # co-moving sample equals the plain deposit of particles moved to X + tau V with
    # velocity V + qm tau E_n(X); total momentum = sum w (V + qm tau E_n(X))
    ncell, dx, tau, qm = 64, 0.5, 3.7, 1.0
    c, t, v, w = _state(2000, ncell, 8)
    E0 = inputs.random_field(ncell, 3)
    st = orc.State(c, t, v, w)
    d, m = orc.restrict_sample(st, v, E0, ncell, dx, tau, qm)
    X = (c + t) * dx + tau * v
    Xg = np.mod(X, ncell * dx) / dx
    cm = np.floor(Xg).astype(np.int32)
    Eg = orc.gather(E0, c, t)
    vt = v + qm * tau * Eg
    d2, m2 = orc.deposit_f64(cm, Xg - cm, w, ncell, vel=vt)
    assert np.allclose(d, d2, atol=1e-11) and np.allclose(m, m2, atol=1e-11)
    assert m.sum() == pytest.approx(np.sum(w * vt), rel=1e-12)


# ----------------------------------------------------------------- wavelets (App. A)


@pytest.mark.parametrize("wav", ["haar", "d4", "coif4"])
def test_filter_is_orthonormal(wav):
    h = orc.FILTERS[wav]
    L = len(h)
    assert h.sum() == pytest.approx(np.sqrt(2), abs=1e-15)
    for s in range(0, L, 2):
        assert np.dot(h[: L - s], h[s:]) == pytest.approx(1.0 if s == 0 else 0.0, abs=1e-15)
    g = np.array([(-1) ** m * h[L - 1 - m] for m in range(L)])
    moments = {"haar": 1, "d4": 2, "coif4": 4}[wav]  # Daubechies: L/2; the coiflet trades two for phi's
    for q in range(moments):  # vanishing moments of the wavelet
        assert np.dot(np.arange(L) ** q, g) == pytest.approx(0.0, abs=1e-13)


@pytest.mark.parametrize("wav", ["haar", "d4", "coif4"])
def test_dwt_round_trip_and_parseval(wav):
    x = np.random.default_rng(1).standard_normal(64)
    a, d = orc.dwt_level(x, wav)
    assert np.sum(a**2) + np.sum(d**2) == pytest.approx(np.sum(x**2), rel=1e-14)
    assert np.max(np.abs(orc.idwt_level(a, d, wav) - x)) < 1e-14


def test_coif4_moments_through_the_transform():
    # four vanishing wavelet moments: the interior detail coefficients of a cubic vanish
    # (Daubechies-4, with two, does not annihilate it)
    n = 128
    x = np.arange(n, dtype=np.float64)
    cubic = 0.3 + 0.02 * x - 1e-3 * x**2 + 2e-5 * x**3
    _, d = orc.dwt_level(cubic, "coif4")
    inner = slice(0, n // 2 - 6)  # away from the periodic wrap of the 12-tap filter
    assert np.max(np.abs(d[inner])) < 1e-12 * np.max(np.abs(cubic))
    _, d4 = orc.dwt_level(cubic, "d4")
    assert np.max(np.abs(d4[inner])) > 1e-6


@pytest.mark.parametrize("wav,order", [("coif4", 4), ("haar", 1)])
def test_coarse_scaling_coefficients_sample_the_function(wav, order):
    # coiflet property (vanishing scaling-function moments 1..3): after L analysis levels the
    # scaling coefficient k is 2^{L/2} f(2^L k + s_L) up to O(h^4), with s_L = 4 (2^L - 1) for
    # taps stored from k = -4; Haar's block mean is only first order about its block centre.
    L = 2
    errs = []
    for n in (64, 128, 256):
        t = np.arange(n) / n
        f = np.sin(2 * np.pi * 3 * t) + 0.5 * np.cos(2 * np.pi * 5 * t)
        c = orc.coarsen(f, n >> L, wav) * 2.0 ** (np.log2(n) / 2)  # undo the 2^{-J_f/2} of the fine level
        shift = 4 * (2**L - 1) if wav == "coif4" else 0
        tk = ((2**L * np.arange(n >> L) + shift) % n) / n
        want = 2 ** (L / 2) * (np.sin(2 * np.pi * 3 * tk) + 0.5 * np.cos(2 * np.pi * 5 * tk))
        errs.append(np.max(np.abs(c - want)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > order - 0.3), rates


def test_coif4_is_the_concentrated_solution():
    # the coiflet equations have four real solutions; the one used has the largest central
    # tap (its scaling function peaks at 0), and its taps solve the equations to rounding
    h = orc.FILTERS["coif4"]
    assert np.max(np.abs(orc.coif4_equations(h))) < 1e-14
    assert np.argmax(np.abs(h)) == 4 and h[4] > 0.8
    from scipy.optimize import least_squares

    rng = np.random.default_rng(0)
    for _ in range(40):
        r = least_squares(orc.coif4_equations, rng.standard_normal(12) * 0.5, xtol=1e-15, ftol=1e-15, gtol=1e-15)
        if np.max(np.abs(orc.coif4_equations(r.x))) < 1e-12:
            assert r.x[4] <= h[4] + 1e-12


def test_haar_coarsen_is_scaled_block_mean():
    nf, nc = 256, 16
    f = np.random.default_rng(2).standard_normal(nf)
    c = orc.coarsen(f, nc, "haar")
    Jc = 4
    assert np.allclose(c, 2.0 ** (-Jc / 2) * f.reshape(nc, -1).mean(axis=1), atol=1e-14)
    back = orc.refine(c, nf, "haar")
    assert np.allclose(back, np.repeat(f.reshape(nc, -1).mean(axis=1), nf // nc), atol=1e-13)


@pytest.mark.parametrize("wav", ["haar", "d4", "coif4"])
def test_coarsen_constant_and_refine_coarsen_identity(wav):
    nf, nc = 128, 16
    c = orc.coarsen(np.full(nf, 3.0), nc, wav)
    assert np.allclose(c, 3.0 * 2.0 ** (-4 / 2), atol=1e-13)
    cc = np.random.default_rng(4).standard_normal(nc)
    assert np.allclose(orc.coarsen(orc.refine(cc, nf, wav), nc, wav), cc, atol=1e-13)


# ----------------------------------------------------------------- projection (Section 3.3)


def test_ls_weights_match_paper_golden():
    rows = read_golden("ls_weights_Ne6.txt")
    K = 6
    for p, num, den in rows:
        p = int(p)
        # the slope of the unit sample at K-p is the weight of pair p
        w_p = orc.ls_slope(np.eye(K + 1)[K - p], 1.0)
        assert w_p == pytest.approx(int(num) / int(den), abs=1e-15)


def test_ls_slope_matches_paired_form_and_polyfit():
    rng = np.random.default_rng(5)
    for K in (1, 2, 5, 6, 20, 31):
        y = rng.standard_normal(K + 1)
        dt = 0.1
        paired = sum(6 * (K - 2 * p) / (K * (K + 1) * (K + 2) * dt) * (y[K - p] - y[p]) for p in range(K // 2 + 1))
        s = orc.ls_slope(y, dt)
        assert s == pytest.approx(paired, rel=1e-12, abs=1e-12)
        assert s == pytest.approx(np.polyfit(np.arange(K + 1) * dt, y, 1)[0], rel=1e-10)


def test_ls_project_exact_on_linear_data_and_conserves_charge():
    K, nc, dt, dT = 20, 8, 0.1, 20.0
    rng = np.random.default_rng(6)
    a, b = rng.standard_normal(nc), rng.standard_normal(nc)
    t = np.arange(K + 1) * dt
    samples = a[None, :] + b[None, :] * t[:, None]
    out, slope = orc.ls_project(samples, dt, dT)
    assert np.allclose(slope, b, atol=1e-12)
    assert np.allclose(out, a + b * dT, atol=1e-11)
    # Remark (charge conservation): constant column sums give constant projected sum
    noisy = rng.standard_normal((K + 1, nc))
    noisy -= noisy.sum(axis=1, keepdims=True) / nc
    noisy += 1.0
    out, _ = orc.ls_project(noisy, dt, dT)
    assert out.sum() == pytest.approx(nc * 1.0, abs=1e-11)


# ----------------------------------------------------------------- lifting (App. C)


def test_ndtri_matches_scipy():
    p = np.concatenate([np.linspace(1e-6, 1 - 1e-6, 301), [1e-12, 2.3e-10, 0.5, 1 - 1e-9]])
    assert np.allclose(orc.ndtri(p), scipy.special.ndtri(p), rtol=1e-13, atol=1e-14)


def test_quiet_start_hammersley_velocities_and_positions():
    # the loaded points are the Hammersley pairs ((2i+1)/2N, phi_2(i) + shift) of the golden
    # table; a power-of-two cell stores them in ascending order of the velocity quantile
    N, ncell, seed = 16, 1, 99
    st = orc.quiet_start(N, ncell, np.ones(1), np.zeros(1), 1.0, seed)
    shift = orc.splitmix64(seed) >> 32
    B = np.rint(scipy.special.ndtr(st.v) * 2.0**32 - 0.5).astype(np.int64)
    phi2 = ((B - shift - (2**31 // N)) % 2**32) / 2**28
    gold = {int(i): int(v) for i, v in read_golden("hammersley_base2.txt")}
    pairs = sorted(zip(np.rint(st.theta * 2 * N).astype(int), np.rint(phi2).astype(int)))
    assert pairs == sorted((2 * i + 1, gold[i]) for i in range(N))
    assert np.all(np.diff(phi2) > 0)  # ascending velocity quantile inside the cell


def test_quiet_start_weights_sum_and_moments():
    ncell, ppc = 64, 256
    nprof, uprof = orc.sine_profile(ncell, 32.0, 0.3)
    st = orc.quiet_start(ncell * ppc, ncell, nprof, uprof, 1.0, 7)
    assert st.w.sum() == pytest.approx(nprof.sum(), rel=1e-13)
    # Hammersley velocities: per cell the v_th-normalised thermal part has ~zero mean, unit variance
    X = st.cell + st.theta
    u_at = np.interp(X, np.arange(ncell + 1), np.append(uprof, uprof[0]))
    therm = st.v - u_at
    assert abs(therm.mean()) < 1e-3
    assert therm.var() == pytest.approx(1.0, rel=2e-3)


def test_lift_profile_clamps_and_conserves_mass():
    n = np.array([1.0, -0.2, 0.5, 2.0])
    m = np.array([0.5, 0.1, -0.5, 1.0])
    nn, u = orc.lift_profile(n, m)
    assert np.all(nn >= 0) and nn.sum() == pytest.approx(n.sum())
    assert u[1] == 0.0 and u[0] == pytest.approx(0.5 / nn[0])


def test_restrict_of_lift_reproduces_coarse_state():
    cfg = inputs.workload("iaw_small")
    ncell, nc = cfg["ncell"], cfg["n_coarse"]
    nprof, uprof = orc.sine_profile(ncell, cfg["L"], 0.3)
    coarse = np.stack([orc.coarsen(nprof, nc), orc.coarsen(nprof * uprof, nc)])
    st = orc.lift(coarse, cfg, seed=1)
    d, m = orc.deposit_f64(st.cell, st.theta, st.w, ncell, vel=st.v)
    back = np.stack([orc.coarsen(d, nc), orc.coarsen(m, nc)])
    assert np.max(np.abs(back[0] - coarse[0])) / np.max(np.abs(coarse[0])) < 2e-3
    assert np.max(np.abs(back[1] - coarse[1])) / np.max(np.abs(coarse[1])) < 2e-2


# ----------------------------------------------------------------- whole bursts


def _cfg(**kw):
    base = dict(ncell=32, L=16.0, N=32 * 64, dt=0.1, qm=1.0, K=10, M=2, n_coarse=8, v_th=0.0)
    base.update(kw)
    base["dT"] = base["M"] * base["K"] * base["dt"]
    base["s_w"] = orc.fx_shift(4.0 * base["ncell"] / base["N"])
    return base


def test_burst_cold_drifting_plasma_is_a_fixed_point():
    # uniform density, uniform drift: E == 0, slope 0, projection reproduces the state
    cfg = _cfg(v_th=0.0)
    ncell = cfg["ncell"]
    st = orc.quiet_start(cfg["N"], ncell, np.ones(ncell), np.full(ncell, 0.25), 0.0, 1)
    coarse, cs, phi = orc.efpi_macro_step(st, cfg, np.zeros(ncell))
    assert np.max(np.abs(phi)) < 1e-13
    expect_n = 2.0 ** (-3 / 2) * 1.0
    assert np.allclose(coarse[0], expect_n, atol=1e-12)
    assert np.allclose(coarse[1], 0.25 * expect_n, atol=1e-12)


def test_burst_without_leap_equals_restriction_of_final_state():
    # Appendix B: the co-moving sample at s = t_{n+1} is f(t_{n+1}); with dT = K dt there is no leap
    cfg = _cfg(v_th=1.0, M=1)
    ncell = cfg["ncell"]
    nprof, uprof = orc.sine_profile(ncell, cfg["L"], 0.2)
    st = orc.quiet_start(cfg["N"], ncell, nprof, uprof, 1.0, 3)
    st2 = st.copy()
    coarse, cs, phi = orc.efpi_macro_step(st, cfg, np.zeros(ncell))
    # integer-time velocity of the final state
    dx = cfg["L"] / ncell
    phi2, _ = orc.pic_steps(st2, ncell, dx, cfg["dt"], 1.0, cfg["K"], cfg["s_w"], np.zeros(ncell))
    rho = orc.deposit_fx(st2.cell, st2.theta, st2.w, ncell, cfg["s_w"]) * 2.0 ** -(cfg["s_w"] + 24)
    phi3, _, _ = orc.newton_pb(rho, dx, phi0=phi2)
    E = orc.efield(phi3, dx)
    Eg = orc.gather(E, st2.cell, st2.theta)
    vbar = st2.v + 0.5 * cfg["dt"] * Eg
    d, m = orc.deposit_f64(st2.cell, st2.theta, st2.w, ncell, vel=vbar)
    assert np.allclose(coarse[0], orc.coarsen(d, cfg["n_coarse"]), atol=1e-12)
    assert np.allclose(coarse[1], orc.coarsen(m, cfg["n_coarse"]), atol=1e-11)


def test_linearised_mode_conserves_momentum():
    ncell = 64
    cfg = _cfg(ncell=ncell, L=32.0, N=ncell * 64)
    nprof, uprof = orc.sine_profile(ncell, cfg["L"], 0.3)
    st = orc.quiet_start(cfg["N"], ncell, nprof, uprof, 1.0, 11)
    dx = cfg["L"] / ncell
    P0 = np.sum(st.w * st.v)
    # a fine fixed-point scale (weights ~2^28 quanta) so that the deposit's quantisation,
    # the one non-conservative term, stays far below the tolerance
    orc.pic_steps(st, ncell, dx, cfg["dt"], 1.0, 40, 34, np.zeros(ncell), mode=1, vel_at_integer=False)
    P1 = np.sum(st.w * st.v)
    assert abs(P1 - P0) < 1e-11 * np.sum(st.w * np.abs(st.v))


@pytest.mark.parametrize("mode", [0, 1])
def test_cold_ion_acoustic_dispersion(mode):
    # linear ion-acoustic wave, cold ions, Boltzmann electrons (Eq. poisson2rescaled linearised):
    # W_d^2 = qm k kappa S^2 / (1 + K^2), kappa = sin(k dx)/dx, S = sinc^2(k dx / 2),
    # K = (2/dx) sin(k dx / 2); leapfrog: sin(W dt / 2) = W_d dt / 2.
    ncell, L, ppc, dt, delta = 32, 16.0, 64, 0.1, 1e-3
    dx = L / ncell
    k = 2 * np.pi / L
    nprof, uprof = orc.sine_profile(ncell, L, delta)
    st = orc.quiet_start(ncell * ppc, ncell, nprof, np.zeros(ncell), 0.0, 0)
    s_w = orc.fx_shift(2.0 / ppc)
    x = np.arange(ncell) * dx
    phi = np.zeros(ncell)
    amps = []
    nsteps = 600
    for s in range(nsteps):
        rho = orc.deposit_fx(st.cell, st.theta, st.w, ncell, s_w) * 2.0 ** -(s_w + 24)
        amps.append(np.sum((rho - 1.0) * np.cos(k * x)))
        phi, _, fail = orc.newton_pb(rho, dx, phi0=phi, mode=mode, tol=1e-14)
        assert fail == 0
        orc.push(st, orc.efield(phi, dx), ncell, dx, dt, 1.0, kick=0.5 if s == 0 else 1.0)
    a = np.array(amps)
    t = np.arange(nsteps) * dt
    z = np.where(np.sign(a[:-1]) != np.sign(a[1:]))[0]
    tz = t[z] - a[z] * dt / (a[z + 1] - a[z])
    W = np.pi / np.mean(np.diff(tz))
    S = np.sinc(k * dx / 2 / np.pi) ** 2
    kappa = np.sin(k * dx) / dx
    K2 = (2 / dx * np.sin(k * dx / 2)) ** 2
    Wd = np.sqrt(k * kappa * S**2 / (1 + K2))
    W_leap = 2 * np.arcsin(Wd * dt / 2) / dt
    assert len(tz) >= 5
    assert W == pytest.approx(W_leap, rel=3e-3)
    # the continuum answer k/sqrt(1+k^2) differs by more than the tolerance used above
    assert abs(k / np.sqrt(1 + k * k) - W_leap) / W_leap > 3e-3


# ----------------------------------------------------------------- diagnostics (Section 4)


def test_moments_closed_forms():
    ncell, L = 32, 16.0
    dx = L / ncell
    x = np.arange(ncell) * dx
    A = 0.7
    E = A * np.sin(2 * np.pi * x / L)
    # one particle at rest in the middle of cell 5, weight 0.25, field sampled there
    st = orc.State([5], [0.5], [0.0], [0.25])
    s_w = 20
    zero = np.zeros(ncell)
    m = orc.moments(st, E, zero, ncell, dx, 0.1, 1.0, 0.5, s_w)
    # discrete sum of sin^2 over a whole period is ncell / 2
    assert m["field_energy"] == pytest.approx(A * A * L / 4, rel=1e-14)
    assert m["electron_energy"] == 0.0
    assert m["charge"] == pytest.approx(0.25 * dx, rel=1e-15)
    assert m["charge_fx"] == round(0.25 * 2**s_w) * 2**24
    assert m["momentum"] == 0.0 and m["kinetic"] == 0.0
    # kick = 1: the half kick of a half-integer velocity, E(X) = mean of the two nodes
    st2 = orc.State([5], [0.5], [0.3], [0.25])
    Ex = 0.5 * (E[5] + E[6])
    m = orc.moments(st2, E, zero, ncell, dx, 0.1, 2.0, 1.0, s_w)
    vb = 0.3 + 0.5 * 2.0 * 0.1 * Ex
    assert m["momentum"] == pytest.approx(0.25 * vb * dx, rel=1e-14)
    assert m["kinetic"] == pytest.approx(0.5 * 0.25 * vb * vb * dx, rel=1e-14)
    assert m["cfl"] == pytest.approx(abs(vb) * 0.1 / dx, rel=1e-14)
    # constant potential c: Boltzmann free energy (c e^c - e^c + 1) L, linearised c^2 L / 2
    c = 0.4
    phi = np.full(ncell, c)
    m0 = orc.moments(st, zero, phi, ncell, dx, 0.1, 1.0, 0.5, s_w, mode=0)
    m1 = orc.moments(st, zero, phi, ncell, dx, 0.1, 1.0, 0.5, s_w, mode=1)
    assert m0["electron_energy"] == pytest.approx((c * np.exp(c) - np.exp(c) + 1) * L, rel=1e-13)
    assert m1["electron_energy"] == pytest.approx(0.5 * c * c * L, rel=1e-13)


def test_moments_of_quiet_start_maxwellian():
    ncell, L, ppc, u0, vth = 32, 16.0, 1024, 0.3, 0.8
    st = orc.quiet_start(ncell * ppc, ncell, np.ones(ncell), np.full(ncell, u0), vth, 7)
    m = orc.moments(st, np.zeros(ncell), np.zeros(ncell), ncell, L / ncell, 0.1, 1.0, 0.5, 16)
    assert m["charge"] == pytest.approx(L, rel=1e-12)
    assert m["momentum"] == pytest.approx(u0 * L, rel=2e-3)
    assert m["kinetic"] == pytest.approx(0.5 * L * (u0 * u0 + vth * vth), rel=2e-3)
    # the charge in fixed point is the sum of the deposit
    rho = orc.deposit_fx(st.cell, st.theta, st.w, ncell, 16)
    assert m["charge_fx"] == int(rho.sum())


@pytest.mark.parametrize("mode", [0, 1])
def test_moments_energy_conserved_by_resolved_pic(mode):
    """Ion kinetic + field + electron free energy stays constant while field and kinetic
    energy exchange a much larger amount (Boltzmann and linearised electrons)."""
    ncell, L, ppc, dt = 64, 32.0, 128, 0.1
    dx = L / ncell
    n, u = orc.sine_profile(ncell, L, 0.3)
    st = orc.quiet_start(ncell * ppc, ncell, n, u, 0.1, 3)
    s_w = orc.fx_shift(8.0 / ppc)
    phi = np.zeros(ncell)
    E = orc.field_of(st, ncell, dx, s_w, phi, mode=mode)
    hist = [orc.moments(st, E, phi, ncell, dx, dt, 1.0, 0.5, s_w, mode)]
    vint = True
    for _ in range(6):
        phi = orc.pic_steps(st, ncell, dx, dt, 1.0, 20, s_w, phi, mode=mode, vel_at_integer=vint)[0]
        vint = False
        E = orc.field_of(st, ncell, dx, s_w, phi, mode=mode)
        hist.append(orc.moments(st, E, phi, ncell, dx, dt, 1.0, 1.0, s_w, mode))
    H = np.array([h["total_energy"] for h in hist])
    pot = np.array([h["field_energy"] + h["electron_energy"] for h in hist])
    kin = np.array([h["kinetic"] for h in hist])
    assert np.ptp(pot) > 0.05 and np.ptp(kin) > 0.05
    assert np.abs(H - H[0]).max() < 0.05 * np.ptp(pot)


def test_rel_l2_closed_forms():
    a = np.array([1.0, -2.0, 3.0])
    assert orc.rel_l2(a, a) == 0.0
    assert orc.rel_l2(a, np.zeros(3)) == pytest.approx(1.0, rel=1e-15)
    assert orc.rel_l2(a, -a) == pytest.approx(np.sqrt(2.0), rel=1e-15)
    assert orc.rel_l2([1.0, 0.0], [0.0, 1.0]) == pytest.approx(1.0, rel=1e-15)
    assert orc.rel_l2([3.0], [1.0]) == pytest.approx(np.sqrt(4.0 / 10.0), rel=1e-15)
