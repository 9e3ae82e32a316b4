"""Pins of the bounded-domain oracle (Section 4.2: the slab expansion with an absorbing
boundary and phi' = 0 at the walls). Walls sit at node 0 and node ncell-1; the wall
nodes' densities are twice their deposits (half control volumes). No GPU needed.

The pins are closed forms (cosine eigenvectors of the Neumann Laplacian), invariants
(the discrete Gauss law with Neumann walls, mirror symmetry of a mirrored particle set),
brute force (free-streaming absorption) and the linear ion-acoustic standing wave, whose
bounded-domain frequency equals that of the periodic wave of twice the length.
"""
import numpy as np
import pytest

import oracle as orc


def _cos_mode(ncell, m):
    j = np.arange(ncell)
    return np.cos(np.pi * m * j / (ncell - 1))


def _K2(ncell, dx, m):
    # eigenvalue of -D2 with mirror ghosts on the cosine mode m: (2/dx)^2 sin^2(pi m / (2 (ncell-1)))
    return (2.0 / dx * np.sin(np.pi * m / (2 * (ncell - 1)))) ** 2


def _dep_from_density(n):
    dep = np.array(n, dtype=np.float64)
    dep[[0, -1]] *= 0.5
    return dep


@pytest.mark.parametrize("mode", [0, 1])
def test_newton_walls_manufactured_cosine_solution(mode):
    # phi* = a cos(pi m x / L_w) + b cos(pi m' x / L_w) satisfies phi' = 0 at both walls and
    # the mirror ghosts exactly; n = K^2 phi* + g(phi*) from the closed-form eigenvalues.
    ncell, dx = 256, 0.5
    phi_star = 0.7 * _cos_mode(ncell, 3) - 0.3 * _cos_mode(ncell, 10)
    g = np.exp(phi_star) if mode == 0 else 1.0 + phi_star
    n = _K2(ncell, dx, 3) * 0.7 * _cos_mode(ncell, 3) - _K2(ncell, dx, 10) * 0.3 * _cos_mode(ncell, 10) + g
    phi, iters, fail = orc.newton_pb_walls(_dep_from_density(n), dx, phi0=np.zeros(ncell), mode=mode, tol=1e-13)
    assert fail == 0
    assert np.max(np.abs(phi - phi_star)) < 1e-12
    # the periodic solver on the same data does not give phi* (the walls matter)
    phi_p, _, _ = orc.newton_pb(n, dx, phi0=np.zeros(ncell), mode=mode, tol=1e-13)
    assert np.max(np.abs(phi_p - phi_star)) > 1e-3


def test_newton_walls_linear_limit_cosine_multiplier():
    ncell, dx, m, eps = 128, 0.5, 4, 1e-7
    n = 1.0 + eps * _cos_mode(ncell, m)
    phi, _, fail = orc.newton_pb_walls(_dep_from_density(n), dx, tol=1e-15)
    assert fail == 0
    assert np.allclose(phi, eps * _cos_mode(ncell, m) / (1 + _K2(ncell, dx, m)), rtol=0, atol=1e-13)


def test_newton_walls_gauss_law_with_neumann_walls():
    # summing the equations with the trapezoid weights (1/2 at the walls) telescopes the
    # Laplacian to the wall fluxes, which vanish: sum dep = sum_j omega_j exp(phi_j)
    ncell, dx = 512, 0.5
    rng = np.random.default_rng(4)
    dens = np.zeros(ncell)
    dens[200:300] = 1.0 + 0.3 * rng.random(100)
    dep = _dep_from_density(dens)
    phi, _, fail = orc.newton_pb_walls(dep, dx, tol=1e-13)
    assert fail == 0
    omega = np.ones(ncell)
    omega[[0, -1]] = 0.5
    assert np.sum(omega * np.exp(phi)) == pytest.approx(dep.sum(), rel=1e-11)
    # vacuum potential is monotone towards the walls and flat at them
    assert phi[0] < phi[100] < phi[199] and phi[-1] < phi[400] < phi[300]


def test_efield_walls_closed_form_and_zero_at_walls():
    ncell, dx, m = 64, 0.5, 5
    j = np.arange(ncell)
    E = orc.efield_walls(_cos_mode(ncell, m), dx)
    a = np.pi * m / (ncell - 1)
    assert np.allclose(E, np.sin(a * j) * np.sin(a) / dx, atol=1e-14)
    assert E[0] == 0.0 and E[-1] == 0.0


def _single(cell, theta, v, w=1.0):
    return orc.State(np.array([cell]), np.array([theta]), np.array([v]), np.array([w]))


def test_push_walls_free_streaming_absorption_brute_force():
    ncell, dx, dt = 32, 0.5, 0.1
    Lw = (ncell - 1) * dx
    rng = np.random.default_rng(1)
    n = 400
    X0 = rng.random(n) * Lw
    v0 = rng.standard_normal(n) * 2.0
    cell = np.floor(X0 / dx).astype(np.int32)
    st = orc.State(cell, X0 / dx - cell, v0, np.full(n, 0.25))
    E = np.zeros(ncell)
    nsteps = 40
    for s in range(nsteps):
        orc.push_walls(st, E, ncell, dx, dt, 1.0, kick=0.5 if s == 0 else 1.0)
    # brute force: the straight line leaves [0, Lw) at the first step k with X0 + k v dt outside
    k = np.arange(1, nsteps + 1)
    Xk = X0[:, None] + v0[:, None] * dt * k[None, :]
    out = (Xk < 0) | (Xk >= Lw)
    absorbed = out.any(axis=1)
    assert absorbed.any() and (~absorbed).any()
    assert np.array_equal(st.w == 0.0, absorbed)
    alive = ~absorbed
    X = (st.cell + st.theta) * dx
    assert np.allclose(X[alive], Xk[alive, -1], atol=1e-11)
    assert np.all(st.v[absorbed] == 0.0) and np.all(st.theta[absorbed] == 0.0)
    left = absorbed & (Xk[np.arange(n), np.argmax(out, axis=1)] < 0)
    assert np.all(st.cell[left] == 0) and np.all(st.cell[absorbed & ~left] == ncell - 1)


def test_push_walls_uniform_field_parabola_then_absorbed():
    ncell, dx, dt, qm, E0 = 64, 0.5, 0.1, 1.0, -0.2
    E = np.full(ncell, E0)
    E[[0, -1]] = E0  # a prescribed field (not a Neumann solution): the push only gathers
    x0, v0 = 6.0, 0.3
    st = _single(int(x0 // dx), (x0 % dx) / dx, v0)
    orc.push_walls(st, E, ncell, dx, dt, qm, kick=0.5)
    n = 1
    while st.w[0] != 0.0:
        T = n * dt
        x = (st.cell[0] + st.theta[0]) * dx
        assert x == pytest.approx(x0 + v0 * T + 0.5 * qm * E0 * T * T, abs=1e-11)
        orc.push_walls(st, E, ncell, dx, dt, qm, kick=1.0)
        n += 1
    # absorbed at the first step whose exact parabola is below 0
    T = np.arange(1, n + 1) * dt
    xs = x0 + v0 * T + 0.5 * qm * E0 * T * T
    assert np.argmax(xs < 0) == n - 1
    assert st.cell[0] == 0 and st.v[0] == 0.0
    before = st.copy()
    orc.push_walls(st, E, ncell, dx, dt, qm, kick=1.0)  # frozen
    assert st.cell[0] == before.cell[0] and st.theta[0] == before.theta[0] and st.v[0] == 0.0


def test_restrict_sample_walls_is_deposit_of_moved_particles_inside():
    ncell, dx, tau, qm = 64, 0.5, 2.3, 1.0
    Lw = (ncell - 1) * dx
    rng = np.random.default_rng(2)
    n = 3000
    X0 = rng.random(n) * Lw
    cell = np.floor(X0 / dx).astype(np.int32)
    th = X0 / dx - cell
    v = rng.standard_normal(n) * 1.5
    w = rng.random(n)
    w[::17] = 0.0
    E0 = 0.1 * np.sin(np.arange(ncell) * 0.3)
    st = orc.State(cell, th, v, w)
    d, m = orc.restrict_sample_walls(st, v, E0, ncell, dx, tau, qm)
    Xt = X0 + tau * v
    keep = (Xt >= 0) & (Xt < Lw) & (w > 0)
    cm = np.floor(Xt[keep] / dx).astype(np.int32)
    vt = v + qm * tau * orc.gather(E0, cell, th)
    d2, m2 = orc.deposit_f64(cm, Xt[keep] / dx - cm, w[keep], ncell, vel=vt[keep])
    assert np.allclose(d, d2, atol=1e-11) and np.allclose(m, m2, atol=1e-11)
    assert (~keep & (w > 0)).sum() > 100  # the walls removed a part of the sample


def _point_order(N, bits=12):
    """Point index held by each storage slot: the low 12 bits reversed inside full blocks of 4096."""
    s = np.arange(N)
    rev = np.zeros(N, np.int64)
    for b in range(bits):
        rev |= ((s >> b) & 1) << (bits - 1 - b)
    full = (s | ((1 << bits) - 1)) < N
    return np.where(full, (s & ~((1 << bits) - 1)) | rev, s)


def _by_point(arr, N):
    out = np.empty_like(arr)
    out[_point_order(N)] = arr
    return out


def test_quiet_start_equal_uniform_profile_is_uniform_lattice():
    ncell, N = 33, 3 * 4096 + 17  # a ragged last block
    dx = 0.5
    st = orc.quiet_start_equal(N, ncell, np.ones(ncell), np.zeros(ncell), 1.0, 5)
    X = _by_point((st.cell + st.theta) * dx, N)
    assert np.allclose(X, (np.arange(N) + 0.5) / N * (ncell - 1) * dx, atol=1e-12)
    assert np.all(st.w == (ncell - 1) / N)
    # storage: every full block of 4096 slots holds its points in ascending velocity quantile,
    # cyclically (the Cranley-Patterson shift wraps the quantiles once)
    v = st.v[: (N // 4096) * 4096].reshape(-1, 4096)
    assert np.all(np.sum(np.diff(v, axis=1) < 0, axis=1) <= 1)


def test_quiet_start_equal_counts_follow_mass_and_ramp_is_sqrt():
    ncell, N = 64, 6400
    n, u = orc.slab_profile(ncell)
    st = orc.quiet_start_equal(N, ncell, n, u, 1.0, 11)
    m = 0.5 * (n[:-1] + n[1:])
    C = np.concatenate([[0.0], np.cumsum(m)])
    M = C[-1]
    assert st.w.sum() == pytest.approx(M, rel=1e-13)
    counts = np.bincount(st.cell, minlength=ncell)
    cell_p, theta_p = _by_point(st.cell, N), _by_point(st.theta, N)
    # particle i sits in cell c iff C_c <= (i + 1/2) M / N < C_{c+1}
    want = np.ceil(C[1:] * N / M - 0.5) - np.ceil(C[:-1] * N / M - 0.5)
    assert np.array_equal(counts[:-1], want.astype(int)) and counts[-1] == 0
    assert counts[: 7 * ncell // 16 - 1].sum() == 0 and counts[9 * ncell // 16 + 1:].sum() == 0
    # rising ramp cell (density 0 -> 1): mass up to t is t^2 / 2, so t = sqrt(r)
    c0 = 7 * ncell // 16 - 1
    idx = np.nonzero(cell_p == c0)[0]
    r = ((idx + 0.5) * M / N - C[c0]) / m[c0]
    assert np.allclose(theta_p[idx], np.sqrt(r), atol=1e-13)
    # falling ramp (1 -> 0): t = 1 - sqrt(1 - r)
    c1 = 9 * ncell // 16
    idx = np.nonzero(cell_p == c1)[0]
    r = ((idx + 0.5) * M / N - C[c1]) / m[c1]
    assert np.allclose(theta_p[idx], 1 - np.sqrt(1 - r), atol=1e-12)


def test_quiet_start_equal_deposit_reproduces_profile():
    ncell, N = 128, 1 << 17
    j = np.arange(ncell)
    n = 1.0 + 0.4 * np.cos(np.pi * 3 * j / (ncell - 1))
    st = orc.quiet_start_equal(N, ncell, n, np.zeros(ncell), 1.0, 1)
    dep = orc.deposit_f64(st.cell, st.theta, st.w, ncell)
    dens = dep.copy()
    dens[[0, -1]] *= 2.0
    # CIC of a linear-in-cell density at quantile points: second-order in dx, the nodal
    # value error is the curvature term (dx^2 / 6) |n''| plus the ~1/ppc quadrature error
    curv = 0.4 * (np.pi * 3 / (ncell - 1)) ** 2
    assert np.max(np.abs(dens - n)) < curv / 6 + 2e-3
    v = st.v
    assert abs(v.mean()) < 1e-3 and v.var() == pytest.approx(1.0, rel=2e-3)


def _mirror(st, ncell):
    """x -> L_w - x, v -> -v of a particle set (cell c, theta t) -> (ncell - 2 - c, 1 - t)."""
    c = ncell - 2 - st.cell
    t = 1.0 - st.theta
    wrap = t >= 1.0
    c = np.where(wrap, c + 1, c)
    t = np.where(wrap, 0.0, t)
    return orc.State(c, t, -st.v, st.w)


def test_burst_walls_preserves_mirror_symmetry():
    # a mirror-symmetric particle set stays mirror-symmetric: any asymmetry between the two
    # walls (ghosts, doubling, absorption side) breaks it
    ncell, dx, dt, K = 128, 0.5, 0.1, 30
    n, u = orc.slab_profile(ncell)
    half = orc.quiet_start_equal(8192, ncell, n, u, 1.0, 3)
    half.v *= 3.0  # fast enough that some ions reach the walls within the burst
    mir = _mirror(half, ncell)
    st = orc.State(np.concatenate([half.cell, mir.cell]), np.concatenate([half.theta, mir.theta]),
                   np.concatenate([half.v, mir.v]), np.concatenate([half.w, mir.w]))
    s_w = orc.fx_shift(4 * st.w.max())
    samples, phi, fails = orc.burst_walls(st, ncell, dx, dt, 1.0, K, 2.0 * K * dt, s_w, np.zeros(ncell), tol=1e-13)
    assert fails == 0
    assert np.allclose(phi, phi[::-1], atol=1e-9)
    assert np.allclose(samples[:, 0], samples[:, 0, ::-1], atol=1e-9)
    assert np.allclose(samples[:, 1], -samples[:, 1, ::-1], atol=1e-9)
    absorbed = st.w == 0.0
    assert absorbed.sum() > 10
    X = (st.cell + st.theta) * dx
    Lw = (ncell - 1) * dx
    a, b = absorbed[: half.n], absorbed[half.n:]
    assert np.array_equal(a, b)
    assert np.allclose(X[: half.n][~a], Lw - X[half.n:][~b], atol=1e-9)


@pytest.mark.parametrize("mode", [0, 1])
def test_cold_ion_acoustic_standing_wave_dispersion(mode):
    # cos(k x) with k = pi m / L_w: the bounded system equals the mirror-extended periodic one of
    # length 2 L_w while no ion reaches a wall, so the periodic dispersion relation holds:
    # W_d^2 = qm k kappa S^2 / (1 + K^2), kappa = sin(k dx)/dx, S = sinc^2(k dx / 2),
    # K = (2/dx) sin(k dx / 2); leapfrog: sin(W dt / 2) = W_d dt / 2.
    ncell, dx, ppc, dt, delta = 33, 0.5, 64, 0.1, 1e-3
    Lw = (ncell - 1) * dx
    k = 2 * np.pi / Lw  # standing-wave mode m = 2
    j = np.arange(ncell)
    nprof = 1.0 + delta * np.cos(k * j * dx)
    st = orc.quiet_start_equal((ncell - 1) * ppc, ncell, nprof, np.zeros(ncell), 0.0, 0)
    s_w = orc.fx_shift(2.0 / ppc)
    omega = np.ones(ncell)
    omega[[0, -1]] = 0.5
    phi = np.zeros(ncell)
    amps = []
    nsteps = 700
    for s in range(nsteps):
        dep = orc.deposit_fx(st.cell, st.theta, st.w, ncell, s_w) * 2.0 ** -(s_w + 24)
        dens = dep.copy()
        dens[[0, -1]] *= 2.0
        amps.append(np.sum(omega * (dens - 1.0) * np.cos(k * j * dx)))
        phi, _, fail = orc.newton_pb_walls(dep, dx, phi0=phi, mode=mode, tol=1e-14)
        assert fail == 0
        orc.push_walls(st, orc.efield_walls(phi, dx), ncell, dx, dt, 1.0, kick=0.5 if s == 0 else 1.0)
    assert np.all(st.w > 0)
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
    assert abs(k / np.sqrt(1 + k * k) - W_leap) / W_leap > 3e-3


def test_pic_walls_charge_accounting_is_exact():
    # the fixed-point charge of the live ions plus that of the absorbed ones is the initial
    # charge, to the bit
    ncell, dx, dt = 64, 0.5, 0.1
    n, u = orc.slab_profile(ncell)
    st = orc.quiet_start_equal(20000, ncell, n, u, 2.0, 9)
    s_w = orc.fx_shift(4 * st.w.max())
    wq = np.rint(st.w * 2.0**s_w).astype(np.int64)
    q0 = int(orc.deposit_fx(st.cell, st.theta, st.w, ncell, s_w).sum())
    assert q0 == int(wq.sum()) << 24
    phi, fails = orc.pic_steps_walls(st, ncell, dx, dt, 1.0, 150, s_w, np.zeros(ncell))
    assert fails == 0
    gone = st.w == 0.0
    assert gone.sum() > 100
    q1 = int(orc.deposit_fx(st.cell, st.theta, st.w, ncell, s_w).sum())
    assert q1 + (int(wq[gone].sum()) << 24) == q0
    assert np.all((st.cell[~gone] >= 0) & (st.cell[~gone] < ncell - 1))


def test_restrict_of_lift_walls_reproduces_coarse_state():
    # lifting (refine, clamp, wall deposits doubled to densities, equal-weight loading) followed
    # by the tau = 0 restriction returns the coarse state up to the loading's quadrature error;
    # the coarse state is non-zero at the walls, so the wall doubling is exercised
    ncell, nc, N = 256, 32, 256 * 512
    dx = 0.5
    j = np.arange(ncell)
    dens = 1.0 + 0.4 * np.cos(np.pi * 3 * j / (ncell - 1))
    dep = dens.copy()
    dep[[0, -1]] *= 0.5
    mom = 0.1 * dep
    c = np.stack([orc.coarsen(dep, nc), orc.coarsen(mom, nc)])
    cfg = dict(ncell=ncell, N=N, v_th=0.0, wavelet="haar")
    st = orc.lift_walls(c, cfg, seed=3)
    d, m = orc.restrict_sample_walls(st, st.v, np.zeros(ncell), ncell, dx, 0.0, 1.0)
    back = np.stack([orc.coarsen(d, nc), orc.coarsen(m, nc)])
    assert np.max(np.abs(back - c)) < 2e-3 * np.max(np.abs(c))
    # total charge is exact: sum of the weights = sum of the refined deposits
    assert st.w.sum() == pytest.approx(orc.refine(c[0], ncell).sum(), rel=1e-12)


# ----------------------------------------------------------------- phase space on the bounded grid


def test_ps_quiet_start_equal_uniform_tables_closed_form():
    # equal bin masses and identical uniform velocity histograms: positions on the uniform
    # lattice and V = v_min + (n_v dv) b_i exactly (the inverse CDF of a uniform histogram)
    ncell, b, nv, N, seed = 64, 3, 16, 3 * 4096 + 5, 7
    H = np.ones((ncell >> b, nv))
    mass, cdf, bad = orc.ps_lift_tables(H)
    assert bad == 0
    vmin, dv = -4.0, 0.5
    st = orc.ps_quiet_start_equal(N, ncell, b, mass, cdf, vmin, dv, seed)
    X = _by_point(st.cell + st.theta, N)
    # every bin's density is its mass over its width inside the domain (the wall bins are half
    # a node narrower): the ends of the profile are denser, and the lattice follows the mass
    width = 1 << b
    wid = np.full(ncell >> b, float(width))
    wid[[0, -1]] -= 0.5
    assert np.all(np.diff(X) > 0) and X[0] > 0 and X[-1] < ncell - 1
    i = np.arange(N, dtype=np.uint64)
    rev = np.zeros(N, np.uint64)
    for k in range(32):
        rev |= ((i >> np.uint64(k)) & np.uint64(1)) << np.uint64(31 - k)
    B = (rev + np.uint64(2**31 // N) + np.uint64(orc.splitmix64(seed) >> 32)) % np.uint64(2**32)
    bq = (B.astype(np.float64) + 0.5) * 2.0**-32
    interior = (bq > 1.0 / nv) & (bq < 1.0 - 1.0 / nv)  # edge cells carry a density slope
    assert np.allclose(_by_point(st.v, N)[interior], (vmin + nv * dv * bq)[interior], atol=1e-12)
    assert st.w.sum() == pytest.approx(mass.sum(), rel=1e-13) and np.all(st.w == st.w[0])


def test_ps_lift_walls_restrict_reproduces_the_masses():
    # smooth phase-space density, non-zero at the walls: the tau = 0 sample of the loaded ions
    # returns each bin's mass to the interpolation and quadrature error, and the total exactly
    ncell, b, nv, N = 128, 3, 32, 128 * 512
    nxc = ncell >> b
    vmin, dv = -6.0, 12.0 / nv
    x = (np.arange(nxc) + 0.5) / nxc
    vc = vmin + dv * (np.arange(nv) + 0.5)
    n = 8.0 * (1.2 + 0.5 * np.cos(np.pi * x))
    H = n[:, None] * np.exp(-0.5 * (vc[None, :] - 0.3) ** 2) * dv / np.sqrt(2 * np.pi)
    mass, cdf, _ = orc.ps_lift_tables(H)
    st = orc.ps_quiet_start_equal(N, ncell, b, mass, cdf, vmin, dv, 3)
    s_w = orc.fx_shift(4 * st.w.max())
    F = orc.ps_sample_fx_walls(st, st.v, np.zeros(ncell), ncell, 0.5, 0.0, 1.0, b, vmin, dv, nv, s_w)
    got = F * 2.0 ** -(s_w + 24)
    assert got.sum() == pytest.approx(mass.sum(), rel=1e-6)
    # the profile linear between bin midpoints is not conservative bin by bin: its error is the
    # reconstruction's (curvature x width^2, ~1 % for this profile), the total is exact
    assert np.max(np.abs(got.sum(axis=1) - mass) / mass) < 0.02
    vel_marg = got.sum(axis=0) / got.sum()
    want_marg = H.sum(axis=0) / H.sum()
    assert np.max(np.abs(vel_marg - want_marg)) < 0.01 * want_marg.max()


def test_ps_sample_walls_reduces_to_the_periodic_sample_inside():
    ncell, b, nv, N = 64, 2, 16, 3000
    rng = np.random.default_rng(5)
    X = 10 + rng.random(N) * 40  # far from the walls; tau v below 4 cells
    cell = np.floor(X).astype(np.int32)
    st = orc.State(cell, X - cell, rng.standard_normal(N) * 0.5, 0.5 + rng.random(N))
    E0 = 0.05 * np.sin(np.arange(ncell) * 0.2)
    a = orc.ps_sample_fx_walls(st, st.v, E0, ncell, 0.5, 3.0, 1.0, b, -4.0, 0.5, nv, 20)
    p = orc.ps_sample_fx(st, st.v, E0, ncell, 0.5, 3.0, 1.0, b, -4.0, 0.5, nv, 20)
    assert np.array_equal(a, p)


@pytest.mark.parametrize("filt", [0, 1, 2, 3, 6, 7])
def test_ps_project_filters(filt):
    rng = np.random.default_rng(filt)
    K, nxc, nv, dt, dT = 6, 12, 16, 0.1, 4.0
    y = rng.standard_normal((K + 1, nxc, nv))
    y[:, :, :2] = y[:, :, -2:] = 0.0  # empty velocity edges: the v filter then keeps both moments
    out, s = orc.ps_project(y, dt, dT, filt)
    c0, raw = orc.ls_project(y.reshape(K + 1, -1), dt, dT)
    raw = raw.reshape(nxc, nv)
    if filt == 0:
        assert np.allclose(out, c0.reshape(nxc, nv), atol=1e-13)
    # the slope's total is kept (charge), and with the v filter its first v moment (momentum)
    assert s.sum() == pytest.approx(raw.sum(), abs=1e-12)
    j = np.arange(nv)
    assert np.allclose((s * j).sum(axis=1).sum(), (raw * j).sum(axis=1).sum(), atol=1e-11)
    if filt & 2 and not filt & 4:  # periodic x: each velocity cell's x-sum is kept too
        assert np.allclose(s.sum(axis=0), (orc.ps_project(y, dt, dT, filt & 1)[1]).sum(axis=0), atol=1e-12)
    # a smooth (linear) slope in v passes the v filter unchanged away from the edges
    assert np.allclose(out, y[-1] + (dT - K * dt) * s, atol=1e-13)


def test_ps_burst_walls_mirror_symmetry():
    ncell, b, nv, dx, dt, K = 128, 3, 16, 0.5, 0.1, 12
    n, u = orc.slab_profile(ncell)
    half = orc.quiet_start_equal(4096, ncell, n, u, 1.0, 3)
    half.v *= 10.0
    mir = _mirror(half, ncell)
    st = orc.State(np.concatenate([half.cell, mir.cell]), np.concatenate([half.theta, mir.theta]),
                   np.concatenate([half.v, mir.v]), np.concatenate([half.w, mir.w]))
    s_w = orc.fx_shift(4 * st.w.max())
    K = 30
    samples, phi, fails = orc.ps_burst_walls(st, ncell, dx, dt, 1.0, K, 4.0, s_w, np.zeros(ncell), b, -32.0, 4.0,
                                             nv, tol=1e-13)
    assert fails == 0
    # mirror: x-bin i <-> nxc-1-i, velocity cell j <-> nv-1-j (symmetric velocity range)
    assert np.array_equal(samples, samples[:, ::-1, ::-1])
    assert (st.w == 0).sum() > 0


def test_ps_quiet_start_equal_empty_bins_lend_no_velocities():
    # ions next to the expansion front take their velocities from the occupied bins only: bins
    # without ions have a placeholder (uniform) table that must not leak into the blend
    ncell, b, nv, N = 128, 3, 32, 1 << 15
    nxc = ncell >> b
    vmin, dv = -8.0, 0.5
    vc = vmin + dv * (np.arange(nv) + 0.5)
    H = np.zeros((nxc, nv))
    H[4:10] = np.exp(-0.5 * ((vc - 2.0) / 0.3) ** 2)[None, :]  # a cold beam at v = 2 in bins 4..9
    mass, cdf, _ = orc.ps_lift_tables(H)
    st = orc.ps_quiet_start_equal(N, ncell, b, mass, cdf, vmin, dv, 4)
    occupied = vc[H[4] > 1e-12 * H[4].max()]
    assert st.v.min() >= occupied.min() - dv and st.v.max() <= occupied.max() + dv
    assert np.all((st.cell >= 4 * 8 - 5) & (st.cell < 10 * 8 + 4))
