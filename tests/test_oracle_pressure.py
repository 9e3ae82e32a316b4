"""Pins of the oracle's ion-pressure variable (Section 3.2, EFREE's n, V, P; no GPU).

The restriction adds the ions' second velocity moment S_j = sum_p w V~^2 S_j(X~) to the density
and momentum samples; the lift takes P = S - (nV)^2 / n and loads Maxwellians of the local
temperature T = P / n. The pins do not restate that arithmetic: a single particle worked out by
hand (with the co-moving shift), the Galilean identity S(v + u0) = S + 2 u0 M + u0^2 n, the sum
rule sum_j S_j dx = 2 x kinetic energy of the diagnostics, closed-form Maxwellian fields, the
loader at a uniform temperature against the pinned loader at v_th = sqrt(T), quadrature of the
loaded variance, and a cold drifting plasma as a fixed point of the macro step.
"""
import numpy as np

import oracle as orc


def _dyadic_particles(N, ncell, seed):
    rng = np.random.default_rng(seed)
    cell = rng.integers(0, ncell, N).astype(np.int32)
    theta = rng.integers(0, 256, N) / 256.0
    v = rng.integers(-512, 512, N) / 128.0
    w = rng.integers(1, 16, N) / 16.0
    return orc.State(cell, theta, v, w)


def test_second_moment_single_particle_by_hand():
    st = orc.State(np.array([3], np.int32), np.array([0.25]), np.array([2.0]), np.array([0.5]))
    # tau = 0: w V^2 = 2 split 3/4, 1/4 between nodes 3 and 4
    got = orc.restrict_second_moment(st, [2.0], np.zeros(16), 16, 0.5, 0.0, 1.0)
    want = np.zeros(16)
    want[3], want[4] = 1.5, 0.5
    assert np.array_equal(got, want)
    # tau = 2, dx = 0.5, uniform E0 = 0.5, qm = 1: X~ = X + tau V moves 8 cells (to 11, theta
    # 1/4) and V~ = V + qm tau E0 = 3, so w V~^2 = 4.5 split 3/4, 1/4 between nodes 11 and 12
    got = orc.restrict_second_moment(st, [2.0], np.full(16, 0.5), 16, 0.5, 2.0, 1.0)
    want = np.zeros(16)
    want[11], want[12] = 3.375, 1.125
    assert np.allclose(got, want, rtol=0, atol=1e-15)


def test_second_moment_galilean_shift():
    ncell, N, u0 = 32, 5000, 0.375
    st = _dyadic_particles(N, ncell, 7)
    E0 = np.zeros(ncell)
    n, M = orc.restrict_sample(st, st.v, E0, ncell, 0.5, 0.0, 1.0)
    S = orc.restrict_second_moment(st, st.v, E0, ncell, 0.5, 0.0, 1.0)
    S_shift = orc.restrict_second_moment(st, st.v + u0, E0, ncell, 0.5, 0.0, 1.0)
    assert np.allclose(S_shift, S + 2 * u0 * M + u0 * u0 * n, rtol=1e-13, atol=1e-12)


def test_second_moment_sum_is_twice_the_kinetic_energy():
    ncell, N, dx, dt = 64, 20000, 0.5, 0.1
    rng = np.random.default_rng(11)
    st = orc.State(rng.integers(0, ncell, N).astype(np.int32), rng.random(N), rng.normal(0.3, 1.2, N),
                   rng.random(N) * 0.01)
    E = rng.normal(0, 0.1, ncell)
    S = orc.restrict_second_moment(st, st.v, E, ncell, dx, 0.0, 1.0)
    # kick 1/2: the diagnostics' integer-time velocity is v itself
    mom = orc.moments(st, E, np.zeros(ncell), ncell, dx, dt, 1.0, 0.5, 20)
    assert abs(S.sum() * dx - 2.0 * mom["kinetic"]) <= 1e-12 * 2.0 * mom["kinetic"]


def test_lift_profile_pressure_recovers_maxwellian_fields():
    ncell = 128
    x = np.arange(ncell) / ncell
    n = 1.0 + 0.4 * np.cos(2 * np.pi * x)
    u = 0.3 * np.sin(2 * np.pi * x)
    T = 0.8 + 0.3 * np.cos(4 * np.pi * x)
    n_out, u_out, T_out = orc.lift_profile_pressure(n, n * u, n * (u * u + T))
    assert np.array_equal(n_out, n)
    assert np.allclose(u_out, u, rtol=0, atol=1e-15)
    assert np.allclose(T_out, T, rtol=0, atol=1e-14)


def test_lift_profile_pressure_clamps():
    n = np.array([1.0, 1.0, -0.5, 2.0, 0.0, 1.5, 1.0, 1.0])
    m = np.array([0.5, -0.5, 0.1, 1.0, 0.0, 0.0, 0.0, 0.0])
    s = np.array([0.5, 0.20, 0.3, 3.0, 0.0, 0.0, 1.0, 1.0])
    n_out, u_out, T_out = orc.lift_profile_pressure(n, m, s)
    assert n_out[2] == 0.0 and np.isclose(n_out.sum(), n.sum(), rtol=1e-15)  # clamped, mass kept
    assert T_out[1] == 0.0  # S below the kinetic part n u^2: cold, not negative
    assert T_out[2] == 0.0 and T_out[4] == 0.0  # no ions: no temperature
    resc = n.sum() / np.maximum(n, 0).sum()
    assert np.isclose(T_out[0], 0.5 / resc - (0.5 / resc) ** 2, rtol=1e-14)
    assert np.isclose(T_out[3], 3.0 / (2 * resc) - (1.0 / (2 * resc)) ** 2, rtol=1e-14)


def test_quiet_start_thermal_at_uniform_temperature_is_the_loader_at_sqrt_t():
    ncell, N = 32, 32 * 64
    x = np.arange(ncell) / ncell
    n = 1.0 + 0.5 * np.cos(2 * np.pi * x)
    u = 0.25 * np.sin(2 * np.pi * x)
    a = orc.quiet_start_thermal(N, ncell, n, u, np.full(ncell, 4.0), 99)
    b = orc.quiet_start(N, ncell, n, u, 2.0, 99)
    for p, q in zip((a.cell, a.theta, a.v, a.w), (b.cell, b.theta, b.v, b.w)):
        assert np.array_equal(p, q)


def test_quiet_start_thermal_loads_the_local_temperature():
    ncell, ppc = 128, 1024
    N = ncell * ppc
    x = np.arange(ncell) / ncell
    n = 1.0 + 0.3 * np.cos(2 * np.pi * x)
    u = 0.2 * np.cos(2 * np.pi * x)
    T = 1.0 + 0.5 * np.sin(2 * np.pi * x)
    st = orc.quiet_start_thermal(N, ncell, n, u, T, 5)
    dens, mom = orc.restrict_sample(st, st.v, np.zeros(ncell), ncell, 0.5, 0.0, 1.0)
    sec = orc.restrict_second_moment(st, st.v, np.zeros(ncell), ncell, 0.5, 0.0, 1.0)
    _, u_got, T_got = orc.lift_profile_pressure(dens, mom, sec)
    # quadrature of the Hammersley velocities (the loader at uniform temperature shows the same
    # 6e-3 in u on this grid) and the CIC mixing of neighbouring cells
    assert np.max(np.abs(u_got - u)) < 1e-2
    assert np.max(np.abs(T_got - T)) < 2e-2
    assert np.max(np.abs(T_got - T)) > 0.0


def test_burst_pressure_density_and_momentum_are_the_two_moment_burst():
    cfg = dict(ncell=64, L=32.0, dt=0.1, qm=1.0, K=4, dT=2.0)
    x = np.arange(cfg["ncell"]) / cfg["ncell"]
    st0 = orc.quiet_start(64 * 64, cfg["ncell"], 1.0 + 0.2 * np.cos(2 * np.pi * x), 0.1 * np.cos(2 * np.pi * x),
                          1.0, 3)
    s_w = orc.fx_shift(8.0 * cfg["ncell"] / st0.n)
    dx = cfg["L"] / cfg["ncell"]
    a, b = st0.copy(), st0.copy()
    phi0 = np.zeros(cfg["ncell"])
    s2, phi2, _ = orc.burst(a, cfg["ncell"], dx, cfg["dt"], cfg["qm"], cfg["K"], cfg["dT"], s_w, phi0)
    s3, phi3, _ = orc.burst_pressure(b, cfg["ncell"], dx, cfg["dt"], cfg["qm"], cfg["K"], cfg["dT"], s_w, phi0)
    assert np.array_equal(s3[:, :2], s2) and np.array_equal(phi3, phi2)
    for p, q in zip((a.cell, a.theta, a.v), (b.cell, b.theta, b.v)):
        assert np.array_equal(p, q)
    # sample 0 is the second moment of the initial ions (v at integer time) along the
    # characteristics of the field at burst start
    E0 = orc.field_of(st0.copy(), cfg["ncell"], dx, s_w, np.zeros(cfg["ncell"]))
    want = orc.restrict_second_moment(st0, st0.v, E0, cfg["ncell"], dx, cfg["dT"], cfg["qm"])
    assert np.allclose(s3[0, 2], want, rtol=1e-12, atol=1e-15)


def test_cold_drifting_plasma_is_a_fixed_point():
    ncell, ppc, u0 = 64, 64, 0.5
    cfg = dict(ncell=ncell, n_coarse=8, L=32.0, dt=0.1, qm=1.0, K=5, dT=2.0, N=ncell * ppc)
    st = orc.quiet_start(cfg["N"], ncell, np.ones(ncell), np.full(ncell, u0), 0.0, 1)
    cfg["s_w"] = orc.fx_shift(8.0 * ncell / cfg["N"])
    coarse, cs, _ = orc.efpi_macro_step_pressure(st, cfg, np.zeros(ncell))
    c_n = orc.coarsen(np.ones(ncell), 8)
    assert np.allclose(coarse[0], c_n, rtol=1e-12)
    assert np.allclose(coarse[1], u0 * c_n, rtol=1e-12)
    assert np.allclose(coarse[2], u0 * u0 * c_n, rtol=1e-12)
    # the lift of that state is the cold drifting plasma again
    lifted = orc.lift_pressure(coarse, cfg, 2)
    assert np.allclose(lifted.v, u0, rtol=0, atol=1e-12)


def test_restrict_of_lift_returns_the_coarse_state():
    ncell, nc, ppc = 128, 16, 1024
    cfg = dict(ncell=ncell, n_coarse=nc, N=ncell * ppc)
    x = np.arange(ncell) / ncell
    n = 1.0 + 0.3 * np.cos(2 * np.pi * x)
    u = 0.2 * np.sin(2 * np.pi * x)
    T = 1.0 + 0.3 * np.cos(2 * np.pi * x)
    coarse = np.stack([orc.coarsen(f, nc) for f in (n, n * u, n * (u * u + T))])
    st = orc.lift_pressure(coarse, cfg, 17)
    E0 = np.zeros(ncell)
    dens, mom = orc.restrict_sample(st, st.v, E0, ncell, 0.5, 0.0, 1.0)
    sec = orc.restrict_second_moment(st, st.v, E0, ncell, 0.5, 0.0, 1.0)
    back = np.stack([orc.coarsen(f, nc) for f in (dens, mom, sec)])
    # the bounds of the two-moment round trip: 2e-3 of the density, 2e-2 of the momentum scale
    rel = np.max(np.abs(back - coarse), axis=1) / np.abs(coarse).max(axis=1)
    assert rel[0] < 2e-3 and rel[1] < 2e-2 and rel[2] < 2e-3
