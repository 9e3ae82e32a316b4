"""Pins of the kinetic-electron oracle (Section 4.1: in the paper's ion-acoustic runs both
species are particles during the bursts, q_e/m_e = -1800, q_i/m_i = 1, and the field is the
plain Poisson equation for the net charge). No GPU needed.

The pins: the periodic Poisson solve against a least-squares solve of the dense Laplacian
(another method), its Fourier eigenmodes in closed form, the discrete Gauss law; total
momentum of the two-species system (conserved by CIC deposit, CIC gather and the centred
field); the cold Langmuir oscillation at the electron plasma frequency sqrt(n_0 |q_e/m_e|);
and the Boltzmann electrons of the lifting, whose charge balances the ions'.
"""
import numpy as np
import pytest

import oracle as orc

QM_E = -1800.0


def _laplacian(n, dx):
    A = np.zeros((n, n))
    for j in range(n):
        A[j, j] = 2.0 / dx**2
        A[j, (j + 1) % n] = -1.0 / dx**2
        A[j, (j - 1) % n] = -1.0 / dx**2
    return A


@pytest.mark.parametrize("n,dx", [(8, 0.5), (64, 0.3), (256, 1.0)])
def test_poisson_periodic_matches_least_squares(n, dx):
    r = np.random.default_rng(n).normal(size=n) + 0.7  # nonzero mean: the background is removed
    phi, E = orc.poisson_periodic(r, dx)
    ref = np.linalg.lstsq(_laplacian(n, dx), r - r.mean(), rcond=None)[0]
    ref -= ref.mean()
    scale = np.abs(ref).max()
    assert np.abs(phi - ref).max() <= 1e-12 * scale
    Eref = -(np.roll(ref, -1) - np.roll(ref, 1)) / (2 * dx)
    assert np.abs(E - Eref).max() <= 1e-12 * np.abs(Eref).max()
    assert abs(phi.sum()) <= 1e-12 * scale * n


@pytest.mark.parametrize("m", [1, 3, 17])
def test_poisson_fourier_mode_closed_form(m):
    # r_j = cos(k x_j), k = 2 pi m / L: phi_j = r_j dx^2 / (2 - 2 cos(k dx)) and
    # E_j = phi_amp sin(k x_j) sin(k dx) / dx
    n, dx = 128, 0.4
    kdx = 2 * np.pi * m / n
    j = np.arange(n)
    r = np.cos(kdx * j)
    phi, E = orc.poisson_periodic(r, dx)
    amp = dx**2 / (2 - 2 * np.cos(kdx))
    assert np.abs(phi - amp * r).max() <= 1e-12 * amp
    assert np.abs(E - amp * np.sin(kdx * j) * np.sin(kdx) / dx).max() <= 1e-12 * amp / dx


def test_poisson_gauss_law_and_neutral_background():
    n, dx = 96, 0.25
    r = np.random.default_rng(5).uniform(0.5, 1.5, n)
    phi, E = orc.poisson_periodic(r, dx)
    F = -(np.roll(phi, -1) - phi) / dx  # face fields F_{j+1/2}
    assert np.allclose(F - np.roll(F, 1), dx * (r - r.mean()), atol=1e-12)
    assert abs(F.sum()) < 1e-11
    phi0, E0 = orc.poisson_periodic(np.full(n, 3.0), dx)  # uniform charge: no field
    assert np.abs(phi0).max() == 0.0 and np.abs(E0).max() == 0.0


def _uniform(N, ncell, v_th, seed, amp=0.0, L=None):
    n = np.ones(ncell)
    u = np.zeros(ncell) if L is None else amp * np.sin(2 * np.pi * np.arange(ncell) / ncell)
    return orc.quiet_start(N, ncell, n, u, v_th, seed)


def test_two_species_momentum_is_conserved():
    # CIC deposit + CIC gather + centred field on a periodic grid exert no net self-force:
    # sum_s m_s v_s (m = w / (q/m) per unit |charge|) is conserved up to the fixed-point
    # rounding of the deposit; a sign error in either species' charge or acceleration breaks it
    ncell, ppc, dx, dt = 64, 64, 0.5, 0.25 / np.sqrt(-QM_E)
    N = ncell * ppc
    ions = _uniform(N, ncell, 0.05, 3)
    L = ncell * dx
    x = (ions.cell + ions.theta) * dx
    ions.v += 0.3 * np.cos(2 * np.pi * x / L)
    elec = _uniform(N, ncell, np.sqrt(-QM_E), 4)
    s_w = orc.fx_shift(8.0 / ppc)

    def momentum(i, e, kick_half):
        _, E = orc.field_kinetic(i, e, ncell, dx, s_w)
        # integer-time velocities: v + (kick - 1/2) qm dt E(X) with kick 1 after a step
        vi = i.v - 0.5 * dt * orc.gather(E, i.cell, i.theta) if kick_half else i.v
        ve = e.v - 0.5 * QM_E * dt * orc.gather(E, e.cell, e.theta) if kick_half else e.v
        return np.sum(i.w * vi) + np.sum(e.w * ve / -QM_E), np.sum(np.abs(i.w * vi))

    p0, scale = momentum(ions, elec, False)
    orc.pic_steps_kinetic(ions, elec, ncell, dx, dt, 1.0, QM_E, 60, s_w)
    p1, _ = momentum(ions, elec, True)
    assert abs(p1 - p0) <= 1e-5 * scale, (p0, p1, scale)


def test_cold_langmuir_oscillation_at_electron_plasma_frequency():
    # immobile ions (q/m = 0), cold electrons with a small velocity wave: the wave's momentum
    # oscillates at omega_pe = sqrt(n_0 |q_e/m_e|) (n_0 = 1), up to O((k dx)^2, (omega dt)^2)
    ncell, ppc, dx = 256, 16, 0.5
    N = ncell * ppc
    wpe = np.sqrt(-QM_E)
    dt = 0.1 / wpe
    ions = _uniform(N, ncell, 0.0, 1)
    elec = _uniform(N, ncell, 0.0, 2)
    L = ncell * dx
    k = 2 * np.pi / L
    elec.v += 1e-3 * np.sin(k * (elec.cell + elec.theta) * dx)
    s_w = orc.fx_shift(8.0 / ppc)
    proj = []
    steps = 400  # about 6.4 plasma periods
    for s in range(steps):
        orc.pic_steps_kinetic(ions, elec, ncell, dx, dt, 0.0, QM_E, 1, s_w, vel_at_integer=(s == 0))
        proj.append(np.sum(elec.w * elec.v * np.sin(k * (elec.cell + elec.theta) * dx)))
    proj = np.array(proj)
    # the projection follows cos(omega t): time its zero crossings by linear interpolation
    t = (np.arange(steps) + 0.5) * dt  # velocities sit at half steps
    z = [t[i] - proj[i] * (t[i + 1] - t[i]) / (proj[i + 1] - proj[i])
         for i in range(steps - 1) if proj[i] * proj[i + 1] < 0]
    assert len(z) >= 10
    omega = np.pi / np.mean(np.diff(z))
    assert abs(omega / wpe - 1.0) < 5e-3, omega / wpe


def test_boltzmann_electrons_balance_the_ion_charge():
    # Eq. electronpassive: n_e = exp(phi) with phi the Poisson-Boltzmann potential of the ions;
    # sum_j exp(phi_j) = sum_j n_j (the periodic Laplacian sums to zero), so the loaded
    # electrons carry the ions' charge and deposit the Boltzmann profile
    ncell, ppc, dx = 128, 32, 0.5
    n, _ = orc.sine_profile(ncell, ncell * dx, 0.3)
    phi, _, fail = orc.newton_pb(n, dx, tol=1e-13)
    assert not fail
    e = orc.boltzmann_electrons(ncell * ppc, ncell, phi, np.sqrt(-QM_E), seed=9)
    assert np.sum(e.w) == pytest.approx(np.sum(n), rel=1e-12)
    dens = np.asarray(orc.deposit_f64(e.cell, e.theta, e.w, ncell))
    dens = dens[0] if dens.ndim == 2 else dens
    assert np.abs(dens - np.exp(phi)).max() < 2e-3  # quiet start: CIC of the linear profile
    v = e.v
    assert abs(np.mean(v)) < 1e-2 * np.sqrt(-QM_E) and np.std(v) == pytest.approx(np.sqrt(-QM_E), rel=2e-2)


def test_kinetic_burst_runs_the_same_steps_as_plain_pic():
    # the burst's particle trajectory is that of plain two-species PIC, and its first sample
    # (p = 0, tau = dT) is the co-moving sample of the initial ions in the initial field
    ncell, ppc, dx = 64, 32, 0.5
    N = ncell * ppc
    dt = 0.25 / np.sqrt(-QM_E)
    n, u = orc.sine_profile(ncell, ncell * dx, 0.2)
    ions = orc.quiet_start(N, ncell, n, u, 0.22, 7)
    phi, _, _ = orc.newton_pb(n, dx, tol=1e-13)
    elec = orc.boltzmann_electrons(N, ncell, phi, np.sqrt(-QM_E), 8)
    s_w = orc.fx_shift(8.0 / ppc)
    K, dT = 6, 40 * dt
    a_i, a_e, b_i, b_e = ions.copy(), elec.copy(), ions.copy(), elec.copy()
    samples, _ = orc.burst_kinetic(a_i, a_e, ncell, dx, dt, 1.0, QM_E, K, dT, s_w)
    orc.pic_steps_kinetic(b_i, b_e, ncell, dx, dt, 1.0, QM_E, K, s_w)
    for a, b in ((a_i, b_i), (a_e, b_e)):
        assert np.array_equal(a.cell, b.cell) and np.array_equal(a.theta, b.theta) and np.array_equal(a.v, b.v)
    _, E = orc.field_kinetic(ions, elec, ncell, dx, s_w)
    vbar = ions.v  # loaded at integer time
    dens, mom = orc.restrict_sample(ions, vbar, E, ncell, dx, dT, 1.0)
    assert np.array_equal(samples[0, 0], dens) and np.array_equal(samples[0, 1], mom)


def test_boltzmann_electrons_drift_with_the_ions():
    # Eq. electronpassive: V_e = V_i. A uniform ion drift gives the electrons exactly that drift
    # on top of their symmetric quiet-start Maxwellian; a sinusoidal one is reproduced node by node
    ncell, ppc, dx = 64, 64, 0.5
    N = ncell * ppc
    ions = orc.quiet_start(N, ncell, np.ones(ncell), np.full(ncell, 0.3), 0.0, 3)  # cold: V_i = 0.3
    phi = np.zeros(ncell)
    e = orc.boltzmann_electrons(N, ncell, phi, np.sqrt(-QM_E), 5, ions=ions)
    e0 = orc.boltzmann_electrons(N, ncell, phi, np.sqrt(-QM_E), 5)
    assert np.allclose(e.v - e0.v, 0.3, rtol=0, atol=1e-12)  # the same draws, shifted by the drift
    n, u = orc.sine_profile(ncell, ncell * dx, 0.2)
    ions = orc.quiet_start(N, ncell, n, u, 0.0, 3)  # cold ions: V_i(x) = u(x)
    e = orc.boltzmann_electrons(N, ncell, phi, 1e-9, 6, ions=ions)
    d, m = orc.deposit_f64(e.cell, e.theta, e.w, ncell, vel=e.v)
    # up to the O((k dx)^2) smoothing of the CIC deposits and the linear profile interpolation
    kdx = 2 * np.pi / ncell
    assert np.abs(m / d - u).max() < 0.2 * kdx**2 / 2


def test_temperature_lift_solves_the_boltzmann_relation_at_t_e():
    # psi from -T_e psi'' + e^psi = n at the step dx / sqrt(T_e); phi = T_e psi satisfies the
    # printed relation -phi'' + exp(phi / T_e) = n on the grid step dx (residual ~ Newton tol)
    ncell, L, Te = 64, 32.0, 0.6
    dx = L / ncell
    x = np.arange(ncell) * dx
    n = 1.0 + 0.3 * np.cos(2 * np.pi * x / L)
    _, psi = orc.boltzmann_electrons_te(ncell * 64, ncell, n, dx, Te, 2.0, 5)
    phi = Te * psi
    lap = (np.roll(phi, -1) - 2 * phi + np.roll(phi, 1)) / dx ** 2
    assert np.max(np.abs(-lap + np.exp(phi / Te) - n)) < 1e-9


def test_temperature_lift_scales_the_thermal_energy():
    # a uniform ion density gives psi = 0 at any T_e: the same weights and quantiles, velocities
    # scaled by sqrt(T_e), so the kinetic energy scales by T_e exactly
    ncell, L, N = 32, 16.0, 32 * 128
    dx = L / ncell
    n = np.ones(ncell)
    e1, _ = orc.boltzmann_electrons_te(N, ncell, n, dx, 1.0, 3.0, 9)
    e2, psi = orc.boltzmann_electrons_te(N, ncell, n, dx, 1.7, 3.0, 9)
    assert np.max(np.abs(psi)) < 1e-12
    E = np.zeros(ncell)
    k1 = orc.electron_kinetic_energy(e1, E, ncell, dx, 0.1, -1800.0, 0.5)
    k2 = orc.electron_kinetic_energy(e2, E, ncell, dx, 0.1, -1800.0, 0.5)
    assert k2 / k1 == pytest.approx(1.7, rel=1e-12)
    assert orc.lift_electron_temperature(k2, k1) == pytest.approx(1.7, rel=1e-12)
    # the quiet start's thermal energy: sum w v^2 dx / 2 = (sum w dx) v_th^2 / 2 to the
    # Hammersley quadrature's accuracy
    q = float(np.sum(e1.w)) * dx
    assert k1 == pytest.approx(0.5 * q * 9.0, rel=2e-3)
