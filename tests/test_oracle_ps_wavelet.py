"""Pins of the oracle's wavelet form of the phase-space variable (Section 3.3 as stated:
Eqs. waveletapproximation, restriction, interpolation; Appendices A, B, C) against closed
forms, brute force and textbook special cases."""
import numpy as np
import pytest

import oracle as orc


def _tent_deposit(y, w, ncell, b):
    """Brute force: weight of a particle at fine position y (in nodes) on coarse node k is
    w 2^-b max(0, 1 - d / 2^b), d the periodic distance from y to fine node k 2^b."""
    nxc = ncell >> b
    out = np.zeros(nxc)
    width = float(1 << b)
    for yi, wi in zip(y, w):
        for k in range(nxc):
            d = abs(yi - k * width)
            d = min(d, ncell - d)
            out[k] += wi * max(0.0, 1.0 - d / width) / width
    return out


def _state(n, ncell, rng, vmax=3.0):
    y = rng.uniform(0, ncell, n)
    cell = np.floor(y).astype(np.int32)
    theta = y - cell
    v = rng.uniform(-vmax, vmax, n)
    w = rng.uniform(0.5, 1.5, n)
    return orc.State(cell, theta, v, w), y


@pytest.mark.parametrize("b", [1, 2, 3])
def test_repeated_121_restriction_of_the_cic_histogram_is_the_coarse_tent(b):
    # Eq. (restriction) applied b times to a CIC deposit equals a hat of half-width 2^b
    # around each coarse node, scaled by 2^-b (brute force over the particles)
    rng = np.random.default_rng(3)
    ncell = 32
    st, y = _state(57, ncell, rng)
    H = orc.ps_hist_fine(st, st.v, np.zeros(ncell), ncell, 1.0, 0.0, 1.0, -1e9, 2e9, 1)
    got = orc.restrict_121(H[:, 0], b)
    want = _tent_deposit(y, st.w, ncell, b)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
    assert abs(got.sum() - st.w.sum() / 2 ** b) < 1e-12  # each level halves the sum (an average)


def test_121_restriction_one_level_stencil():
    f = np.zeros(16)
    f[5] = 1.0  # odd fine node 2k+1 between coarse nodes 2 and 3
    np.testing.assert_allclose(orc.restrict_121(f, 1), np.eye(8)[2] * 0.25 + np.eye(8)[3] * 0.25)
    f = np.zeros(16)
    f[6] = 1.0  # even fine node = coarse node 3
    np.testing.assert_allclose(orc.restrict_121(f, 1), np.eye(8)[3] * 0.5)
    f = np.zeros(16)
    f[15] = 1.0  # periodic wrap: last fine node lies between coarse nodes 7 and 0
    np.testing.assert_allclose(orc.restrict_121(f, 1), np.eye(8)[7] * 0.25 + np.eye(8)[0] * 0.25)


def test_restriction_after_interpolation_is_the_1_6_1_stencil():
    # Eqs. (interpolation) then (restriction): g_k = f_{k-1}/8 + 3 f_k/4 + f_{k+1}/8
    rng = np.random.default_rng(5)
    f = rng.normal(size=16)
    got = orc.restrict_121(orc.interpolate_x(f, 1), 1)
    want = np.roll(f, 1) / 8 + 0.75 * f + np.roll(f, -1) / 8
    np.testing.assert_allclose(got, want, atol=1e-14)


def test_repeated_interpolation_is_linear_between_coarse_nodes():
    rng = np.random.default_rng(7)
    M = rng.normal(size=8)
    b = 3
    fine = orc.interpolate_x(M, b)
    j = np.arange(8 << b)
    i0 = j >> b
    phi = (j & ((1 << b) - 1)) / float(1 << b)
    want = (1 - phi) * M[i0] + phi * M[(i0 + 1) % 8]
    np.testing.assert_allclose(fine, want, atol=1e-14)


def test_haar_coarsening_in_v_is_block_sums():
    rng = np.random.default_rng(9)
    H = rng.normal(size=(4, 64))
    got = orc.ps_coarsen_v(H, 16, "haar")
    np.testing.assert_allclose(got, H.reshape(4, 16, 4).sum(-1), atol=1e-13)


@pytest.mark.parametrize("wav", ["d4", "coif4"])
def test_coarsening_in_v_keeps_the_mass_and_inverts_the_refinement(wav):
    rng = np.random.default_rng(11)
    H = rng.normal(size=(3, 128))
    C = orc.ps_coarsen_v(H, 32, wav)
    np.testing.assert_allclose(C.sum(-1), H.sum(-1), rtol=1e-12, atol=1e-12)
    C2 = rng.normal(size=(3, 16))
    np.testing.assert_allclose(orc.ps_coarsen_v(orc.ps_refine_v(C2, 128, wav), 16, wav), C2, atol=1e-12)


def test_coif4_projection_keeps_velocity_moments_0_to_3():
    # Appendix A: psi has four vanishing moments, so discarding the details keeps the first
    # four moments of a histogram whose support stays clear of the periodic wrap
    k = np.arange(256, dtype=np.float64)
    rng = np.random.default_rng(15)
    f = np.where((k >= 80) & (k < 176), rng.uniform(0.0, 1.0, 256), 0.0)  # rough, clear of the wrap
    for L in (1, 2, 3):
        nvc = 256 >> L
        P = orc.ps_refine_v(orc.ps_coarsen_v(f, nvc, "coif4"), 256, "coif4")
        for p in range(4):
            a, b = np.sum(k ** p * f), np.sum(k ** p * P)
            assert abs(a - b) <= 1e-11 * abs(a), (L, p)
        # the fourth moment is not protected: the projection is not the identity
        assert np.max(np.abs(P - f)) > 1e-6
    # Daubechies-4 has two vanishing moments: the second moment moves
    P = orc.ps_refine_v(orc.ps_coarsen_v(f, 64, "d4"), 256, "d4")
    assert abs(np.sum(k * P) - np.sum(k * f)) <= 1e-10 * np.sum(k * f)
    assert abs(np.sum(k * k * P) - np.sum(k * k * f)) > 1e-6 * np.sum(k * k * f)


def test_fine_histogram_of_one_particle_at_its_co_moving_target():
    ncell, dx, nvf, vmin, dv = 16, 0.5, 32, -4.0, 0.25
    st = orc.State(np.array([3], np.int32), np.array([0.25]), np.array([1.3]), np.array([2.0]))
    E0 = np.full(ncell, 0.4)
    tau, qm = 2.5, 1.0
    H = orc.ps_hist_fine(st, st.v, E0, ncell, dx, tau, qm, vmin, dv, nvf)
    x = (3 + 0.25) + tau * 1.3 / dx  # target position in nodes: 9.75
    kv = int(np.floor((1.3 + qm * tau * 0.4 - vmin) / dv))  # V~ = 2.3 -> cell 25
    want = np.zeros((ncell, nvf))
    want[9, kv] = 2.0 * 0.25
    want[10, kv] = 2.0 * 0.75
    np.testing.assert_allclose(H, want, atol=1e-14)
    assert abs(x - 9.75) < 1e-14
    # velocities beyond the range count in the edge cells
    st.v[:] = 50.0
    H = orc.ps_hist_fine(st, st.v, np.zeros(ncell), ncell, dx, 0.0, qm, vmin, dv, nvf)
    assert H[:, nvf - 1].sum() == pytest.approx(2.0) and H.sum() == pytest.approx(2.0)


def test_node_loader_on_uniform_tables():
    # every coarse node holds the same uniform velocity histogram: V = vmin + nvf dv b
    # exactly, and the weights follow the interpolated node values
    ncell, b, nvf, N = 32, 2, 16, 32 * 64
    nxc = ncell >> b
    rng = np.random.default_rng(13)
    mass = rng.uniform(0.5, 1.5, nxc)
    cdf = np.tile(np.linspace(0, 1, nvf + 1), (nxc, 1))
    st = orc.ps_quiet_start_nodes(N, ncell, b, mass, cdf, -2.0, 0.25, 17)
    ref = orc.quiet_start(N, ncell, np.ones(ncell), np.zeros(ncell), 1.0, 17)  # same points and order
    np.testing.assert_array_equal(st.cell, ref.cell)
    np.testing.assert_allclose(st.theta, ref.theta, atol=0)
    # recover b from the moment loader's velocities (V = Phi^-1(b) there)
    from scipy.stats import norm

    bb = norm.cdf(ref.v)
    np.testing.assert_allclose(st.v, -2.0 + 4.0 * bb, atol=1e-9)
    nfine = orc.interpolate_x(mass, b)
    want_w = ((1 - st.theta) * nfine[st.cell] + st.theta * nfine[(st.cell + 1) % ncell]) / (N // ncell)
    np.testing.assert_allclose(st.w, want_w, atol=1e-14)
    # total weight = the interpolated profile's sum (midpoint offsets are symmetric)
    assert abs(st.w.sum() - nfine.sum()) < 1e-10


def test_node_loader_mixes_the_two_coarse_distributions():
    # coarse node 0 holds all its velocity mass in cell 0, node 1 in the last cell. Fine node j
    # at phi_j between them holds the mixture (Eq. interpolation of the histograms): its CDF is
    # 1 - phi on cells 1..7, so V_j(b) = b / (1 - phi) for b < 1 - phi, else
    # 7 + (b - 1 + phi) / phi; a particle takes (1 - theta) V_c + theta V_{c+1} (closed form)
    from scipy.stats import norm

    ncell, b, nvf, ppc = 8, 2, 8, 256
    nxc = ncell >> b
    cdf = np.ones((nxc, nvf + 1))
    cdf[:, 0] = 0.0
    cdf[1, :-1] = 0.0
    mass = np.array([1.0, 1.0])
    N = ncell * ppc
    st = orc.ps_quiet_start_nodes(N, ncell, b, mass, cdf, 0.0, 1.0, 3)
    bb = norm.cdf(orc.quiet_start(N, ncell, np.ones(ncell), np.zeros(ncell), 1.0, 3).v)

    def node_v(j, bq):
        i0 = j >> b
        phi = (j & 3) / 4.0
        phi = np.where(i0 == 1, 1.0 - phi, phi)  # from node 1 (last cell) back to node 0: mirrored
        lo = 1.0 - phi  # weight of the cell-0 component
        return np.where(bq < lo, bq / np.maximum(lo, 1e-300), 7.0 + (bq - lo) / np.maximum(1.0 - lo, 1e-300))

    want = (1 - st.theta) * node_v(st.cell, bb) + st.theta * node_v((st.cell + 1) % ncell, bb)
    np.testing.assert_allclose(st.v, want, atol=1e-8)


def test_wavelet_macro_step_conserves_charge_and_keeps_a_cold_uniform_plasma():
    # Section 3.3 Remark on charge: the least-squares weights sum to zero, and the restriction
    # keeps the total (1/2 per level of Eq. restriction); a uniform plasma at rest with a
    # Maxwellian in v stays uniform in x
    ncell, nc, N, K = 32, 8, 32 * 256, 4
    cfg = dict(ncell=ncell, n_coarse=nc, N=N, K=K, L=16.0, dt=0.1, dT=0.8, qm=1.0, v_max=6.0, n_v=64, n_v_coarse=16,
               wavelet="coif4", s_w=orc.fx_shift(8.0 * ncell / N))
    st = orc.quiet_start(N, ncell, np.ones(ncell), np.zeros(ncell), 1.0, 21)
    coarse, cs, phi = orc.efpi_ps_wavelet_macro_step(st, cfg, np.zeros(ncell))
    b = 2
    tot = st.w.sum() / 2 ** b
    for p in range(K + 1):
        assert abs(cs[p].sum() - tot) < 1e-10 * tot
    assert abs(coarse.sum() - tot) < 1e-10 * tot
    dens = coarse.sum(1)
    assert np.max(np.abs(dens / dens.mean() - 1)) < 2e-3
    # the lift of that state reloads the same total weight and a zero-mean velocity
    new, bad = orc.ps_wavelet_lift(coarse, cfg, 5)
    assert abs(new.w.sum() - st.w.sum()) < 1e-9 * st.w.sum()
    assert abs(np.sum(new.w * new.v)) < 2e-3 * new.w.sum()
