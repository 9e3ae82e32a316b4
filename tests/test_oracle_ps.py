"""Pins of the phase-space coarse variable of the oracle (Section 3.3, Appendices B and C):
the momentum-conserving CDF reconstruction, its inverse, the co-moving phase-space sample,
the lifting tables, the phase-space quiet start and the free-streaming burst. No GPU."""
import numpy as np
import pytest

import oracle as orc
from paper_1610_01071_gb300 import inputs


def _m1(F):
    N = F.shape[0] - 1
    return float(np.sum(np.arange(1, N + 1) * np.diff(F)))


def test_cdf_reconstruction_worked_example():
    # F = [0, .5, .4, .8, 1]: from below the dip [.5, .4] becomes the ramp 0, .3, .6 (slope
    # 2/2 (0.9/3 - 0) = 0.3, first moment kept); from above (mirrored) .333, .567; the result
    # is their mean.
    F, bad = orc.cdf_reconstruct(np.array([0.0, 0.5, 0.4, 0.8, 1.0]))
    assert bad == 0
    assert np.allclose(F, [0.0, 0.95 / 3, 1.75 / 3, 0.8, 1.0], rtol=0, atol=1e-15)


def test_cdf_reconstruction_keeps_monotone_input():
    F = np.concatenate([[0.0], np.sort(np.random.default_rng(0).random(15)), [1.0]])
    G, bad = orc.cdf_reconstruct(F)
    assert bad == 0 and np.array_equal(G, F)


@pytest.mark.parametrize("seed", range(12))
def test_cdf_reconstruction_monotone_bounded_and_moment_conserving(seed):
    rng = np.random.default_rng(seed)
    N = 32
    v = np.linspace(-4, 4, N + 1)
    F = 0.5 * (1 + np.tanh(v / 1.5))
    F = (F - F[0]) / (F[-1] - F[0])
    F = F + 0.01 * rng.standard_normal(N + 1)  # overshoots below 0, above 1 and dips
    F[0], F[-1] = 0.0, 1.0
    G, bad = orc.cdf_reconstruct(F)
    assert G[0] == 0.0 and G[-1] == 1.0
    assert np.all(np.diff(G) >= -1e-15) and G.min() >= -1e-15 and G.max() <= 1 + 1e-15
    if bad == 0:
        # the Lemma of Appendix C: zeroth and first moments of the histogram are kept
        assert _m1(G) == pytest.approx(_m1(F), rel=1e-12, abs=1e-12)
    else:
        # a descent next to F = 0 or 1 with no admissible ramp is filled flat: only the few
        # values of that descent move
        assert abs(_m1(G) - _m1(F)) <= N * 0.05
    # symmetric by construction: reconstructing the mirrored array mirrors the result
    Gm, _ = orc.cdf_reconstruct(1.0 - F[::-1])
    assert np.allclose(Gm, 1.0 - G[::-1], atol=1e-14)


def test_cdf_reconstruction_interior_dips_keep_both_moments():
    N = 40
    v = np.linspace(-4, 4, N + 1)
    F = 0.5 * (1 + np.tanh(v / 1.5))
    F = (F - F[0]) / (F[-1] - F[0])
    F[12] += 0.03   # an overshoot and a dip in the body of the distribution
    F[25] -= 0.04
    G, bad = orc.cdf_reconstruct(F)
    assert bad == 0
    assert np.all(np.diff(G) >= 0)
    assert _m1(G) == pytest.approx(_m1(F), rel=1e-12)
    assert np.abs(G - F).max() < 0.05


def test_cdf_inverse_matches_linear_interpolation():
    rng = np.random.default_rng(3)
    nv, vmin, dv = 16, -4.0, 0.5
    F = np.concatenate([[0.0], np.cumsum(rng.random(nv))])
    F /= F[-1]
    edges = vmin + dv * np.arange(nv + 1)
    for b in rng.random(50):
        assert orc.cdf_inverse(F, b, vmin, dv) == pytest.approx(np.interp(b, F, edges), rel=1e-13, abs=1e-13)


def test_cdf_inverse_inside_a_cell_with_linear_density():
    rng = np.random.default_rng(8)
    nv, vmin, dv = 8, -2.0, 0.5
    F = np.concatenate([[0.0], np.cumsum(rng.random(nv) + 0.1)])
    F /= F[-1]
    sig = orc.cdf_cell_slopes(F)
    p = np.diff(F)
    pl, pr = np.concatenate([[0.0], p[:-1]]), np.concatenate([p[1:], [0.0]])
    assert np.allclose(sig, np.clip((pr - pl) / (4 * p), -1, 1), rtol=1e-15)
    for b in rng.random(40):
        V = orc.cdf_inverse(F, b, vmin, dv, sig)
        k = min(int(np.searchsorted(F, b, side="right")) - 1, nv - 1)
        t = (V - vmin) / dv - k
        r = (b - F[k]) / (F[k + 1] - F[k])
        assert 0.0 <= t <= 1.0
        # the cell's CDF fraction at t: integral of 1 + sigma (2u - 1) over [0, t]
        assert t + sig[k] * (t * t - t) == pytest.approx(r, abs=1e-12)
    # the edge cases sigma = +-1 (density vanishing at one edge) and sigma = 0
    one = np.array([0.0, 1.0])
    assert orc.cdf_inverse(one, 0.25, 0.0, 1.0, np.array([1.0])) == pytest.approx(0.5, rel=1e-14)
    assert orc.cdf_inverse(one, 0.75, 0.0, 1.0, np.array([-1.0])) == pytest.approx(0.5, rel=1e-14)
    assert orc.cdf_inverse(one, 0.3, 0.0, 1.0, np.array([0.0])) == pytest.approx(0.3, rel=1e-14)


def test_ps_lift_keeps_the_temperature():
    """Uniform sampling inside a velocity cell adds dv^2/12 to the variance (Sheppard's
    correction); the linear-density cells of the lift keep it to a small fraction of that."""
    ncell, b, nv, vmin, dv, ppc = 64, 3, 32, -8.0, 0.5, 1024
    nxc = ncell >> b
    H = _maxwellian_hist(nxc, nv, vmin, dv, float(1 << b), amp=0.0, u0=0.0)
    mass, cdf, _ = orc.ps_lift_tables(H)
    st = orc.ps_quiet_start(ncell * ppc, ncell, b, mass, cdf, vmin, dv, 3)
    var = np.average(st.v ** 2, weights=st.w) - np.average(st.v, weights=st.w) ** 2
    assert abs(var - 1.0) < 0.15 * dv * dv / 12


def _moved(st, vbar, E0, ncell, dx, tau, qm):
    """The co-moving targets of Appendix B computed here with numpy (positions in cells)."""
    E0p = (1 - st.theta) * E0[st.cell] + st.theta * E0[(st.cell + 1) % ncell]
    s = st.cell + st.theta + tau * vbar / dx
    k = np.floor(s)
    return (k.astype(np.int64) % ncell).astype(np.int32), s - k, vbar + qm * tau * E0p


def test_ps_sample_marginals_are_exact():
    ncell, b, nv, vmin, dv, s_w = 64, 3, 16, -4.0, 0.5, 18
    dx, tau, qm = 0.5, 3.7, 1.0
    c, t, v, w = inputs.random_particles(5000, ncell, seed=11)
    st = orc.State(c, t, v, w)
    E0 = inputs.random_field(ncell, 12, 0.2)
    F = orc.ps_sample_fx(st, st.v, E0, ncell, dx, tau, qm, b, vmin, dv, nv, s_w)
    cm, tm, vm = _moved(st, st.v, E0, ncell, dx, tau, qm)
    # summed over velocity: the fixed-point charge deposit of the moved particles, binned
    rho = orc.deposit_fx(cm, tm, st.w, ncell, s_w)
    assert np.array_equal(F.sum(axis=1), rho.reshape(ncell >> b, 1 << b).sum(axis=1))
    # summed over position: whole weights per velocity cell (clamped to the edge cells)
    j = np.clip(np.floor((vm - vmin) / dv), 0, nv - 1).astype(int)
    wq = np.rint(st.w * 2.0 ** s_w).astype(np.int64) * (1 << 24)
    assert np.array_equal(F.sum(axis=0), np.bincount(j, weights=None, minlength=nv) * 0 +
                          np.array([wq[j == k].sum() for k in range(nv)]))


def _maxwellian_hist(nxc, nv, vmin, dv, per_bin, amp=0.3, u0=0.4, vth=1.0):
    """Phase-space cell masses of n(x) Maxwellian(u(x), vth), exact cell integrals in v."""
    from scipy.special import erf
    x = (np.arange(nxc) + 0.5) / nxc
    n = per_bin * (1 + amp * np.cos(2 * np.pi * x))
    u = u0 * np.cos(2 * np.pi * x)
    edges = vmin + dv * np.arange(nv + 1)
    cdf = 0.5 * (1 + erf((edges[None, :] - u[:, None]) / (np.sqrt(2) * vth)))
    H = n[:, None] * np.diff(cdf, axis=1)
    return H


def test_ps_lift_tables_and_clamp():
    H = _maxwellian_hist(8, 16, -6.0, 0.75, 16.0)
    mass, cdf, bad = orc.ps_lift_tables(H)
    assert bad == 0
    assert np.allclose(mass, H.sum(axis=1), rtol=1e-14)
    assert np.allclose(cdf[:, 1:], np.cumsum(H, axis=1) / H.sum(axis=1)[:, None], rtol=1e-13, atol=1e-15)
    # a bin of negative mass carries no particles; the total mass is kept
    H2 = H.copy()
    H2[3] *= -0.1
    mass2, cdf2, _ = orc.ps_lift_tables(H2)
    assert mass2[3] == 0.0 and mass2.sum() == pytest.approx(H2.sum(), rel=1e-14)
    assert np.allclose(cdf2[3], np.linspace(0, 1, 17))


def test_ps_quiet_start_reproduces_the_histogram():
    ncell, b, nv, vmin, dv, ppc = 256, 3, 32, -6.0, 0.375, 256
    nxc = ncell >> b
    H = _maxwellian_hist(nxc, nv, vmin, dv, float(1 << b))
    mass, cdf, _ = orc.ps_lift_tables(H)
    st = orc.ps_quiet_start(ncell * ppc, ncell, b, mass, cdf, vmin, dv, 5)
    assert np.all(np.diff(st.cell) >= 0)
    s_w = 16
    F = orc.ps_sample_fx(st, st.v, np.zeros(ncell), ncell, 0.5, 0.0, 1.0, b, vmin, dv, nv, s_w)
    G = F * 2.0 ** -(s_w + 24)
    assert G.sum() == pytest.approx(H.sum(), rel=1e-6)
    # f(x, v) is lifted linear in x between bin centres, so the bin masses come back smoothed
    # by [1/8, 3/4, 1/8] in x (the bin integrals of the linear interpolant); the rest is the
    # quadrature of the quiet start and the quantile blend between neighbouring bins
    Hs = 0.75 * H + 0.125 * (np.roll(H, 1, axis=0) + np.roll(H, -1, axis=0))
    assert np.allclose(G.sum(axis=1), Hs.sum(axis=1), rtol=3e-3)
    assert np.abs(G - Hs).sum() / H.sum() < 0.03
    # the same quantiles b as the Maxwellian quiet start (same Hammersley points and storage
    # order); V blends the two neighbouring bins' CDF inverses (here from numpy's interp)
    from scipy.stats import norm
    ref = orc.quiet_start(ncell * ppc, ncell, np.ones(ncell), np.zeros(ncell), 1.0, 5)
    assert np.array_equal(ref.cell, st.cell) and np.array_equal(ref.theta, st.theta)
    edges = vmin + dv * np.arange(nv + 1)
    for i in range(0, ncell * ppc, 997):
        bq = norm.cdf(ref.v[i])
        u = st.cell[i] + st.theta[i] + 0.5  # a bin covers x/dx in [i 2^b - 1/2, (i+1) 2^b - 1/2)
        pos = (u % (1 << b)) / (1 << b)
        b0 = int(u // (1 << b)) - (1 if pos < 0.5 else 0)
        phi = pos - 0.5 if pos >= 0.5 else pos + 0.5
        v0 = orc.cdf_inverse(cdf[b0 % nxc], bq, vmin, dv, orc.cdf_cell_slopes(cdf[b0 % nxc]))
        v1 = orc.cdf_inverse(cdf[(b0 + 1) % nxc], bq, vmin, dv, orc.cdf_cell_slopes(cdf[(b0 + 1) % nxc]))
        assert st.v[i] == pytest.approx((1 - phi) * v0 + phi * v1, abs=1e-6)
    m1 = (G * (vmin + dv * (np.arange(nv) + 0.5))[None, :]).sum()
    assert m1 == pytest.approx((H * (vmin + dv * (np.arange(nv) + 0.5))[None, :]).sum(), rel=2e-2, abs=1e-2)


def test_ps_burst_free_streaming_gives_identical_samples():
    """A cold uniform beam with linearised electrons: the density stays exactly uniform
    (dyadic drift of a uniform lattice), phi = E = 0, the approximate characteristics are exact
    and every co-moving sample equals the first (zero slope)."""
    ncell, b, nv, vmin, dv, ppc, K = 32, 2, 16, -6.0, 0.75, 64, 6
    N = ncell * ppc
    st = orc.quiet_start(N, ncell, np.ones(ncell), np.full(ncell, 0.3125), 0.0, 9)
    s_w = orc.fx_shift(8.0 / ppc)
    samples, phi, fails = orc.ps_burst(st, ncell, 0.5, 0.125, 1.0, K, 2.0, s_w, np.zeros(ncell), b, vmin, dv, nv,
                                       mode=1)
    assert fails == 0 and np.all(phi == 0.0)
    assert samples[0].sum(axis=0)[int((0.3125 - vmin) / dv)] == samples[0].sum()
    for p in range(1, K + 1):
        assert np.array_equal(samples[p], samples[0])
