"""Pins of the leap-error estimate behind the adaptive macro step (an estimator of the kind
Section 3.1's remark asks for; the paper keeps Delta t fixed). No GPU needed.

The identity it rests on: on a quadratic trajectory c(t) = a + b t + q t^2 the least-squares
slope of the K+1 burst samples is the derivative at the burst's midpoint, so the forward-Euler
leap of length L from c_K (Section 3.3, Eq. extrapolation2 with the slope of Eq. leastsquares)
misses c(t_K + L) by exactly q L (L + K dt). The oracle's own projection checks it."""
import numpy as np
import pytest

import oracle as orc


@pytest.mark.parametrize("K,L", [(2, 0.3), (6, 1.7), (20, 18.0)])
def test_least_squares_leap_error_of_a_quadratic(K, L):
    dt = 0.1
    rng = np.random.default_rng(K)
    a, b, q = rng.normal(size=(3, 40))
    t = np.arange(K + 1) * dt
    samples = a + np.outer(t, b) + np.outer(t * t, q)
    coarse, slope = orc.ls_project(samples, dt, K * dt + L)
    tK = K * dt
    truth = a + b * (tK + L) + q * (tK + L) ** 2
    assert np.allclose(coarse - truth, -q * L * (L + K * dt), rtol=1e-9, atol=1e-9)
    qn, cn, noise = orc.leap_curvature(samples, dt)
    assert noise < 1e-9 * np.linalg.norm(q)  # exact quadratics leave no residual
    assert qn == pytest.approx(np.linalg.norm(q), rel=1e-9)
    assert cn == pytest.approx(np.linalg.norm(samples[-1]), rel=1e-14)


def test_linear_trajectories_have_no_curvature():
    dt, K = 0.2, 8
    t = np.arange(K + 1) * dt
    samples = 1.0 + np.outer(t, np.linspace(-1, 1, 16))
    qn, _, _ = orc.leap_curvature(samples, dt)
    assert qn < 1e-12
    assert orc.leap_for_tol(0.0, 1.0, K * dt, 1e-4) == float("inf")


@pytest.mark.parametrize("tol", [1e-6, 1e-4, 1e-2])
def test_leap_for_tol_meets_the_tolerance(tol):
    qn, cn, Kdt = 0.37, 5.0, 2.0
    L = orc.leap_for_tol(qn, cn, Kdt, tol)
    assert L > 0 and qn * L * (L + Kdt) / cn == pytest.approx(tol, rel=1e-10)


def test_noise_correction_removes_the_bias_of_the_curvature():
    # pure noise: the raw quadratic coefficients are nonzero, but their expected square is the
    # variance the residuals estimate, so the corrected curvature of many components is ~0;
    # a true curvature well above the noise survives the correction
    rng = np.random.default_rng(7)
    K, dt, n, sig = 20, 0.1, 4000, 1e-2
    t = np.arange(K + 1) * dt
    noise = sig * rng.normal(size=(K + 1, n))
    qn, _, nz = orc.leap_curvature(1.0 + noise, dt)
    raw = np.linalg.norm(np.polyfit(t, 1.0 + noise, 2)[0])
    assert nz == pytest.approx(raw, rel=0.05)  # the noise of q is what the raw norm measured
    assert qn < 0.2 * raw
    q = np.full(n, 5.0 * raw / np.sqrt(n))
    qn2, _, _ = orc.leap_curvature(1.0 + np.outer(t * t, q) + noise, dt)
    assert qn2 == pytest.approx(np.linalg.norm(q), rel=0.05)


def test_slope_noise_of_white_noise_matches_the_least_squares_law():
    # samples = a + b t + noise (std sigma) on 4000 components: the estimated slope noise is
    # sqrt(ncoef 12 sigma^2 / (K (K+1) (K+2) dt^2)) (the variance of a least-squares slope)
    rng = np.random.default_rng(41)
    K, dt, sigma, n = 12, 0.1, 0.3, 4000
    t = np.arange(K + 1) * dt
    y = 1.0 + 0.5 * t[:, None] + sigma * rng.standard_normal((K + 1, n))
    want = np.sqrt(n * 12 * sigma ** 2 / (K * (K + 1) * (K + 2) * dt ** 2))
    assert abs(orc.slope_noise(y, dt) / want - 1) < 0.03
    # noise-free quadratics have no residual
    q = 2.0 - 0.3 * t[:, None] + 0.7 * t[:, None] ** 2 * np.ones((1, 5))
    assert orc.slope_noise(q, dt) < 1e-9


def test_burst_length_for_noise_closed_form():
    # leap sn sqrt(K(K+1)(K+2) / (K'(K'+1)(K'+2))) <= tol cn: with K = 10 (K(K+1)(K+2) = 1320),
    # leap sn / (tol cn) = 4 needs K'(K'+1)(K'+2) >= 16 * 1320 = 21120: K' = 27 (27*28*29 = 21924;
    # 26*27*28 = 19656 is short)
    assert orc.burst_length_for_noise(4.0, 10, 1.0, 1.0, 1.0, 5, 40) == 27
    assert orc.burst_length_for_noise(4.0, 10, 1.0, 1.0, 1.0, 5, 20) == 20  # capped at K_max
    assert orc.burst_length_for_noise(0.01, 10, 1.0, 1.0, 1.0, 5, 40) == 5  # quiet: K_min
    assert orc.burst_length_for_noise(0.0, 10, 1.0, 1.0, 1.0, 5, 40) == 5
