"""GPU checks of the adaptive macro step (pe_leap_curvature, pe_step_adaptive,
pe_set_macro_step): the curvature estimate against the oracle, and the controller's rules
(whole bursts, bounds, rejection and rerun, the next step from the tolerance)."""
import numpy as np
import pytest
import torch

import oracle as orc
import paper_1610_01071_gb300 as pe

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("K,n", [(3, 17), (10, 256), (20, 16384)])
def test_leap_curvature_matches_oracle(K, n):
    rng = np.random.default_rng(K * n)
    dt = 0.1
    t = np.arange(K + 1) * dt
    q = rng.normal(size=n)
    samples = 1.0 + np.outer(t, rng.normal(size=n)) + np.outer(t * t, q) + 1e-3 * rng.normal(size=(K + 1, n))
    got = pe._binding.leap_curvature(torch.from_numpy(samples).to(DEV), dt).cpu().numpy()
    qn, cn, nz = orc.leap_curvature(samples, dt)
    assert got[1] == pytest.approx(cn, rel=1e-12)
    assert got[2] == pytest.approx(nz, rel=1e-9)
    assert got[0] == pytest.approx(qn, rel=1e-9)
    if K > 2:
        assert got[3] == pytest.approx(orc.slope_noise(samples, dt), rel=1e-9)


def make(seed=3, coarse="moments", dT_bursts=4, v_th=1.0):
    K, dt = 10, 0.1
    c = pe.make_config(128, 16, K, 128 * 256, 64.0, dt, dT_bursts * K * dt, v_th=v_th, seed=seed, newton_tol=1e-11,
                       coarse=coarse, n_v=32, v_max=6.0, ps_filter=3 if coarse == "phase_space" else 0)
    ctx = pe.Context(c, device=DEV)
    ctx.load_initial(0.1)
    return ctx, K * dt


@pytest.mark.parametrize("coarse", ["moments", "phase_space"])
def test_adaptive_steps_follow_the_controller(coarse):
    ctx, Kdt = make(coarse=coarse)
    tol, M_min, M_max, safety, grow = 3e-3, 1, 6, 0.8, 2.0
    t, M_prev = 0.0, 4
    for _ in range(8):
        st = ctx.step_adaptive(tol=tol, M_min=M_min, M_max=M_max, safety=safety, grow=grow)
        M = st["dT"] / Kdt
        assert abs(M - round(M)) < 1e-9 and M_min <= round(M) <= M_max
        assert st["fine_steps"] == 10 * (1 + st["rejected"])
        if st["rejected"] == 0:
            assert round(M) == M_prev  # the step the previous one chose
        assert st["err"] <= tol or round(M) == M_min
        L = st["dT"] - Kdt
        Mn = st["dT_next"] / Kdt
        assert abs(Mn - round(Mn)) < 1e-9 and M_min <= round(Mn) <= min(M_max, int(grow * round(M)))
        if L > 0 and st["err"] > 0:  # recompute the next step from the estimate
            r = tol / (st["err"] / (L * (L + Kdt)))  # tol ||c|| / ||q||
            L_tol = 0.5 * (-Kdt + np.sqrt(Kdt * Kdt + 4 * r))
            want = max(M_min, min(M_max, int(grow * round(M)), int(np.floor((Kdt + safety * L_tol) / Kdt + 1e-9))))
            assert round(Mn) == want
        t += st["dT"]
        M_prev = round(Mn)
    assert ctx.diagnostics().time == pytest.approx(t, rel=1e-12)
    assert ctx.sync_status() == 0


def test_a_tight_tolerance_rejects_down_to_the_smallest_step():
    # a cold plasma: smooth samples, so the curvature is not lost in particle noise
    ctx, Kdt = make(seed=5, dT_bursts=4, v_th=0.0)
    st = ctx.step_adaptive(tol=1e-14, M_min=1, M_max=8)
    assert st["rejected"] >= 1 and st["dT"] == pytest.approx(Kdt) and st["err"] == 0.0
    assert st["dT_next"] == pytest.approx(Kdt)
    assert ctx.diagnostics().macro_steps == 1


def test_set_macro_step_and_batches():
    ctx, Kdt = make(seed=7)
    with pytest.raises(pe.PepicError):
        ctx.set_macro_step(0.5 * Kdt)
    ctx.set_macro_step(3 * Kdt)
    ctx.step()
    assert ctx.diagnostics().time == pytest.approx(3 * Kdt)
    with pytest.raises(pe.PepicError):  # the ensemble steps by the configured Delta t only
        b = pe.Batch([ctx])
        b.step()


@pytest.mark.parametrize("expect", ["long", "short"])
def test_adaptive_burst_length_follows_the_noise_rule(expect):
    """Adaptive burst length: every step's K and the next K lie in [K_min, K_max]; the next K is
    the oracle rule applied to the step's reported slope noise; Delta t stays a whole number of
    bursts of the current length. With the tolerance a hundredth of the measured noise effect
    K goes to K_max, with a thousand times it to K_min."""
    ctx, Kdt = make(dT_bursts=3)
    dt, K_min, K_max = 0.1, 4, 10
    probe = ctx.step_adaptive(tol=1.0, M_min=2, M_max=6)  # fixed K: the noise effect of a 2-burst leap
    assert probe["K"] == 10 and probe["K_next"] == 10 and probe["noise"] > 0
    tol = probe["noise"] * (1e-2 if expect == "long" else 1e3)
    for _ in range(5):
        st = ctx.step_adaptive(tol=tol, M_min=2, M_max=6, K_min=K_min, K_max=K_max, noise_frac=0.5)
        K = st["K"]
        assert K_min <= K <= K_max and K_min <= st["K_next"] <= K_max
        assert st["fine_steps"] == K * (1 + st["rejected"])
        M = st["dT"] / (K * dt)
        assert abs(M - round(M)) < 1e-9
        Mn = st["dT_next"] / (st["K_next"] * dt)
        assert abs(Mn - round(Mn)) < 1e-9
        L = st["dT"] - K * dt
        if L > 0 and st["noise"] > 0:
            want = orc.burst_length_for_noise(st["noise"] / L, K, L, 1.0, 0.5 * tol, K_min, K_max)
            assert st["K_next"] == want
    assert ctx.sync_status() == 0
    assert st["K_next"] == (K_max if expect == "long" else K_min)
    # a checkpoint keeps the adapted burst length
    img = ctx.checkpoint()
    ctx2, _ = make(dT_bursts=3)
    ctx2.restore(img)
    a = ctx.step_adaptive(tol=tol, M_min=2, M_max=6, K_min=K_min, K_max=K_max)
    b = ctx2.step_adaptive(tol=tol, M_min=2, M_max=6, K_min=K_min, K_max=K_max)
    assert a["K"] == b["K"] and a["dT"] == b["dT"]
    assert torch.equal(ctx.get_coarse(), ctx2.get_coarse())
