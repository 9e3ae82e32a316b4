"""GPU parity of the diagnostics (charge, momentum, energies, Courant number, Section 4)
and of the Section 4.1.1 error measure against the FP64 CPU oracle, through the C ABI.

Tolerances: charge_fx bit-exact (integer sum of the fixed-point weights); momentum,
kinetic and field/electron energy 1e-6 relative (FP32 gather of the half kick against
FP64, FP64 sums in another order); max speed 1e-6 relative; error measure 1e-13.
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


def _field(ncell, L, seed):
    rng = np.random.default_rng(seed)
    x = np.arange(ncell) * (L / ncell)
    phi = 0.3 * np.cos(2 * np.pi * x / L) + 0.05 * rng.standard_normal(ncell)
    E = orc.efield(phi, L / ncell)
    return phi, E


@pytest.mark.parametrize("ncell,N,kick,mode", [(64, 1, 0.5, 0), (128, (1 << 14) + 3, 1.0, 0),
                                                (4096, (1 << 20) + 77, 1.0, 1), (8192, 1 << 22, 0.5, 0)])
def test_moments_match_oracle(ncell, N, kick, mode):
    L, dt, qm = ncell * 0.5, 0.1, 1.0
    dx = L / ncell
    c, t, v, w = inputs.random_particles(N, ncell, seed=N % 1000 + ncell)
    phi, E = _field(ncell, L, ncell)
    Ef = E.astype(np.float32)
    s_w = orc.fx_shift(2.0 * ncell / max(N, 1))
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    dc, dt_, dv, dw, dEf, dphi, dE = to_dev(c, t, v, w, Ef, phi, E)
    got = pe.compute_moments(dc, dt_, dv, dw, dEf, ncell, dx, dt, qm * dt, kick, s_w, phi=dphi, E=dE,
                             mode=("boltzmann", "linearized")[mode], status=st)
    # the oracle gathers the same FP32 field values, in FP64
    want = orc.moments(orc.State(c, t, v, w), Ef.astype(np.float64), phi, ncell, dx, dt, qm, kick, s_w, mode)
    assert int(st.item()) == 0 and got["invalid"] == 0
    assert got["charge_fx"] == want["charge_fx"]
    # the deposit-unit total is an int64 (it wraps like the oracle's beyond 2^63); charge_wq does not
    assert (((got["charge_wq"] << 24) + (1 << 63)) % (1 << 64)) - (1 << 63) == want["charge_fx"]
    assert got["charge_fixed_point"] == pytest.approx(want["charge_fx"] * 2.0 ** -(s_w + 24) * dx, rel=1e-15)
    for k in ("charge", "momentum", "kinetic", "max_speed", "cfl"):
        assert got[k] == pytest.approx(want[k], rel=1e-6, abs=1e-12), k
    # grid energies come from the FP64 arrays on both sides
    want_g = orc.moments(orc.State(c[:0], t[:0], v[:0], w[:0]), E, phi, ncell, dx, dt, qm, kick, s_w, mode)
    for k in ("field_energy", "electron_energy"):
        assert got[k] == pytest.approx(want_g[k], rel=1e-12), k
    total = want["kinetic"] + want_g["field_energy"] + want_g["electron_energy"]
    assert got["total_energy"] == pytest.approx(total, rel=1e-6)
    # fixed partition: identical bits on a repeat
    again = pe.compute_moments(dc, dt_, dv, dw, dEf, ncell, dx, dt, qm * dt, kick, s_w, phi=dphi, E=dE,
                               mode=("boltzmann", "linearized")[mode])
    assert again == got


def test_moments_empty_and_invalid_particles():
    ncell = 64
    c, t, v, w = inputs.random_particles(1000, ncell, seed=5)
    Ef = np.zeros(ncell, np.float32)
    got = pe.compute_moments(*to_dev(c[:0], t[:0], v[:0], w[:0], Ef), ncell, 0.5, 0.1, 0.1, 0.5, 20)
    assert got["charge_fx"] == 0 and got["invalid"] == 0 and got["kinetic"] == 0.0
    c, t, v = c.copy(), t.copy(), v.copy()
    c[3] = ncell      # cell out of range: counted, skipped (the kernel checks before any read)
    c[10] = -1
    v[20] = np.nan
    t[30] = 1.5
    keep = np.ones(1000, bool)
    keep[[3, 10, 20, 30]] = False
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    got = pe.compute_moments(*to_dev(c, t, v, w, Ef), ncell, 0.5, 0.1, 0.1, 0.5, 20, status=st)
    assert got["invalid"] == 4 and (int(st.item()) & 4)
    want = orc.moments(orc.State(c[keep], t[keep], v[keep], w[keep]), np.zeros(ncell), np.zeros(ncell), ncell, 0.5,
                       0.1, 1.0, 0.5, 20)
    assert got["charge_fx"] == want["charge_fx"]
    assert got["momentum"] == pytest.approx(want["momentum"], rel=1e-9)


@pytest.mark.parametrize("n", [0, 1, 512, 1 << 20])
def test_rel_l2_matches_oracle(n):
    rng = np.random.default_rng(n)
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    got = pe.rel_l2(*to_dev(a, b))
    assert got == pytest.approx(orc.rel_l2(a, b), rel=1e-13, abs=0.0)


def test_context_moments_conserve_charge_and_track_energy():
    """Through the context: the fixed-point charge is invariant to the bit over plain PIC
    steps (sorts included), and the total energy of resolved PIC stays within 2% of the
    energy it exchanges."""
    cfg = pe.make_config(64, 16, 20, 64 * 512, 32.0, 0.1, 20.0, v_th=0.1, seed=3, sort_every=20)
    ctx = pe.Context(cfg, device=DEV)
    ctx.load_initial(0.3)
    m0 = ctx.moments()
    assert m0["invalid"] == 0
    assert m0["charge"] == pytest.approx(32.0, rel=1e-6)
    hist = [m0]
    for _ in range(6):
        ctx.pic_steps(20)
        hist.append(ctx.moments())
    assert ctx.sync_status() == 0
    assert all(h["charge_fx"] == m0["charge_fx"] for h in hist)
    H = np.array([h["total_energy"] for h in hist])
    pot = np.array([h["field_energy"] + h["electron_energy"] for h in hist])
    assert np.ptp(pot) > 0.05
    assert np.abs(H - H[0]).max() < 0.02 * np.ptp(pot) + 1e-3 * abs(H[0])
    assert max(h["cfl"] for h in hist) < 1.0
