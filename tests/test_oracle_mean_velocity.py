"""Pins of the two ion mean-velocity functions of the oracle (no GPU).

Eq. electronpassive places the electrons of a lift with the ions' mean velocity, V_e = V_i.
Section 3.3 obtains the ions' n and V by integrating the coarse distribution along v, so the
oracle has two forms of V_i:

- ``ion_mean_velocity``: the CIC momentum of ion particles over their CIC density, per node;
- ``ps_mean_velocity``: per coarse x-bin, the mean velocity of its reconstructed CDF row (mass
  of each velocity cell at the cell centre), then linear in x between bin midpoints (periodic).

The pins are independent of the oracle's arithmetic: exact symmetry (a distribution symmetric
about u has mean u), the CIC ratio worked out by hand, and the interpolation between midpoints
written as a search over periodic distances. Two planted mistakes (half-bin offset of the
midpoints, cell edges instead of cell centres) are shown to fail the pins.
"""
import numpy as np
import pytest

import oracle as orc


# ------------------------------------------------------------------ ion_mean_velocity (CIC ratio)


def test_ion_mean_velocity_uniform_drift_is_exact():
    # every ion drifts with u: momentum = u * density node by node (dyadic data: no rounding)
    rng = np.random.default_rng(3)
    ncell, N, u = 32, 4096, 0.75
    cell = rng.integers(0, ncell, N).astype(np.int32)
    theta = rng.integers(0, 64, N) / 64.0
    w = rng.integers(1, 8, N) / 8.0
    st = orc.State(cell, theta, np.full(N, u), w)
    got = orc.ion_mean_velocity(st, ncell)
    assert np.all(got == u)


def test_ion_mean_velocity_two_particles_by_hand():
    # A: cell 2, theta 1/4, w 1, v +1. B: cell 2, theta 3/4, w 2, v -1 (ncell 8).
    # node 2: density 1(3/4) + 2(1/4) = 5/4, momentum 3/4 - 1/2 = 1/4  -> u = 1/5
    # node 3: density 1(1/4) + 2(3/4) = 7/4, momentum 1/4 - 3/2 = -5/4 -> u = -5/7
    st = orc.State(np.array([2, 2], np.int32), np.array([0.25, 0.75]), np.array([1.0, -1.0]), np.array([1.0, 2.0]))
    got = orc.ion_mean_velocity(st, 8)
    want = np.zeros(8)
    want[2], want[3] = 0.2, -5.0 / 7.0
    assert np.allclose(got, want, rtol=0, atol=1e-15)


def test_ion_mean_velocity_wraps_and_is_zero_where_empty():
    # an ion in the last cell shares its charge with node 0 (periodic); empty nodes give 0
    st = orc.State(np.array([7], np.int32), np.array([0.5]), np.array([-0.375]), np.array([1.0]))
    got = orc.ion_mean_velocity(st, 8)
    assert got[7] == -0.375 and got[0] == -0.375
    assert np.all(got[1:7] == 0.0)


# ------------------------------------------------------------------ ps_mean_velocity (CDF rows)


def symmetric_cdf(u_edges, vmin, dv, nv, half_width=4, sigma=1.3):
    """CDF rows [nxc][nv + 1] of truncated Gaussians about the cell edges vmin + u_edges[b] dv:
    the masses are symmetric about that edge, so each row's mean over cell centres is exactly
    that edge velocity."""
    F = np.zeros((len(u_edges), nv + 1))
    for b, k in enumerate(u_edges):
        u = vmin + k * dv
        p = np.zeros(nv)
        for j in range(k - half_width, k + half_width):  # the 2 half_width cells around the edge
            vc = vmin + (j + 0.5) * dv
            p[j] = np.exp(-0.5 * ((vc - u) / (sigma * dv)) ** 2)
        F[b, 1:] = np.cumsum(p) / p.sum()
        F[b, -1] = 1.0
    return F


def interpolate_between_midpoints(ub, bin_shift, ncell):
    """Nodal values of per-bin values ub: for node j, the nearest bin midpoint at or to the
    left of j (periodic distance d from midpoint m_b = b B + (B - 1)/2, B = 2^bin_shift),
    then linear towards the next bin's value with weight d / B."""
    B = 1 << bin_shift
    nxc = len(ub)
    out = np.zeros(ncell)
    for j in range(ncell):
        best, bsel = None, None
        for b in range(nxc):
            d = (j - (b * B + 0.5 * (B - 1))) % ncell
            if best is None or d < best:
                best, bsel = d, b
        f = best / B
        out[j] = (1 - f) * ub[bsel] + f * ub[(bsel + 1) % nxc]
    return out


def pin_ps_mean_velocity(fn):
    """The pins applied to a candidate implementation fn(cdf, vmin, dv, bin_shift, ncell);
    returns True when every pin holds."""
    vmin, nv = -4.0, 32
    dv = 8.0 / nv
    ok = True
    # (1) one symmetric row repeated in every bin: its edge velocity at every node
    for k in (16, 11, 21):
        for bin_shift, ncell in ((2, 64), (0, 16), (3, 128)):
            nxc = ncell >> bin_shift
            F = symmetric_cdf([k] * nxc, vmin, dv, nv)
            got = fn(F, vmin, dv, bin_shift, ncell)
            ok &= bool(np.max(np.abs(got - (vmin + k * dv))) < 1e-13)
    # (2) per-bin means linear in the bin index: linear in x between the first and last
    #     midpoints, and the closed-form interpolation (periodic wrap included) everywhere
    for bin_shift, ncell in ((2, 64), (3, 128), (1, 32)):
        nxc = ncell >> bin_shift
        ks = 8 + np.arange(nxc) % 17
        F = symmetric_cdf(list(ks), vmin, dv, nv)
        ub = vmin + ks * dv
        got = fn(F, vmin, dv, bin_shift, ncell)
        ok &= bool(np.max(np.abs(got - interpolate_between_midpoints(ub, bin_shift, ncell))) < 1e-13)
        B = 1 << bin_shift
        j = np.arange(ncell)
        inner = (j >= 0.5 * (B - 1)) & (j <= (nxc - 1) * B + 0.5 * (B - 1))
        if np.all(np.diff(ks) == 1):  # strictly linear stretch
            lin = vmin + (8 + (j - 0.5 * (B - 1)) / B) * dv
            ok &= bool(np.max(np.abs(got[inner] - lin[inner])) < 1e-13)
    # (3) a strictly linear table over the bins (no wrap in the bin values' slope inside)
    bin_shift, ncell = 2, 64
    nxc = ncell >> bin_shift
    ks = 8 + np.arange(nxc)
    F = symmetric_cdf(list(ks), vmin, dv, nv)
    got = fn(F, vmin, dv, bin_shift, ncell)
    B = 1 << bin_shift
    j = np.arange(ncell)
    inner = (j >= 0.5 * (B - 1)) & (j <= (nxc - 1) * B + 0.5 * (B - 1))
    lin = vmin + (8 + (j - 0.5 * (B - 1)) / B) * dv
    ok &= bool(np.max(np.abs(got[inner] - lin[inner])) < 1e-13)
    # wrap stretch: nodes after the last midpoint and before the first one interpolate between
    # the last bin's value and the first bin's
    wrap = ~inner
    want = interpolate_between_midpoints(vmin + ks * dv, bin_shift, ncell)
    ok &= bool(np.max(np.abs(got[wrap] - want[wrap])) < 1e-13)
    return ok


def test_ps_mean_velocity_pins_hold():
    assert pin_ps_mean_velocity(orc.ps_mean_velocity)


def _planted_half_bin(cdf, vmin, dv, bin_shift, ncell):
    # planted mistake: midpoints at the bin edges (t = j / B) instead of the bin centres
    nxc, nv = cdf.shape[0], cdf.shape[1] - 1
    vc = vmin + (np.arange(nv) + 0.5) * dv
    ub = np.sum(vc * np.diff(cdf, axis=1), axis=1)
    t = np.arange(ncell) / (2**bin_shift)
    b0 = np.floor(t)
    f = t - b0
    b0 = b0.astype(np.int64) % nxc
    return (1 - f) * ub[b0] + f * ub[(b0 + 1) % nxc]


def _planted_cell_edges(cdf, vmin, dv, bin_shift, ncell):
    # planted mistake: the mass of a velocity cell placed at its left edge
    out = orc.ps_mean_velocity(cdf, vmin, dv, bin_shift, ncell)
    return out - 0.5 * dv


@pytest.mark.parametrize("planted", [_planted_half_bin, _planted_cell_edges])
def test_ps_mean_velocity_pins_reject_planted_mistakes(planted):
    assert not pin_ps_mean_velocity(planted)
