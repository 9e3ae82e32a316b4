"""Plain FP64 CPU oracle for the projective-integration PIC hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference legs of ``bench.py`` may import this package. The
product path (``paper_1610_01071_gb300``) never imports it and shares no code
with it; the C source lives in ``pepic_oracle.c`` and every function there cites
the section, equation or appendix of Cazeaux & Hesthaven it follows.

This module only compiles the C file with gcc and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pepic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

THETA_ONE = 1 << 24


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = force or not os.path.exists(_LIB_PATH)
    if not stale:
        src_m = max(os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pepic_oracle.h")))
        stale = os.path.getmtime(_LIB_PATH) < src_m
    if stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
             "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, i64, u64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            P = ctypes.c_void_p
            sig = {
                "orc_splitmix64": (u64, [u64]),
                "orc_fx_shift": (i32, [dbl]),
                "orc_deposit_fx": (None, [i64, P, P, P, i32, i32, P]),
                "orc_deposit_f64": (None, [i64, P, P, P, P, i32, P, P]),
                "orc_cyclic_tridiag": (None, [i32, dbl, P, dbl, P, P]),
                "orc_newton_pb": (ctypes.c_int, [i32, dbl, i32, P, P, dbl, i32, P]),
                "orc_efield": (None, [i32, dbl, P, P]),
                "orc_gather": (dbl, [P, i32, i32, dbl]),
                "orc_push": (None, [i64, P, P, P, P, i32, dbl, dbl, dbl, dbl]),
                "orc_restrict_sample": (None, [i64, P, P, P, P, P, i32, dbl, dbl, dbl, P, P]),
                "orc_dwt_level": (None, [P, i32, P, i32, P, P]),
                "orc_idwt_level": (None, [P, i32, P, P, i32, P]),
                "orc_coarsen": (None, [P, i32, P, i32, P, i32]),
                "orc_refine": (None, [P, i32, P, i32, P, i32]),
                "orc_ls_slope": (dbl, [i32, dbl, P, i64]),
                "orc_ls_project": (None, [i32, i32, dbl, dbl, P, P, P]),
                "orc_ndtri": (dbl, [dbl]),
                "orc_quiet_start": (None, [i64, i32, P, P, dbl, u64, P, P, P, P]),
                "orc_lift_profile": (None, [i32, P, P, P]),
                "orc_burst": (ctypes.c_int, [i64, P, P, P, P, i32, dbl, dbl, dbl, i32, dbl,
                                             i32, i32, i32, dbl, i32, i32, P, P]),
                "orc_pic_steps": (ctypes.c_int, [i64, P, P, P, P, i32, dbl, dbl, dbl, i32,
                                                 i32, i32, dbl, i32, i32, P]),
                "orc_moments": (None, [i64, P, P, P, P, P, P, i32, dbl, dbl, dbl, dbl, i32, i32, P, P]),
                "orc_rel_l2": (dbl, [i64, P, P]),
                "orc_ps_sample_fx": (None, [i64, P, P, P, P, P, i32, dbl, dbl, dbl, i32, dbl, dbl, i32, i32, P]),
                "orc_cdf_reconstruct": (ctypes.c_int, [i32, P]),
                "orc_ps_lift_tables": (ctypes.c_int, [i32, i32, P, P, P]),
                "orc_cdf_inverse": (dbl, [i32, P, P, dbl, dbl, dbl]),
                "orc_cdf_cell_slopes": (None, [i32, P, P]),
                "orc_ps_quiet_start": (None, [i64, i32, i32, P, P, i32, dbl, dbl, u64, P, P, P, P]),
                "orc_ps_burst": (ctypes.c_int, [i64, P, P, P, P, i32, dbl, dbl, dbl, i32, dbl, i32, i32, dbl, i32,
                                                i32, i32, dbl, dbl, i32, P, P]),
                "orc_newton_pb_walls": (ctypes.c_int, [i32, dbl, i32, P, P, dbl, i32, P]),
                "orc_efield_walls": (None, [i32, dbl, P, P]),
                "orc_push_walls": (None, [i64, P, P, P, P, P, i32, dbl, dbl, dbl, dbl]),
                "orc_restrict_sample_walls": (None, [i64, P, P, P, P, P, i32, dbl, dbl, dbl, P, P]),
                "orc_quiet_start_equal": (None, [i64, i32, P, P, dbl, u64, P, P, P, P]),
                "orc_burst_walls": (ctypes.c_int, [i64, P, P, P, P, i32, dbl, dbl, dbl, i32, dbl,
                                                   i32, i32, i32, dbl, i32, i32, P, P]),
                "orc_pic_steps_walls": (ctypes.c_int, [i64, P, P, P, P, i32, dbl, dbl, dbl, i32,
                                                       i32, i32, dbl, i32, i32, P]),
                "orc_ps_sample_fx_walls": (None, [i64, P, P, P, P, P, i32, dbl, dbl, dbl, i32, dbl, dbl, i32, i32,
                                                  P]),
                "orc_ps_quiet_start_equal": (None, [i64, i32, i32, P, P, i32, dbl, dbl, u64, P, P, P, P]),
                "orc_ps_burst_walls": (ctypes.c_int, [i64, P, P, P, P, i32, dbl, dbl, dbl, i32, dbl, i32, i32, dbl,
                                                      i32, i32, i32, dbl, dbl, i32, P, P]),
                "orc_ps_hist_fine": (None, [i64, P, P, P, P, P, i32, dbl, dbl, dbl, dbl, dbl, i32, P]),
                "orc_ps_burst_fine": (ctypes.c_int, [i64, P, P, P, P, i32, dbl, dbl, dbl, i32, dbl, i32, i32, dbl,
                                                     i32, i32, dbl, dbl, i32, P, P]),
                "orc_ps_quiet_start_nodes": (None, [i64, i32, i32, P, P, i32, dbl, dbl, u64, P, P, P, P]),
                "orc_poisson_periodic": (None, [i32, dbl, P, P, P]),
                "orc_field_kinetic": (None, [i64, P, P, P, i64, P, P, P, i32, dbl, i32, P, P]),
                "orc_pic_steps_kinetic": (None, [i64, P, P, P, P, i64, P, P, P, P, i32, dbl, dbl, dbl, dbl, i32,
                                                 i32, i32, i32, P]),
                "orc_burst_kinetic": (None, [i64, P, P, P, P, i64, P, P, P, P, i32, dbl, dbl, dbl, dbl, i32, dbl,
                                             i32, i32, i32, dbl, dbl, i32, P, P, P]),
                "orc_boltzmann_electrons": (None, [i64, i32, P, P, dbl, u64, P, P, P, P]),
                "orc_restrict_second_moment": (None, [i64, P, P, P, P, P, i32, dbl, dbl, dbl, P]),
                "orc_burst_pressure": (ctypes.c_int, [i64, P, P, P, P, i32, dbl, dbl, dbl, i32, dbl,
                                                      i32, i32, i32, dbl, i32, i32, P, P]),
                "orc_lift_profile_pressure": (None, [i32, P, P, P, P, P]),
                "orc_quiet_start_thermal": (None, [i64, i32, P, P, P, u64, P, P, P, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ------------------------------------------------------------------ filters
# Orthonormal scaling filters (sum h = sqrt 2). Haar; Daubechies' 4-tap filter
# from its closed form (two vanishing moments of the wavelet); the coiflet of order 4
# (Appendix A: four vanishing moments of the wavelet, and of the scaling function the
# moments 1..3) from its defining equations.
_S3 = np.sqrt(3.0)


def coif4_equations(h):
    """Residuals of the order-4 coiflet conditions for 12 taps h_k, k = -4..7: sum h = sqrt 2;
    sum k^p h_k = 0 (p = 1, 2, 3: scaling-function moments about 0); sum (-1)^k k^p h_k = 0
    (p = 0..3: wavelet moments, the wavelet filter being (-1)^k h_{1-k}); sum_k h_k h_{k+2m} =
    delta_m (m = 0..5: orthonormal translates)."""
    k = np.arange(-4, 8, dtype=np.float64)
    r = [np.sum(h) - np.sqrt(2.0)]
    r += [np.sum(k**p * h) for p in (1, 2, 3)]
    r += [np.sum((-1.0) ** k * k**p * h) for p in (0, 1, 2, 3)]
    r += [np.dot(h[: 12 - 2 * m], h[2 * m:]) - (1.0 if m == 0 else 0.0) for m in range(6)]
    return np.array(r)


def _coif4_jacobian(h):
    k = np.arange(-4, 8, dtype=np.float64)
    rows = [np.ones(12)]
    rows += [k**p for p in (1, 2, 3)]
    rows += [(-1.0) ** k * k**p for p in (0, 1, 2, 3)]
    for m in range(6):
        r = np.zeros(12)
        r[: 12 - 2 * m] += h[2 * m:]
        r[2 * m:] += h[: 12 - 2 * m]
        rows.append(r)
    return np.array(rows)


def _coif4():
    """Solves the 14 coiflet equations for 12 taps by Gauss-Newton (numpy least-squares
    steps, halved until the residual decreases). The real solutions of the system are few
    (four); the coiflet is the one concentrated at k = 0 (the largest central tap h_0),
    Daubechies' choice. The Newton path from one start can reach another root depending on
    rounding, so several starts centred on k = 0 are tried and the solution with the largest
    h_0 is kept. Taps returned in the order k = -4..7."""
    best = None
    for start in ([0.5, 1.0, 0.5], [0.0, 2.0, 0.0], [0.0, 1.0, 1.0], [1.0, 0.5, 0.0], [0.0, 0.5, 1.0]):
        h = np.zeros(12)
        h[3:6] = np.array(start) / np.sqrt(2.0)
        for _ in range(200):
            r = coif4_equations(h)
            if np.max(np.abs(r)) < 1e-15:
                break
            d = np.linalg.lstsq(_coif4_jacobian(h), -r, rcond=None)[0]
            t = 1.0
            while t > 1e-6 and np.sum(coif4_equations(h + t * d) ** 2) >= np.sum(r**2):
                t *= 0.5
            h = h + t * d
        if np.max(np.abs(coif4_equations(h))) < 1e-13 and (best is None or h[4] > best[4]):
            best = h
    if best is None or not best[4] > 0.8:
        raise RuntimeError("coiflet equations not solved")
    return best


FILTERS = {
    "haar": np.array([1.0, 1.0]) / np.sqrt(2.0),
    "d4": np.array([1 + _S3, 3 + _S3, 3 - _S3, 1 - _S3]) / (4 * np.sqrt(2.0)),
    "coif4": _coif4(),
}
WAVELET_IDS = {0: "haar", 1: "d4", 2: "coif4"}


def splitmix64(x: int) -> int:
    return int(_load().orc_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def fx_shift(cap: float) -> int:
    return int(_load().orc_fx_shift(float(cap)))


class State:
    """FP64 particle state (cell, theta, v, w)."""

    def __init__(self, cell, theta, v, w):
        self.cell = _i32(cell).copy()
        self.theta = _f64(theta).copy()
        self.v = _f64(v).copy()
        self.w = _f64(w).copy()

    @property
    def n(self):
        return self.cell.shape[0]

    def copy(self):
        return State(self.cell, self.theta, self.v, self.w)


def deposit_fx(cell, theta, w, ncell, s_w):
    cell, theta, w = _i32(cell), _f64(theta), _f64(w)
    rho = np.zeros(ncell, np.int64)
    _load().orc_deposit_fx(cell.shape[0], _p(cell), _p(theta), _p(w), ncell, s_w, _p(rho))
    return rho


def deposit_f64(cell, theta, w, ncell, vel=None):
    cell, theta, w = _i32(cell), _f64(theta), _f64(w)
    dens = np.zeros(ncell)
    mom = np.zeros(ncell) if vel is not None else None
    vel_a = _f64(vel) if vel is not None else None
    _load().orc_deposit_f64(cell.shape[0], _p(cell), _p(theta), _p(w),
                            _p(vel_a) if vel is not None else None, ncell, _p(dens),
                            _p(mom) if mom is not None else None)
    return (dens, mom) if vel is not None else dens


def cyclic_tridiag(a, b, c, d):
    b, d = _f64(b), _f64(d)
    x = np.zeros_like(b)
    _load().orc_cyclic_tridiag(b.shape[0], float(a), _p(b), float(c), _p(d), _p(x))
    return x


def newton_pb(n, dx, phi0=None, mode=0, tol=1e-11, maxit=50):
    n = _f64(n)
    phi = _f64(phi0).copy() if phi0 is not None else np.log(np.maximum(n, 1e-8))
    iters = np.zeros(1, np.int32)
    fail = _load().orc_newton_pb(n.shape[0], float(dx), int(mode), _p(n), _p(phi), float(tol), int(maxit), _p(iters))
    return phi, int(iters[0]), int(fail)


def efield(phi, dx):
    phi = _f64(phi)
    E = np.zeros_like(phi)
    _load().orc_efield(phi.shape[0], float(dx), _p(phi), _p(E))
    return E


def gather(F, cell, theta):
    """CIC gather of nodal field F at each (cell, theta)."""
    F = _f64(F)
    fn = _load().orc_gather
    return np.array([fn(_p(F), F.shape[0], int(c), float(t)) for c, t in zip(cell, theta)])


def push(st: State, E, ncell, dx, dt, qm, kick=1.0):
    E = _f64(E)
    _load().orc_push(st.n, _p(st.cell), _p(st.theta), _p(st.v), _p(E), ncell, float(dx), float(dt),
                     float(qm), float(kick))


def restrict_sample(st: State, vbar, E0, ncell, dx, tau, qm):
    vbar, E0 = _f64(vbar), _f64(E0)
    dens, mom = np.zeros(ncell), np.zeros(ncell)
    _load().orc_restrict_sample(st.n, _p(st.cell), _p(st.theta), _p(vbar), _p(st.w), _p(E0), ncell,
                                float(dx), float(tau), float(qm), _p(dens), _p(mom))
    return dens, mom


def dwt_level(x, wavelet="haar"):
    h = FILTERS[wavelet]
    x = _f64(x)
    a, d = np.zeros(x.shape[0] // 2), np.zeros(x.shape[0] // 2)
    _load().orc_dwt_level(_p(h), h.shape[0], _p(x), x.shape[0], _p(a), _p(d))
    return a, d


def idwt_level(a, d, wavelet="haar"):
    h = FILTERS[wavelet]
    a = _f64(a)
    d = _f64(d) if d is not None else None
    x = np.zeros(2 * a.shape[0])
    _load().orc_idwt_level(_p(h), h.shape[0], _p(a), _p(d) if d is not None else None, a.shape[0], _p(x))
    return x


def coarsen(fine, ncoarse, wavelet="haar"):
    h = FILTERS[wavelet]
    fine = _f64(fine)
    out = np.zeros(ncoarse)
    _load().orc_coarsen(_p(h), h.shape[0], _p(fine), fine.shape[0], _p(out), ncoarse)
    return out


def refine(coarse, nfine, wavelet="haar"):
    h = FILTERS[wavelet]
    coarse = _f64(coarse)
    out = np.zeros(nfine)
    _load().orc_refine(_p(h), h.shape[0], _p(coarse), coarse.shape[0], _p(out), nfine)
    return out


def ls_slope(y, dt):
    y = _f64(y)
    return float(_load().orc_ls_slope(y.shape[0] - 1, float(dt), _p(y), 1))


def ls_project(samples, dt, dT):
    """samples: [K+1, ncoef]. Returns (coarse, slope)."""
    s = _f64(samples)
    K, ncoef = s.shape[0] - 1, s.shape[1]
    out, slope = np.zeros(ncoef), np.zeros(ncoef)
    _load().orc_ls_project(K, ncoef, float(dt), float(dT), _p(s), _p(out), _p(slope))
    return out, slope


def ndtri(p):
    lib = _load()
    return np.array([lib.orc_ndtri(float(x)) for x in np.atleast_1d(p)])


def quiet_start(N, ncell, nprof, uprof, v_th, seed):
    nprof, uprof = _f64(nprof), _f64(uprof)
    cell = np.zeros(N, np.int32)
    theta, v, w = np.zeros(N), np.zeros(N), np.zeros(N)
    _load().orc_quiet_start(N, ncell, _p(nprof), _p(uprof), float(v_th), seed & 0xFFFFFFFFFFFFFFFF,
                            _p(cell), _p(theta), _p(v), _p(w))
    return State(cell, theta, v, w)


def lift_profile(n, m):
    n = _f64(n).copy()
    m = _f64(m)
    u = np.zeros_like(n)
    _load().orc_lift_profile(n.shape[0], _p(n), _p(m), _p(u))
    return n, u


def burst(st: State, ncell, dx, dt, qm, K, dT, s_w, phi, comoving=True, mode=0, tol=1e-11,
          maxit=50, vel_at_integer=True):
    """Runs K steps in place on st; returns (samples [(K+1),2,ncell], phi, fails)."""
    phi = _f64(phi).copy()
    samples = np.zeros((K + 1, 2, ncell))
    fails = _load().orc_burst(st.n, _p(st.cell), _p(st.theta), _p(st.v), _p(st.w), ncell, float(dx),
                              float(dt), float(qm), int(K), float(dT), int(comoving), int(mode), int(s_w),
                              float(tol), int(maxit), int(vel_at_integer), _p(phi), _p(samples))
    return samples, phi, int(fails)


def pic_steps(st: State, ncell, dx, dt, qm, nsteps, s_w, phi, mode=0, tol=1e-11, maxit=50,
              vel_at_integer=True):
    phi = _f64(phi).copy()
    fails = _load().orc_pic_steps(st.n, _p(st.cell), _p(st.theta), _p(st.v), _p(st.w), ncell, float(dx),
                                  float(dt), float(qm), int(nsteps), int(mode), int(s_w), float(tol),
                                  int(maxit), int(vel_at_integer), _p(phi))
    return phi, int(fails)


# ------------------------------------------------------------------ composite steps


def sine_profile(ncell, L, amplitude):
    """Section 4.1 initial condition on nodes: n = 1 + d cos(2 pi x/L), u = d cos(2 pi x/L)."""
    x = np.arange(ncell) * (L / ncell)
    c = amplitude * np.cos(2 * np.pi * x / L)
    return 1.0 + c, c


def efpi_macro_step(st: State, cfg: dict, phi, vel_at_integer=True):
    """One forward-Euler projective step (Section 3.1/3.3): burst with co-moving
    restriction, coarsening, least-squares slope, leap. Returns (coarse [2,nc], samples_c, phi)."""
    ncell, nc, K = cfg["ncell"], cfg["n_coarse"], cfg["K"]
    dx = cfg["L"] / ncell
    samples, phi, fails = burst(st, ncell, dx, cfg["dt"], cfg["qm"], K, cfg["dT"], cfg["s_w"], phi,
                                comoving=cfg.get("comoving", True), mode=cfg.get("mode", 0),
                                vel_at_integer=vel_at_integer)
    wav = cfg.get("wavelet", "haar")
    cs = np.zeros((K + 1, 2, nc))
    for p in range(K + 1):
        for m in range(2):
            cs[p, m] = coarsen(samples[p, m], nc, wav)
    coarse, _ = ls_project(cs.reshape(K + 1, 2 * nc), cfg["dt"], cfg["dT"])
    return coarse.reshape(2, nc), cs, phi


def lift(coarse, cfg: dict, seed):
    """Lifting (Section 3.3 + Appendix C): refine with zero details, clamp, quiet start."""
    ncell = cfg["ncell"]
    wav = cfg.get("wavelet", "haar")
    nf = refine(coarse[0], ncell, wav)
    mf = refine(coarse[1], ncell, wav)
    nf, uf = lift_profile(nf, mf)
    return quiet_start(cfg["N"], ncell, nf, uf, cfg["v_th"], seed)


MOMENT_KEYS = ("charge", "momentum", "kinetic", "field_energy", "electron_energy", "total_energy",
               "max_speed", "cfl")


def moments(st: State, E, phi, ncell, dx, dt, qm, kick, s_w, mode=0):
    """Conserved quantities and CFL number of a state (orc_moments); dict incl. charge_fx."""
    E, phi = _f64(E), _f64(phi)
    q = np.zeros(1, np.int64)
    out = np.zeros(8)
    _load().orc_moments(st.n, _p(st.cell), _p(st.theta), _p(st.v), _p(st.w), _p(E), _p(phi), ncell, dx, dt, qm,
                        kick, s_w, mode, _p(q), _p(out))
    d = dict(zip(MOMENT_KEYS, out.tolist()))
    d["charge_fx"] = int(q[0])
    return d


def rel_l2(a, b):
    """Section 4.1.1 error measure sqrt(sum (a-b)^2 / sum (a^2 + b^2))."""
    a, b = _f64(a).ravel(), _f64(b).ravel()
    assert a.shape == b.shape
    return float(_load().orc_rel_l2(a.size, _p(a), _p(b)))


def field_of(st: State, ncell, dx, s_w, phi, mode=0, tol=1e-12, maxit=50):
    """Deposit + Newton + E of a state (the field step of a PIC step); phi updated in place."""
    rho = deposit_fx(st.cell, st.theta, st.w, ncell, s_w)
    dens = rho.astype(np.float64) * 2.0 ** -(s_w + 24)
    phi[:] = newton_pb(dens, dx, phi0=phi, mode=mode, tol=tol, maxit=maxit)[0]
    return efield(phi, dx)


# ------------------------------------------------------------------ phase-space coarse variable


def ps_sample_fx(st: State, vbar, E0, ncell, dx, tau, qm, bin_shift, vmin, dv, nv, s_w):
    """Co-moving phase-space sample in fixed point: int64 [(ncell >> b), nv]."""
    vbar, E0 = _f64(vbar), _f64(E0)
    F = np.zeros((ncell >> bin_shift, nv), np.int64)
    _load().orc_ps_sample_fx(st.n, _p(st.cell), _p(st.theta), _p(vbar), _p(st.w), _p(E0), ncell, float(dx),
                             float(tau), float(qm), int(bin_shift), float(vmin), float(dv), int(nv), int(s_w), _p(F))
    return F


def cdf_reconstruct(F):
    """Appendix C reconstruction of a CDF array (copy); returns (F, pathological flag)."""
    F = _f64(F).copy()
    bad = _load().orc_cdf_reconstruct(F.shape[0] - 1, _p(F))
    return F, int(bad)


def ps_lift_tables(H):
    """H [nxc, nv] (FP64 masses) -> (mass [nxc], cdf [nxc, nv+1], pathological flag)."""
    H = _f64(H)
    nxc, nv = H.shape
    mass = np.zeros(nxc)
    cdf = np.zeros((nxc, nv + 1))
    bad = _load().orc_ps_lift_tables(nxc, nv, _p(H), _p(mass), _p(cdf))
    return mass, cdf, int(bad)


def cdf_cell_slopes(F):
    F = _f64(F)
    sig = np.zeros(F.shape[0] - 1)
    _load().orc_cdf_cell_slopes(F.shape[0] - 1, _p(F), _p(sig))
    return sig


def cdf_inverse(F, b, vmin, dv, sigma=None):
    """Inverse CDF; sigma (per-cell density slopes) None: uniform inside each cell."""
    F = _f64(F)
    sg = _f64(sigma) if sigma is not None else None
    return float(_load().orc_cdf_inverse(F.shape[0] - 1, _p(F), _p(sg) if sg is not None else None, float(b),
                                         float(vmin), float(dv)))


def ps_quiet_start(N, ncell, bin_shift, mass, cdf, vmin, dv, seed):
    mass, cdf = _f64(mass), _f64(cdf)
    nv = cdf.shape[1] - 1
    cell = np.zeros(N, np.int32)
    theta, v, w = np.zeros(N), np.zeros(N), np.zeros(N)
    _load().orc_ps_quiet_start(N, ncell, int(bin_shift), _p(mass), _p(cdf), nv, float(vmin), float(dv),
                               seed & 0xFFFFFFFFFFFFFFFF, _p(cell), _p(theta), _p(v), _p(w))
    return State(cell, theta, v, w)


def ps_burst(st: State, ncell, dx, dt, qm, K, dT, s_w, phi, bin_shift, vmin, dv, nv, mode=0, tol=1e-11,
             maxit=50, vel_at_integer=True):
    """K fine steps in place with phase-space co-moving samples; returns (samples int64
    [(K+1), nxc, nv], phi, fails)."""
    phi = _f64(phi).copy()
    samples = np.zeros((K + 1, ncell >> bin_shift, nv), np.int64)
    fails = _load().orc_ps_burst(st.n, _p(st.cell), _p(st.theta), _p(st.v), _p(st.w), ncell, float(dx), float(dt),
                                 float(qm), int(K), float(dT), int(mode), int(s_w), float(tol), int(maxit),
                                 int(vel_at_integer), int(bin_shift), float(vmin), float(dv), int(nv), _p(phi),
                                 _p(samples))
    return samples, phi, int(fails)


# ------------------------------------------------------------------ phase space, wavelet form
# Section 3.3 as the paper states it (Eqs. waveletapproximation, restriction, interpolation;
# Appendices A-C): the coarse variable is the array of coarse scaling coefficients
# C[i, m] (coarse x node i, velocity coefficient m) of the phase-space histogram.


def ps_hist_fine(st: State, vbar, E0, ncell, dx, tau, qm, vmin, dv, nvf):
    """Fine co-moving histogram [ncell, nvf] (FP64): hat weights on the fine nodes in x,
    nearest cell in v (Appendix B)."""
    vbar, E0 = _f64(vbar), _f64(E0)
    H = np.zeros((ncell, nvf))
    _load().orc_ps_hist_fine(st.n, _p(st.cell), _p(st.theta), _p(vbar), _p(st.w), _p(E0), ncell, float(dx),
                             float(tau), float(qm), float(vmin), float(dv), int(nvf), _p(H))
    return H


def ps_burst_fine(st: State, ncell, dx, dt, qm, K, dT, s_w, phi, vmin, dv, nvf, mode=0, tol=1e-11, maxit=50,
                  vel_at_integer=True):
    """K fine steps in place with the fine co-moving histograms; returns (samples
    [(K+1), ncell, nvf], phi, fails)."""
    phi = _f64(phi).copy()
    samples = np.zeros((K + 1, ncell, nvf))
    fails = _load().orc_ps_burst_fine(st.n, _p(st.cell), _p(st.theta), _p(st.v), _p(st.w), ncell, float(dx),
                                      float(dt), float(qm), int(K), float(dT), int(mode), int(s_w), float(tol),
                                      int(maxit), int(vel_at_integer), float(vmin), float(dv), int(nvf), _p(phi),
                                      _p(samples))
    return samples, phi, int(fails)


def restrict_121(f, levels):
    """Eq. (restriction) along axis 0, `levels` times: coarse node k (fine node 2k) takes
    (f[2k-1] + 2 f[2k] + f[2k+1]) / 4, periodic."""
    f = np.asarray(f, dtype=np.float64)
    for _ in range(levels):
        left = np.roll(f, 1, axis=0)[0::2]   # f[2k - 1]
        mid = f[0::2]                         # f[2k]
        right = np.roll(f, -1, axis=0)[0::2]  # f[2k + 1]
        f = 0.25 * (left + 2.0 * mid + right)
    return f


def interpolate_x(f, levels):
    """Eq. (interpolation) along axis 0, `levels` times: fine node 2k takes f[k], fine node
    2k+1 the mean of f[k] and f[k+1], periodic."""
    f = np.asarray(f, dtype=np.float64)
    for _ in range(levels):
        out = np.empty((2 * f.shape[0],) + f.shape[1:])
        out[0::2] = f
        out[1::2] = 0.5 * (f + np.roll(f, -1, axis=0))
        f = out
    return f


def ps_coarsen_v(H, nvc, wavelet="coif4"):
    """Periodized DWT along the last axis from nvf cells to nvc scaling coefficients
    (Section 3.3; Appendix A), details discarded, scaled by 2^(L/2) for L levels so that
    the coefficients of a row sum to its mass (each analysis level multiplies a row's sum
    by 1/sqrt 2)."""
    H = np.asarray(H, dtype=np.float64)
    nvf = H.shape[-1]
    L = int(np.log2(nvf // nvc))
    rows = H.reshape(-1, nvf)
    out = np.zeros((rows.shape[0], nvc))
    for r in range(rows.shape[0]):
        a = rows[r]
        for _ in range(L):
            a, _d = dwt_level(a, wavelet)
        out[r] = a * 2.0 ** (L / 2)
    return out.reshape(H.shape[:-1] + (nvc,))


def ps_refine_v(C, nvf, wavelet="coif4"):
    """Synthesis along the last axis with zero details from nvc coefficients to nvf cells,
    scaled by 2^(-L/2): the inverse of ps_coarsen_v on its range."""
    C = np.asarray(C, dtype=np.float64)
    nvc = C.shape[-1]
    L = int(np.log2(nvf // nvc))
    rows = C.reshape(-1, nvc)
    out = np.zeros((rows.shape[0], nvf))
    for r in range(rows.shape[0]):
        a = rows[r]
        for _ in range(L):
            a = idwt_level(a, None, wavelet)
        out[r] = a * 2.0 ** (-L / 2)
    return out.reshape(C.shape[:-1] + (nvf,))


def ps_wavelet_restrict(hist, bin_shift, nvc, wavelet="coif4"):
    """Coarse coefficients [.., nxc, nvc] of fine histograms [.., ncell, nvf]: Eq.
    (restriction) in x (bin_shift levels), then ps_coarsen_v."""
    hist = np.asarray(hist, dtype=np.float64)
    if hist.ndim == 2:
        return ps_coarsen_v(restrict_121(hist, bin_shift), nvc, wavelet)
    return np.stack([ps_coarsen_v(restrict_121(h, bin_shift), nvc, wavelet) for h in hist])


def ps_quiet_start_nodes(N, ncell, bin_shift, mass, cdf, vmin, dv, seed):
    """Appendix C loading of the wavelet form on coarse-node tables (mass [nxc], cdf
    [nxc, nvf+1])."""
    mass, cdf = _f64(mass), _f64(cdf)
    nvf = cdf.shape[1] - 1
    cell = np.zeros(N, np.int32)
    theta, v, w = np.zeros(N), np.zeros(N), np.zeros(N)
    _load().orc_ps_quiet_start_nodes(N, ncell, int(bin_shift), _p(mass), _p(cdf), nvf, float(vmin), float(dv),
                                     seed & 0xFFFFFFFFFFFFFFFF, _p(cell), _p(theta), _p(v), _p(w))
    return State(cell, theta, v, w)


def ps_wavelet_lift(coarse, cfg: dict, seed):
    """Lifting of the wavelet form (Section 3.3): synthesis in v to the fine velocity cells,
    the Appendix C reconstruction per coarse node (negative node masses clamped, total kept),
    then the loading with the linear interpolation in x. Returns (state, pathological flag)."""
    nvf, wav = cfg["n_v"], cfg.get("wavelet", "coif4")
    H = ps_refine_v(coarse, nvf, wav)
    mass, cdf, bad = ps_lift_tables(H)
    b = int(np.log2(cfg["ncell"] // cfg["n_coarse"]))
    vmin, dv = -cfg["v_max"], 2.0 * cfg["v_max"] / nvf
    return ps_quiet_start_nodes(cfg["N"], cfg["ncell"], b, mass, cdf, vmin, dv, seed), bad


def efpi_ps_wavelet_macro_step(st: State, cfg: dict, phi, vel_at_integer=True):
    """One projective step of the wavelet form: burst with fine co-moving histograms, Eq.
    (restriction) and the DWT in v, least-squares slope, leap (Eqs. extrapolation2 and
    leastsquares). Returns (coarse [nxc, nvc], coarse samples [(K+1), nxc, nvc], phi)."""
    ncell, nc, K, nvf, nvc = cfg["ncell"], cfg["n_coarse"], cfg["K"], cfg["n_v"], cfg["n_v_coarse"]
    dx = cfg["L"] / ncell
    vmin, dv = -cfg["v_max"], 2.0 * cfg["v_max"] / nvf
    samples, phi, fails = ps_burst_fine(st, ncell, dx, cfg["dt"], cfg["qm"], K, cfg["dT"], cfg["s_w"], phi, vmin, dv,
                                        nvf, mode=cfg.get("mode", 0), vel_at_integer=vel_at_integer)
    b = int(np.log2(ncell // nc))
    cs = ps_wavelet_restrict(samples, b, nvc, cfg.get("wavelet", "coif4"))
    coarse, _ = ls_project(cs.reshape(K + 1, nc * nvc), cfg["dt"], cfg["dT"])
    return coarse.reshape(nc, nvc), cs, phi


# ------------------------------------------------------------------ bounded domain (Section 4.2)
# Walls at node 0 and node ncell-1, absorbing for the ions, phi' = 0 for the potential.


def newton_pb_walls(dep, dx, phi0=None, mode=0, tol=1e-11, maxit=50):
    """Newton for Poisson-Boltzmann with mirror ghosts; dep is the nodal deposit (the wall
    nodes count twice in the density)."""
    dep = _f64(dep)
    if phi0 is not None:
        phi = _f64(phi0).copy()
    else:
        dens = dep.copy()
        dens[[0, -1]] *= 2.0
        phi = np.log(np.maximum(dens, 1e-8))
    iters = np.zeros(1, np.int32)
    fail = _load().orc_newton_pb_walls(dep.shape[0], float(dx), int(mode), _p(dep), _p(phi), float(tol), int(maxit),
                                       _p(iters))
    return phi, int(iters[0]), int(fail)


def efield_walls(phi, dx):
    phi = _f64(phi)
    E = np.zeros_like(phi)
    _load().orc_efield_walls(phi.shape[0], float(dx), _p(phi), _p(E))
    return E


def push_walls(st: State, E, ncell, dx, dt, qm, kick=1.0):
    E = _f64(E)
    _load().orc_push_walls(st.n, _p(st.cell), _p(st.theta), _p(st.v), _p(st.w), _p(E), ncell, float(dx), float(dt),
                           float(qm), float(kick))


def restrict_sample_walls(st: State, vbar, E0, ncell, dx, tau, qm):
    vbar, E0 = _f64(vbar), _f64(E0)
    dens, mom = np.zeros(ncell), np.zeros(ncell)
    _load().orc_restrict_sample_walls(st.n, _p(st.cell), _p(st.theta), _p(vbar), _p(st.w), _p(E0), ncell,
                                      float(dx), float(tau), float(qm), _p(dens), _p(mom))
    return dens, mom


def quiet_start_equal(N, ncell, nprof, uprof, v_th, seed):
    nprof, uprof = _f64(nprof), _f64(uprof)
    cell = np.zeros(N, np.int32)
    theta, v, w = np.zeros(N), np.zeros(N), np.zeros(N)
    _load().orc_quiet_start_equal(N, ncell, _p(nprof), _p(uprof), float(v_th), seed & 0xFFFFFFFFFFFFFFFF,
                                  _p(cell), _p(theta), _p(v), _p(w))
    return State(cell, theta, v, w)


def burst_walls(st: State, ncell, dx, dt, qm, K, dT, s_w, phi, comoving=True, mode=0, tol=1e-11, maxit=50,
                vel_at_integer=True):
    phi = _f64(phi).copy()
    samples = np.zeros((K + 1, 2, ncell))
    fails = _load().orc_burst_walls(st.n, _p(st.cell), _p(st.theta), _p(st.v), _p(st.w), ncell, float(dx),
                                    float(dt), float(qm), int(K), float(dT), int(comoving), int(mode), int(s_w),
                                    float(tol), int(maxit), int(vel_at_integer), _p(phi), _p(samples))
    return samples, phi, int(fails)


def pic_steps_walls(st: State, ncell, dx, dt, qm, nsteps, s_w, phi, mode=0, tol=1e-11, maxit=50,
                    vel_at_integer=True):
    phi = _f64(phi).copy()
    fails = _load().orc_pic_steps_walls(st.n, _p(st.cell), _p(st.theta), _p(st.v), _p(st.w), ncell, float(dx),
                                        float(dt), float(qm), int(nsteps), int(mode), int(s_w), float(tol),
                                        int(maxit), int(vel_at_integer), _p(phi))
    return phi, int(fails)


def slab_profile(ncell):
    """Section 4.2 slab in vacuum, uniform variant: n = 1 on the nodes of the central eighth,
    7 ncell/16 <= j <= 9 ncell/16, and 0 elsewhere; u = 0."""
    n = np.zeros(ncell)
    n[7 * ncell // 16: 9 * ncell // 16 + 1] = 1.0
    return n, np.zeros(ncell)


def field_of_walls(st: State, ncell, dx, s_w, phi, mode=0, tol=1e-12, maxit=50):
    rho = deposit_fx(st.cell, st.theta, st.w, ncell, s_w)
    dens = rho.astype(np.float64) * 2.0 ** -(s_w + 24)
    phi[:] = newton_pb_walls(dens, dx, phi0=phi, mode=mode, tol=tol, maxit=maxit)[0]
    return efield_walls(phi, dx)


def efpi_macro_step_walls(st: State, cfg: dict, phi, vel_at_integer=True):
    """efpi_macro_step in the bounded domain."""
    ncell, nc, K = cfg["ncell"], cfg["n_coarse"], cfg["K"]
    dx = cfg["L"] / ncell
    samples, phi, fails = burst_walls(st, ncell, dx, cfg["dt"], cfg["qm"], K, cfg["dT"], cfg["s_w"], phi,
                                      comoving=cfg.get("comoving", True), mode=cfg.get("mode", 0),
                                      vel_at_integer=vel_at_integer)
    wav = cfg.get("wavelet", "haar")
    cs = np.zeros((K + 1, 2, nc))
    for p in range(K + 1):
        for m in range(2):
            cs[p, m] = coarsen(samples[p, m], nc, wav)
    coarse, _ = ls_project(cs.reshape(K + 1, 2 * nc), cfg["dt"], cfg["dT"])
    return coarse.reshape(2, nc), cs, phi


def lift_walls(coarse, cfg: dict, seed):
    """Lifting in the bounded domain: refine, clamp, the wall nodes' deposits doubled to
    densities, equal-weight loading."""
    ncell = cfg["ncell"]
    wav = cfg.get("wavelet", "haar")
    nf = refine(coarse[0], ncell, wav)
    mf = refine(coarse[1], ncell, wav)
    nf, uf = lift_profile(nf, mf)
    nf[[0, -1]] *= 2.0
    return quiet_start_equal(cfg["N"], ncell, nf, uf, cfg["v_th"], seed)


# ------------------------------------------------------------------ phase space on the bounded grid


def ps_sample_fx_walls(st: State, vbar, E0, ncell, dx, tau, qm, bin_shift, vmin, dv, nv, s_w):
    vbar, E0 = _f64(vbar), _f64(E0)
    F = np.zeros((ncell >> bin_shift, nv), np.int64)
    _load().orc_ps_sample_fx_walls(st.n, _p(st.cell), _p(st.theta), _p(vbar), _p(st.w), _p(E0), ncell, float(dx),
                                   float(tau), float(qm), int(bin_shift), float(vmin), float(dv), int(nv), int(s_w),
                                   _p(F))
    return F


def ps_quiet_start_equal(N, ncell, bin_shift, mass, cdf, vmin, dv, seed):
    mass, cdf = _f64(mass), _f64(cdf)
    nv = cdf.shape[1] - 1
    cell = np.zeros(N, np.int32)
    theta, v, w = np.zeros(N), np.zeros(N), np.zeros(N)
    _load().orc_ps_quiet_start_equal(N, ncell, int(bin_shift), _p(mass), _p(cdf), nv, float(vmin), float(dv),
                                     seed & 0xFFFFFFFFFFFFFFFF, _p(cell), _p(theta), _p(v), _p(w))
    return State(cell, theta, v, w)


def ps_burst_walls(st: State, ncell, dx, dt, qm, K, dT, s_w, phi, bin_shift, vmin, dv, nv, mode=0, tol=1e-11,
                   maxit=50, vel_at_integer=True):
    phi = _f64(phi).copy()
    samples = np.zeros((K + 1, ncell >> bin_shift, nv), np.int64)
    fails = _load().orc_ps_burst_walls(st.n, _p(st.cell), _p(st.theta), _p(st.v), _p(st.w), ncell, float(dx),
                                       float(dt), float(qm), int(K), float(dT), int(mode), int(s_w), float(tol),
                                       int(maxit), int(vel_at_integer), int(bin_shift), float(vmin), float(dv),
                                       int(nv), _p(phi), _p(samples))
    return samples, phi, int(fails)


def ps_project(samples, dt, dT, filt=0):
    """Projective step of the phase-space masses samples [(K+1), nxc, nv] (Section 3.3, Eqs.
    extrapolation2 and leastsquares) with the least-squares slope filtered before the leap:
    filt bit 0 smooths every x-bin's slope along v by (1/4, 1/2, 1/4) with zero beyond the
    velocity range; bit 1 smooths every velocity cell's slope along x, periodically, or with
    bit 2 reflecting at the walls (the edge value repeated, which keeps the sum). Returns
    (out, filtered slope), both [nxc, nv]."""
    y = _f64(samples)
    K1, nxc, nv = y.shape
    _, raw = ls_project(y.reshape(K1, nxc * nv), dt, dT)
    raw = raw.reshape(nxc, nv)
    s = raw
    if filt & 1:
        pad = np.zeros((nxc, nv + 2))
        pad[:, 1:-1] = s
        s = 0.25 * pad[:, :-2] + 0.5 * pad[:, 1:-1] + 0.25 * pad[:, 2:]
    if filt & 2:
        if filt & 4:
            left = np.concatenate([s[:1], s[:-1]])
            right = np.concatenate([s[1:], s[-1:]])
        else:
            left, right = np.roll(s, 1, axis=0), np.roll(s, -1, axis=0)
        s = 0.25 * left + 0.5 * s + 0.25 * right
    out = y[-1] + (dT - (K1 - 1) * dt) * s
    return out, s


# ------------------------------------------------------------------ kinetic electrons (Section 4.1)
# Both species as particles in the bursts; ions q/m = qm_i, electrons q/m = qm_e (-1800 in the
# paper's runs). The field is the periodic Poisson equation for the net charge n_i - n_e.


def poisson_periodic(r, dx):
    """-(phi_{j+1} - 2 phi_j + phi_{j-1}) / dx^2 = r_j - <r>, <phi> = 0; returns (phi, E)."""
    r = _f64(r)
    phi, E = np.zeros_like(r), np.zeros_like(r)
    _load().orc_poisson_periodic(r.shape[0], float(dx), _p(r), _p(phi), _p(E))
    return phi, E


def field_kinetic(ions: State, electrons: State, ncell, dx, s_w):
    """Fixed-point deposits of both species, net density, periodic Poisson: (phi, E)."""
    phi, E = np.zeros(ncell), np.zeros(ncell)
    _load().orc_field_kinetic(ions.n, _p(ions.cell), _p(ions.theta), _p(ions.w), electrons.n, _p(electrons.cell),
                              _p(electrons.theta), _p(electrons.w), ncell, float(dx), int(s_w), _p(phi), _p(E))
    return phi, E


def pic_steps_kinetic(ions: State, electrons: State, ncell, dx, dt, qm_i, qm_e, nsteps, s_w, vel_at_integer=True,
                      e_vel_at_integer=None):
    """nsteps two-species leapfrog steps in place; returns the last step's phi. The electrons'
    first kick is a half kick if e_vel_at_integer (default: vel_at_integer)."""
    phi = np.zeros(ncell)
    ev = vel_at_integer if e_vel_at_integer is None else e_vel_at_integer
    _load().orc_pic_steps_kinetic(ions.n, _p(ions.cell), _p(ions.theta), _p(ions.v), _p(ions.w), electrons.n,
                                  _p(electrons.cell), _p(electrons.theta), _p(electrons.v), _p(electrons.w), ncell,
                                  float(dx), float(dt), float(qm_i), float(qm_e), int(nsteps), int(s_w),
                                  int(vel_at_integer), int(ev), _p(phi))
    return phi


def burst_kinetic(ions: State, electrons: State, ncell, dx, dt, qm_i, qm_e, K, dT, s_w, vel_at_integer=True,
                  nv=0, bin_shift=0, vmin=0.0, dv=1.0):
    """K two-species steps in place with the ions' co-moving restriction; returns (samples, phi):
    moments [(K+1), 2, ncell] (double) for nv = 0, else phase-space int64 [(K+1), nxc, nv]."""
    phi = np.zeros(ncell)
    if nv > 0:
        sfx = np.zeros((K + 1, ncell >> bin_shift, nv), np.int64)
        sd = np.zeros(1)
    else:
        sd = np.zeros((K + 1, 2, ncell))
        sfx = np.zeros(1, np.int64)
    _load().orc_burst_kinetic(ions.n, _p(ions.cell), _p(ions.theta), _p(ions.v), _p(ions.w), electrons.n,
                              _p(electrons.cell), _p(electrons.theta), _p(electrons.v), _p(electrons.w), ncell,
                              float(dx), float(dt), float(qm_i), float(qm_e), int(K), float(dT), int(s_w),
                              int(vel_at_integer), int(bin_shift), float(vmin), float(dv), int(nv), _p(phi), _p(sd),
                              _p(sfx))
    return (sfx if nv > 0 else sd), phi


def ion_mean_velocity(ions: State, ncell):
    """The ions' nodal mean velocity: CIC momentum over CIC density (0 where the density is 0)."""
    d, m = deposit_f64(ions.cell, ions.theta, ions.w, ncell, vel=ions.v)
    return np.where(d > 0, m / np.where(d > 0, d, 1.0), 0.0)


def boltzmann_electrons(N, ncell, phi, v_th_e, seed, u=None, ions: State = None):
    """Electrons of the lifting: quiet start on n_e = exp(phi) drifting with the ions' mean
    velocity u (V_e = V_i), or with that of the particles `ions`; no drift without either."""
    phi = _f64(phi)
    if u is None and ions is not None:
        u = ion_mean_velocity(ions, ncell)
    ua = _f64(u) if u is not None else None
    cell = np.zeros(N, np.int32)
    theta, v, w = np.zeros(N), np.zeros(N), np.zeros(N)
    _load().orc_boltzmann_electrons(N, ncell, _p(phi), _p(ua) if ua is not None else None, float(v_th_e),
                                    seed & 0xFFFFFFFFFFFFFFFF, _p(cell), _p(theta), _p(v), _p(w))
    return State(cell, theta, v, w)


def electron_kinetic_energy(electrons: State, E, ncell, dx, dt, qm_e, kick):
    """The electrons' total kinetic energy sum w Vbar^2 dx / 2 at integer time (Vbar = v +
    (kick - 1/2) qm_e dt E(X)): the global active variable of Section 4.2's runs."""
    return moments(electrons, E, np.zeros(ncell), ncell, dx, dt, qm_e, kick, 0, mode=1)["kinetic"]


def lift_electron_temperature(we_proj, we_ref):
    """T_e / T_e0 at a lift from the projected electron kinetic energy we_proj and the energy
    we_ref of the same electrons at T_e0 (the initial load); the electrons' drift energy, a
    fraction (V_i / v_th_e)^2 of the thermal one, is counted in both."""
    return float(we_proj) / float(we_ref)


def boltzmann_electrons_te(N, ncell, n_ions, dx, T_e, v_th_e, seed, u=None, tol=1e-12):
    """Electrons of a lifting at temperature T_e (units of T_e0): the Poisson-Boltzmann potential
    with n_e = exp(phi / T_e), written for psi = phi / T_e as -T_e psi'' + e^psi = n (Newton at
    the grid step dx / sqrt(T_e)), then the quiet start on exp(psi) with thermal speed
    v_th_e sqrt(T_e). Returns (electrons, psi)."""
    psi, _, fail = newton_pb(n_ions, dx / np.sqrt(T_e), tol=tol)
    assert fail == 0
    return boltzmann_electrons(N, ncell, psi, v_th_e * np.sqrt(T_e), seed, u=u), psi


def ps_mean_velocity(cdf, vmin, dv, bin_shift, ncell):
    """Nodal mean ion velocity of a phase-space state: per x-bin the mean of its reconstructed
    CDF row over cell centres, then linear between bin midpoints (periodic)."""
    cdf = _f64(cdf)
    nxc, nv = cdf.shape[0], cdf.shape[1] - 1
    vc = vmin + (np.arange(nv) + 0.5) * dv
    ub = np.sum(vc * np.diff(cdf, axis=1), axis=1)
    B = 2 ** bin_shift
    t = (np.arange(ncell) - 0.5 * (B - 1)) / B
    b0 = np.floor(t)
    f = t - b0
    b0 = b0.astype(np.int64) % nxc
    return (1 - f) * ub[b0] + f * ub[(b0 + 1) % nxc]


# ------------------------------------------------------------------ adaptive macro step


def leap_curvature(samples, dt):
    """(qn, ||c_K||, noise) for coarse samples [(K+1), ncoef] at t_p = p dt: q the quadratic
    coefficient of the least-squares fit c ~ a + b t + q t^2 of each component (numpy.polyfit),
    var_q = (residual sum of squares / (K - 2)) / sum_p g_p^2 with g_p the quadratic basis
    orthogonal to {1, t} on the samples (the variance of the leading coefficient), and
    qn = sqrt(max(0, sum q^2 - sum var_q)), noise = sqrt(sum var_q)."""
    samples = _f64(samples)
    K = samples.shape[0] - 1
    t = np.arange(K + 1) * float(dt)
    coef, res, _, _, _ = np.polyfit(t, samples, 2, full=True)
    q = coef[0]
    tau = t - t.mean()
    g = tau * tau - np.mean(tau * tau)
    if K > 2:
        fit = np.polyval(coef, t[:, None]) if samples.ndim == 2 else np.polyval(coef, t)
        rss = np.sum((samples - fit) ** 2, axis=0)
        var = rss / (K - 2) / np.sum(g * g)
    else:
        var = np.zeros_like(q)
    qn = float(np.sqrt(max(0.0, np.sum(q * q) - np.sum(var))))
    return qn, float(np.sqrt(np.sum(samples[-1] ** 2))), float(np.sqrt(np.sum(var)))


def slope_noise(samples, dt):
    """Norm of the standard errors of the least-squares slopes of a burst's samples
    [(K+1), ncoef] at t_p = p dt: per component s^2 = (residual sum of squares of the quadratic
    fit) / (K - 2) and var(slope) = s^2 / sum_p (t_p - tbar)^2; returns sqrt(sum var). K >= 3."""
    samples = _f64(samples)
    K = samples.shape[0] - 1
    t = np.arange(K + 1) * float(dt)
    coef = np.polyfit(t, samples, 2)
    fit = np.polyval(coef, t[:, None]) if samples.ndim == 2 else np.polyval(coef, t)
    rss = np.sum((samples - fit) ** 2, axis=0)
    tau = t - t.mean()
    return float(np.sqrt(np.sum(rss / (K - 2) / np.sum(tau * tau))))


def burst_length_for_noise(sn, K, leap, cn, tol, K_min, K_max):
    """Smallest burst length K' in [K_min, K_max] whose slope noise, scaled from the measured
    sn at K by the least-squares variance law var ~ 1 / (K (K+1) (K+2)), moves a leap of the
    given length by at most tol relative to cn: leap sn sqrt(K(K+1)(K+2) / (K'(K'+1)(K'+2)))
    <= tol cn; K_max when none does."""
    if not (leap > 0 and sn > 0 and cn > 0):
        return int(K_min)
    base = float(K) * (K + 1) * (K + 2)
    for Kp in range(int(K_min), int(K_max) + 1):
        if leap * sn * np.sqrt(base / (float(Kp) * (Kp + 1) * (Kp + 2))) <= tol * cn:
            return Kp
    return int(K_max)


def leap_for_tol(qn, cn, Kdt, tol):
    """Leap L >= 0 with qn L (L + K dt) = tol cn (infinite without curvature)."""
    if not qn > 0:
        return float("inf")
    return 0.5 * (-Kdt + np.sqrt(Kdt * Kdt + 4.0 * tol * cn / qn))


# ------------------------------------------------------------------ ion pressure (Section 3.2)
# EFREE's active ion variables are n, V and P. The restriction adds the second velocity moment
# S = sum_p w V~^2 S_j(X~) to the density and momentum samples; the coarse state is the
# wavelet scaling coefficients of the three, [3][n_coarse]; the lift loads Maxwellians of the
# local temperature T = S / n - u^2.


def restrict_second_moment(st: State, vbar, E0, ncell, dx, tau, qm):
    vbar, E0 = _f64(vbar), _f64(E0)
    sec = np.zeros(ncell)
    _load().orc_restrict_second_moment(st.n, _p(st.cell), _p(st.theta), _p(vbar), _p(st.w), _p(E0), ncell,
                                       float(dx), float(tau), float(qm), _p(sec))
    return sec


def burst_pressure(st: State, ncell, dx, dt, qm, K, dT, s_w, phi, comoving=True, mode=0, tol=1e-11,
                   maxit=50, vel_at_integer=True):
    """Runs K steps in place on st; returns (samples [(K+1),3,ncell], phi, fails)."""
    phi = _f64(phi).copy()
    samples = np.zeros((K + 1, 3, ncell))
    fails = _load().orc_burst_pressure(st.n, _p(st.cell), _p(st.theta), _p(st.v), _p(st.w), ncell, float(dx),
                                       float(dt), float(qm), int(K), float(dT), int(comoving), int(mode),
                                       int(s_w), float(tol), int(maxit), int(vel_at_integer), _p(phi),
                                       _p(samples))
    return samples, phi, int(fails)


def lift_profile_pressure(n, m, s):
    """Returns (n clamped, u, T) of the lifting (orc_lift_profile_pressure)."""
    n = _f64(n).copy()
    m, s = _f64(m), _f64(s)
    u, T = np.zeros_like(n), np.zeros_like(n)
    _load().orc_lift_profile_pressure(n.shape[0], _p(n), _p(m), _p(s), _p(u), _p(T))
    return n, u, T


def quiet_start_thermal(N, ncell, nprof, uprof, tprof, seed):
    nprof, uprof, tprof = _f64(nprof), _f64(uprof), _f64(tprof)
    cell = np.zeros(N, np.int32)
    theta, v, w = np.zeros(N), np.zeros(N), np.zeros(N)
    _load().orc_quiet_start_thermal(N, ncell, _p(nprof), _p(uprof), _p(tprof), seed & 0xFFFFFFFFFFFFFFFF,
                                    _p(cell), _p(theta), _p(v), _p(w))
    return State(cell, theta, v, w)


def efpi_macro_step_pressure(st: State, cfg: dict, phi, vel_at_integer=True):
    """efpi_macro_step with the ion pressure active: burst with three-moment co-moving
    samples, coarsening of each, least-squares slope and leap. Returns (coarse [3,nc],
    samples_c [(K+1),3,nc], phi)."""
    ncell, nc, K = cfg["ncell"], cfg["n_coarse"], cfg["K"]
    dx = cfg["L"] / ncell
    samples, phi, fails = burst_pressure(st, ncell, dx, cfg["dt"], cfg["qm"], K, cfg["dT"], cfg["s_w"], phi,
                                         comoving=cfg.get("comoving", True), mode=cfg.get("mode", 0),
                                         vel_at_integer=vel_at_integer)
    wav = cfg.get("wavelet", "haar")
    cs = np.zeros((K + 1, 3, nc))
    for p in range(K + 1):
        for m in range(3):
            cs[p, m] = coarsen(samples[p, m], nc, wav)
    coarse, _ = ls_project(cs.reshape(K + 1, 3 * nc), cfg["dt"], cfg["dT"])
    return coarse.reshape(3, nc), cs, phi


def lift_pressure(coarse, cfg: dict, seed):
    """Lifting of the three moments: refine each with zero details, n clamped, u = nV / n,
    T = S / n - u^2 clamped at 0, quiet start at the local temperature."""
    ncell = cfg["ncell"]
    wav = cfg.get("wavelet", "haar")
    nf, mf, sf = (refine(coarse[k], ncell, wav) for k in range(3))
    nf, uf, Tf = lift_profile_pressure(nf, mf, sf)
    return quiet_start_thermal(cfg["N"], ncell, nf, uf, Tf, seed)
