"""ctypes binding of libpepic.so (C ABI in include/pepic.h).

Argument marshalling only: torch provides the device memory and the stream, every
step of the method runs in the CUDA library. There is no CPU fallback: if the
library is missing, or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libpepic.so")

PE_OK, PE_EINVAL, PE_ECUDA, PE_ENOCONV, PE_EOVERFLOW, PE_ERANGE, PE_ESTATE = range(7)
PE_WAVELET = {"haar": 0, "d4": 1, "coif4": 2}
PE_POISSON = {"boltzmann": 0, "linearized": 1}
PE_PROFILE_SINE = 0
PE_PROFILE_SLAB = 1
PE_BOUNDARY = {"periodic": 0, "absorbing": 1}
PE_NBUF = 20
# launch kinds of the context's kernel timing, in the order of PE_PROF_* (include/pepic.h)
PROFILE_KINDS = ("push_sample", "push", "sample", "deposit", "load", "push_sample_ps", "field")
BUF = dict(particles_a=0, particles_b=1, rho=2, phi=3, E=4, Ef=5, E0f=6, samples_fx=7, coarse_samples=8,
           coarse=9, slope=10, profile=11, sort=12, status=13, diag=14, surrogate=15, phase=16, electrons_a=17,
           electrons_b=18, rho_e=19)
PE_ELECTRONS = {"boltzmann": 0, "kinetic": 1}
PE_COARSE = {"moments": 0, "phase_space": 1, "moments_pressure": 2}
PE_MLP_NBUF = 7
MLP_BUF = dict(params=0, params_bf16=1, grads=2, adam_m=3, adam_v=4, norm=5, work=6)
PE_MOMENTS_SCRATCH_BYTES = 65536

_lock = threading.Lock()
_lib = None


class PepicError(RuntimeError):
    pass


class SampleArgs(ctypes.Structure):
    _fields_ = [("E0f", ctypes.c_void_p), ("tau", ctypes.c_float), ("qm", ctypes.c_float),
                ("inv_dx", ctypes.c_float), ("s_w", ctypes.c_int32), ("s_p", ctypes.c_int32),
                ("bin_shift", ctypes.c_int32), ("sample_fx", ctypes.c_void_p), ("n_v", ctypes.c_int32),
                ("v_min", ctypes.c_float), ("inv_dv", ctypes.c_float), ("boundary", ctypes.c_int32),
                ("x_tent", ctypes.c_int32), ("second_moment", ctypes.c_int32), ("s_e", ctypes.c_int32)]


class Config(ctypes.Structure):
    _fields_ = [("ncell", ctypes.c_int32), ("n_coarse", ctypes.c_int32), ("wavelet", ctypes.c_int32),
                ("K", ctypes.c_int32), ("nparticles", ctypes.c_int64), ("L", ctypes.c_double),
                ("dt", ctypes.c_double), ("dT", ctypes.c_double), ("qm", ctypes.c_double),
                ("v_th", ctypes.c_double), ("comoving", ctypes.c_int32), ("poisson", ctypes.c_int32),
                ("newton_tol", ctypes.c_double), ("newton_maxit", ctypes.c_int32), ("sort_every", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("w_cap", ctypes.c_double), ("v_cap", ctypes.c_double),
                ("coarse_kind", ctypes.c_int32), ("n_v", ctypes.c_int32), ("v_max", ctypes.c_double),
                ("ps_filter", ctypes.c_int32), ("boundary", ctypes.c_int32), ("electrons", ctypes.c_int32),
                ("reset_every", ctypes.c_int32), ("qm_e", ctypes.c_double), ("v_th_e", ctypes.c_double),
                ("n_v_coarse", ctypes.c_int32), ("te_active", ctypes.c_int32)]


class Layout(ctypes.Structure):
    _fields_ = [("total_bytes", ctypes.c_size_t), ("offset", ctypes.c_size_t * PE_NBUF),
                ("bytes", ctypes.c_size_t * PE_NBUF)]


class Diag(ctypes.Structure):
    _fields_ = [("macro_steps", ctypes.c_int64), ("fine_steps", ctypes.c_int64), ("time", ctypes.c_double),
                ("particle_bank", ctypes.c_int32), ("v_at_integer", ctypes.c_int32), ("s_w", ctypes.c_int32),
                ("s_p", ctypes.c_int32), ("newton_iters", ctypes.c_int32), ("status", ctypes.c_uint32),
                ("electron_bank", ctypes.c_int32), ("e_v_at_integer", ctypes.c_int32), ("T_e", ctypes.c_double),
                ("W_e", ctypes.c_double)]


class Moments(ctypes.Structure):
    _fields_ = [("charge_fx", ctypes.c_int64), ("invalid", ctypes.c_int64)] + [
        (k, ctypes.c_double) for k in ("charge_fixed_point", "charge", "momentum", "kinetic", "field_energy",
                                       "electron_energy", "total_energy", "max_speed", "cfl")] + [
        ("charge_wq", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MLPLayout(ctypes.Structure):
    _fields_ = [("total_bytes", ctypes.c_size_t), ("offset", ctypes.c_size_t * PE_MLP_NBUF),
                ("bytes", ctypes.c_size_t * PE_MLP_NBUF), ("nparams", ctypes.c_int64)]


class GateCfg(ctypes.Structure):
    _fields_ = [("K_probe", ctypes.c_int32), ("tol", ctypes.c_double), ("noise_sigmas", ctypes.c_double)]


class GateStats(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_int32), ("fine_steps", ctypes.c_int32), ("err", ctypes.c_double),
                ("floor", ctypes.c_double), ("norm", ctypes.c_double), ("sigma", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AdaptCfg(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("M_min", ctypes.c_int32), ("M_max", ctypes.c_int32),
                ("safety", ctypes.c_double), ("grow", ctypes.c_double), ("K_min", ctypes.c_int32),
                ("K_max", ctypes.c_int32), ("noise_frac", ctypes.c_double)]


class AdaptStats(ctypes.Structure):
    _fields_ = [("dT", ctypes.c_double), ("err", ctypes.c_double), ("dT_next", ctypes.c_double),
                ("rejected", ctypes.c_int32), ("fine_steps", ctypes.c_int32), ("noise", ctypes.c_double),
                ("K", ctypes.c_int32), ("K_next", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# exported symbol -> (restype, argtypes); the test-suite checks this against include/pepic.h
P, i32, i64, u64, f32, f64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                  ctypes.c_float, ctypes.c_double, ctypes.c_size_t)
SIGNATURES = {
    "pe_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "pe_version": (ctypes.c_char_p, []),
    "pe_deposit": (ctypes.c_int, [P, P, P, i64, i32, i32, P, P, P]),
    "pe_field": (ctypes.c_int, [P, i32, f64, i32, i32, f64, i32, P, P, P, P, P, P]),
    "pe_field_ex": (ctypes.c_int, [P, i32, f64, i32, i32, i32, f64, i32, P, P, P, P, P, P]),
    "pe_field_kinetic": (ctypes.c_int, [P, P, i32, f64, i32, P, P, P, P]),
    "pe_boltzmann_profile": (ctypes.c_int, [P, P, i32, i32, i32, P, P, P]),
    "pe_ps_mean_velocity": (ctypes.c_int, [P, i32, i32, f64, f64, i32, i32, P, P]),
    "pe_push": (ctypes.c_int, [P, P, P, P, i64, P, i32, f32, f32, f32, i32, P, ctypes.POINTER(SampleArgs), P, P]),
    "pe_push_ex": (ctypes.c_int, [P, P, P, P, i64, P, i32, f32, f32, f32, i32, i32, P, ctypes.POINTER(SampleArgs),
                                  P, P]),
    "pe_sample": (ctypes.c_int, [P, P, P, P, i64, P, i32, f32, f32, ctypes.POINTER(SampleArgs), P, P]),
    "pe_coarsen": (ctypes.c_int, [P, i32, i32, i32, i32, i32, i32, i32, P, P]),
    "pe_ls_project": (ctypes.c_int, [P, i32, i32, f64, f64, P, P, P]),
    "pe_refine": (ctypes.c_int, [P, i32, i32, i32, P, P, P]),
    "pe_quiet_start": (ctypes.c_int, [P, P, P, P, i64, i32, P, P, f32, u64, i32, P, P, P]),
    "pe_quiet_start_slice": (ctypes.c_int, [P, P, P, P, i64, i64, i64, i32, P, P, f32, u64, i32, P, P, P]),
    "pe_refine_f64": (ctypes.c_int, [P, i32, i32, i32, P, P, P]),
    "pe_push_f64": (ctypes.c_int, [P, P, P, P, i64, P, i32, f64, f64, f64, i32, P, P, f64, f64, i32, P, P, P]),
    "pe_sample_f64": (ctypes.c_int, [P, P, P, P, i64, P, i32, f64, f64, i32, P, f64, f64, i32, P, P, P]),
    "pe_quiet_start_f64": (ctypes.c_int, [P, P, P, P, i64, i32, P, P, f64, u64, i32, P, P, P]),
    "pe_fixed_point_shifts": (ctypes.c_int, [i64, i32, f64, f64, P, P]),
    "pe_second_moment_shift": (ctypes.c_int, [i64, i32, f64, f64, P]),
    "pe_coarsen_pressure": (ctypes.c_int, [P, i32, i32, i32, i32, i32, i32, i32, i32, P, P]),
    "pe_refine_pressure": (ctypes.c_int, [P, i32, i32, i32, P, P, P, P]),
    "pe_quiet_start_thermal": (ctypes.c_int, [P, P, P, P, i64, i32, P, P, P, u64, i32, P, P, P]),
    "pe_initial_profile": (ctypes.c_int, [i32, i32, f64, f64, P, P]),
    "pe_quiet_start_equal": (ctypes.c_int, [P, P, P, P, i64, i32, P, P, f32, f32, u64, i32, P, P, P, P]),
    "pe_sort": (ctypes.c_int, [P, P, P, P, i64, i32, P, P, P, P, P, P, P]),
    "pe_sort_noalloc": (ctypes.c_int, [P, P, P, P, i64, i32, P, P, P, P, P, P]),
    "pe_layout_for": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(Layout)]),
    "pe_create": (ctypes.c_int, [ctypes.POINTER(Config), P, sz, P, ctypes.POINTER(P)]),
    "pe_destroy": (None, [P]),
    "pe_load_initial": (ctypes.c_int, [P, i32, f64]),
    "pe_burst": (ctypes.c_int, [P]),
    "pe_restrict": (ctypes.c_int, [P]),
    "pe_project": (ctypes.c_int, [P]),
    "pe_lift": (ctypes.c_int, [P]),
    "pe_step": (ctypes.c_int, [P]),
    "pe_pic_steps": (ctypes.c_int, [P, i32]),
    "pe_measure": (ctypes.c_int, [P, P, i32]),
    "pe_get_coarse": (ctypes.c_int, [P, P, i32]),
    "pe_set_coarse": (ctypes.c_int, [P, P, i32]),
    "pe_sync_status": (ctypes.c_int, [P]),
    "pe_diagnostics": (ctypes.c_int, [P, ctypes.POINTER(Diag)]),
    "pe_profile": (ctypes.c_int, [P, i32]),
    "pe_profile_mask": (ctypes.c_int, [P, i32]),
    "pe_profile_read": (ctypes.c_int, [P, P, P, P, P]),
    "pe_profile_read_kinds": (ctypes.c_int, [P, P, P]),
    "pe_launch_count": (i64, []),
    "pe_compute_moments": (ctypes.c_int, [P, P, P, P, i64, P, P, P, i32, f64, f64, f32, f32, i32, i32, P, P, P, P]),
    "pe_rel_l2": (ctypes.c_int, [P, P, i64, P, P]),
    "pe_state_moments": (ctypes.c_int, [P, ctypes.POINTER(Moments), i32]),
    "pe_get_slope": (ctypes.c_int, [P, P, i32]),
    "pe_export_f32": (ctypes.c_int, [P, i32, P]),
    "pe_step_surrogate": (ctypes.c_int, [P, P, ctypes.POINTER(GateCfg), ctypes.POINTER(GateStats)]),
    "pe_leap_curvature": (ctypes.c_int, [P, i32, i32, f64, P, P, P]),
    "pe_step_adaptive": (ctypes.c_int, [P, ctypes.POINTER(AdaptCfg), ctypes.POINTER(AdaptStats)]),
    "pe_set_macro_step": (ctypes.c_int, [P, f64]),
    "pe_checkpoint_bytes": (ctypes.c_int, [P, ctypes.POINTER(sz)]),
    "pe_checkpoint_save": (ctypes.c_int, [P, P, sz]),
    "pe_checkpoint_restore": (ctypes.c_int, [P, P, sz]),
    "pe_gate": (ctypes.c_int, [P, i32, i32, f64, f64, P, f64, f64, P, P, P, P]),
    "pe_ps_coarsen": (ctypes.c_int, [P, i32, i64, i32, P, P]),
    "pe_ps_project": (ctypes.c_int, [P, i32, i32, i32, f64, f64, i32, P, P, P, P]),
    "pe_ps_lift_tables": (ctypes.c_int, [P, i32, i32, P, P, P, P, P, P]),
    "pe_ps_coarsen_v": (ctypes.c_int, [P, i64, i32, i32, i32, i32, i32, P, P]),
    "pe_tc_gemm_bf16": (ctypes.c_int, [P, i64, P, i64, P, i64, i32, i32, i32, P, P]),
    "pe_kinetic_energy": (ctypes.c_int, [P, P, P, P, i64, P, i32, f64, f32, f32, P, P, P, P]),
    "pe_ps_refine_v": (ctypes.c_int, [P, i64, i32, i32, i32, P, P]),
    "pe_ps_node_tables": (ctypes.c_int, [P, P, i32, i32, i32, P, P, P]),
    "pe_ps_quiet_start_nodes": (ctypes.c_int, [P, P, P, P, i64, i32, P, P, i32, f64, f64, u64, i32, P, P, P]),
    "pe_ps_quiet_start": (ctypes.c_int, [P, P, P, P, i64, i32, i32, P, P, i32, f64, f64, u64, i32, P, P, P]),
    "pe_ps_quiet_start_equal": (ctypes.c_int, [P, P, P, P, i64, i32, i32, P, P, i32, f64, f64, u64, i32, P, P, P,
                                               P]),
    "pe_mlp_layout_for": (ctypes.c_int, [i32, P, i32, ctypes.POINTER(MLPLayout)]),
    "pe_mlp_sync_status": (ctypes.c_int, [P]),
    "pe_mlp_create": (ctypes.c_int, [i32, P, i32, P, sz, P, ctypes.POINTER(P)]),
    "pe_mlp_destroy": (None, [P]),
    "pe_mlp_init": (ctypes.c_int, [P, u64]),
    "pe_mlp_fit_norm": (ctypes.c_int, [P, P, P, i64, i32]),
    "pe_mlp_forward": (ctypes.c_int, [P, P, i32, i32, P, i32]),
    "pe_mlp_grad": (ctypes.c_int, [P, P, P, i64, P, i32, P]),
    "pe_mlp_adam": (ctypes.c_int, [P, f64, f64, f64, f64]),
    "pe_mlp_train": (ctypes.c_int, [P, P, P, i64, i32, i32, u64, i32, f32, P]),
    "pe_mlp_set_params": (ctypes.c_int, [P, P]),
    "pe_mlp_info": (ctypes.c_int, [P, P, P, P, P]),
    "pe_batch_scratch_bytes": (ctypes.c_int, [P, i32, ctypes.POINTER(sz)]),
    "pe_batch_create": (ctypes.c_int, [P, i32, P, sz, P, ctypes.POINTER(P)]),
    "pe_batch_step": (ctypes.c_int, [P]),
    "pe_batch_tune": (ctypes.c_int, [P, ctypes.POINTER(i64)]),
    "pe_batch_tuned": (ctypes.c_int, [P, P, P, P]),
    "pe_batch_group_mean": (ctypes.c_int, [P, P, i32, P]),
    "pe_batch_destroy": (None, [P]),
}


def launch_count() -> int:
    return int(load().pe_launch_count())


def load(path: str = LIB_PATH):
    """Loads libpepic.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise PepicError(f"{path} is missing: build it with paper_1610_01071_gb300._build.build()")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(rc: int, what: str = ""):
    if rc != PE_OK:
        msg = load().pe_strerror(rc).decode()
        raise PepicError(f"{what}: {msg} (code {rc})")


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise PepicError("device tensor expected (the library has no CPU path)")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _status(status, dev):
    return status if status is not None else torch.zeros(1, dtype=torch.int32, device=dev)


# ------------------------------------------------------------------ stateless kernels


def deposit(cell, theta, w, ncell, s_w, rho=None, status=None, stream=None):
    dev = cell.device
    rho = rho if rho is not None else torch.empty(ncell, dtype=torch.int64, device=dev)
    status = _status(status, dev)
    check(load().pe_deposit(_ptr(cell), _ptr(theta), _ptr(w), cell.numel(), ncell, s_w, _ptr(rho), _ptr(status),
                            _stream(stream)), "pe_deposit")
    return rho


def field(rho, ncell, dx, s_w, phi, mode="boltzmann", tol=1e-11, maxit=50, status=None, stream=None,
          boundary="periodic"):
    dev = rho.device
    E = torch.empty(ncell, dtype=torch.float64, device=dev)
    Ef = torch.empty(ncell, dtype=torch.float32, device=dev)
    diag = torch.zeros(4, dtype=torch.int32, device=dev)
    status = _status(status, dev)
    if boundary == "periodic":
        check(load().pe_field(_ptr(rho), ncell, float(dx), s_w, PE_POISSON[mode], float(tol), int(maxit), _ptr(phi),
                              _ptr(E), _ptr(Ef), _ptr(diag), _ptr(status), _stream(stream)), "pe_field")
    else:
        check(load().pe_field_ex(_ptr(rho), ncell, float(dx), s_w, PE_POISSON[mode], PE_BOUNDARY[boundary],
                                 float(tol), int(maxit), _ptr(phi), _ptr(E), _ptr(Ef), _ptr(diag), _ptr(status),
                                 _stream(stream)), "pe_field_ex")
    return E, Ef, diag


def field_kinetic(rho_i, rho_e, ncell, dx, s_w, phi=None, stream=None):
    """Periodic Poisson field of the net charge of ions and electrons (both fixed-point
    deposits with positive weights); returns (phi, E, Ef)."""
    dev = rho_i.device
    phi = phi if phi is not None else torch.empty(ncell, dtype=torch.float64, device=dev)
    E = torch.empty(ncell, dtype=torch.float64, device=dev)
    Ef = torch.empty(ncell, dtype=torch.float32, device=dev)
    check(load().pe_field_kinetic(_ptr(rho_i), _ptr(rho_e), ncell, float(dx), int(s_w), _ptr(phi), _ptr(E), _ptr(Ef),
                                  _stream(stream)), "pe_field_kinetic")
    return phi, E, Ef


def ps_mean_velocity(cdf, v_min, dv, bin_shift, ncell, stream=None):
    """Nodal mean ion velocity (float32 [ncell]) of phase-space CDF rows cdf [nxc, n_v + 1]."""
    nxc, nv1 = cdf.shape
    u = torch.empty(ncell, dtype=torch.float32, device=cdf.device)
    check(load().pe_ps_mean_velocity(_ptr(cdf), nxc, nv1 - 1, float(v_min), float(dv), int(bin_shift), ncell, _ptr(u),
                                     _stream(stream)), "pe_ps_mean_velocity")
    return u


def leap_curvature(samples, dt, stream=None):
    """(noise-corrected ||q||, ||c_K||, noise of q, noise of the least-squares slope) of coarse
    samples [(K+1), ncoef] (pe_leap_curvature), as a device tensor."""
    K1, n = samples.shape
    out = torch.empty(4, dtype=torch.float64, device=samples.device)
    scratch = torch.empty(4 * 1024, dtype=torch.float64, device=samples.device)
    check(load().pe_leap_curvature(_ptr(samples), K1 - 1, n, float(dt), _ptr(scratch), _ptr(out), _stream(stream)),
          "pe_leap_curvature")
    return out


def boltzmann_profile(phi, ncell, ion_moments=None, s_w=0, s_p=0, stream=None):
    """Boltzmann electron profile: exp(phi) and the ions' mean velocity from their nodal moment
    sample ion_moments (int64 [2, ncell]; zero drift without it), float32 [2, ncell]."""
    prof = torch.empty(2 * ncell, dtype=torch.float32, device=phi.device)
    mom = _ptr(ion_moments) if ion_moments is not None else None
    check(load().pe_boltzmann_profile(_ptr(phi), mom, int(s_w), int(s_p), ncell, _ptr(prof), _ptr(prof[ncell:]),
                                      _stream(stream)), "pe_boltzmann_profile")
    return prof.view(2, ncell)


def make_sample_args(E0f, tau, qm, inv_dx, s_w, s_p, sample_fx, bin_shift=0, n_v=0, v_min=0.0, dv=1.0,
                     boundary="periodic", x_tent=False, s_e=None):
    """Restriction-sample arguments; n_v > 0 selects the phase-space sample (n_v velocity
    cells of width dv from v_min) instead of the density and momentum moments; x_tent rows
    are coarse nodes with the hat weights of the repeated 1-2-1 rule instead of Haar bins;
    s_e (not None) adds the second velocity moment as a third nodal row."""
    return SampleArgs(ctypes.c_void_p(E0f.data_ptr()), float(tau), float(qm), float(inv_dx), int(s_w), int(s_p),
                      int(bin_shift), ctypes.c_void_p(sample_fx.data_ptr()), int(n_v), float(v_min),
                      float(1.0 / dv), PE_BOUNDARY[boundary], int(bool(x_tent)), int(s_e is not None),
                      int(s_e or 0))


def push(cell, theta, v, w, Ef, ncell, dt_over_dx, qm_dt, kick, s_w, rho=None, sample=None, status=None,
         stream=None, boundary="periodic"):
    """Leapfrog push fused with the deposit (and the sample); boundary="absorbing" writes w of
    the absorbed particles."""
    dev = cell.device
    rho = rho if rho is not None else torch.empty(ncell, dtype=torch.int64, device=dev)
    status = _status(status, dev)
    sp = ctypes.byref(sample) if sample is not None else None
    if boundary == "periodic":
        check(load().pe_push(_ptr(cell), _ptr(theta), _ptr(v), _ptr(w), cell.numel(), _ptr(Ef), ncell,
                             float(dt_over_dx), float(qm_dt), float(kick), s_w, _ptr(rho), sp, _ptr(status),
                             _stream(stream)), "pe_push")
    else:
        check(load().pe_push_ex(_ptr(cell), _ptr(theta), _ptr(v), _ptr(w), cell.numel(), _ptr(Ef), ncell,
                                float(dt_over_dx), float(qm_dt), float(kick), s_w, PE_BOUNDARY[boundary], _ptr(rho),
                                sp, _ptr(status), _stream(stream)), "pe_push_ex")
    return rho


def sample(cell, theta, v, w, Ef, ncell, qm_dt, kick, args, status=None, stream=None):
    status = _status(status, cell.device)
    check(load().pe_sample(_ptr(cell), _ptr(theta), _ptr(v), _ptr(w), cell.numel(), _ptr(Ef), ncell, float(qm_dt),
                           float(kick), ctypes.byref(args), _ptr(status), _stream(stream)), "pe_sample")


def coarsen(sample_fx, nsamples, ncell, s_w, s_p, n_coarse, wavelet="haar", out=None, stream=None, bin_shift=0):
    out = out if out is not None else torch.empty((nsamples, 2, n_coarse), dtype=torch.float64,
                                                  device=sample_fx.device)
    check(load().pe_coarsen(_ptr(sample_fx), nsamples, ncell, s_w, s_p, PE_WAVELET[wavelet], n_coarse, bin_shift,
                            _ptr(out), _stream(stream)), "pe_coarsen")
    return out


def second_moment_shift(nparticles, ncell, w_cap=0.0, v_cap=0.0):
    s_e = ctypes.c_int32()
    check(load().pe_second_moment_shift(int(nparticles), int(ncell), float(w_cap), float(v_cap), ctypes.byref(s_e)),
          "pe_second_moment_shift")
    return s_e.value


def coarsen_pressure(sample_fx, nsamples, ncell, s_w, s_p, s_e, n_coarse, wavelet="haar", out=None, stream=None,
                     bin_shift=0):
    """Three moments [nsamples][3][ncell >> bin_shift] -> [nsamples][3][n_coarse] (pe_coarsen_pressure)."""
    out = out if out is not None else torch.empty((nsamples, 3, n_coarse), dtype=torch.float64,
                                                  device=sample_fx.device)
    check(load().pe_coarsen_pressure(_ptr(sample_fx), nsamples, ncell, s_w, s_p, s_e, PE_WAVELET[wavelet], n_coarse,
                                     int(bin_shift), _ptr(out), _stream(stream)), "pe_coarsen_pressure")
    return out


def refine_pressure(coarse, ncell, wavelet="haar", stream=None):
    """coarse: [3, n_coarse] float64. Returns float32 (n, u, T) profiles."""
    nc = coarse.shape[-1]
    prof = [torch.empty(ncell, dtype=torch.float32, device=coarse.device) for _ in range(3)]
    check(load().pe_refine_pressure(_ptr(coarse), nc, PE_WAVELET[wavelet], ncell, *[_ptr(p) for p in prof],
                                    _stream(stream)), "pe_refine_pressure")
    return tuple(prof)


def quiet_start_thermal(n, ncell, prof_n, prof_u, prof_T, seed, s_w, with_rho=True, status=None, stream=None):
    """pe_quiet_start at the local temperature prof_T (pe_quiet_start_thermal)."""
    dev = prof_n.device
    cell = torch.empty(n, dtype=torch.int32, device=dev)
    theta = torch.empty(n, dtype=torch.float32, device=dev)
    v = torch.empty_like(theta)
    w = torch.empty_like(theta)
    rho = torch.empty(ncell, dtype=torch.int64, device=dev) if with_rho else None
    status = _status(status, dev)
    check(load().pe_quiet_start_thermal(_ptr(cell), _ptr(theta), _ptr(v), _ptr(w), n, ncell, _ptr(prof_n),
                                        _ptr(prof_u), _ptr(prof_T), int(seed) & 0xFFFFFFFFFFFFFFFF, s_w, _ptr(rho),
                                        _ptr(status), _stream(stream)), "pe_quiet_start_thermal")
    return cell, theta, v, w, rho


def ls_project(samples, dt, dT, stream=None):
    """samples: [(K+1), ncoef] float64 on the device. Returns (out, slope)."""
    K, ncoef = samples.shape[0] - 1, samples.shape[1]
    out = torch.empty(ncoef, dtype=torch.float64, device=samples.device)
    slope = torch.empty_like(out)
    check(load().pe_ls_project(_ptr(samples), K, ncoef, float(dt), float(dT), _ptr(out), _ptr(slope),
                               _stream(stream)), "pe_ls_project")
    return out, slope


def refine(coarse, ncell, wavelet="haar", stream=None):
    """coarse: [2, n_coarse] float64. Returns float32 (n, u) profiles."""
    nc = coarse.shape[-1]
    prof_n = torch.empty(ncell, dtype=torch.float32, device=coarse.device)
    prof_u = torch.empty_like(prof_n)
    check(load().pe_refine(_ptr(coarse), nc, PE_WAVELET[wavelet], ncell, _ptr(prof_n), _ptr(prof_u),
                           _stream(stream)), "pe_refine")
    return prof_n, prof_u


def quiet_start(n, ncell, prof_n, prof_u, v_th, seed, s_w, with_rho=True, status=None, stream=None):
    dev = prof_n.device
    cell = torch.empty(n, dtype=torch.int32, device=dev)
    theta = torch.empty(n, dtype=torch.float32, device=dev)
    v = torch.empty_like(theta)
    w = torch.empty_like(theta)
    rho = torch.empty(ncell, dtype=torch.int64, device=dev) if with_rho else None
    status = _status(status, dev)
    check(load().pe_quiet_start(_ptr(cell), _ptr(theta), _ptr(v), _ptr(w), n, ncell, _ptr(prof_n), _ptr(prof_u),
                                float(v_th), int(seed) & 0xFFFFFFFFFFFFFFFF, s_w, _ptr(rho), _ptr(status),
                                _stream(stream)), "pe_quiet_start")
    return cell, theta, v, w, rho


def quiet_start_equal(n, ncell, prof_n, prof_u, v_th, seed, s_w, wall_factor=1.0, with_rho=True, status=None,
                      stream=None):
    """Equal-weight loading of a bounded grid (pe_quiet_start_equal)."""
    dev = prof_n.device
    cell = torch.empty(n, dtype=torch.int32, device=dev)
    theta = torch.empty(n, dtype=torch.float32, device=dev)
    v = torch.empty_like(theta)
    w = torch.empty_like(theta)
    rho = torch.empty(ncell, dtype=torch.int64, device=dev) if with_rho else None
    scratch = torch.empty((16 * ncell + 16 + 15) // 8, dtype=torch.float64, device=dev)
    status = _status(status, dev)
    check(load().pe_quiet_start_equal(_ptr(cell), _ptr(theta), _ptr(v), _ptr(w), n, ncell, _ptr(prof_n),
                                      _ptr(prof_u), float(wall_factor), float(v_th), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                      s_w, _ptr(scratch), _ptr(rho), _ptr(status), _stream(stream)),
          "pe_quiet_start_equal")
    return cell, theta, v, w, rho


def sort(cell, theta, v, w, ncell, status=None, stream=None):
    dev = cell.device
    oc, ot, ov, ow = torch.empty_like(cell), torch.empty_like(theta), torch.empty_like(v), torch.empty_like(w)
    scratch = torch.empty(2 * ncell + 64, dtype=torch.int32, device=dev)
    status = _status(status, dev)
    check(load().pe_sort(_ptr(cell), _ptr(theta), _ptr(v), _ptr(w), cell.numel(), ncell, _ptr(oc), _ptr(ot),
                         _ptr(ov), _ptr(ow), _ptr(scratch), _ptr(status), _stream(stream)), "pe_sort")
    return oc, ot, ov, ow


def sort_noalloc(cell, theta, v, w, ncell, status=None, stream=None, out=None):
    """pe_sort without a scratch argument: its counters live in the library's static
    device array (for callers that cannot allocate device memory when they sort). With
    `out` = (cell, theta, v, w) and `status` given, this wrapper allocates nothing either.
    The call runs with the particles' device current, on `stream` or that device's current
    stream."""
    dev = cell.device
    with torch.cuda.device(dev):
        if out is None:
            out = (torch.empty_like(cell), torch.empty_like(theta), torch.empty_like(v), torch.empty_like(w))
        oc, ot, ov, ow = out
        status = _status(status, dev)
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        check(load().pe_sort_noalloc(_ptr(cell), _ptr(theta), _ptr(v), _ptr(w), cell.numel(), ncell, _ptr(oc),
                                     _ptr(ot), _ptr(ov), _ptr(ow), _ptr(status), _stream(s)), "pe_sort_noalloc")
    return oc, ot, ov, ow


def compute_moments(cell, theta, v, w, Ef, ncell, dx, dt, qm_dt, kick, s_w, phi=None, E=None, mode="boltzmann",
                    status=None, stream=None) -> dict:
    """Conserved quantities and Courant number of a particle state (pe_compute_moments)."""
    dev = cell.device
    scratch = torch.empty(PE_MOMENTS_SCRATCH_BYTES // 8, dtype=torch.float64, device=dev)
    out = torch.empty(ctypes.sizeof(Moments) // 8, dtype=torch.float64, device=dev)
    status = _status(status, dev)
    check(load().pe_compute_moments(_ptr(cell), _ptr(theta), _ptr(v), _ptr(w), cell.numel(), _ptr(Ef), _ptr(phi),
                                    _ptr(E), ncell, float(dx), float(dt), float(qm_dt), float(kick), int(s_w),
                                    PE_POISSON[mode], _ptr(scratch), _ptr(out), _ptr(status), _stream(stream)),
          "pe_compute_moments")
    m = Moments.from_buffer_copy(out.cpu().numpy().tobytes())
    return m.as_dict()


def rel_l2(a, b, stream=None) -> float:
    """Section 4.1.1 error measure of two device FP64 vectors (pe_rel_l2)."""
    a, b = a.contiguous(), b.contiguous()
    assert a.dtype == torch.float64 and b.dtype == torch.float64 and a.numel() == b.numel()
    out = torch.empty(1, dtype=torch.float64, device=a.device)
    check(load().pe_rel_l2(_ptr(a), _ptr(b), a.numel(), _ptr(out), _stream(stream)), "pe_rel_l2")
    return float(out.item())


def ps_coarsen(sample_fx, s_w, stream=None):
    """Fixed-point phase-space samples (int64 [..., nxc, nv]) -> FP64 masses."""
    out = torch.empty(sample_fx.shape, dtype=torch.float64, device=sample_fx.device)
    nrow = sample_fx.shape[0] if sample_fx.dim() == 3 else 1
    ncoef = sample_fx.numel() // nrow
    check(load().pe_ps_coarsen(_ptr(sample_fx), nrow, ncoef, int(s_w), _ptr(out), _stream(stream)), "pe_ps_coarsen")
    return out


def ps_lift_tables(H, stream=None):
    """H [nxc, nv] FP64 (device) -> (mass [nxc], cdf [nxc, nv+1] FP64, sampling table
    [nxc, 3 nv + 1] FP32, flag)."""
    H = H.contiguous()
    nxc, nv = H.shape
    mass = torch.empty(nxc, dtype=torch.float64, device=H.device)
    cdf = torch.empty((nxc, nv + 1), dtype=torch.float64, device=H.device)
    table = torch.empty((nxc, 3 * nv + 1), dtype=torch.float32, device=H.device)
    scratch = torch.empty(2 * nxc * (nv + 1), dtype=torch.float64, device=H.device)
    flags = torch.zeros(1, dtype=torch.int32, device=H.device)
    check(load().pe_ps_lift_tables(_ptr(H), nxc, nv, _ptr(mass), _ptr(cdf), _ptr(table), _ptr(scratch), _ptr(flags),
                                   _stream(stream)), "pe_ps_lift_tables")
    return mass, cdf, table, int(flags.item())


def ps_quiet_start(n, ncell, bin_shift, mass, table, v_min, dv, seed, s_w, with_rho=True, status=None, stream=None):
    """Phase-space quiet start on the FP64 masses and the FP32 sampling table of ps_lift_tables."""
    dev = mass.device
    cell = torch.empty(n, dtype=torch.int32, device=dev)
    theta = torch.empty(n, dtype=torch.float32, device=dev)
    v = torch.empty_like(theta)
    w = torch.empty_like(theta)
    rho = torch.empty(ncell, dtype=torch.int64, device=dev) if with_rho else None
    status = _status(status, dev)
    check(load().pe_ps_quiet_start(_ptr(cell), _ptr(theta), _ptr(v), _ptr(w), n, ncell, int(bin_shift), _ptr(mass),
                                   _ptr(table), (table.shape[1] - 1) // 3, float(v_min), float(dv),
                                   int(seed) & 0xFFFFFFFFFFFFFFFF, int(s_w), _ptr(rho), _ptr(status),
                                   _stream(stream)), "pe_ps_quiet_start")
    return cell, theta, v, w, rho


def ps_coarsen_v(sample_fx, s_w, bin_shift, n_vc, wavelet="coif4", stream=None):
    """Hat rows of fixed-point phase-space samples (int64 [..., nxc, n_vf]) -> coarse
    coefficients (FP64 [..., nxc, n_vc]): pe_ps_coarsen_v."""
    n_vf = sample_fx.shape[-1]
    nrows = sample_fx.numel() // n_vf
    out = torch.empty(sample_fx.shape[:-1] + (n_vc,), dtype=torch.float64, device=sample_fx.device)
    check(load().pe_ps_coarsen_v(_ptr(sample_fx), nrows, n_vf, int(s_w), int(bin_shift), PE_WAVELET[wavelet], n_vc,
                                 _ptr(out), _stream(stream)), "pe_ps_coarsen_v")
    return out


def ps_refine_v(coarse, n_vf, wavelet="coif4", stream=None):
    """Coarse coefficients (FP64 [..., n_vc]) -> fine velocity histograms (FP64 [..., n_vf])."""
    coarse = coarse.contiguous()
    n_vc = coarse.shape[-1]
    nrows = coarse.numel() // n_vc
    out = torch.empty(coarse.shape[:-1] + (n_vf,), dtype=torch.float64, device=coarse.device)
    check(load().pe_ps_refine_v(_ptr(coarse), nrows, n_vc, PE_WAVELET[wavelet], n_vf, _ptr(out), _stream(stream)),
          "pe_ps_refine_v")
    return out


def ps_node_tables(mass, cdf, ncell, stream=None):
    """Fine-node sampling tables (FP32 [ncell, 3 n_v + 1]) and densities (FP32 [ncell]) of the
    coarse-node tables of ps_lift_tables (pe_ps_node_tables)."""
    nxc, nv = cdf.shape[0], cdf.shape[1] - 1
    table = torch.empty((ncell, 3 * nv + 1), dtype=torch.float32, device=mass.device)
    dens = torch.empty(ncell, dtype=torch.float32, device=mass.device)
    check(load().pe_ps_node_tables(_ptr(mass), _ptr(cdf), nxc, ncell, nv, _ptr(table), _ptr(dens), _stream(stream)),
          "pe_ps_node_tables")
    return table, dens


def ps_quiet_start_nodes(n, ncell, table, dens, v_min, dv, seed, s_w, with_rho=True, status=None, stream=None):
    """Wavelet-form quiet start on fine-node tables (pe_ps_quiet_start_nodes)."""
    dev = table.device
    cell = torch.empty(n, dtype=torch.int32, device=dev)
    theta = torch.empty(n, dtype=torch.float32, device=dev)
    v = torch.empty_like(theta)
    w = torch.empty_like(theta)
    rho = torch.empty(ncell, dtype=torch.int64, device=dev) if with_rho else None
    status = _status(status, dev)
    check(load().pe_ps_quiet_start_nodes(_ptr(cell), _ptr(theta), _ptr(v), _ptr(w), n, ncell, _ptr(table), _ptr(dens),
                                         (table.shape[1] - 1) // 3, float(v_min), float(dv),
                                         int(seed) & 0xFFFFFFFFFFFFFFFF, int(s_w), _ptr(rho), _ptr(status),
                                         _stream(stream)), "pe_ps_quiet_start_nodes")
    return cell, theta, v, w, rho


def tc_gemm(A, B, status=None, stream=None):
    """C = A B^T (FP32) for BF16 A [M, K] and B [N, K] on the tensor cores (pe_tc_gemm_bf16)."""
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16 and A.shape[1] == B.shape[1]
    A, B = A.contiguous(), B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    status = _status(status, A.device)
    check(load().pe_tc_gemm_bf16(_ptr(A), K, _ptr(B), K, _ptr(C), N, M, N, K, _ptr(status), _stream(stream)),
          "pe_tc_gemm_bf16")
    return C, status


def ps_project(samples, dt, dT, filt=0, stream=None):
    """Filtered phase-space projective step (pe_ps_project) of samples [(K+1), nxc, n_v] (FP64,
    device); returns (out, filtered slope), each [nxc, n_v]."""
    K, nxc, nv = samples.shape[0] - 1, samples.shape[1], samples.shape[2]
    out = torch.empty((nxc, nv), dtype=torch.float64, device=samples.device)
    slope, work = torch.empty_like(out), torch.empty_like(out)
    check(load().pe_ps_project(_ptr(samples), K, nxc, nv, float(dt), float(dT), int(filt), _ptr(work), _ptr(out),
                               _ptr(slope), _stream(stream)), "pe_ps_project")
    return out, slope


def ps_quiet_start_equal(n, ncell, bin_shift, mass, table, v_min, dv, seed, s_w, with_rho=True, status=None,
                         stream=None):
    """Phase-space loading of a bounded grid with equal weights (pe_ps_quiet_start_equal)."""
    dev = mass.device
    cell = torch.empty(n, dtype=torch.int32, device=dev)
    theta = torch.empty(n, dtype=torch.float32, device=dev)
    v = torch.empty_like(theta)
    w = torch.empty_like(theta)
    rho = torch.empty(ncell, dtype=torch.int64, device=dev) if with_rho else None
    scratch = torch.empty((28 * ncell + 64 + 7) // 8, dtype=torch.float64, device=dev)
    status = _status(status, dev)
    check(load().pe_ps_quiet_start_equal(_ptr(cell), _ptr(theta), _ptr(v), _ptr(w), n, ncell, int(bin_shift),
                                         _ptr(mass), _ptr(table), (table.shape[1] - 1) // 3, float(v_min), float(dv),
                                         int(seed) & 0xFFFFFFFFFFFFFFFF, int(s_w), _ptr(scratch), _ptr(rho),
                                         _ptr(status), _stream(stream)), "pe_ps_quiet_start_equal")
    return cell, theta, v, w, rho


# ------------------------------------------------------------------ context


def make_config(ncell, n_coarse, K, nparticles, L, dt, dT, qm=1.0, v_th=1.0, wavelet="haar", comoving=True,
                poisson="boltzmann", newton_tol=1e-10, newton_maxit=50, sort_every=0, seed=0, w_cap=0.0,
                v_cap=0.0, coarse="moments", n_v=64, v_max=8.0, ps_filter=0, boundary="periodic",
                electrons="boltzmann", reset_every=0, qm_e=0.0, v_th_e=0.0, n_v_coarse=0, te_active=False) -> Config:
    """coarse="moments": density and momentum coefficients (2 n_coarse); "moments_pressure": those and
    the second velocity moment's (3 n_coarse; the ion pressure of Section 3.2 active); "phase_space": the
    masses of n_coarse x n_v phase-space cells over velocities [-v_max, v_max); ps_filter: 1-2-1
    filter of the projected phase-space slope (bit 0 along v, bit 1 along x); boundary:
    "periodic" or "absorbing" (walls at nodes 0 and ncell-1, Section 4.2); electrons:
    "boltzmann" (fluid) or "kinetic" (particles of charge-to-mass ratio qm_e, default -1800,
    thermal speed v_th_e, default sqrt(-qm_e); plain PIC reloads them in Boltzmann equilibrium
    every reset_every steps if > 0); n_v_coarse > 0 selects the wavelet form of the phase-space
    variable (Section 3.3 as stated: coarse nodes by the 1-2-1 rule in x, n_v fine velocity
    cells reduced by the DWT of `wavelet` to n_v_coarse coefficients)."""
    return Config(int(ncell), int(n_coarse), PE_WAVELET[wavelet], int(K), int(nparticles), float(L), float(dt),
                  float(dT), float(qm), float(v_th), int(bool(comoving)), PE_POISSON[poisson], float(newton_tol),
                  int(newton_maxit), int(sort_every), int(seed) & 0xFFFFFFFFFFFFFFFF, float(w_cap), float(v_cap),
                  PE_COARSE[coarse], int(n_v), float(v_max), int(ps_filter), PE_BOUNDARY[boundary],
                  PE_ELECTRONS[electrons], int(reset_every), float(qm_e), float(v_th_e), int(n_v_coarse),
                  int(bool(te_active)))


def layout(cfg: Config) -> Layout:
    lay = Layout()
    check(load().pe_layout_for(ctypes.byref(cfg), ctypes.byref(lay)), "pe_layout_for")
    return lay


class Context:
    """One realisation: a caller-owned device arena (torch) bound to a pe_ctx."""

    def __init__(self, cfg: Config, device="cuda", stream=None):
        self.cfg = cfg
        self.lay = layout(cfg)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.arena = torch.empty(self.lay.total_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self.arena.data_ptr()
        self._pad = (-base) % 256
        self._h = ctypes.c_void_p()
        check(load().pe_create(ctypes.byref(cfg), ctypes.c_void_p(base + self._pad), self.lay.total_bytes,
                               _stream(self.stream), ctypes.byref(self._h)), "pe_create")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.pe_destroy(h)
            self._h = None

    def _call(self, name, *args):
        check(getattr(load(), name)(self._h, *args), name)

    # -- cycle
    def load_initial(self, amplitude=0.0, profile="sine"):
        """profile "sine" (amplitude of the Section 4.1 wave) or "slab" (Section 4.2, bounded grids)."""
        self._call("pe_load_initial", PE_PROFILE_SLAB if profile == "slab" else PE_PROFILE_SINE, float(amplitude))

    def burst(self):
        self._call("pe_burst")

    def restrict(self):
        self._call("pe_restrict")

    def project(self):
        self._call("pe_project")

    def lift(self):
        self._call("pe_lift")

    def step(self):
        self._call("pe_step")

    def pic_steps(self, nsteps):
        self._call("pe_pic_steps", int(nsteps))

    def measure(self, out=None):
        out = out if out is not None else torch.empty((2, self.cfg.n_coarse), dtype=torch.float64,
                                                      device=self.device)
        self._call("pe_measure", _ptr(out), 1)
        return out

    def coarse_shape(self):
        """(2, n_coarse) for the moments, (n_coarse, n_v) for the phase-space cells."""
        if self.cfg.coarse_kind == PE_COARSE["phase_space"]:
            return (self.cfg.n_coarse, self.cfg.n_v_coarse if self.cfg.n_v_coarse > 0 else self.cfg.n_v)
        if self.cfg.coarse_kind == PE_COARSE["moments_pressure"]:
            return (3, self.cfg.n_coarse)
        return (2, self.cfg.n_coarse)

    def get_coarse(self):
        out = torch.empty(self.coarse_shape(), dtype=torch.float64, device=self.device)
        self._call("pe_get_coarse", _ptr(out), 1)
        return out

    def set_coarse(self, coarse):
        c = coarse.to(self.device, torch.float64).contiguous()
        self._call("pe_set_coarse", _ptr(c), 1)

    def get_coarse_host(self, out):
        """Copies the coarse state into a (pinned) host tensor [2, n_coarse] through the C ABI."""
        assert out.device.type == "cpu" and out.dtype == torch.float64 and out.is_contiguous()
        check(load().pe_get_coarse(self._h, ctypes.c_void_p(out.data_ptr()), 0), "pe_get_coarse")
        return out

    def set_coarse_host(self, src):
        assert src.device.type == "cpu" and src.dtype == torch.float64 and src.is_contiguous()
        check(load().pe_set_coarse(self._h, ctypes.c_void_p(src.data_ptr()), 0), "pe_set_coarse")

    def sync_status(self):
        return load().pe_sync_status(self._h)

    def get_slope(self):
        out = torch.empty(self.coarse_shape(), dtype=torch.float64, device=self.device)
        self._call("pe_get_slope", _ptr(out), 1)
        return out

    def export_f32(self, what, out):
        """FP32 copy of the coarse state (what=0) or last slope (what=1) into out[2 n_coarse] (device)."""
        assert out.dtype == torch.float32 and out.is_contiguous()
        assert out.numel() == self.coarse_shape()[0] * self.coarse_shape()[1]
        self._call("pe_export_f32", int(what), _ptr(out))

    def step_surrogate(self, net, K_probe=5, tol=1e-2, noise_sigmas=3.0) -> dict:
        """Gated surrogate macro step (pe_step_surrogate); returns the gate statistics."""
        g = GateCfg(int(K_probe), float(tol), float(noise_sigmas))
        st = GateStats()
        self._call("pe_step_surrogate", net._h, ctypes.byref(g), ctypes.byref(st))
        return st.as_dict()

    def step_adaptive(self, tol=1e-4, M_min=1, M_max=16, safety=0.8, grow=2.0, K_min=0, K_max=0,
                      noise_frac=0.5) -> dict:
        """Macro step with the curvature-controlled Delta t (pe_step_adaptive) and, with K_max > 0,
        the noise-controlled burst length; returns its statistics."""
        a = AdaptCfg(float(tol), int(M_min), int(M_max), float(safety), float(grow), int(K_min), int(K_max),
                     float(noise_frac))
        st = AdaptStats()
        self._call("pe_step_adaptive", ctypes.byref(a), ctypes.byref(st))
        return st.as_dict()

    def checkpoint(self) -> bytes:
        """Checkpoint image (bytes) of the context between macro steps (pe_checkpoint_save)."""
        n = ctypes.c_size_t()
        self._call("pe_checkpoint_bytes", ctypes.byref(n))
        buf = ctypes.create_string_buffer(n.value)
        self._call("pe_checkpoint_save", buf, n.value)
        return buf.raw

    def restore(self, image: bytes):
        """Resume from a checkpoint image of a context of the same configuration."""
        buf = ctypes.create_string_buffer(bytes(image), len(image))
        self._call("pe_checkpoint_restore", buf, len(image))

    def set_macro_step(self, dT):
        """Delta t of the next macro steps (>= K dt)."""
        self._call("pe_set_macro_step", float(dT))

    def moments(self) -> dict:
        """Charge, momentum, energies and Courant number of the current particles (pe_state_moments)."""
        m = Moments()
        check(load().pe_state_moments(self._h, ctypes.byref(m), 0), "pe_state_moments")
        return m.as_dict()

    def diagnostics(self) -> Diag:
        d = Diag()
        check(load().pe_diagnostics(self._h, ctypes.byref(d)), "pe_diagnostics")
        return d

    def profile(self, enable=True, kinds=None):
        """Time every launch kind (enable), or only the named kinds (PROFILE_KINDS names)."""
        if kinds is None:
            self._call("pe_profile", int(bool(enable)))
        else:
            mask = 0
            for k in kinds:
                mask |= 1 << PROFILE_KINDS.index(k)
            self._call("pe_profile_mask", mask if enable else 0)

    def profile_read(self):
        """Summed event time (ms) and launch counts of particle kernels and field solves."""
        pm, pl, fm, fl = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int64()
        check(load().pe_profile_read(self._h, ctypes.byref(pm), ctypes.byref(pl), ctypes.byref(fm),
                                     ctypes.byref(fl)), "pe_profile_read")
        return dict(push_ms=pm.value, push_launches=pl.value, field_ms=fm.value, field_launches=fl.value)

    def profile_read_kinds(self):
        """Summed event time (ms) and launch count per launch kind (PROFILE_KINDS), then reset."""
        ms = (ctypes.c_double * len(PROFILE_KINDS))()
        n = (ctypes.c_int64 * len(PROFILE_KINDS))()
        check(load().pe_profile_read_kinds(self._h, ms, n), "pe_profile_read_kinds")
        return {k: dict(ms=ms[i], launches=n[i]) for i, k in enumerate(PROFILE_KINDS)}

    # -- typed views into the arena (for tests and inspection)
    def view(self, buf: str, dtype, count=None):
        i = BUF[buf]
        off = self._pad + self.lay.offset[i]
        nbytes = self.lay.bytes[i]
        t = self.arena[off:off + nbytes].view(dtype)
        return t if count is None else t[:count]

    def particles(self, bank=None, species="ions"):
        """(cell, theta, v, w) views of the current (or given) particle bank of the ions, or
        of the kinetic electrons (species="electrons")."""
        d = self.diagnostics() if bank is None else None
        if species == "electrons":
            if bank is None:
                bank = d.electron_bank
            first = BUF["electrons_a"]
        else:
            if bank is None:
                bank = d.particle_bank
            first = BUF["particles_a"]
        N = self.cfg.nparticles
        stride = ((4 * N + 255) // 256) * 256
        off = self._pad + self.lay.offset[first + bank]
        seg = [self.arena[off + k * stride: off + k * stride + 4 * N] for k in range(4)]
        return (seg[0].view(torch.int32), seg[1].view(torch.float32), seg[2].view(torch.float32),
                seg[3].view(torch.float32))


class Batch:
    """Ensemble of Context objects advanced together (pe_batch_*)."""

    def __init__(self, contexts, stream=None):
        self.contexts = list(contexts)
        dev = self.contexts[0].device
        # a created stream (the legacy default stream cannot be captured into a graph)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        self._arr = arr
        nbytes = ctypes.c_size_t()
        check(load().pe_batch_scratch_bytes(arr, len(self.contexts), ctypes.byref(nbytes)), "pe_batch_scratch_bytes")
        self.scratch = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=dev)
        base = self.scratch.data_ptr()
        pad = (-base) % 256
        self._h = ctypes.c_void_p()
        check(load().pe_batch_create(arr, len(self.contexts), ctypes.c_void_p(base + pad), nbytes.value,
                                     _stream(self.stream), ctypes.byref(self._h)), "pe_batch_create")

    def step(self):
        check(load().pe_batch_step(self._h), "pe_batch_step")

    def tune(self):
        chunk = ctypes.c_int64()
        check(load().pe_batch_tune(self._h, ctypes.byref(chunk)), "pe_batch_tune")
        return chunk.value

    def tuned(self) -> dict:
        """The particle launch shape in use: chunk, threads per block, shared-memory deposit window."""
        chunk, block, priv = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        check(load().pe_batch_tuned(self._h, ctypes.byref(chunk), ctypes.byref(block), ctypes.byref(priv)),
              "pe_batch_tuned")
        return dict(chunk=chunk.value, block=block.value, privatised=bool(priv.value))

    def group_mean(self, members, out=None):
        """Mean coarse state [2, n_coarse] of the realisations `members` (indices into the batch)."""
        nc = self.contexts[members[0]].cfg.n_coarse
        out = out if out is not None else torch.empty((2, nc), dtype=torch.float64, device=self.contexts[0].device)
        idx = (ctypes.c_int32 * len(members))(*members)
        check(load().pe_batch_group_mean(self._h, idx, len(members), _ptr(out)), "pe_batch_group_mean")
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.pe_batch_destroy(h)
            self._h = None


# ------------------------------------------------------------------ learned surrogate


def gate(samples, dt, dT, s_mlp, coarse, slope, tol=1e-2, noise_sigmas=3.0, stream=None) -> dict:
    """pe_gate on device tensors: samples [(Ks+1)][n], s_mlp [n]; coarse, slope [n] updated on
    acceptance. Returns the decision and statistics."""
    Ks, n = samples.shape[0] - 1, samples.shape[1]
    res = torch.zeros(5, dtype=torch.float64, device=samples.device)
    check(load().pe_gate(_ptr(samples), Ks, n, float(dt), float(dT), _ptr(s_mlp), float(tol), float(noise_sigmas),
                         _ptr(coarse), _ptr(slope), _ptr(res), _stream(stream)), "pe_gate")
    r = res.cpu().numpy()
    return dict(err=float(r[0]), floor=float(r[1]), norm=float(r[2]), sigma=float(r[3]),
                accepted=int(r[4:5].view("int32")[0]))


class MLP:
    """The surrogate network (pe_mlp) in a caller-owned device arena (torch)."""

    def __init__(self, dims, max_batch=256, device="cuda", stream=None):
        self.dims = [int(d) for d in dims]
        self.L = len(self.dims) - 1
        self.max_batch = int(max_batch)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._dims_c = (ctypes.c_int32 * (self.L + 1))(*self.dims)
        self.lay = MLPLayout()
        check(load().pe_mlp_layout_for(self.L, self._dims_c, self.max_batch, ctypes.byref(self.lay)),
              "pe_mlp_layout_for")
        self.nparams = int(self.lay.nparams)
        self.arena = torch.empty(self.lay.total_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self.arena.data_ptr()
        self._pad = (-base) % 256
        self._h = ctypes.c_void_p()
        check(load().pe_mlp_create(self.L, self._dims_c, self.max_batch, ctypes.c_void_p(base + self._pad),
                                   self.lay.total_bytes, _stream(self.stream), ctypes.byref(self._h)),
              "pe_mlp_create")
        self.loss_dev = torch.zeros(1, dtype=torch.float32, device=self.device)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.pe_mlp_destroy(h)
            self._h = None

    def _view(self, buf, dtype, count):
        off = self._pad + self.lay.offset[MLP_BUF[buf]]
        esz = torch.tensor([], dtype=dtype).element_size()
        return self.arena[off:off + count * esz].view(dtype)

    def params(self):
        return self._view("params", torch.float32, self.nparams)

    def params_bf16(self):
        return self._view("params_bf16", torch.bfloat16, self.nparams)

    def params_bf16_transposed(self):
        """The per-layer transposes of the BF16 weights (W_l^T at W_l's offset; biases unused)."""
        return self._view("params_bf16", torch.bfloat16, 2 * self.nparams)[self.nparams:]

    def grads(self):
        return self._view("grads", torch.float32, self.nparams)

    def adam_state(self):
        return self._view("adam_m", torch.float32, self.nparams), self._view("adam_v", torch.float32, self.nparams)

    def norm(self):
        """[4][dmax] FP32: mu_in, sd_in, mu_out, sd_out."""
        dmax = max(self.dims)
        return self._view("norm", torch.float32, 4 * dmax).view(4, dmax)

    def init(self, seed):
        torch.cuda.synchronize(self.device)
        check(load().pe_mlp_init(self._h, int(seed) & 0xFFFFFFFFFFFFFFFF), "pe_mlp_init")

    def set_params(self, flat):
        src = flat.to(self.device).contiguous()
        assert src.dtype == torch.float32 and src.numel() == self.nparams
        check(load().pe_mlp_set_params(self._h, _ptr(src)), "pe_mlp_set_params")
        self.stream.synchronize()

    def fit_norm(self, X, Y, period=0):
        assert X.dtype == torch.float32 and Y.dtype == torch.float32 and X.shape[0] == Y.shape[0]
        check(load().pe_mlp_fit_norm(self._h, _ptr(X), _ptr(Y), X.shape[0], int(period)), "pe_mlp_fit_norm")
        self.stream.synchronize()

    def forward(self, x):
        """x [B][d0] FP32 or FP64 on the device -> y [B][dL] of the same dtype (de-normalised)."""
        x = x.contiguous()
        is64 = x.dtype == torch.float64
        y = torch.empty((x.shape[0], self.dims[-1]), dtype=x.dtype, device=self.device)
        check(load().pe_mlp_forward(self._h, _ptr(x), int(is64), x.shape[0], _ptr(y), int(is64)), "pe_mlp_forward")
        self.stream.synchronize()
        return y

    def grad(self, X, Y, rows=None, B=None) -> float:
        B = int(B if B is not None else (rows.numel() if rows is not None else X.shape[0]))
        check(load().pe_mlp_grad(self._h, _ptr(X), _ptr(Y), X.shape[0], _ptr(rows), B, _ptr(self.loss_dev)),
              "pe_mlp_grad")
        self.stream.synchronize()
        return float(self.loss_dev.item())

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        check(load().pe_mlp_adam(self._h, float(lr), float(beta1), float(beta2), float(eps)), "pe_mlp_adam")
        self.stream.synchronize()

    def train(self, X, Y, B, nsteps, lr, seed=0, shift_period=0) -> float:
        check(load().pe_mlp_train(self._h, _ptr(X), _ptr(Y), X.shape[0], int(B), int(shift_period),
                                  int(seed) & 0xFFFFFFFFFFFFFFFF, int(nsteps), float(lr), _ptr(self.loss_dev)),
              "pe_mlp_train")
        self.stream.synchronize()
        return float(self.loss_dev.item())

    def sync_status(self) -> int:
        """PE_OK, or PE_ETIMEOUT if a tensor-core GEMM's bounded wait expired (status cleared)."""
        return int(load().pe_mlp_sync_status(self._h))
