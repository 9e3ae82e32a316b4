"""Projective macro steps of a periodic realisation with FP64 particles.

The small workload of the method (128 cells, 2^17 ions) is also run with the particle state
(theta, v, w) in double precision: against an FP64 reference this separates the error of a
run into the FP32 particles' precision and the method itself (the fixed-point deposit and
restriction rules are the FP32 path's). Every step runs in the library's kernels
(pe_quiet_start_f64, pe_push_f64, pe_sample_f64, pe_field, pe_coarsen, pe_ls_project,
pe_refine_f64); this module only sequences the calls, as the context API does for FP32
particles (Section 3.1 cycle: lift, burst with co-moving restriction, coarsening, leap).
"""
from __future__ import annotations

import torch

from . import _binding as pb
from .sharded import fixed_point_shifts, lift_seed


class FP64Realisation:
    """One realisation (periodic, Boltzmann electrons) with FP64 particles and nodal
    restriction samples (any wavelet)."""

    def __init__(self, ncell, n_coarse, K, N, L, dt, dT, qm=1.0, v_th=1.0, seed=1, newton_tol=1e-12,
                 newton_maxit=50, wavelet="haar", device=None, stream=None):
        self.ncell, self.nc, self.K, self.N = int(ncell), int(n_coarse), int(K), int(N)
        self.L, self.dt, self.dT, self.qm, self.v_th = float(L), float(dt), float(dT), float(qm), float(v_th)
        self.seed, self.tol, self.maxit, self.wavelet = int(seed), float(newton_tol), int(newton_maxit), wavelet
        self.dx = self.L / self.ncell
        self.dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream
        self.s_w, self.s_p = fixed_point_shifts(self.N, self.ncell)
        z = dict(device=self.dev)
        self.cell = torch.empty(self.N, dtype=torch.int32, **z)
        self.theta = torch.empty(self.N, dtype=torch.float64, **z)
        self.v = torch.empty(self.N, dtype=torch.float64, **z)
        self.w = torch.empty(self.N, dtype=torch.float64, **z)
        self.rho = torch.zeros(self.ncell, dtype=torch.int64, **z)
        self.samples = torch.zeros((self.K + 1, 2, self.ncell), dtype=torch.int64, **z)
        self.phi = torch.zeros(self.ncell, dtype=torch.float64, **z)
        self.E = torch.zeros(self.ncell, dtype=torch.float64, **z)
        self.E0 = torch.zeros(self.ncell, dtype=torch.float64, **z)
        self.coarse = torch.zeros((2, self.nc), dtype=torch.float64, **z)
        self.status = torch.zeros(1, dtype=torch.int32, **z)
        self.macro_steps = 0
        self.fresh = False
        self.v_at_integer = True

    def _s(self):
        return pb._stream(self.stream)

    def load(self, prof_n, prof_u, seed=None):
        """Appendix C loading on FP64 nodal profiles (device tensors)."""
        pb.check(pb.load().pe_quiet_start_f64(
            pb._ptr(self.cell), pb._ptr(self.theta), pb._ptr(self.v), pb._ptr(self.w), self.N, self.ncell,
            pb._ptr(prof_n), pb._ptr(prof_u), self.v_th, (self.seed if seed is None else seed) & (2**64 - 1),
            self.s_w, pb._ptr(self.rho), pb._ptr(self.status), self._s()), "pe_quiet_start_f64")
        self.fresh = True
        self.v_at_integer = True

    def load_initial(self, amplitude):
        """The ion-wave initial profile of the context API (pe_initial_profile)."""
        from .sharded import initial_profile

        n, u = initial_profile(self.ncell, self.L, amplitude)
        self.phi.zero_()
        self.macro_steps = 0
        self.load(n.to(self.dev, torch.float64), u.to(self.dev, torch.float64))

    def lift(self):
        prof_n = torch.empty(self.ncell, dtype=torch.float64, device=self.dev)
        prof_u = torch.empty_like(prof_n)
        pb.check(pb.load().pe_refine_f64(pb._ptr(self.coarse), self.nc, pb.PE_WAVELET[self.wavelet], self.ncell,
                                         pb._ptr(prof_n), pb._ptr(prof_u), self._s()), "pe_refine_f64")
        self.load(prof_n, prof_u, lift_seed(self.seed, self.macro_steps))

    def field(self):
        E, _, _ = pb.field(self.rho, self.ncell, self.dx, self.s_w, self.phi, tol=self.tol, maxit=self.maxit,
                           status=self.status, stream=self.stream)
        self.E.copy_(E)

    def push(self, kick, sample_row=None, tau=0.0):
        """One fine step (kick, drift, deposit), with the co-moving sample of the state before it."""
        E0 = pb._ptr(self.E0) if sample_row is not None else None
        samp = pb._ptr(self.samples[sample_row]) if sample_row is not None else None
        pb.check(pb.load().pe_push_f64(
            pb._ptr(self.cell), pb._ptr(self.theta), pb._ptr(self.v), pb._ptr(self.w), self.N, pb._ptr(self.E),
            self.ncell, self.dt / self.dx, self.qm * self.dt, float(kick), self.s_w, pb._ptr(self.rho), E0,
            tau / self.dx, self.qm * tau, self.s_p, samp, pb._ptr(self.status), self._s()), "pe_push_f64")

    def pic_steps(self, nsteps):
        """Plain (resolved) PIC: field of the current charge, then kick and drift."""
        for _ in range(nsteps):
            self.field()
            self.push(0.5 if self.v_at_integer else 1.0)
            self.v_at_integer = False
        self.fresh = False

    def burst(self):
        """K fine steps with the co-moving restriction sample of each of the K + 1 states (Appendix B)."""
        self.field()
        self.E0.copy_(self.E)
        kick = 0.5 if self.v_at_integer else 1.0
        for p in range(self.K + 1):
            tau = self.dT - p * self.dt
            if p < self.K:
                self.push(kick, p, tau)
                self.field()
                kick = 1.0
            else:
                pb.check(pb.load().pe_sample_f64(
                    pb._ptr(self.cell), pb._ptr(self.theta), pb._ptr(self.v), pb._ptr(self.w), self.N,
                    pb._ptr(self.E), self.ncell, self.qm * self.dt, kick, self.s_w, pb._ptr(self.E0), tau / self.dx,
                    self.qm * tau, self.s_p, pb._ptr(self.samples[p]), pb._ptr(self.status), self._s()),
                    "pe_sample_f64")
        self.v_at_integer = False
        self.fresh = False

    def restrict_project(self):
        cs = pb.coarsen(self.samples.reshape(self.K + 1, 2 * self.ncell), self.K + 1, self.ncell, self.s_w,
                        self.s_p, self.nc, self.wavelet, stream=self.stream)
        out, _ = pb.ls_project(cs.reshape(self.K + 1, 2 * self.nc), self.dt, self.dT, stream=self.stream)
        self.coarse.copy_(out.reshape(2, self.nc))
        self.macro_steps += 1

    def step(self):
        """One projective macro step: lift (unless just loaded), burst, restriction, leap."""
        if not self.fresh:
            self.lift()
        self.burst()
        self.restrict_project()

    def sync_status(self) -> int:
        torch.cuda.synchronize(self.dev)
        st = int(self.status.item())
        self.status.zero_()
        return st

