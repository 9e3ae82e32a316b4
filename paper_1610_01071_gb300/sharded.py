"""One realisation of the periodic ion-wave workload with its ions split over ranks.

Appendix C's point set, Section 2.2's fine steps and Appendix B's co-moving restriction are
defined per particle, so the particles of one realisation can live on several GPUs. Every
quantity that couples particles is an integer sum: the fixed-point charge deposit and the
fixed-point restriction samples. Each rank therefore deposits and samples its own slice,
and one exact all-reduce (sum, int64) per fine step of the deposit grid, and one per
burst of the samples, gives every rank the grids of the whole realisation, bit for bit as
one GPU holding all particles would compute them (integer addition is associative). The
field solve, the coarsening and the projective leap then run redundantly on every rank
and agree bit for bit.

Every step of the path runs in the library's kernels (`libpepic.so`, through
`_binding`); this module only sequences those calls and the collectives. The collective
is `torch.distributed.all_reduce` (NCCL between GPUs); `local_shards > 1` splits a rank's
slice further and sums the shards' grids on the device before the collective (used to
check the decomposition on one GPU).
"""
from __future__ import annotations

import ctypes

import torch

from . import _binding as pb

PE_PROFILE_SINE = 0


def shard_range(n_total: int, world: int, rank: int, align: int = 4):
    """Storage slots [first, first + n) of rank `rank` among `world` ranks: contiguous slices
    that partition [0, n_total), each starting at a multiple of `align` (the particle passes
    read 16-byte groups of four particles)."""
    if world < 1 or not 0 <= rank < world or n_total < 1:
        raise ValueError("invalid decomposition")
    units = (n_total + align - 1) // align
    lo = units * rank // world
    hi = units * (rank + 1) // world
    first = min(lo * align, n_total)
    last = min(hi * align, n_total)
    return first, last - first


def fixed_point_shifts(n_total: int, ncell: int):
    """The deposit rule's shifts (s_w, s_p) of a realisation of n_total ions (the same on every rank)."""
    s_w, s_p = ctypes.c_int32(), ctypes.c_int32()
    pb.check(pb.load().pe_fixed_point_shifts(int(n_total), int(ncell), 0.0, 0.0, ctypes.byref(s_w),
                                             ctypes.byref(s_p)), "pe_fixed_point_shifts")
    return s_w.value, s_p.value


def initial_profile(ncell: int, L: float, amplitude: float):
    """The ion-wave initial profiles (host FP32 tensors) of pe_initial_profile."""
    n = torch.empty(ncell, dtype=torch.float32)
    u = torch.empty(ncell, dtype=torch.float32)
    pb.check(pb.load().pe_initial_profile(PE_PROFILE_SINE, int(ncell), float(L), float(amplitude),
                                          ctypes.c_void_p(n.data_ptr()), ctypes.c_void_p(u.data_ptr())),
             "pe_initial_profile")
    return n, u


def lift_seed(seed: int, macro_steps: int) -> int:
    """Seed of the lifting that starts macro step `macro_steps` (the context API's rule)."""
    return (seed + 0x632BE59BD9B4E019 * (macro_steps + 1)) & 0xFFFFFFFFFFFFFFFF


class ShardedRealisation:
    """Projective macro steps (moment coarse variables, Haar, Boltzmann electrons, periodic)
    of one realisation whose N ions are split over the ranks of `group` (or the default
    process group); `local_shards` further slices per rank. reduce(t) sums an int64 device
    tensor over the ranks in place (default: all_reduce over the process group when it has
    more than one rank)."""

    def __init__(self, ncell, n_coarse, K, N, L, dt, dT, qm=1.0, v_th=1.0, seed=1, newton_tol=1e-10,
                 newton_maxit=50, device=None, rank=0, world=1, local_shards=1, reduce=None, stream=None):
        if ncell % n_coarse or (ncell // n_coarse) & (ncell // n_coarse - 1):
            raise ValueError("n_coarse must divide ncell by a power of two")
        self.ncell, self.nc, self.K, self.N = int(ncell), int(n_coarse), int(K), int(N)
        self.L, self.dt, self.dT, self.qm, self.v_th = float(L), float(dt), float(dT), float(qm), float(v_th)
        self.seed, self.tol, self.maxit = int(seed), float(newton_tol), int(newton_maxit)
        self.dx = self.L / self.ncell
        self.bin_shift = (self.ncell // self.nc).bit_length() - 1
        self.nb = self.ncell >> self.bin_shift
        self.dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream
        self.rank, self.world = int(rank), int(world)
        self.reduce = reduce if reduce is not None else self._all_reduce
        self.s_w, self.s_p = fixed_point_shifts(self.N, self.ncell)
        first, n = shard_range(self.N, self.world, self.rank)
        self.shards = []
        for k in range(local_shards):
            f, m = shard_range(n, local_shards, k)
            if m == 0:
                continue
            self.shards.append(dict(first=first + f, n=m, cell=torch.empty(m, dtype=torch.int32, device=self.dev),
                                    theta=torch.empty(m, dtype=torch.float32, device=self.dev),
                                    v=torch.empty(m, dtype=torch.float32, device=self.dev),
                                    w=torch.empty(m, dtype=torch.float32, device=self.dev),
                                    rho=torch.zeros(self.ncell, dtype=torch.int64, device=self.dev),
                                    samples=torch.zeros((self.K + 1, 2 * self.nb), dtype=torch.int64,
                                                        device=self.dev)))
        z = dict(device=self.dev)
        self.rho = torch.zeros(self.ncell, dtype=torch.int64, **z)
        self.samples = torch.zeros((self.K + 1, 2 * self.nb), dtype=torch.int64, **z)
        self.phi = torch.zeros(self.ncell, dtype=torch.float64, **z)
        self.E0f = torch.zeros(self.ncell, dtype=torch.float32, **z)
        self.Ef = torch.zeros(self.ncell, dtype=torch.float32, **z)
        self.coarse = torch.zeros((2, self.nc), dtype=torch.float64, **z)
        self.status = torch.zeros(1, dtype=torch.int32, **z)
        self.macro_steps = 0
        self.fresh = False

    # -- collectives ---------------------------------------------------------------------
    def _all_reduce(self, t):
        if self.world > 1:
            import torch.distributed as dist

            dist.all_reduce(t, op=dist.ReduceOp.SUM)

    def _sum_shards(self, key, out):
        """The rank's grid: the sum of its shards' integer grids (exact), then the all-ranks sum."""
        if len(self.shards) == 1:
            out.copy_(self.shards[0][key])
        else:
            torch.sum(torch.stack([s[key] for s in self.shards]), dim=0, out=out)
        self.reduce(out)

    # -- the hot path ----------------------------------------------------------------------
    def _load(self, prof_n, prof_u, seed):
        for s in self.shards:
            pb.check(pb.load().pe_quiet_start_slice(
                pb._ptr(s["cell"]), pb._ptr(s["theta"]), pb._ptr(s["v"]), pb._ptr(s["w"]), s["first"], s["n"], self.N,
                self.ncell, pb._ptr(prof_n), pb._ptr(prof_u), self.v_th, seed, self.s_w, pb._ptr(s["rho"]),
                pb._ptr(self.status), pb._stream(self.stream)), "pe_quiet_start_slice")
        self._sum_shards("rho", self.rho)
        self.fresh = True

    def load_initial(self, amplitude):
        """Appendix C loading of the ion-wave initial profile (every rank its slice)."""
        n, u = initial_profile(self.ncell, self.L, amplitude)
        self.phi.zero_()
        self.macro_steps = 0
        self._load(n.to(self.dev), u.to(self.dev), self.seed)

    def lift(self):
        """Section 3.3 lifting from the coarse state (the same profile on every rank)."""
        prof_n, prof_u = pb.refine(self.coarse, self.ncell, "haar", stream=self.stream)
        self._load(prof_n, prof_u, lift_seed(self.seed, self.macro_steps))

    def _field(self):
        _, Ef, _ = pb.field(self.rho, self.ncell, self.dx, self.s_w, self.phi, tol=self.tol, maxit=self.maxit,
                            status=self.status, stream=self.stream)
        self.Ef.copy_(Ef)

    def burst(self):
        """K fine steps (fused push, deposit and co-moving sample on every shard), the exact
        all-reduce of the deposit after each, the redundant field solve; then the last sample
        and the all-reduce of the K + 1 sample rows."""
        self._field()
        self.E0f.copy_(self.Ef)
        kick = 0.5
        dt_dx, qm_dt = self.dt / self.dx, self.qm * self.dt
        for p in range(self.K + 1):
            tau = self.dT - p * self.dt
            for s in self.shards:
                args = pb.make_sample_args(self.E0f, tau, self.qm, 1.0 / self.dx, self.s_w, self.s_p, s["samples"][p],
                                           bin_shift=self.bin_shift)
                if p < self.K:
                    pb.push(s["cell"], s["theta"], s["v"], s["w"], self.Ef, self.ncell, dt_dx, qm_dt, kick, self.s_w,
                            rho=s["rho"], sample=args, status=self.status, stream=self.stream)
                else:
                    pb.sample(s["cell"], s["theta"], s["v"], s["w"], self.Ef, self.ncell, qm_dt, kick, args,
                              status=self.status, stream=self.stream)
            if p < self.K:
                self._sum_shards("rho", self.rho)
                self._field()
                kick = 1.0
        self._sum_shards("samples", self.samples)
        self.fresh = False

    def restrict_project(self):
        """Coarsening of the summed samples and the least-squares leap (redundant, identical)."""
        cs = pb.coarsen(self.samples, self.K + 1, self.ncell, self.s_w, self.s_p, self.nc, "haar",
                        stream=self.stream, bin_shift=self.bin_shift)
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
