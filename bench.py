#!/usr/bin/env python
"""Benchmark: projective-integration PIC on the ion-wave steepening workload at scale
(periodic, 4096 cells, 2^24 ions, amplitude 0.5, v_th 1, burst K = 20, projective
ratio M = 10, 256 Haar coefficients per moment).

One benchmark step is one projective macro step (Section 3.1): lift -> 20 fine PIC
steps with a co-moving restriction sample after each (Appendix B) -> coarsening ->
least-squares slope -> forward-Euler leap over Delta t = M K dt. ``value`` is the
fine particle-steps executed per second; the simulated time per wall-second of the
projective path and of plain (resolved) GPU PIC are reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent realisation (replicas, weak
scaling, no data-path collective); timing is the maximum over ranks.
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s and simulated time per wall-second, projective vs plain PIC"
UNIT = "particle-steps/s"
FALLBACK_HBM_GBS = 6800.0
# Algorithmic bytes per particle of each particle kernel (reads and writes of the particle
# arrays; the grids stay in shared memory and L2).
KERNEL_BYTES = {
    "push_sample": (28, "k_particles<push + binned moment sample> (gather, kick, drift, deposit, co-moving sample)"),
    "push": (28, "k_particles<push> (gather, kick, drift, deposit; plain PIC)"),
    "sample": (16, "k_particles<binned moment sample> (last co-moving sample of a burst, read only)"),
    "deposit": (12, "k_particles<deposit> (charge deposit alone: cell, theta, w read)"),
    "load": (16, "k_quiet_start (lifting: quiet-start loading with the deposit fused, write only)"),
    "push_sample_ps": (28, "k_particles<push + phase-space sample> (64 x-bins x 64 velocity cells window)"),
    "push_sample_psw": (28, "k_particles<push + phase-space sample, hat rows> (wavelet form: 16 coarse nodes x "
                            "256 velocity cells window)"),
    "load_psw": (16, "k_ps_quiet_start on fine-node tables (wavelet-form lifting, write only)"),
    "push_sample_pressure": (28, "k_particles<push + binned sample of density, momentum and second moment> "
                                 "(ion pressure active)"),
    "load_thermal": (16, "k_quiet_start<thermal> (lifting at the local temperature, deposit fused, write only)"),
    "push_sample_slab": (28, "k_particles<push + binned moment sample, walls> on the slab (2^25 ions, 8192 cells)"),
    "push_sample_ps_slab": (28, "k_particles<push + phase-space sample, walls> on the slab (2^25 ions)"),
}
# DRAM bytes (read + write) per launch on the 2^24-ion workload from the ncu captures
# summarised in profiles/, each valid while the particle kernels' device code
# (kernel_source_hash) hashes to the value it was taken with.
NCU_TRAFFIC = {
    "push_sample": {"source_hash": "173582129c21fd7b", "bytes": 270.715904e6 + 145.457152e6},
    "push": {"source_hash": "173582129c21fd7b", "bytes": 270.730496e6 + 145.774336e6},
    "sample": {"source_hash": "173582129c21fd7b", "bytes": 270.679552e6 + 3.367168e6},
    "deposit": {"source_hash": "173582129c21fd7b", "bytes": 203.015936e6 + 2.963968e6},
    "push_sample_ps": {"source_hash": "173582129c21fd7b", "bytes": 270.272256e6 + 145.230080e6},
    "push_sample_psw": {"source_hash": "173582129c21fd7b", "bytes": 270.507520e6 + 145.440768e6},
    "push_sample_pressure": {"source_hash": "173582129c21fd7b", "bytes": 270.752512e6 + 145.262592e6},
    "load": {"source_hash": "173582129c21fd7b", "bytes": 0.574720e6 + 207.112192e6},
}


def kernel_source_hash():
    """Hash of the particle kernels' device code: pe_particles.cu up to its host-side section,
    and the device headers it includes (host-side edits leave the counters valid)."""
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1610_01071_gb300", "csrc")
    with open(os.path.join(csrc, "pe_particles.cu"), "rb") as fh:
        src = fh.read()
    cut = src.find(b"// ------------------------------------------------------------------ host side")
    h.update(src if cut < 0 else src[:cut])
    for f in ("pe_common.cuh", "pe_eq.cuh"):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        for k in ("hbm_gbs", "hbm_GBps", "hbm"):
            if k in d and isinstance(d[k], (int, float)):
                return float(d[k]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


def peak_bf16():
    """Dense bf16 tensor peak: the measured burst figure (the training loop is timed alone)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        if isinstance(d.get("bf16_tflops"), (int, float)):
            return float(d["bf16_tflops"]), "measured (bf16 burst)"
    except (OSError, ValueError):
        pass
    return 1900.0, "fallback (bf16 burst)"


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the benchmark runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.tmp = tempfile.NamedTemporaryFile(prefix="clocks_", suffix=".csv", delete=False)
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.tmp,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.tmp.name) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for name, val in zip(names, f[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        os.unlink(self.tmp.name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def workload_cfg():
    from paper_1610_01071_gb300 import inputs

    return inputs.workload("iaw_large")


# ------------------------------------------------------------------ oracle (CPU) legs


def oracle_macro_step(cfg, n_sample, seed):
    """One projective macro step of the workload with n_sample particles; returns the
    number of fine particle-steps done and the wall time."""
    import numpy as np

    import oracle as orc

    ncell = cfg["ncell"]
    ocfg = dict(cfg, N=n_sample, s_w=orc.fx_shift(8.0 * ncell / n_sample))
    nprof, uprof = orc.sine_profile(ncell, cfg["L"], cfg["amplitude"])
    coarse = np.stack([orc.coarsen(nprof, cfg["n_coarse"]), orc.coarsen(nprof * uprof, cfg["n_coarse"])])
    t0 = time.perf_counter()
    st = orc.lift(coarse, ocfg, seed)
    orc.efpi_macro_step(st, ocfg, np.zeros(ncell))
    return n_sample * cfg["K"], time.perf_counter() - t0


def host_cores():
    """Host cores this process may run on (the all-core oracle leg uses one process per core)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _oracle_worker(cfg, n_sample, seeds, barrier, out):
    import oracle as orc

    orc._load()  # compile/load before the common start
    for k, seed in enumerate(seeds):
        barrier.wait()
        t0 = time.perf_counter()
        ps, _ = oracle_macro_step(cfg, n_sample, seed)
        out.put((k, ps, t0, time.perf_counter()))


def oracle_all_cores(cfg, n_sample, seed0, cores, steps=1):
    """The oracle as it stands, one independent macro step per host core and step (processes
    started once with spawn; each step released together by a barrier). Returns per step the
    whole-host particle-steps and the wall time from the common start to the last worker's end
    (perf_counter is the system-wide monotonic clock, so the processes' readings compare)."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(cores), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker,
                         args=(cfg, n_sample, [seed0 + 1000 * k + j for k in range(steps)], barrier, out))
             for j in range(cores)]
    for p in procs:
        p.start()
    res = [out.get() for _ in range(cores * steps)]
    for p in procs:
        p.join()
    per_step = []
    for k in range(steps):
        rk = [r for r in res if r[0] == k]
        per_step.append((sum(r[1] for r in rk), max(r[3] for r in rk) - min(r[2] for r in rk)))
    return per_step


def cpu_baseline(cfg, n_single=1 << 23, n_each=1 << 22):
    """The FP64 oracle on the host cores: one thread on a 2^23-particle sample, and all cores
    (one process per core, each a 2^22-particle sample with its own seed)."""
    ps1, t1 = oracle_macro_step(cfg, n_single, seed=1)
    cores = host_cores()
    psn, tn = oracle_all_cores(cfg, n_each, 50, cores)[0]
    return {"value": psn / tn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"all {cores} host cores, one process each: one projective macro step (lift, {cfg['K']}-step "
                       f"burst with co-moving restriction, coarsening, projection) of the {cfg['ncell']}-cell workload "
                       f"with {n_each} of its {cfg['N']} particles per process (own seed), FP64; {tn:.1f} s wall"),
            "single_core": {"value": ps1 / t1, "unit": UNIT, "cores": 1,
                            "sample": f"one thread, one macro step with {n_single} particles; {t1:.1f} s"}}


def bench_config(cfg, world):
    """The workload entry of the JSON line (the same for the GPU arm and the reference arm)."""
    return {"workload": "iaw_large", "ncell": cfg["ncell"], "particles": cfg["N"], "K": cfg["K"], "M": cfg["M"],
            "n_coarse": cfg["n_coarse"], "wavelet": cfg["wavelet"], "dt": cfg["dt"], "dT": cfg["dT"],
            "l2": "inputs larger than L2 (268 MB of particles per realisation), no flush",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = workload_cfg()
    cores = host_cores()
    n_each = 1 << 20
    runs = oracle_all_cores(cfg, n_each, 100, cores, steps=args.warmup + args.steps)[args.warmup:]
    tot_ps, tot_t = sum(r[0] for r in runs), sum(r[1] for r in runs)
    value = tot_ps / tot_t
    sample = (f"each step: one projective macro step of the iaw_large workload per host core ({cores} processes), "
              f"each with {n_each} of its {cfg['N']} particles and its own seed (FP64 oracle)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            # the GPU arm's workload and config; each step a bounded sample of it (cpu_baseline.sample)
            "config": bench_config(cfg, args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ranks (replicas)


def reduce_over_ranks(x, op, world, device):
    """Max or sum of one float over the ranks of the process group (identity with one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replica_totals(t_local, work_local, world, device):
    """Whole-job throughput of weakly scaled replicas: the work of all ranks over the slowest
    rank's time. Returns (throughput, max time, total work)."""
    t = reduce_over_ranks(t_local, "max", world, device)
    w = reduce_over_ranks(work_local, "sum", world, device)
    return w / t, t, w


# ------------------------------------------------------------------ GPU leg


def run_gpu(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    from paper_1610_01071_gb300 import _binding as pb
    from paper_1610_01071_gb300 import _build

    _build.build()
    cfg = workload_cfg()
    N, K, ncell = cfg["N"], cfg["K"], cfg["ncell"]
    stream = torch.cuda.Stream(device=dev)
    c = pb.make_config(ncell, cfg["n_coarse"], K, N, cfg["L"], cfg["dt"], cfg["dT"], qm=cfg["qm"], v_th=cfg["v_th"],
                       wavelet=cfg["wavelet"], seed=1000 + rank, sort_every=20, newton_tol=1e-10)
    ctx = pb.Context(c, device=dev, stream=stream)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(x):
        return reduce_over_ranks(x, "max", world, dev)

    def sum_over_ranks(x):
        return reduce_over_ranks(x, "sum", world, dev)

    sampler = ClockSampler(local)
    sampler.start()
    with torch.cuda.stream(stream):
        ctx.load_initial(cfg["amplitude"])
        for _ in range(args.warmup):
            ctx.step()
        if ctx.sync_status() != 0:
            raise RuntimeError("device status after warm-up: " + pb.load().pe_strerror(ctx.sync_status()).decode())
        # ---------------- timed region: projective macro steps, inputs resident in HBM
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ctx.profile_read()
        ctx.profile(True, kinds=("push_sample",))  # the roofline kernel only: events cost stream time
        launches0 = pb.launch_count()
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            ctx.step()
        ev1.record(stream)
        barrier()
        launches = pb.launch_count() - launches0
        ctx.profile(False)
        prof = ctx.profile_read_kinds()
        newton_iters = ctx.diagnostics().newton_iters
        t_proj = ev0.elapsed_time(ev1) / 1e3
        st = ctx.sync_status()
        if st != 0:
            raise RuntimeError("device status after the timed region: " + pb.load().pe_strerror(st).decode())
        # the other kernels of a macro step (field solve, last sample, lifting), timed on
        # steps after the timed region
        ctx.profile(True)
        for _ in range(min(args.steps, 5)):
            ctx.step()
        ctx.profile(False)
        prof_rest = ctx.profile_read_kinds()
        # ---------------- plain (resolved) GPU PIC on the same workload, same context
        ctx.load_initial(cfg["amplitude"])
        ctx.pic_steps(max(3, args.warmup) * K)
        n_plain = max(args.steps, 1) * K
        ctx.profile_read_kinds()
        ctx.profile(True, kinds=("push",))
        barrier()
        ev0.record(stream)
        ctx.pic_steps(n_plain)
        ev1.record(stream)
        barrier()
        ctx.profile(False)
        prof_plain = ctx.profile_read_kinds()
        t_plain = ev0.elapsed_time(ev1) / 1e3
        ctx.profile(True, kinds=("field",))
        ctx.pic_steps(K)
        ctx.profile(False)
        prof_plain["field"] = ctx.profile_read_kinds()["field"]
        # ---------------- the deposit alone and the phase-space pass, for their rooflines
        kern = time_kernels(ctx, cfg, pb, stream)
        # ---------------- end to end through the C ABI with host buffers
        host = torch.empty((2, cfg["n_coarse"]), dtype=torch.float64).pin_memory()
        ctx.load_initial(cfg["amplitude"])
        ctx.step()  # every timed step then lifts, as in the timed region
        ctx.get_coarse_host(host)
        ctx.profile(True, kinds=("push_sample",))  # the timed region's event pairs too
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.set_coarse_host(host)
            ctx.step()
            ctx.get_coarse_host(host)
        t_e2e = time.perf_counter() - t0
        barrier()
        ctx.profile(False)
        ctx.profile_read_kinds()
        # ---------------- time to solution and accuracy against a resolved plain-PIC run
        acc, want, checks = run_accuracy(dev, cfg, pb) if not args.no_accuracy else (None, None, None)
        sur = run_surrogate(dev, cfg, pb, want, checks) if (acc is not None and not args.no_surrogate) else None
        slab = run_slab(dev, pb) if not args.no_slab else None
        kin = run_kinetic(dev, pb) if not args.no_kinetic else None
        # ---------------- ensemble of 64 realisations of log-uniform sizes (pe_batch)
        ens = run_ensemble(dev, max(args.steps // 2, 2), 3, rank) if not args.no_ensemble else None
    clocks = sampler.stop()

    value, t_proj_max, ps_proj = replica_totals(t_proj, float(N) * K * args.steps, world, dev)
    t_plain_max = max_over_ranks(t_plain)
    t_e2e_max = max_over_ranks(t_e2e)
    ps_plain = sum_over_ranks(float(N) * n_plain)
    sim_proj = cfg["dT"] * args.steps / t_proj_max
    sim_plain = cfg["dt"] * n_plain / t_plain_max
    peak, peak_kind = peak_hbm()
    src_hash = kernel_source_hash()
    means = {k: (v["ms"] / v["launches"], v["launches"]) for k, v in prof_rest.items()
             if v["launches"] and k not in ("field", "push_sample")}
    means["push_sample"] = (prof["push_sample"]["ms"] / max(prof["push_sample"]["launches"], 1),
                            prof["push_sample"]["launches"])
    means["push"] = (prof_plain["push"]["ms"] / max(prof_plain["push"]["launches"], 1), prof_plain["push"]["launches"])
    means.update(kern)
    roof = {k: roofline_entry(k, ms, n, N, peak, peak_kind, src_hash) for k, (ms, n) in means.items()}
    slab_roof = []
    if slab is not None:  # the bounded-grid workload's fused passes (2^25 ions), timed inside its bursts
        from paper_1610_01071_gb300 import inputs as _inp

        n_slab = _inp.workload("slab")["N"]
        for r in slab["projective"]:
            if r["coarse"] == "moments" or r["K"] == 30:
                kk = r["pass_kind"] + "_slab"
                if r["pass_launches"] and kk not in [e.get("key") for e in slab_roof]:
                    e = roofline_entry(kk, r["pass_ms"], r["pass_launches"], n_slab, peak, peak_kind, src_hash)
                    e["key"] = kk
                    slab_roof.append(e)
    if rank != 0:
        dist.destroy_process_group()
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_proj_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": bench_config(cfg, world),
        "sim_time_per_wall_s": {"projective": sim_proj, "plain_pic": sim_plain,
                                "ratio": sim_proj / sim_plain},
        "plain_pic": {"value": ps_plain / t_plain_max, "unit": UNIT, "steps": n_plain,
                      "ms_per_step": 1e3 * t_plain_max / n_plain, "sort_every": 20},
        "field_solve_us": 1e3 * prof_rest["field"]["ms"] / max(prof_rest["field"]["launches"], 1),
        "field_solve_us_plain_pic": 1e3 * prof_plain["field"]["ms"] / max(prof_plain["field"]["launches"], 1),
        "newton_iters_last": newton_iters,
        # the dominant kernel: the fused pass of the bursts, from its own launches only
        "roofline": roof["push_sample"],
        "roofline_kernels": [roof[k] for k in KERNEL_BYTES if k in roof and k != "push_sample"] + slab_roof,
        "e2e": {"value": ps_proj / t_e2e_max, "unit": UNIT, "h2d_bytes_per_step": 8 * 2 * cfg["n_coarse"],
                "d2h_bytes_per_step": 8 * 2 * cfg["n_coarse"]},
        "gpu_launches": launches,
        "clocks": clocks,
    }
    if acc is not None:
        line["time_to_solution"] = acc
    if sur is not None:
        line["surrogate"] = sur
    if slab is not None:
        line["slab"] = slab
    if kin is not None:
        line["kinetic_electrons"] = kin
    if ens is not None:
        t_ens = max_over_ranks(ens["seconds"])
        line["ensemble"] = {"workload": "64 realisations, 2^9..2^13 cells, 2^18..2^22 ions (log-uniform), K=20, M=10, "
                                        "odd: periodic sinusoid, even: bounded slab",
                            "value": sum_over_ranks(ens["particle_steps"]) / t_ens, "unit": UNIT,
                            "ms_per_step": 1e3 * t_ens / ens["steps"], "particles": ens["particles"],
                            "tuned_chunk": ens["tuned_chunk"], "tuned_shape": ens["tuned_shape"],
                            "groups": ens["groups"], "steps": ens["steps"]}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def roofline_entry(kind, ms, launches, N, peak, peak_kind, src_hash):
    """Roofline of one particle kernel: algorithmic bytes per launch (bytes per particle x N)
    over its mean CUDA-event launch time, against the measured HBM copy bandwidth."""
    bpp, name = KERNEL_BYTES[kind]
    achieved = bpp * N / (ms / 1e3) / 1e9
    t = NCU_TRAFFIC.get(kind)
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind,
            "traffic": t["bytes"] if t and t["source_hash"] == src_hash else None,
            "bytes_per_particle": bpp, "algorithmic_bytes": bpp * N, "launch_us": 1e3 * ms, "launches": launches}


def time_kernels(ctx, cfg, pb, stream, reps=10):
    """Mean launch time (ms) of the charge deposit alone on the context's particles, and of the
    fused push + phase-space sample in a phase-space context of the same workload (two macro
    steps with the context's own event pairs), for the per-kernel rooflines."""
    import torch

    dev = stream.device
    N, ncell = cfg["N"], cfg["ncell"]
    ctx.load_initial(cfg["amplitude"])  # a freshly loaded (velocity-ordered) state, as a lift leaves it
    d = ctx.diagnostics()
    cell, theta, _, w = ctx.particles(d.particle_bank)
    rho = torch.empty(ncell, dtype=torch.int64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    out = {}
    with torch.cuda.stream(stream):
        for _ in range(3):
            pb.deposit(cell, theta, w, ncell, d.s_w, rho=rho, status=st, stream=stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            pb.deposit(cell, theta, w, ncell, d.s_w, rho=rho, status=st, stream=stream)
        e1.record(stream)
        stream.synchronize()
        out["deposit"] = (e0.elapsed_time(e1) / reps, reps)
        c = pb.make_config(ncell, cfg["n_coarse"], cfg["K"], N, cfg["L"], cfg["dt"], 8.0, qm=cfg["qm"],
                           v_th=cfg["v_th"], seed=13, newton_tol=1e-10, coarse="phase_space", n_v=64, v_max=8.0,
                           ps_filter=3)
        ps = pb.Context(c, device=dev, stream=stream)
        ps.load_initial(cfg["amplitude"])
        ps.step()
        ps.profile_read_kinds()
        ps.profile(True)
        for _ in range(2):
            ps.step()
        ps.profile(False)
        k = ps.profile_read_kinds()["push_sample_ps"]
        out["push_sample_ps"] = (k["ms"] / max(k["launches"], 1), k["launches"])
        if int(st.item()) != 0 or ps.sync_status() != 0:
            raise RuntimeError("device status set while timing the deposit / phase-space pass")
        del ps
        # the wavelet form of the phase-space variable (hat rows, 256 velocity cells -> 64 Coif4)
        c = pb.make_config(ncell, cfg["n_coarse"], cfg["K"], N, cfg["L"], cfg["dt"], 10.0, qm=cfg["qm"],
                           v_th=cfg["v_th"], seed=13, newton_tol=1e-10, coarse="phase_space", n_v=256, v_max=8.0,
                           n_v_coarse=64, wavelet="coif4")
        pw = pb.Context(c, device=dev, stream=stream)
        pw.load_initial(cfg["amplitude"])
        pw.step()
        pw.profile_read_kinds()
        pw.profile(True)
        for _ in range(2):
            pw.step()
        pw.profile(False)
        kk = pw.profile_read_kinds()
        out["push_sample_psw"] = (kk["push_sample_ps"]["ms"] / max(kk["push_sample_ps"]["launches"], 1),
                                  kk["push_sample_ps"]["launches"])
        out["load_psw"] = (kk["load"]["ms"] / max(kk["load"]["launches"], 1), kk["load"]["launches"])
        if pw.sync_status() != 0:
            raise RuntimeError("device status set while timing the wavelet-form passes")
        del pw
        # the moment variable with the ion pressure (three Haar-binned moments, thermal lifting)
        c = pb.make_config(ncell, cfg["n_coarse"], cfg["K"], N, cfg["L"], cfg["dt"], cfg["dT"], qm=cfg["qm"],
                           v_th=cfg["v_th"], seed=13, newton_tol=1e-10, coarse="moments_pressure")
        pp = pb.Context(c, device=dev, stream=stream)
        pp.load_initial(cfg["amplitude"])
        pp.step()
        pp.profile_read_kinds()
        pp.profile(True)
        for _ in range(2):
            pp.step()
        pp.profile(False)
        kk = pp.profile_read_kinds()
        out["push_sample_pressure"] = (kk["push_sample"]["ms"] / max(kk["push_sample"]["launches"], 1),
                                       kk["push_sample"]["launches"])
        out["load_thermal"] = (kk["load"]["ms"] / max(kk["load"]["launches"], 1), kk["load"]["launches"])
        if pp.sync_status() != 0:
            raise RuntimeError("device status set while timing the pressure variable's passes")
    return out


def run_kernel_slab(args):
    """The fused push + phase-space sample on the bounded slab (2^25 ions, 8192 cells), on the
    state after two phase-space macro steps (Delta t = 6, bursts of 30), timed alone."""
    import torch

    from paper_1610_01071_gb300 import _binding as pb
    from paper_1610_01071_gb300 import _build, inputs

    _build.build()
    dev = torch.device("cuda", 0)
    w = inputs.workload("slab")
    N, ncell, nv = w["N"], w["ncell"], 64
    c = pb.make_config(ncell, w["n_coarse"], 30, N, w["L"], w["dt"], 6.0, qm=w["qm"], v_th=w["v_th"], seed=21,
                       newton_tol=1e-10, newton_maxit=80, boundary="absorbing", coarse="phase_space", n_v=nv,
                       v_max=8.0, ps_filter=3)
    ctx = pb.Context(c, device=dev)
    ctx.load_initial(profile="slab")
    for _ in range(2):
        ctx.step()
    d = ctx.diagnostics()
    cell, theta, v, wt = ctx.particles(d.particle_bank)
    rho = ctx.view("rho", torch.int64, ncell)
    Ef = ctx.view("Ef", torch.float32, ncell)
    E0f = ctx.view("E0f", torch.float32, ncell)
    bshift = (ncell // w["n_coarse"]).bit_length() - 1
    samp = torch.zeros(((ncell >> bshift), nv), dtype=torch.int64, device=dev)
    dx = w["L"] / ncell
    sa = pb.make_sample_args(E0f, 6.0, w["qm"], 1.0 / dx, d.s_w, d.s_p, samp, bin_shift=bshift, n_v=nv, v_min=-8.0,
                             dv=16.0 / nv, boundary="absorbing")
    status = torch.zeros(1, dtype=torch.int32, device=dev)

    def once():
        pb.push(cell, theta, v, wt, Ef, ncell, w["dt"] / dx, w["dt"], 1.0, d.s_w, rho=rho, sample=sa, status=status,
                boundary="absorbing")

    for _ in range(args.warmup):
        once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        once()
    e1.record()
    torch.cuda.synchronize()
    us = 1e3 * e0.elapsed_time(e1) / args.steps
    print(json.dumps({"kernel": args.kernel, "particles": N, "ncell": ncell, "launch_us": us,
                      "algorithmic_GBps": 28 * N / (us * 1e-6) / 1e9, "status": int(status.item())}), flush=True)
    return 0


def run_kernel_kinetic(args):
    """Kinetic-electron workload (iaw_kinetic) for profiling: `warmup` then `steps` phase-space
    projective macro steps, then 150 plain two-species PIC steps, each timed with CUDA events;
    the push and field-solve launch times come from the context's own event pairs."""
    import torch

    from paper_1610_01071_gb300 import _binding as pb
    from paper_1610_01071_gb300 import _build, inputs

    _build.build()
    dev = torch.device("cuda", 0)
    w = inputs.workload("iaw_kinetic")
    c = pb.make_config(w["ncell"], w["n_coarse"], w["K"], w["N"], w["L"], w["dt"], w["dT"], qm=w["qm"], v_th=w["v_th"],
                       seed=11, sort_every=20, newton_tol=1e-10, coarse="phase_space", n_v=w["n_v"],
                       v_max=w["v_max"], ps_filter=3, electrons="kinetic", qm_e=w["qm_e"])
    ctx = pb.Context(c, device=dev)
    ctx.load_initial(w["amplitude"])
    for _ in range(args.warmup):
        ctx.step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ctx.profile_read()
    ctx.profile(True)
    e0.record()
    for _ in range(args.steps):
        ctx.step()
    e1.record()
    torch.cuda.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read()
    ms_macro = e0.elapsed_time(e1) / args.steps
    e0.record()
    ctx.pic_steps(150)
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"kernel": "kinetic", "ions": w["N"], "electrons": w["N"], "ncell": w["ncell"],
                      "ms_per_macro_step": ms_macro, "plain_pic_us_per_step": 1e3 * e0.elapsed_time(e1) / 150,
                      "particle_pass_us": 1e3 * prof["push_ms"] / max(prof["push_launches"], 1),
                      "particle_passes": prof["push_launches"],
                      "field_us": 1e3 * prof["field_ms"] / max(prof["field_launches"], 1),
                      "status": ctx.sync_status()}), flush=True)
    return 0


def run_kernel(args):
    """Times one hot-path kernel alone on the workload's particle state (for profiling):
    ``--kernel push_sample|push|deposit|sample|field|quiet_start|push_sample_ps|push_sample_psw|
    push_sample_pressure|ps_tables|ps_quiet_start|push_sample_ps_slab|kinetic|ensemble|tc_gemm``."""
    import torch

    if args.kernel == "push_sample_ps_slab":
        return run_kernel_slab(args)
    if args.kernel == "ensemble":
        import torch

        from paper_1610_01071_gb300 import _build

        _build.build()
        ens = run_ensemble(torch.device("cuda", 0), args.steps, args.warmup)
        ens["value"] = ens["particle_steps"] / ens["seconds"]
        print(json.dumps(dict(kernel="ensemble", **ens)), flush=True)
        return 0
    if args.kernel == "kinetic":
        return run_kernel_kinetic(args)
    if args.kernel == "tc_gemm":
        return run_kernel_tc_gemm(args)

    from paper_1610_01071_gb300 import _binding as pb
    from paper_1610_01071_gb300 import _build

    _build.build()
    dev = torch.device("cuda", 0)
    cfg = workload_cfg()
    N, K, ncell = cfg["N"], cfg["K"], cfg["ncell"]
    c = pb.make_config(ncell, cfg["n_coarse"], K, N, cfg["L"], cfg["dt"], cfg["dT"], qm=cfg["qm"], v_th=cfg["v_th"],
                       seed=7, newton_tol=1e-10)
    ctx = pb.Context(c, device=dev)
    ctx.load_initial(cfg["amplitude"])
    d = ctx.diagnostics()
    cell, theta, v, w = ctx.particles(d.particle_bank)
    rho = ctx.view("rho", torch.int64, ncell)
    phi = ctx.view("phi", torch.float64, ncell)
    samp = ctx.view("samples_fx", torch.int64, 2 * ncell)
    prof = ctx.view("profile", torch.float32, 2 * ncell)
    E, Ef, _ = pb.field(rho, ncell, cfg["L"] / ncell, d.s_w, phi)
    dx = cfg["L"] / ncell
    bshift = (ncell // cfg["n_coarse"]).bit_length() - 1 if cfg["wavelet"] == "haar" else 0
    args_s = pb.make_sample_args(Ef, cfg["dT"], cfg["qm"], 1.0 / dx, d.s_w, d.s_p, samp, bin_shift=bshift)
    args_f = pb.make_sample_args(Ef, cfg["dT"], cfg["qm"], 1.0 / dx, d.s_w, d.s_p, samp, bin_shift=0)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    nv = 64
    nxc = ncell >> bshift
    samp_ps = torch.zeros((nxc, nv), dtype=torch.int64, device=dev)
    args_ps = pb.make_sample_args(Ef, cfg["dT"], cfg["qm"], 1.0 / dx, d.s_w, d.s_p, samp_ps, bin_shift=bshift, n_v=nv,
                                  v_min=-8.0, dv=16.0 / nv)
    samp_psw = torch.zeros((nxc, 256), dtype=torch.int64, device=dev)
    args_psw = pb.make_sample_args(Ef, 10.0, cfg["qm"], 1.0 / dx, d.s_w, d.s_p, samp_psw, bin_shift=bshift, n_v=256,
                                   v_min=-8.0, dv=16.0 / 256, x_tent=True)
    samp3 = torch.zeros(3 * (ncell >> bshift), dtype=torch.int64, device=dev)
    args_e = pb.make_sample_args(Ef, cfg["dT"], cfg["qm"], 1.0 / dx, d.s_w, d.s_p, samp3, bin_shift=bshift,
                                 s_e=pb.second_moment_shift(N, ncell))
    if args.kernel in ("ps_tables", "ps_quiet_start"):
        pb.sample(cell, theta, v, w, Ef, ncell, cfg["dt"], 0.5, args_ps, status=status)
        H = pb.ps_coarsen(samp_ps, d.s_w)
        mass, cdf, table, _ = pb.ps_lift_tables(H)
        scratch = torch.empty(2 * nxc * (nv + 1), dtype=torch.float64, device=dev)
        flags = torch.zeros(1, dtype=torch.int32, device=dev)

    def once():
        if args.kernel == "push_sample_ps":
            pb.push(cell, theta, v, w, Ef, ncell, cfg["dt"] / dx, cfg["dt"], 1.0, d.s_w, rho=rho, sample=args_ps,
                    status=status)
        elif args.kernel == "push_sample_psw":
            pb.push(cell, theta, v, w, Ef, ncell, cfg["dt"] / dx, cfg["dt"], 1.0, d.s_w, rho=rho, sample=args_psw,
                    status=status)
        elif args.kernel == "ps_tables":
            pb.load().pe_ps_lift_tables(pb._ptr(H), nxc, nv, pb._ptr(mass), pb._ptr(cdf), pb._ptr(table),
                                        pb._ptr(scratch), pb._ptr(flags), pb._stream())
        elif args.kernel == "ps_quiet_start":
            pb.load().pe_ps_quiet_start(pb._ptr(cell), pb._ptr(theta), pb._ptr(v), pb._ptr(w), N, ncell, bshift,
                                        pb._ptr(mass), pb._ptr(table), nv, -8.0, 16.0 / nv, 7, d.s_w, pb._ptr(rho),
                                        pb._ptr(status), pb._stream())
        elif args.kernel in ("push_sample", "push_sample_nodal"):
            pb.push(cell, theta, v, w, Ef, ncell, cfg["dt"] / dx, cfg["dt"], 1.0, d.s_w, rho=rho,
                    sample=args_s if args.kernel == "push_sample" else args_f, status=status)
        elif args.kernel == "push_sample_pressure":
            pb.push(cell, theta, v, w, Ef, ncell, cfg["dt"] / dx, cfg["dt"], 1.0, d.s_w, rho=rho, sample=args_e,
                    status=status)
        elif args.kernel == "push":
            pb.push(cell, theta, v, w, Ef, ncell, cfg["dt"] / dx, cfg["dt"], 1.0, d.s_w, rho=rho, status=status)
        elif args.kernel == "deposit":
            pb.deposit(cell, theta, w, ncell, d.s_w, rho=rho, status=status)
        elif args.kernel == "sample":
            pb.sample(cell, theta, v, w, Ef, ncell, cfg["dt"], 1.0, args_s, status=status)
        elif args.kernel == "field":
            pb.field(rho, ncell, dx, d.s_w, phi)
        elif args.kernel == "quiet_start":
            pb.load().pe_quiet_start(pb._ptr(cell), pb._ptr(theta), pb._ptr(v), pb._ptr(w), N, ncell, pb._ptr(prof),
                                     pb._ptr(prof[ncell:]), 1.0, 7, d.s_w, pb._ptr(rho), pb._ptr(status),
                                     pb._stream())
        else:
            raise SystemExit(f"unknown kernel {args.kernel}")

    for _ in range(args.warmup):
        once()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        once()
    e1.record()
    torch.cuda.synchronize()
    us = 1e3 * e0.elapsed_time(e1) / args.steps
    bytes_per = {"push_sample": 28, "push_sample_nodal": 28, "push": 28, "deposit": 12, "sample": 16, "quiet_start": 16,
                 "field": 0, "push_sample_ps": 28, "push_sample_psw": 28, "ps_tables": 0, "ps_quiet_start": 16,
                 "push_sample_pressure": 28}
    gbs = bytes_per[args.kernel] * N / (us * 1e-6) / 1e9
    print(json.dumps({"kernel": args.kernel, "particles": N, "ncell": ncell, "launch_us": us, "algorithmic_GBps": gbs,
                      "status": int(status.item())}), flush=True)
    return 0


def run_kernel_tc_gemm(args):
    """The surrogate's tensor-core product alone: C = A B^T for BF16 A [2048, 512], B [512, 512]
    (one forward layer of a training batch), timed with CUDA events over --steps launches."""
    import torch

    from paper_1610_01071_gb300 import _binding as pb
    from paper_1610_01071_gb300 import _build

    _build.build()
    dev = torch.device("cuda", 0)
    g = torch.Generator(device="cpu").manual_seed(3)
    M, N, K = 2048, 512, 512
    A = torch.randn((M, K), generator=g).to(torch.bfloat16).to(dev)
    B = torch.randn((N, K), generator=g).to(torch.bfloat16).to(dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    for _ in range(args.warmup):
        pb.tc_gemm(A, B, status=status)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        pb.tc_gemm(A, B, status=status)
    e1.record()
    torch.cuda.synchronize()
    us = 1e3 * e0.elapsed_time(e1) / args.steps
    print(json.dumps({"kernel": "tc_gemm", "M": M, "N": N, "K": K, "launch_us": us,
                      "TFLOPs": 2.0 * M * N * K / (us * 1e-6) / 1e12, "status": int(status.item())}), flush=True)
    return 0


def ensemble_sizes(count=64, seed=4):
    """Ensemble workload: grids of 2^U cells, U uniform in 9..13, and 2^V ions, V uniform
    in 18..22 (log-uniform sizes); odd realisations a periodic sinusoid of amplitude
    U(0.05, 0.6), even ones the bounded slab (absorbing walls, uniform central eighth)."""
    import numpy as np

    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        ncell = 1 << int(rng.integers(9, 14))
        n = 1 << int(rng.integers(18, 23))
        out.append((ncell, max(n, ncell), float(rng.uniform(0.05, 0.6)), i % 2 == 0))
    return out


def run_accuracy(dev, cfg, pb):
    """Time to the ion-wave end time T = macro_steps * Delta t, projective vs plain GPU PIC,
    and the relative L2 error of the coarse density (Section 4.1.1, Eq. errormeasures)."""
    import numpy as np
    import torch

    c = pb.make_config(cfg["ncell"], cfg["n_coarse"], cfg["K"], cfg["N"], cfg["L"], cfg["dt"], cfg["dT"],
                       qm=cfg["qm"], v_th=cfg["v_th"], wavelet=cfg["wavelet"], seed=11, sort_every=20,
                       newton_tol=1e-10)
    steps = cfg["macro_steps"]
    per = int(round(cfg["dT"] / cfg["dt"]))
    checks = sorted({max(1, steps // 5), steps // 2, steps})
    ef, ref = pb.Context(c, device=dev), pb.Context(c, device=dev)
    ef.load_initial(cfg["amplitude"])
    ref.load_initial(cfg["amplitude"])
    got = {}
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for m in range(1, steps + 1):
        ef.step()
        if m in checks:
            got[m] = ef.get_coarse()[0].clone()
    torch.cuda.synchronize(dev)
    t_proj = time.perf_counter() - t0
    want = {}
    t0 = time.perf_counter()
    done = 0
    for m in checks:
        ref.pic_steps((m - done) * per)
        done = m
        want[m] = ref.measure()[0].clone()
    torch.cuda.synchronize(dev)
    t_plain = time.perf_counter() - t0
    eps = {}
    for m in checks:
        a, b = got[m].cpu().numpy(), want[m].cpu().numpy()
        eps[str(round(m * cfg["dT"]))] = float(np.sqrt(np.sum((a - b) ** 2) / np.sum(a * a + b * b)))
    out = {"T_end": steps * cfg["dT"], "projective_s": t_proj, "plain_pic_s": t_plain,
           "speedup": t_plain / t_proj, "eps_coarse_density_at_T": eps,
           "status": [ef.sync_status(), ref.sync_status()]}
    runs = []
    # Haar-bin form with the slope filter: bursts of 20 and 10 at Delta t = 8, bursts of 20 at
    # Delta t = 10 and 20; the wavelet form of Section 3.3 (1-2-1 rule in x, 256 velocity cells
    # reduced by Coif4 to 64 coefficients, no filter) at Delta t = 8, 10 and 20
    wav = dict(n_v=256, n_v_coarse=64, ps_filter=0, wavelet="coif4")
    variants = [(cfg["K"], 8.0, {}), (cfg["K"] // 2, 8.0, {}), (cfg["K"], 10.0, {}), (cfg["K"], 20.0, {}),
                (cfg["K"], 8.0, wav), (cfg["K"], 10.0, wav), (cfg["K"] // 2, 10.0, wav), (cfg["K"], 20.0, wav)]
    for K, dT, kw in variants:
        ps = run_phase_space(dev, cfg, pb, want, checks, K=K, dT=dT, **kw)
        ps["speedup_vs_plain_pic"] = t_plain / ps["seconds"]
        ps["eps_at_T_end_below_2pct"] = ps["eps_coarse_density_at_T"][str(round(steps * cfg["dT"]))] <= 0.02
        runs.append(ps)
    for kk in ((0, 0, 8), (5, cfg["K"], 32)):  # adaptive Delta t; adaptive Delta t and burst length
        ad = run_phase_space_adaptive(dev, cfg, pb, want, [m for m in checks if m in (steps // 5, steps)],
                                      K_min=kk[0], K_max=kk[1], M_max=kk[2])
        ad["speedup_vs_plain_pic"] = t_plain / ad["seconds"]
        ad["eps_at_T_end_below_2pct"] = ad["eps_coarse_density_at_T"][str(round(steps * cfg["dT"]))] <= 0.02
        runs.append(ad)
    out["phase_space"] = runs
    # the ion pressure active (Section 3.2, EFREE's n, V, P): three nodal moments, lifting at the
    # local temperature, bursts of K at Delta t = 20, 10 and 8
    out["pressure"] = [run_pressure(dev, cfg, pb, want, checks, dT=dT) for dT in (cfg["dT"], 10.0, 8.0)]
    for r in out["pressure"]:
        r["speedup_vs_plain_pic"] = t_plain / r["seconds"]
        r["eps_at_T_end_below_2pct"] = r["eps_coarse_density_at_T"][str(round(steps * cfg["dT"]))] <= 0.02
    return out, want, checks


def run_pressure(dev, cfg, pb, want, checks, dT=20.0, K=None):
    """The moment variable with the ion pressure active (coarse kind moments_pressure): density,
    momentum and second-moment coefficients projected, Maxwellians of the local temperature at
    each lift; timed to the end time and compared with the resolved states `want` (coarse
    density, Section 4.1.1) at the check times this macro step lands on."""
    import torch

    K = K or cfg["K"]
    c = pb.make_config(cfg["ncell"], cfg["n_coarse"], K, cfg["N"], cfg["L"], cfg["dt"], dT, qm=cfg["qm"],
                       v_th=cfg["v_th"], wavelet=cfg["wavelet"], seed=11, newton_tol=1e-10, coarse="moments_pressure")
    ctx = pb.Context(c, device=dev)
    ctx.load_initial(cfg["amplitude"])
    checks = [m for m in checks if abs((m * cfg["dT"] / dT) - round(m * cfg["dT"] / dT)) < 1e-9]
    targets = {m: m * cfg["dT"] for m in checks}
    got, t, wall = {}, 0.0, 0.0
    for m in checks:
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        while t < targets[m] - 1e-9:
            ctx.step()
            t += dT
        torch.cuda.synchronize(dev)
        wall += time.perf_counter() - t0
        got[m] = ctx.get_coarse()[0].cpu().numpy()
    T_end = cfg["macro_steps"] * cfg["dT"]
    eps = {str(round(targets[m])): _eps(got[m], want[m].cpu().numpy()) for m in checks}
    return {"coarse": "moments + ion pressure", "dT": dT, "K": K, "T_end": T_end, "seconds": wall,
            "sim_time_per_wall_s": T_end / wall, "eps_coarse_density_at_T": eps, "status": ctx.sync_status()}


def run_phase_space(dev, cfg, pb, want, checks, dT=8.0, n_v=64, v_max=8.0, ps_filter=3, K=None, n_v_coarse=0,
                    wavelet="haar"):
    """The paper's own coarse variable (Section 3.3): masses of n_coarse x n_v phase-space
    cells (n_v_coarse = 0), or the wavelet form (n_v fine velocity cells reduced to n_v_coarse
    coefficients, coarse nodes in x), co-moving restriction, projective step (slope filter
    ps_filter), Appendix C lifting; timed to the end time and compared with the resolved
    states `want` (coarse density, Section 4.1.1)."""
    import numpy as np
    import torch

    nc, ncell = cfg["n_coarse"], cfg["ncell"]
    K = K or cfg["K"]
    c = pb.make_config(ncell, nc, K, cfg["N"], cfg["L"], cfg["dt"], dT, qm=cfg["qm"], v_th=cfg["v_th"],
                       seed=11, newton_tol=1e-10, coarse="phase_space", n_v=n_v, v_max=v_max, ps_filter=ps_filter,
                       n_v_coarse=n_v_coarse, wavelet=wavelet)
    ctx = pb.Context(c, device=dev)
    ctx.load_initial(cfg["amplitude"])
    b = int(np.log2(ncell // nc))
    scale = 2.0 ** (-(np.log2(ncell) + b) / 2)  # bin mass -> Haar density coefficient

    def density(coarse):
        d = coarse.sum(1).cpu().numpy()
        if n_v_coarse == 0:
            return d * scale
        # wavelet form: node values (mass per fine node) -> the lifted profile, linear between
        # coarse nodes (Eq. interpolation) -> sums over the resolved run's bins of 2^b nodes
        phi = np.arange(1 << b) / float(1 << b)
        fine = (1 - phi)[None, :] * d[:, None] + phi[None, :] * np.roll(d, -1)[:, None]
        return fine.sum(1) * scale
    T_end = cfg["macro_steps"] * cfg["dT"]
    # compare at the resolved-run check times that this macro step lands on exactly
    checks = [m for m in checks if abs((m * cfg["dT"] / dT) - round(m * cfg["dT"] / dT)) < 1e-9]
    if cfg["macro_steps"] not in checks:
        raise ValueError("the phase-space macro step must divide the end time")
    targets = {m: m * cfg["dT"] for m in checks}
    got, t, wall = {}, 0.0, 0.0
    for m in checks:
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        while t < targets[m] - 1e-9:
            ctx.step()
            t += dT
        torch.cuda.synchronize(dev)
        wall += time.perf_counter() - t0
        got[m] = density(ctx.get_coarse())
    eps = {str(round(targets[m])): _eps(got[m], want[m].cpu().numpy()) for m in checks}
    form = ("wavelet form, %s in v: %d cells -> %d coefficients, 1-2-1 rule in x" % (wavelet, n_v, n_v_coarse)
            if n_v_coarse else "Haar bins x %d velocity cells" % n_v)
    return {"form": form, "dT": dT, "K": K, "M": dT / (K * cfg["dt"]), "n_v": n_v, "v_max": v_max,
            "slope_filter": ps_filter,
            "T_end": T_end, "seconds": wall, "sim_time_per_wall_s": T_end / wall, "eps_coarse_density_at_T": eps,
            "status": ctx.sync_status()}


def run_phase_space_adaptive(dev, cfg, pb, want, checks, tol=1e-2, M_max=8, K=None, K_min=0, K_max=0):
    """The phase-space run with the curvature-controlled macro step (pe_step_adaptive): Delta t
    in whole bursts of K steps between K dt and M_max K dt, landing on the check times; timed to
    the end time and compared with the resolved states `want` as run_phase_space does."""
    import numpy as np
    import torch

    nc, ncell = cfg["n_coarse"], cfg["ncell"]
    K = K or cfg["K"]
    Kdt = K * cfg["dt"]
    c = pb.make_config(ncell, nc, K, cfg["N"], cfg["L"], cfg["dt"], 4 * Kdt, qm=cfg["qm"], v_th=cfg["v_th"],
                       seed=11, newton_tol=1e-10, coarse="phase_space", n_v=64, v_max=8.0, ps_filter=3)
    ctx = pb.Context(c, device=dev)
    ctx.load_initial(cfg["amplitude"])
    b = int(np.log2(ncell // nc))
    scale = 2.0 ** (-(np.log2(ncell) + b) / 2)
    got, t, wall, steps, rejected, dT_next = {}, 0.0, 0.0, 0, 0, 4 * Kdt
    dts, Ks = [], []
    for m in checks:
        T = m * cfg["dT"]
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        while t < T - 1e-9:
            if dT_next > T - t + 1e-9:  # land on the check time (a whole number of bursts away)
                ctx.set_macro_step(T - t)
            st = ctx.step_adaptive(tol=tol, M_min=1, M_max=M_max, safety=0.8, grow=2.0, K_min=K_min, K_max=K_max)
            t += st["dT"]
            dT_next = st["dT_next"]
            steps += 1
            rejected += st["rejected"]
            dts.append(st["dT"])
            Ks.append(st["K"])
        torch.cuda.synchronize(dev)
        wall += time.perf_counter() - t0
        got[m] = (ctx.get_coarse().sum(1) * scale).cpu().numpy()
    eps = {str(round(m * cfg["dT"])): _eps(got[m], want[m].cpu().numpy()) for m in checks}
    T_end = cfg["macro_steps"] * cfg["dT"]
    return {"dT": "adaptive", "tol": tol, "K": K if not K_max else "adaptive %d..%d" % (K_min, K_max),
            "mean_K": float(np.mean(Ks)), "M_max": M_max, "T_end": T_end, "seconds": wall,
            "macro_steps": steps, "rejected": rejected, "mean_dT": float(np.mean(dts)), "max_dT": float(np.max(dts)),
            "sim_time_per_wall_s": T_end / wall, "eps_coarse_density_at_T": eps, "status": ctx.sync_status()}


def _eps(a, b):
    import numpy as np

    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(a * a + b * b)))


def run_slab(dev, pb, variants=(("phase_space", 6.0, 30), ("phase_space", 6.0, 20), ("phase_space", 6.0, 15))):
    """Slab expansion into vacuum (bounded grid, absorbing walls): projective steps with the
    moment coarse variables (the workload's K = 30, M = 8), then with the phase-space variable
    at the given (Delta t, K), against plain GPU PIC to the same end time: time to solution and
    the coarse-density error (Section 4.1.1's measure) at three times."""
    import numpy as np
    import torch

    from paper_1610_01071_gb300 import inputs

    w = inputs.workload("slab")
    steps = w["macro_steps"]
    T_end = steps * w["dT"]

    def make(coarse="moments", dT=None, K=None):
        return pb.make_config(w["ncell"], w["n_coarse"], K or w["K"], w["N"], w["L"], w["dt"], dT or w["dT"],
                              qm=w["qm"], v_th=w["v_th"], wavelet=w["wavelet"], seed=21, sort_every=20,
                              newton_tol=1e-10, newton_maxit=80, boundary="absorbing", coarse=coarse, n_v=64,
                              v_max=8.0, ps_filter=3)

    checks_t = [T_end / 5, T_end / 2, T_end]
    ref = pb.Context(make(), device=dev)
    ref.load_initial(profile="slab")
    q0 = ref.moments()["charge"]
    want, t0, done = {}, time.perf_counter(), 0
    for T in checks_t:
        n = int(round(T / w["dt"]))
        ref.pic_steps(n - done)
        done = n
        want[T] = ref.measure()[0].clone()
    torch.cuda.synchronize(dev)
    t_plain = time.perf_counter() - t0
    q_ref = ref.moments()["charge"]

    def run(coarse, dT, K):
        ctx = pb.Context(make(coarse, dT, K), device=dev)
        ctx.load_initial(profile="slab")
        b = int(np.log2(w["ncell"] // w["n_coarse"]))
        scale = 2.0 ** (-(np.log2(w["ncell"]) + b) / 2)  # bin mass -> Haar density coefficient
        got, t, wall = {}, 0.0, 0.0
        kind = "push_sample_ps" if coarse == "phase_space" else "push_sample"
        ctx.profile_read_kinds()
        ctx.profile(True, kinds=(kind,))  # the fused pass of the bursts, for its roofline
        for T in checks_t:
            torch.cuda.synchronize(dev)
            t1 = time.perf_counter()
            while t < T - 1e-9:
                ctx.step()
                t += dT
            torch.cuda.synchronize(dev)
            wall += time.perf_counter() - t1
            c = ctx.get_coarse()
            got[T] = (c.sum(1) * scale if coarse == "phase_space" else c[0]).cpu().numpy()
        ctx.profile(False)
        pk = ctx.profile_read_kinds()[kind]
        eps = {str(round(T)): _eps(got[T], want[T].cpu().numpy()) for T in checks_t}
        ctx.lift()
        return {"coarse": coarse, "dT": dT, "K": K, "M": dT / (K * w["dt"]), "seconds": wall,
                "pass_kind": kind, "pass_ms": pk["ms"] / max(pk["launches"], 1), "pass_launches": pk["launches"],
                "speedup_vs_plain_pic": t_plain / wall,
                "particle_steps_per_s": float(w["N"]) * K * round(T_end / dT) / wall,
                "eps_coarse_density_at_T": eps, "charge_left": ctx.moments()["charge"] / q0,
                "status": ctx.sync_status()}

    runs = [run("moments", w["dT"], w["K"])] + [run(*v) for v in variants]
    return {"workload": "slab expansion: bounded 8192 cells, absorbing walls, uniform slab on the central "
                        "eighth, 2^25 equal-weight ions, v_th=1, K=30, M=8, 40 macro steps, 512 coarse per moment",
            "T_end": T_end, "plain_pic_s": t_plain,
            "plain_pic_particle_steps_per_s": float(w["N"]) * round(T_end / w["dt"]) / t_plain,
            "charge_left_plain_pic": q_ref / q0, "status_plain_pic": ref.sync_status(), "projective": runs}


def run_kinetic(dev, pb, per_reset=150):
    """Kinetic electrons (Section 4.1: both species as particles, q_e/m_e = -1800, dt resolving
    the electron plasma period): phase-space projective integration against plain two-species
    GPU PIC to the same end time, and against plain PIC whose electrons are reloaded in
    Boltzmann equilibrium with the ions every 150 steps (the paper's reset runs): time to
    solution and the coarse-density error (Section 4.1.1) at a third, two thirds and the end."""
    import numpy as np
    import torch

    from paper_1610_01071_gb300 import inputs

    w = inputs.workload("iaw_kinetic")
    steps, per = w["macro_steps"], int(round(w["dT"] / w["dt"]))
    T_end = steps * w["dT"]
    checks = [steps // 3, 2 * steps // 3, steps]

    def make(coarse="phase_space", reset=0, te_active=False):
        return pb.make_config(w["ncell"], w["n_coarse"], w["K"], w["N"], w["L"], w["dt"], w["dT"], qm=w["qm"],
                              v_th=w["v_th"], seed=11, sort_every=20, newton_tol=1e-10, coarse=coarse, n_v=w["n_v"],
                              v_max=w["v_max"], ps_filter=3, electrons="kinetic", qm_e=w["qm_e"],
                              reset_every=reset, te_active=te_active)

    wants, plain = {}, {}
    for reset in (0, per_reset):
        ref = pb.Context(make("moments", reset), device=dev)
        ref.load_initial(w["amplitude"])
        want, done = {}, 0
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for m in checks:
            ref.pic_steps((m - done) * per)
            done = m
            want[m] = ref.measure()[0].clone()
        torch.cuda.synchronize(dev)
        plain[reset] = {"seconds": time.perf_counter() - t0, "status": ref.sync_status()}
        wants[reset] = want
    t_plain = plain[0]["seconds"]
    b = int(np.log2(w["ncell"] // w["n_coarse"]))
    scale = 2.0 ** (-(np.log2(w["ncell"]) + b) / 2)  # bin mass -> Haar density coefficient
    key = {m: str(round(m * w["dT"])) for m in checks}

    def projective(te_active):
        ctx = pb.Context(make(te_active=te_active), device=dev)
        ctx.load_initial(w["amplitude"])
        got, wall, done = {}, 0.0, 0
        for m in checks:
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for _ in range(m - done):
                ctx.step()
            done = m
            torch.cuda.synchronize(dev)
            wall += time.perf_counter() - t0
            got[m] = (ctx.get_coarse().sum(1) * scale).cpu().numpy()
        return got, wall, ctx.sync_status(), ctx.diagnostics().T_e

    got, wall, status, _ = projective(False)
    got_te, wall_te, status_te, te_end = projective(True)
    eps_plain = {key[m]: _eps(got[m], wants[0][m].cpu().numpy()) for m in checks}
    eps_reset = {key[m]: _eps(got[m], wants[per_reset][m].cpu().numpy()) for m in checks}
    eps_pic = {key[m]: _eps(wants[per_reset][m].cpu().numpy(), wants[0][m].cpu().numpy()) for m in checks}
    particles = 2.0 * w["N"]
    return {"workload": "iaw_kinetic: periodic 1024 cells (L=288), 2^23 ions + 2^23 electrons (q/m -1800), "
                        "amplitude 0.2, dt=0.25/omega_pe, K=30 per macro step of 150 dt, 325 macro steps, "
                        "256 x-bins x 64 velocity cells",
            "T_end": T_end, "fine_steps_plain": steps * per, "plain_pic_s": t_plain,
            "plain_pic_particle_steps_per_s": particles * steps * per / t_plain,
            "plain_pic_reset_s": plain[per_reset]["seconds"], "reset_every": per_reset,
            "projective": {"coarse": "phase_space", "dT": w["dT"], "K": w["K"], "seconds": wall,
                           "speedup_vs_plain_pic": t_plain / wall,
                           "particle_steps_per_s": particles * w["K"] * steps / wall,
                           "eps_vs_plain_pic": eps_plain, "eps_vs_reset_pic": eps_reset,
                           "status": status},
            "projective_electron_energy_active": {
                "coarse": "phase_space + electrons' kinetic energy", "seconds": wall_te,
                "speedup_vs_plain_pic": t_plain / wall_te, "T_e_at_end": te_end,
                "eps_vs_plain_pic": {key[m]: _eps(got_te[m], wants[0][m].cpu().numpy()) for m in checks},
                "eps_vs_reset_pic": {key[m]: _eps(got_te[m], wants[per_reset][m].cpu().numpy()) for m in checks},
                "status": status_te},
            "eps_reset_pic_vs_plain_pic": eps_pic,
            "status_plain_pic": [plain[0]["status"], plain[per_reset]["status"]]}


def run_surrogate(dev, cfg, pb, want, checks):
    """The learned coarse-derivative surrogate on the ion-wave workload: 2^16 training pairs
    (c at the start of a macro step, that step's least-squares slope) from 1024 realisations
    of the 4096-cell wave (2^20 ions each, amplitudes uniform in 0.05..0.6, own seeds) advanced
    64 macro steps each, 64 at a time by pe_batch; training on the GPU (tcgen05 GEMMs, batches
    augmented by circular shifts of the coarse coefficients), then the gated surrogate run
    (probe burst of 5 steps) against the projective run with bursts of K and of 5 steps, each
    timed to the end time and compared with the resolved plain-PIC states `want`."""
    import numpy as np
    import torch

    ncell, nc, K = cfg["ncell"], cfg["n_coarse"], cfg["K"]
    n = 2 * nc
    steps = cfg["macro_steps"]
    n_real, per_batch, msteps, n_ions = 1024, 64, 64, 1 << 20
    rng = np.random.default_rng(17)
    X = torch.empty((n_real * msteps, n), dtype=torch.float32, device=dev)
    Y = torch.empty_like(X)
    row = 0
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for b in range(n_real // per_batch):
        ctxs = []
        for r in range(per_batch):
            c = pb.make_config(ncell, nc, K, n_ions, cfg["L"], cfg["dt"], cfg["dT"], qm=cfg["qm"], v_th=cfg["v_th"],
                               seed=100000 + b * per_batch + r, newton_tol=1e-10)
            ctx = pb.Context(c, device=dev)
            ctx.load_initial(float(rng.uniform(0.05, 0.6)))
            ctxs.append(ctx)
        batch = pb.Batch(ctxs)
        cv = [ctx.view("coarse", torch.float64, n) for ctx in ctxs]
        sv = [ctx.view("slope", torch.float64, n) for ctx in ctxs]
        for m in range(msteps):
            torch.cuda.synchronize(dev)
            X[row:row + per_batch] = torch.stack(cv).float()
            batch.step()
            torch.cuda.synchronize(dev)
            Y[row:row + per_batch] = torch.stack(sv).float()
            row += per_batch
        bad = [i for i, ctx in enumerate(ctxs) if ctx.sync_status() != 0]
        if bad:
            raise RuntimeError(f"device status set in training realisations {bad}")
        del batch, ctxs, cv, sv
    torch.cuda.synchronize(dev)
    t_data = time.perf_counter() - t0
    dims = [n, 512, 512, 512, n]
    B, n1, n2 = 2048, 2000, 1000
    stream = torch.cuda.Stream(dev)
    net = pb.MLP(dims, max_batch=B, device=dev, stream=stream)
    net.init(1)
    net.fit_norm(X, Y, nc)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    loss = net.train(X, Y, B, n1, 1e-3, seed=1, shift_period=nc)
    loss = net.train(X, Y, B, n2, 2e-4, seed=2, shift_period=nc)
    ev1.record(stream)
    stream.synchronize()
    if net.sync_status() != 0:
        raise RuntimeError("a tensor-core GEMM of the training timed out")
    nsteps = n1 + n2
    t_train = ev0.elapsed_time(ev1) / 1e3
    mm = sum(dims[l] * dims[l + 1] for l in range(len(dims) - 1))
    flops = nsteps * 2.0 * B * (2 * mm + (mm - dims[0] * dims[1]))  # forward, weight and data gradients
    tflops = flops / t_train / 1e12
    bf16_peak, bf16_kind = peak_bf16()

    def run(kind, Kb, tol=None):
        c = pb.make_config(ncell, nc, K if kind == "surrogate" else Kb, cfg["N"], cfg["L"], cfg["dt"], cfg["dT"], qm=cfg["qm"], v_th=cfg["v_th"],
                           seed=11, newton_tol=1e-10)
        ctx = pb.Context(c, device=dev)
        ctx.load_initial(cfg["amplitude"])
        got, fine, acc = {}, 0, 0
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for m in range(1, steps + 1):
            if kind == "surrogate":
                st = ctx.step_surrogate(net, K_probe=Kb, tol=tol, noise_sigmas=3.0)
                fine += st["fine_steps"]
                acc += st["accepted"]
            else:
                ctx.step()
                fine += Kb
            if m in checks:
                got[m] = ctx.get_coarse()[0].clone()
        torch.cuda.synchronize(dev)
        t = time.perf_counter() - t0
        eps = {str(round(m * cfg["dT"])): _eps(got[m].cpu().numpy(), want[m].cpu().numpy()) for m in checks}
        out = {"seconds": t, "fine_steps": fine, "eps_coarse_density_at_T": eps, "status": ctx.sync_status()}
        if kind == "surrogate":
            out["accepted"] = acc
            out["gate_tol"] = tol
        return out

    return {
        "network": "MLP %s, GELU, BF16 weights, FP32 accumulation, tcgen05 GEMMs" % "-".join(map(str, dims)),
        "training_pairs": int(X.shape[0]), "augmented_pairs": int(X.shape[0]) * nc, "data_seconds": t_data,
        "training_data": "%d realisations (2^20 ions, amplitude U(0.05, 0.6)) x %d macro steps, pe_batch" % (
            n_real, msteps),
        "train_steps": nsteps, "batch": B, "train_seconds": t_train, "final_loss": loss,
        "train_roofline": {"bound": "tensor", "achieved": tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                           "frac": tflops / bf16_peak, "peak_kind": bf16_kind},
        "projective_K%d" % K: run("efpi", K),
        "projective_K5": run("efpi", 5),
        "surrogate_probe5": run("surrogate", 5, 3e-3),
    }


def run_ensemble(dev, steps, warmup, rank=0):
    """64 realisations advanced by pe_batch (shared launches, replayed CUDA graph)."""
    import torch

    from paper_1610_01071_gb300 import _binding as pb

    K, M, dt = 20, 10, 0.1
    ctxs = []
    for i, (ncell, n, amp, slab) in enumerate(ensemble_sizes()):
        c = pb.make_config(ncell, min(256, ncell // 16), K, n, 0.5 * ncell, dt, M * K * dt, seed=7000 + 97 * i + rank,
                           newton_tol=1e-10, newton_maxit=80, boundary="absorbing" if slab else "periodic")
        ctx = pb.Context(c, device=dev)
        if slab:
            ctx.load_initial(profile="slab")
        else:
            ctx.load_initial(amp)
        ctxs.append(ctx)
    batch = pb.Batch(ctxs)
    t0 = time.perf_counter()
    chunk = batch.tune()
    tune_s = time.perf_counter() - t0
    shape = batch.tuned()
    for _ in range(warmup):
        batch.step()
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(batch.stream)
    for _ in range(steps):
        batch.step()
    ev1.record(batch.stream)
    torch.cuda.synchronize(dev)
    t = ev0.elapsed_time(ev1) / 1e3
    bad = [i for i, c in enumerate(ctxs) if c.sync_status() != 0]
    if bad:
        raise RuntimeError(f"device status set in realisations {bad}")
    total = sum(c.cfg.nparticles for c in ctxs)
    # ensemble groups: realisations of the same grid and initial-condition family, averaged
    groups = {}
    for i, (ncell, n, amp, slab) in enumerate(ensemble_sizes()):
        groups.setdefault((ncell, slab), []).append(i)
    means = {f"{'slab' if k[1] else 'sine'}_{k[0]}": batch.group_mean(v) for k, v in sorted(groups.items())}
    torch.cuda.synchronize(dev)
    return {"realisations": len(ctxs), "particles": int(total), "K": K, "steps": steps, "tuned_chunk": chunk,
            "tuned_shape": shape, "tune_seconds": tune_s,
            "groups": {f"{'slab' if k[1] else 'sine'}_{k[0]}": len(v) for k, v in sorted(groups.items())},
            "group_mean_density_sum": {k: float(m[0].sum().item()) for k, m in means.items()},
            "ms_per_step": 1e3 * t / steps, "seconds": t, "particle_steps": float(total) * K * steps}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--no-slab", action="store_true")
    ap.add_argument("--no-kinetic", action="store_true")
    ap.add_argument("--kernel", default=None, help="time one kernel alone (profiling mode)")
    args = ap.parse_args()
    if args.kernel:
        return run_kernel(args)
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
