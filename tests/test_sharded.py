"""One realisation's particles split over ranks (the multi-GPU particle decomposition), on
the CPU: the slices of the decomposition, and two gloo ranks that each deposit and push their
own slice of the oracle's Appendix C point set, with one exact int64 all-reduce of the charge
deposit per fine step and a redundant field solve, reproducing the single-rank run bit for bit
(integer sums do not depend on their order). No GPU needed."""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import oracle as orc  # noqa: E402
from paper_1610_01071_gb300.sharded import lift_seed, shard_range  # noqa: E402

NCELL, L, PPC, STEPS = 32, 16.0, 64, 6


@pytest.mark.parametrize("n_total", [4, 7, 4096, 4097, 1 << 20])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_ranges_partition_the_point_set(n_total, world):
    slices = [shard_range(n_total, world, r) for r in range(world)]
    pos = 0
    for first, n in slices:
        assert first == pos and n >= 0  # contiguous, in rank order
        assert first % 4 == 0 or n == 0  # 16-byte groups of four particles
        pos += n
    assert pos == n_total


def test_lift_seed_matches_the_context_rule():
    assert lift_seed(17, 1) == (17 + 0x632BE59BD9B4E019 * 2) % 2**64


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(rank, world):
    """Plain PIC steps of one realisation, this rank's slice of the particles; returns its final
    slice and the all-reduced deposits of every step."""
    N = NCELL * PPC
    dx = L / NCELL
    s_w = orc.fx_shift(8.0 * NCELL / N)
    nprof, uprof = orc.sine_profile(NCELL, L, 0.2)
    full = orc.quiet_start(N, NCELL, nprof.astype(np.float32), uprof.astype(np.float32), 1.0, 5)
    first, n = shard_range(N, world, rank)
    st = orc.State(full.cell[first:first + n], full.theta[first:first + n], full.v[first:first + n],
                   full.w[first:first + n])
    phi = np.zeros(NCELL)
    deposits = []
    for step in range(STEPS):
        rho = torch.from_numpy(orc.deposit_fx(st.cell, st.theta, st.w, NCELL, s_w))
        if world > 1:
            dist.all_reduce(rho, op=dist.ReduceOp.SUM)  # exact: int64
        deposits.append(rho.numpy().copy())
        phi, _, fail = orc.newton_pb(rho.numpy() * 2.0 ** -(s_w + 24), dx, phi0=phi, tol=1e-12)
        assert fail == 0
        orc.push(st, orc.efield(phi, dx), NCELL, dx, 0.1, 1.0, kick=0.5 if step == 0 else 1.0)
    return st, np.stack(deposits)


def _rank_main(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        st, dep = _run(rank, world)
        np.savez(os.path.join(outdir, f"rank{rank}.npz"), cell=st.cell, theta=st.theta, v=st.v, dep=dep)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_rank_run_bit_for_bit(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    parts = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    st1, dep1 = _run(0, 1)
    for p in parts:  # every rank holds the whole realisation's deposits
        assert np.array_equal(p["dep"], dep1)
    assert np.array_equal(np.concatenate([p["cell"] for p in parts]), st1.cell)
    assert np.array_equal(np.concatenate([p["theta"] for p in parts]), st1.theta)
    assert np.array_equal(np.concatenate([p["v"] for p in parts]), st1.v)
