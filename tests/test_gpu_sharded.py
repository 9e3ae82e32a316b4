"""One realisation split into slices of its particles (the multi-GPU decomposition, here on
one GPU): the slices of Appendix C's point set load exactly as the whole set does, and
projective macro steps with the deposits and samples of several slices summed exactly give,
bit for bit, the coarse state of the unsplit run; that run matches the oracle's macro step."""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_1610_01071_gb300 import _binding as pb
from paper_1610_01071_gb300.sharded import ShardedRealisation, shard_range

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("ncell,N,parts", [(64, 64 * 128, 3), (4096, 1 << 20, 5), (128, 128 * 64, 2)])
def test_quiet_start_slices_load_the_whole_point_set(ncell, N, parts):
    prof_n = torch.linspace(0.5, 1.5, ncell, device=DEV, dtype=torch.float32)
    prof_u = torch.linspace(-0.2, 0.3, ncell, device=DEV, dtype=torch.float32)
    s_w = 22 - int(np.ceil(np.log2(8.0 * ncell / N)))
    full = pb.quiet_start(N, ncell, prof_n, prof_u, 1.0, 9, s_w)
    rho_sum = torch.zeros(ncell, dtype=torch.int64, device=DEV)
    pieces = []
    for r in range(parts):
        first, n = shard_range(N, parts, r)
        cell = torch.empty(n, dtype=torch.int32, device=DEV)
        th, v, w = (torch.empty(n, dtype=torch.float32, device=DEV) for _ in range(3))
        rho = torch.empty(ncell, dtype=torch.int64, device=DEV)
        st = torch.zeros(1, dtype=torch.int32, device=DEV)
        pb.check(pb.load().pe_quiet_start_slice(pb._ptr(cell), pb._ptr(th), pb._ptr(v), pb._ptr(w), first, n, N, ncell,
                                                 pb._ptr(prof_n), pb._ptr(prof_u), 1.0, 9, s_w, pb._ptr(rho),
                                                 pb._ptr(st), pb._stream()), "pe_quiet_start_slice")
        assert int(st.item()) == 0
        pieces.append((cell, th, v, w))
        rho_sum += rho
    for k in range(4):
        got = torch.cat([p[k] for p in pieces])
        assert torch.equal(got, full[k])
    assert torch.equal(rho_sum, full[4])


def test_quiet_start_slice_rejects_ranges_outside_the_point_set():
    x = torch.empty(64, dtype=torch.float32, device=DEV)
    c = torch.empty(64, dtype=torch.int32, device=DEV)
    prof = torch.ones(64, dtype=torch.float32, device=DEV)
    for first, n, total in ((-4, 16, 64), (56, 16, 64), (0, 0, 64), (0, 16, 63)):
        rc = pb.load().pe_quiet_start_slice(pb._ptr(c), pb._ptr(x), pb._ptr(x), pb._ptr(x), first, n, total, 64,
                                            pb._ptr(prof), pb._ptr(prof), 1.0, 1, 20, None, None, pb._stream())
        assert rc == pb.PE_EINVAL


def make(local_shards, seed=3):
    return ShardedRealisation(256, 16, 8, 256 * 128, 128.0, 0.1, 3.2, seed=seed, device=DEV,
                              local_shards=local_shards)


def test_split_realisation_equals_the_unsplit_one_bit_for_bit():
    runs = [make(k) for k in (1, 3, 7)]
    for r in runs:
        r.load_initial(0.2)
    for step in range(3):  # the first from the load, the next two lifted from the projection
        for r in runs:
            r.step()
        ref = runs[0].coarse.cpu().numpy()
        for r in runs[1:]:
            assert np.array_equal(r.coarse.cpu().numpy(), ref), f"step {step}, {len(r.shards)} shards"
    for r in runs:
        assert r.sync_status() == 0


def test_split_realisation_macro_step_matches_oracle():
    r = make(4)
    r.load_initial(0.2)
    parts = [[s[k].cpu().numpy() for k in ("cell", "theta", "v", "w")] for s in r.shards]
    st = orc.State(*[np.concatenate([p[k] for p in parts]) for k in range(4)])
    r.step()
    got = r.coarse.cpu().numpy()
    assert r.sync_status() == 0
    ocfg = dict(ncell=256, n_coarse=16, K=8, L=128.0, dt=0.1, qm=1.0, dT=3.2, s_w=r.s_w)
    want, _, _ = orc.efpi_macro_step(st, ocfg, np.zeros(256))
    assert np.max(np.abs(got - want)) < 1e-4 * np.max(np.abs(want))
