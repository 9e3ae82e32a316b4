"""Batched ensemble (pe_batch_*): many realisations of different sizes advanced in
shared launches and a replayed CUDA graph must give the coarse states of each realisation
advanced alone with pe_step (to the Newton tolerance: the batch partitions its field solves
for throughput), and each realisation's coarse state must match the oracle's projective macro
step (Section 3.1 cycle) from the same particles. The autotuner and the group means too."""
import numpy as np
import pytest
import torch

import oracle as orc
import paper_1610_01071_gb300 as pe

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")

SIZES = [(512, 1 << 16), (1024, 1 << 17), (256, 1 << 14), (4096, 1 << 18), (2048, 1 << 16), (128, 1 << 12)]


def make(i, ncell, N, slab=False):
    K, M, dt = 6, 3, 0.1
    cfg = pe.make_config(ncell, 16, K, N, ncell * 0.5, dt, M * K * dt, v_th=1.0, seed=100 + i, newton_tol=1e-10,
                         newton_maxit=80, boundary="absorbing" if slab else "periodic")
    ctx = pe.Context(cfg, device=DEV)
    if slab:
        ctx.load_initial(profile="slab")
    else:
        ctx.load_initial(0.1 + 0.05 * i)
    return ctx


def close(ga, gb, rel=1e-8):
    return np.max(np.abs(ga - gb)) <= rel * np.max(np.abs(ga))


def test_batch_matches_individual_contexts():
    alone = [make(i, *s) for i, s in enumerate(SIZES)]
    group = [make(i, *s) for i, s in enumerate(SIZES)]
    batch = pe.Batch(group)
    for step in range(4):  # eager, captured, then replayed graph; tuning before the last
        if step == 3:
            assert batch.tune() in (16384, 32768, 65536)
        batch.step()
        for c in alone:
            c.step()
        for a, b in zip(alone, group):
            ga, gb = a.get_coarse().cpu().numpy(), b.get_coarse().cpu().numpy()
            assert close(ga, gb), f"step {step}: max diff {np.abs(ga - gb).max()}"
    for c in group:
        assert c.sync_status() == 0
        d = c.diagnostics()
        assert d.macro_steps == 4 and d.newton_iters >= 1


def test_batch_of_sinusoids_and_slabs_matches_individual_contexts():
    # the ensemble workload mixes periodic sinusoids and bounded slabs: the batch solves each
    # field with its context's precision (the Jacobian solve of the slabs as alone), pushes with
    # absorbing walls and lifts the slabs with equal weights, all bit for bit as alone
    sizes = [(512, 1 << 16, True), (1024, 1 << 17, False), (256, 1 << 14, True), (4096, 1 << 18, True),
             (2048, 1 << 16, False), (128, 1 << 12, True)]
    alone = [make(i, n, N, slab) for i, (n, N, slab) in enumerate(sizes)]
    group = [make(i, n, N, slab) for i, (n, N, slab) in enumerate(sizes)]
    batch = pe.Batch(group)
    for step in range(3):  # eager, captured, replayed
        batch.step()
        for c in alone:
            c.step()
        for k, (a, b) in enumerate(zip(alone, group)):
            ga, gb = a.get_coarse().cpu().numpy(), b.get_coarse().cpu().numpy()
            assert close(ga, gb), f"step {step}, realisation {k}: max diff {np.abs(ga - gb).max()}"
    for c in group:
        assert c.sync_status() == 0


def test_batch_matches_oracle_per_realisation():
    # a mixed ensemble (periodic sinusoids and bounded slabs of different sizes): one batched
    # macro step from the loaded particles, then a second one that lifts from the projected
    # coarse state, each realisation against the oracle's macro step (efpi_macro_step or its
    # bounded-grid form) at the tolerances of the single-context cycle tests
    sizes = [(256, 1 << 14, False), (512, 1 << 15, True), (128, 1 << 13, False), (256, 1 << 14, True)]
    group = [make(i, n, N, slab) for i, (n, N, slab) in enumerate(sizes)]
    states = [orc.State(*[x.cpu().numpy() for x in c.particles()]) for c in group]
    batch = pe.Batch(group)
    batch.step()
    got1 = [c.get_coarse().cpu().numpy() for c in group]
    batch.step()
    got2 = [c.get_coarse().cpu().numpy() for c in group]
    for i, ((ncell, N, slab), ctx, st) in enumerate(zip(sizes, group, states)):
        assert ctx.sync_status() == 0
        K, M, dt = 6, 3, 0.1
        ocfg = dict(ncell=ncell, n_coarse=16, K=K, L=ncell * 0.5, dt=dt, qm=1.0, dT=M * K * dt, N=N, v_th=1.0,
                    s_w=ctx.diagnostics().s_w)
        macro = orc.efpi_macro_step_walls if slab else orc.efpi_macro_step
        lift = orc.lift_walls if slab else orc.lift
        c1, _, phi = macro(st, ocfg, np.zeros(ncell))
        err1 = np.max(np.abs(got1[i] - c1)) / np.max(np.abs(c1))
        assert err1 < 1e-4, f"realisation {i}, step 1: {err1:.3e}"
        # lifting seed of macro step m: seed + 0x632BE59BD9B4E019 (m + 1)
        seed2 = (100 + i + 0x632BE59BD9B4E019 * 2) % 2**64
        c2, _, _ = macro(lift(c1, ocfg, seed2), ocfg, phi)
        err2 = np.max(np.abs(got2[i] - c2)) / np.max(np.abs(c2))
        assert err2 < 2e-4, f"realisation {i}, step 2: {err2:.3e}"


def test_batch_tuner_shapes_and_cache():
    group = [make(i, *s) for i, s in enumerate(SIZES)]
    b1 = pe.Batch(group)
    chunk = b1.tune()
    t1 = b1.tuned()
    assert t1["chunk"] == chunk and t1["block"] in (128, 256, 512) and isinstance(t1["privatised"], bool)
    b1.step()
    b1.step()  # the tuned shape runs (eager, then captured)
    for c in group:
        assert c.sync_status() == 0
    # a second batch of the same composition takes the cached shape
    again = [make(i + 50, *s) for i, s in enumerate(SIZES)]
    b2 = pe.Batch(again)
    assert b2.tune() == chunk and b2.tuned() == t1


def test_batch_tuner_leaves_the_particles_unchanged():
    # the tuner times the burst's fused pass with a frozen step (dt/dx = 0, kick 0): every particle
    # is rewritten unchanged, periodic and bounded grids alike; a composition not tuned before
    sizes = [(512, 3 << 15, False), (1024, 5 << 14, True), (256, 3 << 13, False)]
    group = [make(i, n, N, slab) for i, (n, N, slab) in enumerate(sizes)]
    before = []
    for c in group:
        before.append([t.clone() for t in c.particles(c.diagnostics().particle_bank)])
    b = pe.Batch(group)
    b.tune()
    torch.cuda.synchronize(DEV)
    for c, ref in zip(group, before):
        for x, y in zip(c.particles(c.diagnostics().particle_bank), ref):
            assert torch.equal(x, y)
        assert c.sync_status() == 0
    b.step()  # the real descriptors are back: the step moves the particles
    for c, ref in zip(group, before):
        assert c.sync_status() == 0
        assert not torch.equal(c.particles(c.diagnostics().particle_bank)[1], ref[1])


def test_group_means_of_coarse_states():
    sizes = [(256, 1 << 14), (256, 1 << 14), (512, 1 << 15), (256, 1 << 14), (512, 1 << 15)]
    group = [make(i, n, N) for i, (n, N) in enumerate(sizes)]
    batch = pe.Batch(group)
    batch.step()
    states = [c.get_coarse().cpu().numpy() for c in group]
    for members in ([0, 1, 3], [2, 4], [3]):
        got = batch.group_mean(members)
        torch.cuda.synchronize()
        want = sum(states[m] for m in members) / len(members)  # summed in the members' order
        assert np.max(np.abs(got.cpu().numpy() - want)) <= 1e-15 * np.max(np.abs(want))
    with pytest.raises(pe.PepicError):  # not a realisation of the batch
        batch.group_mean([0, 7])


def test_batch_rejects_mixed_states():
    a, b = make(0, 256, 1 << 12), make(1, 512, 1 << 13)
    batch = pe.Batch([a, b])
    a.step()  # a alone moves on: the ensemble is no longer in one state
    with pytest.raises(pe.PepicError):
        batch.step()
