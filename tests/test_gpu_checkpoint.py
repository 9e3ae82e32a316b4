"""Checkpoint and resume between macro steps (pe_checkpoint_*): a context restored from a
checkpoint continues bit for bit as the original does, for the moment and phase-space coarse
variables and with kinetic electrons; images of another configuration or of a context whose
particles are the state are refused."""
import numpy as np
import pytest
import torch

import paper_1610_01071_gb300 as pe

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def make(coarse="moments", electrons="boltzmann", ncell=128, seed=9):
    K, dt = (6, 0.25 / np.sqrt(1800.0)) if electrons == "kinetic" else (10, 0.1)
    c = pe.make_config(ncell, 16, K, ncell * 128, ncell * 0.5, dt, 3 * K * dt, v_th=1.0, seed=seed,
                       newton_tol=1e-11, coarse=coarse, n_v=32, v_max=6.0,
                       ps_filter=3 if coarse == "phase_space" else 0, electrons=electrons)
    ctx = pe.Context(c, device=DEV)
    ctx.load_initial(0.2)
    return ctx


@pytest.mark.parametrize("coarse,electrons", [("moments", "boltzmann"), ("phase_space", "boltzmann"),
                                              ("phase_space", "kinetic")])
def test_resumed_context_continues_bit_for_bit(coarse, electrons):
    a = make(coarse, electrons)
    for _ in range(3):
        a.step()
    image = a.checkpoint()
    for _ in range(2):
        a.step()
    b = make(coarse, electrons, seed=9)
    b.restore(image)
    for _ in range(2):
        b.step()
    assert np.array_equal(a.get_coarse().cpu().numpy(), b.get_coarse().cpu().numpy())
    da, db = a.diagnostics(), b.diagnostics()
    assert (da.macro_steps, da.fine_steps, da.time) == (db.macro_steps, db.fine_steps, db.time)
    assert a.sync_status() == 0 and b.sync_status() == 0


def test_checkpoints_are_refused_where_they_cannot_resume():
    a = make()
    with pytest.raises(pe.PepicError):  # just loaded: the particles are the state
        a.checkpoint()
    a.step()
    image = a.checkpoint()
    other = make(ncell=256)
    with pytest.raises(pe.PepicError):  # another grid
        other.restore(image)
    with pytest.raises(pe.PepicError):  # the same grid but another seed: another trajectory
        make(seed=10).restore(image)
    bad = bytearray(image)
    bad[0] ^= 0xFF
    with pytest.raises(pe.PepicError):  # not an image
        make().restore(bytes(bad))
    # a valid header with an impossible clock: header fields at byte offsets 12 (phi history
    # flag, int32), 32 (fine steps, int64) and 40 (time, float64)
    import struct

    for off, fmt, val in ((12, "<i", 2), (32, "<q", -1), (40, "<d", float("nan")), (40, "<d", -1.0)):
        bad = bytearray(image)
        struct.pack_into(fmt, bad, off, val)
        with pytest.raises(pe.PepicError):
            make().restore(bytes(bad))
    make().restore(image)  # the untouched image still loads
    a.pic_steps(3)
    with pytest.raises(pe.PepicError):  # advanced by plain PIC: the particles are the state again
        a.checkpoint()
