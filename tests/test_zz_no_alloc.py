"""The allocation-free sort entry point (pe_sort_noalloc) against pe_sort.

pe_sort_noalloc exists for callers that cannot allocate device memory when they sort
(a host framework that owns every device allocation, a real-time loop that must not take
cudaMalloc's implicit synchronisation, a plugin handed only the particle buffers); its
counters live in a static device array of the library. This file is collected last so
that a run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import paper_1610_01071_gb300 as pe
from paper_1610_01071_gb300 import _binding as pb
from paper_1610_01071_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _canonical(c, t, v, w):
    order = np.lexsort((w, v, t, c))
    return c[order], t[order], v[order], w[order]


def _free_device_bytes():
    # cudaMemGetInfo's free bytes of the device (includes allocations made outside torch)
    return torch.cuda.mem_get_info(DEV)[0]


@pytest.mark.parametrize("ncell,N", [(64, 5003), (4096, (1 << 20) + 7)])
def test_sort_noalloc_matches_sort_twice(ncell, N):
    c, t, v, w = inputs.random_particles(N, ncell, seed=ncell + 17, sort=False)
    dc, dt, dv, dw = [torch.from_numpy(a).to(DEV) for a in (c, t, v, w)]
    ref = [x.cpu().numpy() for x in pe.sort(dc, dt, dv, dw, ncell)]
    out = (torch.empty_like(dc), torch.empty_like(dt), torch.empty_like(dv), torch.empty_like(dw))
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    pb.sort_noalloc(dc, dt, dv, dw, ncell, status=st, out=out)  # first call: module and symbol set-up
    torch.cuda.synchronize()
    for _ in range(2):  # two more calls in a row: the shared counters must be cleared each time
        st.zero_()
        alloc0, free0 = torch.cuda.memory_allocated(DEV), _free_device_bytes()
        pb.sort_noalloc(dc, dt, dv, dw, ncell, status=st, out=out)
        torch.cuda.synchronize()
        # nothing was allocated: not through torch, not by the library behind torch's back
        assert torch.cuda.memory_allocated(DEV) == alloc0
        assert _free_device_bytes() >= free0
        got = [x.cpu().numpy() for x in out]
        assert int(st.item()) == 0
        assert np.all(np.diff(got[0]) >= 0)
        for a, b in zip(_canonical(*ref), _canonical(*got)):
            assert np.array_equal(a, b)  # the same particles, bit for bit


def test_sort_noalloc_rejects_grids_beyond_its_static_size():
    c, t, v, w = inputs.random_particles(100, 64, seed=1)
    dc, dt, dv, dw = [torch.from_numpy(a).to(DEV) for a in (c, t, v, w)]
    with pytest.raises(pb.PepicError):
        pb.sort_noalloc(dc, dt, dv, dw, 16384)
