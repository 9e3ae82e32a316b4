"""The tensor-core GEMM (tcgen05.mma with TMEM accumulators, TMA-staged operands) against an
FP64 product of the same BF16 inputs.

Tolerance: every BF16 x BF16 product is exact in FP32, so the difference is the FP32
accumulation over K: at most K u sum |a b| (u = 2^-24); the test allows 1e-4 of sum |a b| per
element, far below what a transposed operand, a wrong swizzle or a dropped K slice gives."""
import numpy as np
import pytest
import torch

from paper_1610_01071_gb300 import _binding as pb

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 512, 512), (1000, 320, 200), (1, 512, 512), (130, 64, 8),
                                   (4096, 512, 512), (512, 512, 4096)])
def test_tc_gemm_matches_the_fp64_product(M, N, K):
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn((M, K), generator=g).to(torch.bfloat16)
    B = torch.randn((N, K), generator=g).to(torch.bfloat16)
    C, st = pb.tc_gemm(A.to(DEV), B.to(DEV))
    assert int(st.item()) == 0
    a, b = A.double().numpy(), B.double().numpy()
    ref = a @ b.T
    bound = np.abs(a) @ np.abs(b).T
    err = np.abs(C.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= 1e-4 * bound + 1e-30), float((err / np.maximum(bound, 1e-30)).max())


def test_tc_gemm_refuses_bad_shapes():
    A = torch.zeros((64, 64), dtype=torch.bfloat16, device=DEV)
    with pytest.raises(RuntimeError):
        pb.tc_gemm(A, torch.zeros((48, 64), dtype=torch.bfloat16, device=DEV))  # N not a multiple of 64
    with pytest.raises(RuntimeError):
        pb.tc_gemm(torch.zeros((64, 12), dtype=torch.bfloat16, device=DEV),
                   torch.zeros((64, 12), dtype=torch.bfloat16, device=DEV))  # rows not 16-byte multiples
