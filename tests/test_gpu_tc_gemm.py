"""The tcgen05 BF16 GEMM against a plain FP64 matrix product of the same
BF16-rounded operands (products of BF16 values are exact in FP32; the only
difference is the FP32 accumulation order)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K,splits,pad", [(128, 64, 64, 1, 0), (128, 256, 64, 1, 0), (256, 256, 256, 1, 8),
                                              (128, 128, 512, 4, 0), (384, 64, 192, 3, 16), (256, 256, 4096, 8, 0)])
def test_tc_gemm_matches_fp64(fk, M, N, K, splits, pad):
    g = torch.Generator().manual_seed(M * 7 + N + K)
    A = torch.randn((M, K + pad), generator=g).to(torch.bfloat16)
    B = torch.randn((N, K + pad), generator=g).to(torch.bfloat16)
    Ad, Bd = A.cuda(), B.cuda()
    C = fk.fk_tc_gemm_bf16(Ad[:, :K], Bd[:, :K], splits).sum(0).cpu().numpy().astype(np.float64)
    want = A[:, :K].double().numpy() @ B[:, :K].double().numpy().T
    scale = np.abs(A[:, :K].double().numpy()) @ np.abs(B[:, :K].double().numpy()).T
    assert np.all(np.abs(C - want) <= 1e-5 * scale + 1e-6)
