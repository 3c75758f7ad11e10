"""The tcgen05 BF16 GEMM primitive against an FP32 matmul of the same BF16 inputs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (4096, 256, 400), (4096, 176, 256),
                                   (256, 400, 4096), (300, 200, 136), (128, 16, 8)])
def test_gemm_bf16_matches_fp32_matmul(M, N, K):
    import torch
    from paper_2408_10731_b300 import trajbatch as tb
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C = torch.full((M, N), float("nan"), device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    tb.gemm_bf16(A, B, C, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = A.double() @ B.double().T
    diff = (C.double() - ref).abs().max().item()
    assert diff <= 1e-4 * np.sqrt(K) * ref.abs().max().item() + 1e-3, diff
