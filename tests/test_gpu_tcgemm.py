"""The surrogate's tensor-core GEMM (tcgen05, BF16 in, FP32 accumulate)
against a plain PyTorch FP32 matmul of the same BF16 operands, on the layer
shapes of the network (K = 16 first layer, 256 x 256 hidden layers, the
batch dimension as K for weight gradients) and ragged edges."""
import pytest

from paper_2408_00559_gb300 import _lib as B
from paper_2408_00559_gb300 import build as BLD

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    BLD.build()
    B.lib()


@pytest.mark.parametrize("M,N,K", [(128, 64, 16), (256, 256, 128), (200, 48, 64), (384, 512, 256),
                                   (256, 256, 1024), (128, 16, 32)])
def test_tc_gemm_matches_fp32_matmul(M, N, K):
    import torch
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    Bm = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C = torch.full((M, N), float("nan"), device="cuda", dtype=torch.float32)
    B.tc_gemm_bf16(A, Bm, C)
    ref = A.float() @ Bm.float().T
    err = (C - ref).abs().max().item()
    scale = ref.abs().max().item()
    assert err <= 1e-5 * scale * max(1.0, K / 64), (err, scale)
