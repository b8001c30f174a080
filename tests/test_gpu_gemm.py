"""The split-BF16 tensor-core GEMM (tcgen05) against an FP64 product of the same FP32 inputs.

Two BF16 planes per operand and the three leading products give about 2^-16
relative accuracy per product; the tolerance on the Frobenius error is 1e-4.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1803_08333_gb300 as rf  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1803_08333_gb300 import build

    build.build()


@pytest.mark.parametrize(
    "M,N,K",
    [
        (128, 128, 64),  # one tile, one K block
        (128, 128, 256),  # one tile, K blocks through the 3-stage ring
        (300, 200, 1000),  # ragged M, N and K tails
        (1024, 512, 2048),  # many tiles
    ],
)
def test_gemm_matches_fp64(M, N, K):
    g = torch.Generator().manual_seed(M + N + K)
    A = torch.randn((M, K), generator=g, dtype=torch.float32)
    B = torch.randn((N, K), generator=g, dtype=torch.float32)
    D = rf.gemm_bf16x3(A.cuda(), B.cuda()).cpu().double()
    ref = A.double() @ B.double().T
    err = (torch.linalg.norm(D - ref) / torch.linalg.norm(ref)).item()
    assert err <= 1e-4, err


def test_gemm_accumulates():
    g = torch.Generator().manual_seed(7)
    A = torch.randn((256, 192), generator=g)
    B = torch.randn((160, 192), generator=g)
    C = torch.randn((256, 160), generator=g)
    D = rf.gemm_bf16x3(A.cuda(), B.cuda(), C.cuda().clone(), accumulate=True).cpu().double()
    ref = A.double() @ B.double().T + C.double()
    assert (torch.linalg.norm(D - ref) / torch.linalg.norm(ref)).item() <= 1e-4
