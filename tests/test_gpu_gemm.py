"""The split-BF16 tensor-core GEMM (tcgen05) against an FP64 product of the same FP32 inputs.

Two BF16 planes per operand and the three leading products give about 2^-16
relative accuracy per product; the tolerance on the Frobenius error is 1e-4.  The kernel is
persistent (one CTA per SM taking every G-th tile, two tensor-memory accumulators): shapes with
more tiles than SMs check the hand-over between tiles.
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
        (4096, 2048, 320),  # 512 tiles: several per persistent CTA, both accumulators reused
        (600, 20, 700),  # 32-column tiles, ragged
        (700, 60, 900),  # 64-column tiles, ragged
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


def test_gemm_accumulates_over_many_tiles():
    g = torch.Generator().manual_seed(11)
    A = torch.randn((2048, 256), generator=g)
    B = torch.randn((1536, 256), generator=g)
    C = torch.randn((2048, 1536), generator=g)
    D = rf.gemm_bf16x3(A.cuda(), B.cuda(), C.cuda().clone(), accumulate=True).cpu().double()
    ref = A.double() @ B.double().T + C.double()
    assert (torch.linalg.norm(D - ref) / torch.linalg.norm(ref)).item() <= 1e-4
    # every element written: no tile skipped or written twice
    D2 = rf.gemm_bf16x3(A.cuda(), B.cuda(), torch.zeros_like(C).cuda(), accumulate=True).cpu().double()
    assert (torch.linalg.norm(D2 - (ref - C.double())) / torch.linalg.norm(ref - C.double())).item() <= 1e-4
