"""The tcgen05 BF16 GEMM (tensor-memory accumulator) against an FP64 host
product of the same BF16 values and against the mma.sync path."""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SHAPES = [(256, 256, 256), (300, 144, 448), (144, 432, 4096), (4096, 256, 192), (128, 16, 64)]


@pytest.fixture(scope="module")
def bbs():
    from paper_2308_08417_gb300 import _build, bbs as mod

    _build.build()
    return mod


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_tcgen05_gemm_matches_fp64(bbs, M, N, K):
    h = bbs.Handle(0)
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    ref = A.double() @ B.double().T
    # worst-case bound of an FP32 accumulation of K exact products
    bound = (A.double().abs() @ B.double().abs().T) * K * 2 ** -24 + 1e-30
    for kind in ("tcgen05", "mma"):
        C = bbs.bbs_gemm_bf16(h, kind, A.cuda(), B.cuda()).double().cpu()
        err = ((C - ref).abs() / bound).max().item()
        assert err <= 1.0, (kind, err)
