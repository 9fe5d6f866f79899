"""GPU: rq_gemm_bf16, C = A B with bfloat16-rounded inputs and FP32
accumulation (the mixed-precision sketch's product), against the FP64
product of the bfloat16-rounded inputs.

Every product of two bfloat16 values is exact in FP32, so the only error is
the FP32 accumulation: at most K u |A_bf16| |B_bf16| for an accumulation of
K terms (u = 2^-24; the tensor-core path adds chunks of at most 1024 and the
tensor core's own adds truncate), checked elementwise with the chunk length
in place of K, plus a median error far below it.  The shapes cover the
sketch's (72 rows, K split into chunks), ragged tiles, and a leading dimension
that is not a multiple of 4 (the CUDA-core path).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from gpu_util import build_and_handle
    return build_and_handle()


@pytest.mark.parametrize("M,N,K", [(72, 1000, 3000), (256, 300, 512), (130, 257, 64), (9, 5, 1)])
def test_gemm_bf16_matches_the_fp64_product_of_rounded_inputs(H, M, N, K):
    import torch
    from paper_2008_04447_gb300 import colmajor
    g = torch.Generator(device="cpu")
    g.manual_seed(M + N + K)
    A = colmajor(torch.randn((M, K), generator=g, dtype=torch.float32)).cuda()
    B = colmajor(torch.randn((K, N), generator=g, dtype=torch.float32)).cuda()
    C, info = H.gemm_bf16(A, B)
    torch.cuda.synchronize()
    assert int(info.cpu()[0]) == 0
    Ab, Bb = A.bfloat16().double(), B.bfloat16().double()
    ref = Ab @ Bb
    mag = Ab.abs() @ Bb.abs()
    err = (C.double() - ref).abs()
    chunk = min(K, 1024)
    assert bool((err <= 2.0 * chunk * 2.0 ** -24 * mag + 1e-30).all()), float((err / mag).max())
    assert float((err / mag).median()) <= 1e-6


def test_gemm_bf16_argument_checks(H):
    import torch
    from paper_2008_04447_gb300 import _lib
    x = torch.zeros(16, device="cuda")
    assert _lib.rq_gemm_bf16(H.h, 0, 4, 4, x, 4, x, 4, x, 4) == -2
    assert _lib.rq_gemm_bf16(H.h, 4, 4, 4, x, 3, x, 4, x, 4) == -6
    assert _lib.rq_gemm_bf16(H.h, 4, 4, 4, x, 4, x, 3, x, 4) == -8
    assert _lib.rq_gemm_bf16(H.h, 4, 4, 4, x, 4, x, 4, None, 4) == -9
    y = torch.zeros(64, device="cuda")
    assert _lib.rq_gemm_bf16(H.h, 4, 4, 4, y, 4, y[16:], 4, y[8:], 4) == -9       # C overlaps A and B
    # disjoint (A starts one float in: not 16-byte aligned, so the CUDA-core path)
    assert _lib.rq_gemm_bf16(H.h, 4, 4, 4, y[1:], 4, y[20:], 4, y[40:], 4) == 0
    torch.cuda.synchronize()
