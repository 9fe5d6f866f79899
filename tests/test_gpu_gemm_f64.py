"""GPU: rq_gemm_f64, FP64 C = A B on the bfloat16 tensor cores (eight 7-bit
slices per entry, 36 slice pairs, exact FP32 level sums over 128 K steps,
int64 gathering), against the product taken in extended precision
(numpy longdouble) of the same FP64 inputs.

Bound per entry (the error analysis of the split, also checked on the host by
tests/test_f64_slices_host.py): |C - AB| <= (3 K 2^-53 + 2^-52) 2^(ea_i + eb_j)
with 2^ea_i, 2^eb_j the powers of two just above the largest magnitude of
row i of A and column j of B; and the Frobenius error within 10x that of an
FP64 GEMM (numpy).  Shapes: ragged tiles, K = 1, one drain and many drains,
split-K (few tiles, long K), graded and wide-range operands, and long K with
zero, tiny, subnormal, huge and one-entry rows (the row slicer's 2-D path).
A result in the subnormal range adds one unit 2^-1074 to the bound for each
split-K part and one for their sum (each FP64 partial is rounded there).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from gpu_util import build_and_handle
    return build_and_handle()


def _exp2_above(m):
    """2^e with m < 2^e <= 2m (1 for m = 0)."""
    m = np.asarray(m, dtype=np.float64)
    f, e = np.frexp(m)
    return np.where(m > 0, np.ldexp(1.0, e), 1.0)


@pytest.mark.parametrize("M,N,K,kind", [(9, 5, 1, "gaussian"), (130, 70, 200, "gaussian"), (256, 64, 64, "graded"),
                                        (300, 257, 1000, "gaussian"), (64, 64, 4100, "gaussian"),
                                        (200, 90, 333, "wide"), (72, 40, 2000, "rows"), (70, 33, 700, "rows")])
def test_gemm_f64_matches_the_extended_precision_product(H, M, N, K, kind):
    import torch
    from paper_2008_04447_gb300 import colmajor
    g = np.random.default_rng(M * 7 + N * 3 + K)
    A = g.standard_normal((M, K))
    B = g.standard_normal((K, N))
    if kind == "graded":
        A *= np.logspace(0, -12, K)[None, :]
        B *= np.logspace(0, -8, K)[:, None]
    elif kind == "wide":
        A *= 10.0 ** g.uniform(-10, 10, (M, K))
    elif kind == "rows":
        # long K (the row slicer's 2-D path): an all-zero row, a row near the bottom of the
        # normal range, a subnormal row, a huge row and a row with one nonzero entry
        A[0] = 0.0
        A[1] *= 1e-300
        A[2] *= 5e-320
        A[3] *= 1e300
        A[4] = 0.0
        A[4, K - 1] = 3.0
    C, info = H.gemm_f64(colmajor(torch.as_tensor(A)).cuda(), colmajor(torch.as_tensor(B)).cuda())
    torch.cuda.synchronize()
    assert int(info.cpu()[0]) == 0
    C = C.cpu().numpy()
    ref = (A.astype(np.longdouble) @ B.astype(np.longdouble))
    err = np.abs(C.astype(np.longdouble) - ref).astype(np.float64)
    sa = _exp2_above(np.max(np.abs(A), axis=1))[:, None]
    sb = _exp2_above(np.max(np.abs(B), axis=0))[None, :]
    # plus subnormal units: a result below 2^-1022 is rounded to a multiple of 2^-1074 once per
    # split-K part (at most one part per 128 steps of K) and once more by their sum
    parts = -(-K // 128)
    bound = (3 * K * 2.0 ** -53 + 2.0 ** -52) * sa * sb + (parts + 1) * 2.0 ** -1074
    assert np.all(err <= bound), float(np.max(err / bound))
    e_fp64 = float(np.linalg.norm((A @ B).astype(np.longdouble) - ref))
    e_tc = float(np.linalg.norm(err))
    assert e_tc <= max(10 * e_fp64, 2.0 ** -52 * float(np.linalg.norm(np.abs(A) @ np.abs(B)))), (e_tc, e_fp64)


def test_gemm_f64_argument_checks(H):
    import torch
    from paper_2008_04447_gb300 import _lib
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    assert _lib.rq_gemm_f64(H.h, 0, 4, 4, x, 4, x, 4, x, 4) == -2
    assert _lib.rq_gemm_f64(H.h, 4, 4, 4, x, 3, x, 4, x, 4) == -6
    assert _lib.rq_gemm_f64(H.h, 4, 4, 4, x, 4, x, 3, x, 4) == -8
    assert _lib.rq_gemm_f64(H.h, 4, 4, 4, x, 4, x, 4, x[8:], 4) == -9     # C overlaps A and B
    assert _lib.rq_gemm_f64(H.h, 4, 4, 4, x, 4, x[16:], 4, x[32:], 4) == 0
    torch.cuda.synchronize()
