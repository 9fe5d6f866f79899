"""The integer steps of exact FP64 products on bfloat16 tensor cores
(paper_2008_04447_gb300/csrc/f64_slices.cuh), built for the host with g++ and
checked against exact integer and rational arithmetic (no GPU):

* the scale exponent e is tight: m < 2^e <= 2m, for normal and subnormal m;
* trunc(|x| 2^(56 - e)) is exact and below 2^56, and the eight signed 7-bit
  slices put it back together with the sign of x;
* for Gaussian, graded and wide-range operands, FP32 partials of 128 K steps
  per level stay below 2^24 (so an FP32 accumulator adds them exactly), and
  the drained result is within the derived bound of the exact product and
  as accurate as an FP64 GEMM in the Frobenius norm (measured 0.4x to 2.5x
  its error);
* the same header compiles as device code for sm_103a.
"""
import ctypes
import os
import subprocess
from fractions import Fraction

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
S, LEVELS, KC, BITS = 8, 8, 128, 7


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("f64s") / "libf64s.so")
    src = os.path.join(ROOT, "tests", "native", "f64_slices_host.cpp")
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out, src], check=True)
    L = ctypes.CDLL(out)
    P, I = ctypes.c_void_p, ctypes.c_int
    L.f64s_exponents.argtypes = [P, I, P]
    L.f64s_scaled.argtypes = [P, P, I, P]
    L.f64s_slices.argtypes = [P, P, I, P]
    L.f64s_acc_unit.argtypes = [I]
    L.f64s_acc_unit.restype = I
    L.f64s_combine.argtypes = [P, I, I]
    L.f64s_combine.restype = ctypes.c_longlong
    L.f64s_from_acc.argtypes = [ctypes.c_longlong, I, I, I]
    L.f64s_from_acc.restype = ctypes.c_double
    return L


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def exponents(lib, m):
    m = np.ascontiguousarray(m, dtype=np.float64)
    e = np.empty(m.size, dtype=np.int32)
    lib.f64s_exponents(_ptr(m), m.size, _ptr(e))
    return e.reshape(m.shape)


def slices(lib, x, e):
    x = np.ascontiguousarray(x, dtype=np.float64)
    e = np.ascontiguousarray(np.broadcast_to(e, x.shape), dtype=np.int32)
    s = np.empty(x.size * S, dtype=np.int32)
    lib.f64s_slices(_ptr(x), _ptr(e), x.size, _ptr(s))
    return s.reshape(x.shape + (S,))


def test_scale_exponent_is_tight(lib):
    g = np.random.default_rng(0)
    m = np.concatenate([np.abs(g.standard_normal(2000)) * 10.0 ** g.uniform(-300, 300, 2000),
                        [2.0 ** k for k in range(-1074, 1000, 37)], [5e-324, 1e-310, 1.0, 0.75, np.nextafter(1.0, 2)]])
    e = exponents(lib, m)
    for mi, ei in zip(m, e):
        assert Fraction(mi) < Fraction(2) ** int(ei) <= 2 * Fraction(mi), (mi, ei)
    assert exponents(lib, np.zeros(1))[0] == 0


def test_slices_are_exact(lib):
    g = np.random.default_rng(1)
    x = g.standard_normal(3000) * 10.0 ** g.uniform(-30, 30, 3000)
    x[::97] = 0.0
    x[1::101] = 5e-324
    e = exponents(lib, np.abs(x)) + g.integers(0, 40, x.size)      # any e with |x| < 2^e
    xs = np.ascontiguousarray(x)
    es = np.ascontiguousarray(e, dtype=np.int32)
    X = np.empty(x.size, dtype=np.uint64)
    lib.f64s_scaled(_ptr(xs), _ptr(es), x.size, _ptr(X))
    s = slices(lib, x, e)
    for xi, ei, Xi, si in zip(x, e, X, s):
        want = int(abs(Fraction(xi)) * Fraction(2) ** (56 - int(ei)))      # floor of a non-negative value
        assert int(Xi) == want < 2 ** 56
        assert all(abs(int(v)) <= 127 for v in si)
        assert sum(abs(int(v)) << (BITS * (S - 1 - i)) for i, v in enumerate(si)) == want
        assert all(v == 0 or (v < 0) == (xi < 0) for v in si)


def emulated_product(lib, A, B):
    """C = A B through the slices: exact integer level partials per 128-step
    chunk (what an FP32 accumulator holds when they stay below 2^24), drained
    with the library's combination and returned to FP64."""
    M, K = A.shape
    N = B.shape[1]
    ea = exponents(lib, np.max(np.abs(A), axis=1))
    eb = exponents(lib, np.max(np.abs(B), axis=0))
    As = slices(lib, A, ea[:, None]).astype(np.int64)      # M x K x S
    Bs = slices(lib, B, eb[None, :]).astype(np.int64)      # K x N x S
    u = lib.f64s_acc_unit(K)
    nch = (K + KC - 1) // KC
    parts = np.zeros((M, N, nch, LEVELS), dtype=np.int64)
    for c in range(nch):
        k0, k1 = c * KC, min(K, (c + 1) * KC)
        for i in range(S):
            for j in range(S):
                L = (i + 1) + (j + 1)
                if L <= S + 1:
                    parts[:, :, c, L - 2] += As[:, k0:k1, i] @ Bs[k0:k1, :, j]
    assert np.max(np.abs(parts)) < 2 ** 24                 # every FP32 partial is exact
    C = np.empty((M, N))
    for r in range(M):
        for col in range(N):
            P = np.ascontiguousarray(parts[r, col].astype(np.float32).ravel())
            acc = lib.f64s_combine(_ptr(P), nch, u)
            C[r, col] = lib.f64s_from_acc(acc, u, int(ea[r]), int(eb[col]))
    return C, ea, eb


@pytest.mark.parametrize("kind,K", [("gaussian", 64), ("gaussian", 300), ("graded", 64), ("wide", 64)])
def test_emulated_product_is_fp64_accurate(lib, kind, K):
    g = np.random.default_rng(K + len(kind))
    M, N = 12, 10
    A = g.standard_normal((M, K))
    B = g.standard_normal((K, N))
    if kind == "graded":
        A *= np.logspace(0, -12, K)[None, :]
        B *= np.logspace(0, -8, K)[:, None]
    elif kind == "wide":
        A *= 10.0 ** g.uniform(-10, 10, (M, K))
    exact = np.array([[float(sum(Fraction(float(A[r, k])) * Fraction(float(B[k, c])) for k in range(K)))
                       for c in range(N)] for r in range(M)])
    C, ea, eb = emulated_product(lib, A, B)
    scale = np.ldexp(1.0, ea[:, None] + eb[None, :])
    # truncation of both operands (2 K 2^-56), dropped pairs (K 2^-53.4), rounding of the drains and the result
    assert np.all(np.abs(C - exact) <= (3 * K * 2.0 ** -53 + 2.0 ** -52) * scale)
    e_emul = np.linalg.norm(C - exact)
    e_fp64 = np.linalg.norm(A @ B - exact)
    assert e_emul <= max(10 * e_fp64, 2.0 ** -52 * np.linalg.norm(np.abs(A) @ np.abs(B))), (e_emul, e_fp64)


def test_header_compiles_for_the_device(tmp_path):
    import shutil
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = os.path.join(ROOT, "tests", "native", "f64_slices_device.cu")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-c", src, "-o",
                    str(tmp_path / "f64s_device.o")], check=True)
