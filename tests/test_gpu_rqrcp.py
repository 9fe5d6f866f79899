"""GPU parity: rq_rqrcp / rq_qr (CUDA, through the C ABI) against the FP64 oracle.

Bar (FP64): identical pivots while every sample decision is separated by a
relative gap above 1e-6 (a downdated squared norm carries a relative error of
at most about sqrt(eps) = 1.5e-8, so decisions closer than that are
near-ties); R equal to the oracle's within 1e-12 ||A||_F entry by entry;
tau_j and reflector j within 1e-12 ||A||_F / |R_jj| (a Householder vector is
only as well determined as its column is large);
||AP - QR||_F / ||A||_F <= 1e-12 and ||Q^T Q - I||_F <= 1e-12.
"""
import numpy as np
import pytest

import oracle as O
from paper_2008_04447_gb300 import inputs as I

from gpu_util import build_and_handle, factor_quality, first_near_tie, to_dev, to_host

pytestmark = pytest.mark.gpu

TIE = 1e-6


@pytest.fixture(scope="module")
def H():
    return build_and_handle()


def run_gpu_rqrcp(H, a, omega, b, p, k=None, dtype=None):
    import torch
    A = to_dev(a, dtype)
    Om = to_dev(omega, dtype)
    tau, jpvt, info = H.rqrcp(A, Om, b, p, k)
    torch.cuda.synchronize()
    return to_host(A), to_host(tau), jpvt.cpu().numpy().astype(np.int64), int(info.cpu()[0])


CASES = [
    # m, n, b, p, k, decades
    (1000, 1000, 32, 8, None, 8),     # the 1000^2 workload (b=32, p=8)
    (300, 200, 16, 8, None, 8),
    (200, 300, 32, 8, None, 8),
    (129, 97, 10, 4, None, 6),        # ragged last block
    (517, 389, 64, 8, 200, 6),        # truncated k, several CTAs, ragged tiles
    (64, 64, 64, 8, None, 4),         # one block
    (7, 3, 2, 2, None, 2),
    (3, 7, 2, 0, None, 2),            # p = 0
    (1, 1, 1, 0, None, 0),
]


@pytest.mark.parametrize("m,n,b,p,k,dec", CASES)
def test_rqrcp_fp64_matches_oracle(H, m, n, b, p, k, dec):
    a = I.graded(m, n, dec, seed=m * 7 + n)
    omega = I.omega(b + p, m, seed=m + 11)
    F, tau, jpvt, info = run_gpu_rqrcp(H, a, omega, b, p, k)
    ref = O.rqrcp(a, omega, b, k)
    kk = ref.k
    nrm = np.linalg.norm(a)
    tie = first_near_tie(ref.gaps, b, TIE)
    resid, orth = factor_quality(a, F, tau, jpvt, kk)
    assert resid <= 1e-12, resid
    assert orth <= 1e-12, orth
    assert sorted(jpvt.tolist()) == list(range(n))
    assert info == ref.info
    if tie is None:
        assert np.array_equal(jpvt, ref.jpvt)
        assert np.max(np.abs(np.triu(F[:kk]) - np.triu(ref.F[:kk]))) <= 1e-12 * nrm
        # a reflector is determined to about eps ||A|| / |R_jj| (its column's size)
        scale = 1e-12 * nrm / np.maximum(np.abs(np.diag(ref.F[:kk, :kk])), 1e-300)
        assert np.all(np.abs(tau - ref.tau) <= scale)
        dv = np.abs(np.tril(F[:, :kk], -1) - np.tril(ref.F[:, :kk], -1)).max(axis=0)
        assert np.all(dv <= scale)
        if kk < min(m, n):
            assert np.max(np.abs(F[kk:, kk:] - ref.F[kk:, kk:])) <= 1e-12 * nrm
    else:
        assert np.array_equal(jpvt[:tie], ref.jpvt[:tie])


def test_rqrcp_orthonormal_omega_equals_qrcp(H):
    """With Omega of orthonormal columns every sample norm is exact: GPU RQRCP = QRCP."""
    m, n, b = 96, 150, 8
    a = I.graded(m, n, 6, seed=5)
    omega = I.haar(m + 4, m, I.rng(6))
    F, tau, jpvt, info = run_gpu_rqrcp(H, a, omega, b, m + 4 - b)
    Fq, tq, jq = O.qrcp(a)
    assert np.array_equal(jpvt, jq)
    assert np.max(np.abs(np.triu(F) - np.triu(Fq))) <= 1e-12 * np.linalg.norm(a)


def test_zero_matrix_and_rank_deficient(H):
    z = np.zeros((40, 30))
    F, tau, jpvt, info = run_gpu_rqrcp(H, z, I.omega(12, 40, seed=1), 4, 8)
    assert np.array_equal(jpvt, np.arange(30))
    assert np.all(F == 0) and np.all(tau == 0) and info == 1
    g = I.rng(2)
    a = g.standard_normal((90, 6)) @ g.standard_normal((6, 70))
    F, tau, jpvt, info = run_gpu_rqrcp(H, a, I.omega(16, 90, seed=3), 8, 8)
    resid, orth = factor_quality(a, F, tau, jpvt, 70)
    assert resid <= 1e-12 and orth <= 1e-12


@pytest.mark.parametrize("m,n,b", [(300, 200, 32), (200, 333, 16), (1000, 1000, 64), (65, 65, 64)])
def test_unpivoted_qr_matches_oracle(H, m, n, b):
    import torch
    a = I.graded(m, n, 6, seed=m + n)
    A = to_dev(a)
    tau, info = H.qr(A, b)
    torch.cuda.synchronize()
    F, t = to_host(A), to_host(tau)
    Fo, to = O.qr_householder(a)
    nrm = np.linalg.norm(a)
    assert np.max(np.abs(np.triu(F) - np.triu(Fo))) <= 1e-12 * nrm
    k = min(m, n)
    scale = 1e-12 * nrm / np.maximum(np.abs(np.diag(Fo[:k, :k])), 1e-300)
    assert np.all(np.abs(t - to) <= scale)
    resid, orth = factor_quality(a, F, t, np.arange(n), k)
    assert resid <= 1e-12 and orth <= 1e-12


def test_repeatable_bitwise(H):
    a = I.graded(400, 300, 8, seed=9)
    om = I.omega(40, 400, seed=10)
    r1 = run_gpu_rqrcp(H, a, om, 32, 8)
    r2 = run_gpu_rqrcp(H, a, om, 32, 8)
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[2], r2[2])


def test_bad_arguments_return_negative_index(H):
    import torch
    from paper_2008_04447_gb300 import _lib
    A = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    j = torch.zeros(4, dtype=torch.int32, device="cuda")
    i = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _lib.rq_rqrcp(H.h, 0, 4, 4, A, 3, 2, 2, 4, A, 4, t, j, i) == -6   # lda < m
    assert _lib.rq_rqrcp(H.h, 0, 4, 4, A, 4, 2, 2, 5, A, 4, t, j, i) == -9   # k > min(m, n)
    assert _lib.rq_rqrcp(H.h, 0, 4, 4, A, 4, 2, 2, 4, A, 3, t, j, i) == -11  # ldo < l
    assert _lib.rq_rqrcp(H.h, 7, 4, 4, A, 4, 2, 2, 4, A, 4, t, j, i) == -2   # precision
    assert _lib.rq_rqrcp(H.h, 0, 4, 4, A, 4, _lib.RQ_MAX_B + 1, 2, 4, A, 4, t, j, i) == -7   # b > RQ_MAX_B
    assert _lib.rq_rqrcp(H.h, 0, 4, 4, A, 4, 2, _lib.RQ_MAX_L - 1, 4, A, 4, t, j, i) == -8   # b + p > RQ_MAX_L


@pytest.mark.parametrize("mode", ["0", "1"])
def test_fp64_update_engines_agree(mode):
    """The FP64 block reflector products on the bfloat16 tensor cores (the
    default) and on the FP64 pipe (RQ_F64_TC=0) or with only the update on the
    tensor cores (RQ_F64_TC=1) give the same factorisation: identical pivots
    and R within 1e-12 ||A||_F, and each matches the oracle."""
    import os
    import torch
    from paper_2008_04447_gb300 import Handle, build
    build.build()
    m, n, b, p = 700, 600, 32, 8
    a = I.graded(m, n, 8, seed=31)
    om = I.omega(b + p, m, seed=32)
    outs = {}
    for md in ("2", mode):
        old = os.environ.get("RQ_F64_TC")
        os.environ["RQ_F64_TC"] = md
        try:
            h = Handle()
        finally:
            if old is None:
                del os.environ["RQ_F64_TC"]
            else:
                os.environ["RQ_F64_TC"] = old
        outs[md] = run_gpu_rqrcp(h, a, om, b, p)
        h.close()
    ref = O.rqrcp(a, om, b)
    nrm = np.linalg.norm(a)
    for md, (F, tau, jpvt, info) in outs.items():
        assert np.array_equal(jpvt, ref.jpvt), md
        assert np.max(np.abs(np.triu(F) - np.triu(ref.F))) <= 1e-12 * nrm, md
    assert np.array_equal(outs["2"][2], outs[mode][2])
    assert np.max(np.abs(np.triu(outs["2"][0]) - np.triu(outs[mode][0]))) <= 1e-12 * nrm
