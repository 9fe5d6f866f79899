"""GPU parity: rq_trqrcp (Alg. 5, CUDA through the C ABI) against the FP64 oracle.

Same bar as the RQRCP parity tests: identical pivots while every decision's
relative gap exceeds 1e-6; R within 1e-12 ||A||_F entry by entry; reflector j
and tau_j within 1e-12 ||A||_F / |R_jj|; A is left untouched.
"""
import numpy as np
import pytest

import oracle as O
from paper_2008_04447_gb300 import inputs as I

from gpu_util import build_and_handle, first_near_tie, to_dev, to_host

pytestmark = pytest.mark.gpu
TIE = 1e-6


@pytest.fixture(scope="module")
def H():
    return build_and_handle()


def run_gpu(H, a, om, b, p, k):
    import torch
    A = to_dev(a)
    A_before = A.clone()
    Y, tau, R, jpvt, info = H.trqrcp(A, to_dev(om), b, p, k)
    torch.cuda.synchronize()
    assert torch.equal(A, A_before)
    return to_host(Y), to_host(tau), to_host(R), jpvt.cpu().numpy().astype(np.int64), int(info.cpu()[0])


CASES = [
    # m, n, k, b, p, kind
    (600, 400, 128, 32, 8, "graded"),
    (400, 700, 100, 32, 8, "graded"),     # ragged last block (100 = 3*32 + 4)
    (1000, 1000, 200, 32, 8, "graded"),
    (777, 513, 64, 64, 8, "lowrank"),     # single block (k = b)
    (300, 250, 37, 10, 6, "lowrank"),
    (50, 40, 8, 3, 2, "graded"),
]


@pytest.mark.parametrize("m,n,k,b,p,kind", CASES)
def test_trqrcp_fp64_matches_oracle(H, m, n, k, b, p, kind):
    if kind == "graded":
        a = I.graded(m, n, 8, seed=m + n + k)
    else:
        a = I.lowrank_plus_noise(m, n, 3 * k, 1e-6, seed=m + k)
    om = I.omega(b + p, m, seed=k + 5)
    Y, tau, R, jpvt, info = run_gpu(H, a, om, b, p, k)
    ref = O.trqrcp(a, om, b, k)
    nrm = np.linalg.norm(a)
    tie = first_near_tie(ref.gaps, b, TIE)
    assert sorted(jpvt.tolist()) == list(range(n))
    # Y orthogonal reflectors reproduce A P ~ Q R on the chosen columns
    if tie is None:
        assert np.array_equal(jpvt, ref.jpvt)
        assert np.max(np.abs(R - ref.R)) <= 1e-12 * nrm
        scale = 1e-12 * nrm / np.maximum(np.abs(np.diag(ref.R[:, :k])), 1e-300)
        assert np.all(np.abs(tau - ref.tau) <= scale)
        assert np.all(np.abs(Y - ref.Y).max(axis=0) <= scale)
    else:
        assert np.array_equal(jpvt[:tie], ref.jpvt[:tie])
    assert np.allclose(np.triu(R[:, :k]), R[:, :k])
    assert info == ref.info


def test_trqrcp_equals_gpu_rqrcp(H):
    """Sec. 4.1: the truncated reformulation chooses the same pivots and R rows as RQRCP."""
    import torch
    m, n, k, b, p = 800, 600, 160, 32, 8
    a = I.graded(m, n, 8, seed=3)
    om = I.omega(b + p, m, seed=4)
    Y, tau, R, jpvt, info = run_gpu(H, a, om, b, p, k)
    A = to_dev(a)
    tau2, jp2, info2 = H.rqrcp(A, to_dev(om), b, p, k)
    torch.cuda.synchronize()
    F = to_host(A)
    assert np.array_equal(jpvt, jp2.cpu().numpy())
    assert np.max(np.abs(R - np.triu(F[:k]))) <= 1e-12 * np.linalg.norm(a)


@pytest.mark.parametrize("m,n,k,b,p", [(500, 300, 24, 24, 8), (400, 350, 10, 32, 8), (90, 70, 1, 16, 4)])
def test_single_sample_case_is_alg3(H, m, n, k, b, p):
    """k <= b: one sample, one panel, no update (the single-sample algorithm,
    Alg. 3): R = Q(:, 1:k)^T A P to 1e-12 ||A||_F, with the oracle's pivots."""
    a = I.graded(m, n, 8, seed=m + k)
    om = I.omega(b + p, m, seed=k + 3)
    Y, tau, R, jpvt, info = run_gpu(H, a, om, b, p, k)
    T = O.larft(Y, tau)
    Qk = (np.eye(m) - Y @ T @ Y.T)[:, :k]
    nrm = np.linalg.norm(a)
    assert np.max(np.abs(Qk.T @ a[:, jpvt] - R)) <= 1e-12 * nrm
    ref = O.trqrcp(a, om, b, k)
    tie = first_near_tie(ref.gaps, b, TIE)
    upto = k if tie is None else tie
    assert np.array_equal(jpvt[:upto], ref.jpvt[:upto])
