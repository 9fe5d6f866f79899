"""Pins for the oracle's QRCP (Alg. 1) and sample QRCP (Sec. 3.2)."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2008_04447_gb300 import inputs as I


def _greedy_invariant(F, k):
    """|R_jj|^2 >= trailing norm^2 of every later column at step j (Alg. 1 Ensure)."""
    R = np.triu(F)
    m, n = R.shape
    for j in range(k):
        col2 = np.array([np.sum(R[j:min(c, m - 1) + 1, c] ** 2) for c in range(j + 1, n)])
        if col2.size:
            assert R[j, j] ** 2 >= col2.max() * (1 - 1e-12)


@pytest.mark.parametrize("m,n", [(40, 25), (25, 40), (60, 60)])
def test_qrcp_greedy_invariant_and_residual(m, n):
    a = I.graded(m, n, 6, seed=m + n)
    F, tau, jpvt = O.qrcp(a)
    k = min(m, n)
    _greedy_invariant(F, k)
    d = np.abs(np.diag(F[:k, :k]))
    assert np.all(d[:-1] >= d[1:] * (1 - 1e-12))
    Q = O.form_q(F, tau, k)
    assert np.linalg.norm(a[:, jpvt] - Q @ np.triu(F[:k])) <= 1e-13 * np.linalg.norm(a)
    assert sorted(jpvt.tolist()) == list(range(n))


def test_qrcp_matches_lapack_dgeqp3():
    a = I.rng(7).standard_normal((80, 60)) * (1.3 ** np.arange(60))
    F, tau, jpvt = O.qrcp(a)
    _, r, piv = sla.qr(a, pivoting=True)
    assert np.array_equal(jpvt, piv)
    assert np.allclose(np.abs(np.diag(F[:60, :60])), np.abs(np.diag(r)), rtol=1e-12)


def test_qrcp_ties_take_lowest_position():
    a = np.zeros((5, 4))
    a[0, 1] = a[1, 3] = 2.0   # two columns of equal norm
    F, tau, jpvt = O.qrcp(a)
    assert jpvt[0] == 1


@pytest.mark.parametrize("steps", [1, 5, 12])
def test_sample_qrcp_is_qrcp_of_the_sample(steps):
    g = I.rng(11)
    B = g.standard_normal((20, 50)) * np.exp(g.standard_normal(50))
    sq = O.sample_qrcp(B, steps)
    F, tau, jpvt = O.qrcp(B, ncols=steps)
    assert np.array_equal(sq.perm[:steps], jpvt[:steps])
    # the partially factorised sample: same R rows (up to rounding) and U^T B P = S
    assert np.allclose(np.triu(sq.S[:steps]), np.triu(F[:steps]), atol=1e-12 * np.linalg.norm(B))
    U = np.eye(20)
    for i in range(steps):
        U = U @ (np.eye(20) - sq.tau[i] * np.outer(sq.V[:, i], sq.V[:, i]))
    assert np.allclose(U.T @ B[:, sq.perm], sq.S, atol=1e-12 * np.linalg.norm(B))
    # position bookkeeping: applying the swap list reproduces perm
    p = np.arange(50)
    for i, q in enumerate(sq.swaps):
        p[[i, q]] = p[[q, i]]
    assert np.array_equal(p, sq.perm)


def test_sample_qrcp_downdating_recomputes_when_cancellation():
    # column 1 is almost parallel to column 0: its downdated norm collapses
    B = np.zeros((6, 3))
    B[:, 0] = [1, 1, 1, 1, 1, 1]
    B[:, 1] = B[:, 0] * 0.999 + 1e-9 * np.arange(6)
    B[:, 2] = [0.1, -0.1, 0.1, -0.1, 0.1, -0.1]
    sq = O.sample_qrcp(B, 2)
    assert sq.recomputed >= 1
    # after one step, column 2 (norm ~0.245) must beat column 1 (~1e-9)
    assert sq.perm[1] == 2


def test_round_bf16_matches_definition():
    """bfloat16 keeps the top 16 bits of a float32, rounded to nearest even."""
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -3.14159, 0.0, 1e-30])
    r = O.round_bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0 + 2 ** -7 or r[1] == 1.0  # exactly halfway between 1 and 1+2^-7
    assert r[1] == 1.0                           # ties to even mantissa
    assert r[2] == 1.0                           # below half an ulp (ulp = 2^-7)
    assert r[3] == 1.0 + 2 ** -7                 # above half an ulp
    assert abs(r[4] - (-3.140625)) < 1e-12       # -3.14159 -> nearest bf16
    assert r[5] == 0.0
    g = I.rng(3).standard_normal(1000)
    rel = np.abs(O.round_bf16(g) - g) / np.abs(g)
    assert rel.max() <= 2 ** -8 * (1 + 1e-6)
