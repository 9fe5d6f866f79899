"""Pins for the oracle's TRQRCP (Alg. 5), TUXV (Alg. 6) and Jacobi SVD."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2008_04447_gb300 import inputs as I


@pytest.mark.parametrize("m,n,b,p,k", [(200, 150, 16, 8, 64), (150, 220, 10, 6, 37), (90, 90, 8, 8, 8)])
def test_trqrcp_reproduces_rqrcp(m, n, b, p, k):
    """Sec. 4.1: TRQRCP is a reformulation: same pivots, reflectors and R rows."""
    a = I.graded(m, n, 8, seed=m + k)
    om = I.omega(b + p, m, seed=k)
    rr = O.rqrcp(a, om, b, k)
    tr = O.trqrcp(a, om, b, k)
    assert np.array_equal(rr.jpvt, tr.jpvt)
    nrm = np.linalg.norm(a)
    assert np.allclose(np.triu(rr.F[:k]), tr.R, atol=1e-12 * nrm)
    assert np.allclose(O.reflectors_of(rr.F, k), tr.Y, atol=1e-11)
    assert np.allclose(rr.tau, tr.tau, atol=1e-12)


def test_trqrcp_w_recurrence_equals_composite_T():
    """W^T built block by block equals T^T Y^T A P with the composite T (Sec. 4.1)."""
    m, n, b, p, k = 120, 90, 8, 8, 32
    a = I.graded(m, n, 6, seed=21)
    tr = O.trqrcp(a, I.omega(b + p, m, seed=22), b, k)
    T = O.larft(tr.Y, tr.tau)
    Wt = T.T @ tr.Y.T @ a[:, tr.jpvt]
    assert np.allclose(tr.Wt, Wt, atol=1e-12 * np.linalg.norm(a))
    # rows of R are rows of A P - Y W^T
    Ahat = a[:, tr.jpvt] - tr.Y @ tr.Wt
    assert np.allclose(np.triu(Ahat[:k]), tr.R, atol=1e-12 * np.linalg.norm(a))


def test_single_sample_case_alg3():
    """k = b: one sample, R_12 = Q(:,1:k)^T A P (Alg. 3)."""
    m, n, k, p = 100, 80, 12, 6
    a = I.graded(m, n, 6, seed=31)
    tr = O.trqrcp(a, I.omega(k + p, m, seed=32), k, k)
    T = O.larft(tr.Y, tr.tau)
    Qk = (np.eye(m) - tr.Y @ T @ tr.Y.T)[:, :k]
    assert np.allclose(Qk.T @ a[:, tr.jpvt], tr.R, atol=1e-12 * np.linalg.norm(a))


def test_jacobi_svd_matches_lapack():
    x = np.triu(I.rng(41).standard_normal((30, 30)))
    U, s, V = O.jacobi_svd(x)
    s_ref = sla.svd(x, compute_uv=False, lapack_driver="gesvd")
    assert np.allclose(s, s_ref, rtol=1e-13)
    assert np.allclose((U * s) @ V.T, x, atol=1e-13 * np.linalg.norm(x))
    assert np.allclose(U.T @ U, np.eye(30), atol=1e-13)
    assert np.allclose(V.T @ V, np.eye(30), atol=1e-13)


def test_jacobi_svd_graded_and_rank_deficient():
    g = I.rng(42)
    x = I.graded(20, 20, 10, seed=43)
    U, s, V = O.jacobi_svd(x)
    assert np.allclose(s, 10.0 ** (-10 * np.arange(1, 21) / 20), rtol=1e-6)
    y = g.standard_normal((12, 3)) @ g.standard_normal((3, 12))
    U, s, V = O.jacobi_svd(y)
    assert np.all(s[3:] <= 1e-13 * s[0])


@pytest.mark.parametrize("m,n,k,b", [(200, 150, 24, 8), (150, 200, 40, 16)])
def test_tuxv_identities(m, n, k, b):
    a = I.lowrank_plus_noise(m, n, 60, 1e-6, seed=m + n)
    om = I.omega(b + 8, m, seed=51)
    t = O.tuxv(a, om, b, k)
    assert np.allclose(t.U.T @ t.U, np.eye(k), atol=1e-13)
    assert np.allclose(t.V.T @ t.V, np.eye(k), atol=1e-13)
    assert np.allclose(t.X, np.triu(t.X))
    na2 = np.linalg.norm(a) ** 2
    err = np.linalg.norm(a - t.U @ t.X @ t.V.T)
    # A V V^T is an orthogonal projection: ||A - UXV^T||^2 = ||A||^2 - ||X||^2
    assert abs(err ** 2 - (na2 - np.linalg.norm(t.X) ** 2)) <= 1e-10 * na2
    # TUXV beats the TRQRCP truncation; Eckart-Young bounds it below
    err_tr = np.sqrt(max(na2 - np.linalg.norm(t.tr.R) ** 2, 0.0))
    s = np.linalg.svd(a, compute_uv=False)
    err_opt = np.sqrt(np.sum(s[k:] ** 2))
    assert err <= err_tr * (1 + 1e-10)
    assert err >= err_opt * (1 - 1e-10)


def test_tuxv_equals_truncated_rqrcp_qlp():
    """Sec. 4.2: TUXV(j_max=1) = QLP from full RQRCP, without row pivoting, truncated to k."""
    m, n, k, b = 120, 100, 16, 8
    a = I.graded(m, n, 6, seed=61)
    om = I.omega(b + 8, m, seed=62)
    t = O.tuxv(a, om, b, k)
    full = O.rqrcp(a, om, b)             # same Omega, full factorisation
    Q = O.form_q(full.F, full.tau, m)
    R = np.triu(full.F)
    Z = np.zeros_like(R)
    Z[:, full.jpvt] = R                  # R P^T
    F, tau = O.qr_householder(Z.T)       # LQ of R P^T
    V1 = O.form_q(F, tau, k)
    L = np.triu(F).T                     # Z = L V^T
    approx_qlp = Q @ L[:, :k] @ V1.T
    approx_tuxv = t.U @ t.X @ t.V.T
    assert np.allclose(V1, t.V, atol=1e-10)
    assert np.allclose(approx_qlp, approx_tuxv, atol=1e-12 * np.linalg.norm(a))


def test_tuxv_with_core_svd_and_more_iterations():
    m, n, k, b = 150, 120, 20, 10
    a = I.graded(m, n, 8, seed=71)
    om = I.omega(b + 8, m, seed=72)
    t1 = O.tuxv(a, om, b, k)
    ts = O.tuxv(a, om, b, k, svd=True)
    assert np.all(np.diff(ts.sigma) <= 0)
    assert np.allclose(ts.U @ ts.X @ ts.V.T, t1.U @ t1.X @ t1.V.T, atol=1e-12 * np.linalg.norm(a))
    s_true = 10.0 ** (-8 * np.arange(1, k + 1) / n)
    # sigma_i(A V V^T) <= sigma_i(A) (a projection cannot raise singular values);
    # the leading half is resolved closely, the tail more loosely
    assert np.all(ts.sigma <= s_true * (1 + 1e-12))
    assert np.all(np.abs(ts.sigma - s_true)[: k // 2] <= 1e-3 * s_true[: k // 2])
    assert np.all(np.abs(ts.sigma - s_true) <= 0.25 * s_true)
    t2 = O.tuxv(a, om, b, k, jmax=2)
    assert np.allclose(t2.X, np.tril(t2.X))
    e1 = np.linalg.norm(a - t1.U @ t1.X @ t1.V.T)
    e2 = np.linalg.norm(a - t2.U @ t2.X @ t2.V.T)
    assert e2 <= e1 * (1 + 1e-8)


def test_tuxv_iterations_are_subspace_iteration():
    """Alg. 6 with j_max > 1: each step is a projection, A ~= U U^T A or A V V^T,
    so ||A - U X V^T||^2 = ||A||^2 - ||X||^2 at every step; X alternates between
    lower (even j) and upper (odd j) triangular; the error never increases; and
    the alternation is a subspace iteration, so the excess over the
    Eckart-Young error, err^2 - sum_{i>k} sigma_i^2, shrinks by at least
    (sigma_{k+1} / sigma_k)^2 = 1/4 per step once the transient has passed."""
    m, n, k, b = 300, 200, 20, 8
    rng = np.random.default_rng(5)
    Uq, _ = np.linalg.qr(rng.standard_normal((m, n)))
    Vq, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.r_[np.linspace(2.0, 1.0, k), 0.5 * np.linspace(1.0, 0.1, n - k)]
    a = (Uq * s) @ Vq.T
    om = I.omega(b + 8, m, seed=6)
    na2 = np.linalg.norm(a) ** 2
    opt2 = np.sum(s[k:] ** 2)
    excess = []
    for j in range(1, 15):
        t = O.tuxv(a, om, b, k, jmax=j)
        err2 = np.linalg.norm(a - t.U @ t.X @ t.V.T) ** 2
        assert abs(err2 - (na2 - np.linalg.norm(t.X) ** 2)) <= 1e-10 * na2
        assert np.array_equal(t.X, np.tril(t.X) if j % 2 == 0 else np.triu(t.X))
        assert np.allclose(t.U.T @ t.U, np.eye(k), atol=1e-12) and np.allclose(t.V.T @ t.V, np.eye(k), atol=1e-12)
        excess.append(err2 - opt2)
    assert all(e2 <= e1 for e1, e2 in zip(excess, excess[1:]))
    assert all(e2 <= 0.25 * e1 for e1, e2 in zip(excess[2:], excess[3:]))
    assert excess[0] > 0.1 * opt2 and excess[-1] <= 1e-9 * opt2


def test_bf16_sketch_keeps_rank_k_error_on_a_quiet_tail():
    """The reduced-precision reading (the sketch formed from bfloat16-rounded
    Omega and A, everything else FP64) on the low-rank workload with a quiet
    tail (noise 1e-10, where the rank-k error is set by the singular values
    rather than a noise floor): the rank-k error stays within 1.05x of the
    FP64-sketch error, and both are at least the Eckart-Young error."""
    for seed in (3, 4):
        a = I.lowrank_plus_noise(2048, 1024, 512, 1e-10, seed=seed)
        om = I.omega(72, 2048, seed=seed + 100)
        k = 128
        s = np.linalg.svd(a, compute_uv=False)
        nrm = np.linalg.norm(a)
        ey = np.sqrt(np.sum(s[k:] ** 2)) / nrm
        t64 = O.tuxv(a, om, 64, k)
        tbf = O.tuxv(a, om, 64, k, sketch_inputs="bf16")
        e64 = np.linalg.norm(a - t64.U @ t64.X @ t64.V.T) / nrm
        ebf = np.linalg.norm(a - tbf.U @ tbf.X @ tbf.V.T) / nrm
        assert ebf <= 1.05 * e64
        assert min(e64, ebf) >= ey * (1 - 1e-10)
