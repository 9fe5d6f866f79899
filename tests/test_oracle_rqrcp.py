"""Pins for the oracle's RQRCP (Alg. 4) and its sample update (Eq. update1).

The strongest pin: when Omega has orthonormal columns (l >= m), every sample
norm equals the true trailing norm, and the updated compression matrix keeps
orthonormal columns (Omegahat is block upper triangular with orthonormal
columns, so Omegahat_12 = 0 and Omegahat_22 has orthonormal columns).  RQRCP
must then reproduce brute-force QRCP pivot for pivot, which fails for a dropped
term, a wrong sign or a wrong block in the update formula.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2008_04447_gb300 import inputs as I


def _residuals(a, res):
    Q, R = O.unpack_rqrcp(res)
    k = res.k
    nrm = np.linalg.norm(a)
    # full residual includes the trailing block: A P = Q_full [R; 0 A_trail]
    F = res.F
    m, n = F.shape
    Qf = O.form_q(F, res.tau, m)
    Rf = np.triu(F)
    Rf[k:, k:] = F[k:, k:]
    resid = np.linalg.norm(a[:, res.jpvt] - Qf @ Rf) / nrm
    orth = np.linalg.norm(Qf.T @ Qf - np.eye(m))
    return resid, orth


@pytest.mark.parametrize("m,n,b,k", [(40, 60, 8, None), (50, 30, 7, None), (48, 48, 16, 40)])
def test_rqrcp_with_orthonormal_omega_equals_qrcp(m, n, b, k):
    a = I.graded(m, n, 5, seed=3 * m + n)
    l = m + 3
    omega = I.haar(l, m, I.rng(99))          # l x m, orthonormal columns
    res = O.rqrcp(a, omega, b, k)
    kk = res.k
    F, tau, jpvt = O.qrcp(a, ncols=kk)
    assert np.array_equal(res.jpvt[:kk], jpvt[:kk])
    nrm = np.linalg.norm(a)
    assert np.allclose(np.triu(res.F[:kk]), np.triu(F[:kk]), atol=1e-12 * nrm)


def test_rqrcp_orthonormal_omega_catches_planted_update_error(monkeypatch):
    """A dropped S11 R11^-1 R12 term must break the equality with QRCP."""
    m, n, b = 40, 60, 8
    a = I.graded(m, n, 5, seed=3)
    omega = I.haar(m, m, I.rng(98))
    good = O.rqrcp(a, omega, b)
    real = O.sample_update

    def broken(S, bj, R11, R12):
        return np.vstack([S[:bj, bj:], S[bj:, bj:]])

    monkeypatch.setattr(O.rq_oracle, "sample_update", broken)
    bad = O.rqrcp(a, omega, b)
    monkeypatch.setattr(O.rq_oracle, "sample_update", real)
    F, tau, jpvt = O.qrcp(a)
    assert np.array_equal(good.jpvt, jpvt)
    assert not np.array_equal(bad.jpvt, jpvt)


@pytest.mark.parametrize("m,n,b,p", [(300, 200, 16, 8), (200, 300, 32, 8), (129, 97, 10, 4)])
def test_rqrcp_residual_orthogonality(m, n, b, p):
    a = I.graded(m, n, 8, seed=m)
    omega = I.omega(b + p, m, seed=m + 1)
    res = O.rqrcp(a, omega, b)
    resid, orth = _residuals(a, res)
    assert resid <= 1e-14
    assert orth <= 1e-13
    assert sorted(res.jpvt.tolist()) == list(range(n))


def test_update_formula_equals_explicit_compression():
    """Eq. (update1) == applying Omega^[J] = (U^T Omega^[J-1] Q)(b:, b:) explicitly."""
    m, n, b, p = 300, 200, 16, 8
    a = I.graded(m, n, 8, seed=5)
    omega = I.omega(b + p, m, seed=6)
    up = O.rqrcp(a, omega, b, keep_samples=True)
    ex = O.rqrcp(a, omega, b, mode="explicit", keep_samples=True)
    assert np.array_equal(up.jpvt, ex.jpvt)
    # the update cancels entries of the size of the first sample: measure against it
    scale = np.linalg.norm(up.samples[0])
    for s_up, s_ex in zip(up.samples, ex.samples):
        assert np.linalg.norm(s_up - s_ex) <= 1e-13 * scale
    for omh, S, R11 in ex.omegahat:
        bj = R11.shape[0]
        # Omegahat_21 = 0 and Omegahat_11 = S11 R11^{-1} (Sec. 3.2)
        assert np.linalg.norm(omh[bj:, :bj]) <= 1e-12 * np.linalg.norm(omh)
        assert np.allclose(omh[:bj, :bj] @ R11, np.triu(S[:bj, :bj]),
                           atol=1e-11 * np.linalg.norm(S[:bj, :bj]))
        # the sample of the trailing matrix: S22 = Omegahat_22 A^[J]
        assert np.allclose(np.triu(omh[:bj, :bj]), omh[:bj, :bj], atol=1e-12 * np.linalg.norm(omh))


def test_unpivoted_equals_lapack_dgeqrf():
    a = I.graded(120, 90, 6, seed=8)
    res = O.rqrcp(a, np.zeros((1, 120)), 16, pivot=False)
    qr, tau, work, info = sla.lapack.dgeqrf(np.asfortranarray(a))
    assert np.array_equal(res.jpvt, np.arange(90))
    assert np.allclose(np.triu(res.F), np.triu(qr), atol=1e-13 * np.linalg.norm(a))
    assert np.allclose(res.tau, tau, atol=1e-13)


def test_big_gaps_give_identity_pivots_and_dgeqrf():
    m, n = 80, 40
    a = I.rng(9).standard_normal((m, n)) * (1e-3 ** np.arange(n))[None, :] ** 0.25
    a *= (10.0 ** (-np.arange(n) / 2.0))[None, :]
    res = O.rqrcp(a, I.omega(16, m, seed=10), 8)
    assert np.array_equal(res.jpvt, np.arange(n))
    qr, tau, work, info = sla.lapack.dgeqrf(np.asfortranarray(a))
    assert np.allclose(np.abs(np.diag(res.F)), np.abs(np.diag(qr)), rtol=1e-10)


def test_zero_matrix_and_rank_deficient():
    z = np.zeros((20, 15))
    res = O.rqrcp(z, I.omega(10, 20, seed=1), 4)
    assert np.array_equal(res.jpvt, np.arange(15))
    assert np.all(res.F == 0) and np.all(res.tau == 0) and res.info == 1
    g = I.rng(2)
    a = g.standard_normal((60, 5)) @ g.standard_normal((5, 40))
    res = O.rqrcp(a, I.omega(12, 60, seed=3), 8)
    resid, orth = _residuals(a, res)
    assert resid <= 1e-14 and orth <= 1e-13


def test_rqrcp_quality_consistent_with_qrcp():
    """Sec. 5.3: RQRCP truncation error 'consistent with QRCP' (loose statistical bar)."""
    m = n = 160
    a = I.graded(m, n, 8, seed=12)
    _, _, jp = O.qrcp(a)
    Fq, _, _ = O.qrcp(a)
    ratios = []
    for seed in range(6):
        res = O.rqrcp(a, I.omega(24, m, seed=100 + seed), 16)
        for k in (16, 48, 96):
            err_r = np.linalg.norm(np.triu(res.F)[k:, k:])
            err_q = np.linalg.norm(np.triu(Fq)[k:, k:])
            ratios.append(err_r / err_q)
    assert np.median(ratios) <= 1.5 and max(ratios) <= 3.0


def test_rsrqrcp_runs_and_is_valid():
    m, n, b, p = 120, 100, 10, 6
    a = I.graded(m, n, 6, seed=13)
    draws = lambda J, l, mt: I.omega(l, mt, seed=1000 + J)
    res = O.rqrcp(a, I.omega(b + p, m, seed=14), b, mode="resample", resample=draws)
    resid, orth = _residuals(a, res)
    assert resid <= 1e-14


def test_column_norm_property_helper_on_the_oracle():
    """The full-size GPU check uses ||R(:, j)|| = ||A(:, jpvt[j])||; its helper is
    pinned here on the oracle's own factorisation (and a planted error in R)."""
    import sys, os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from gpu_util import column_norm_mismatch, r_column_norms
    a = I.graded(300, 240, 8, seed=5)
    for k in (None, 100):
        res = O.rqrcp(a, I.omega(40, 300, seed=6), 32, k)
        kk = res.k
        rn = r_column_norms(res.F, kk)
        an = np.linalg.norm(a, axis=0)[res.jpvt]
        assert column_norm_mismatch(rn, an) <= 1e-13
        F = res.F.copy()
        F[3, 50] *= 1.001                       # planted error in one R entry
        assert column_norm_mismatch(r_column_norms(F, kk), an) > 1e-7
