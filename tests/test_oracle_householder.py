"""Pins for the oracle's Householder building blocks (Sec. 2, Sec. 4.1).

Checked against LAPACK (dgeqrf through scipy, a second implementation) and
against definitions (H a = beta e_1, orthogonality, compound WY products).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle as O
from paper_2008_04447_gb300 import inputs as I


def test_reflector_maps_to_e1_and_is_orthogonal():
    g = I.rng(1)
    for n in (1, 2, 5, 17):
        a = g.standard_normal(n)
        v, tau, beta = O.reflector(a)
        H = np.eye(n) - tau * np.outer(v, v)
        e = np.zeros(n)
        e[0] = beta
        assert np.allclose(H @ a, e, atol=1e-14 * np.linalg.norm(a))
        assert np.allclose(H.T @ H, np.eye(n), atol=1e-14)
        assert v[0] == 1.0
        # sign rule of Sec. 2: beta = -sign(a_1)||a||
        assert np.sign(beta) == -np.sign(a[0]) or a[0] == 0
        assert abs(abs(beta) - np.linalg.norm(a)) <= 1e-14 * np.linalg.norm(a)


def test_reflector_sign_of_zero_and_zero_vector():
    v, tau, beta = O.reflector(np.array([0.0, 3.0, 4.0]))
    assert beta == -5.0  # sign(0) = +1
    v, tau, beta = O.reflector(np.zeros(4))
    assert tau == 0.0 and beta == 0.0 and v[0] == 1.0


@pytest.mark.parametrize("m,n", [(30, 20), (20, 30), (64, 64), (7, 1)])
def test_qr_householder_matches_lapack_dgeqrf(m, n):
    a = I.rng(m * 100 + n).standard_normal((m, n))
    F, tau = O.qr_householder(a)
    qr, tau_l, work, info = sla.lapack.dgeqrf(np.asfortranarray(a))
    assert info == 0
    # LAPACK dgeqrf uses the same sign rule (beta = -sign(alpha)||x||) and v_1 = 1,
    # except for a reflector of a single entry: LAPACK takes H = I (tau = 0) where
    # the paper's formula reflects (tau = 2, the row changes sign).
    if m <= n:
        assert tau_l[m - 1] == 0.0 and tau[m - 1] == 2.0
        qr = qr.copy()
        qr[m - 1, m - 1:] *= -1.0
        tau_l = tau_l.copy()
        tau_l[m - 1] = 2.0
    assert np.allclose(np.triu(F), np.triu(qr), atol=1e-13 * np.linalg.norm(a))
    assert np.allclose(tau, tau_l, atol=1e-13)
    assert np.allclose(np.tril(F, -1), np.tril(qr, -1), atol=1e-12)


def test_form_q_and_residual():
    a = I.rng(3).standard_normal((50, 30))
    F, tau = O.qr_householder(a)
    Q = O.form_q(F, tau, 30)
    assert np.allclose(Q.T @ Q, np.eye(30), atol=1e-14)
    assert np.linalg.norm(Q @ np.triu(F[:30]) - a) <= 1e-14 * np.linalg.norm(a)


def test_larft_compound_wy_equals_product_of_reflectors():
    m, b = 40, 9
    a = I.rng(4).standard_normal((m, b))
    F, tau = O.qr_householder(a)
    Y = O.reflectors_of(F, b)
    T = O.larft(Y, tau)
    assert np.allclose(T, np.triu(T))
    P = np.eye(m)
    for j in range(b):
        P = P @ (np.eye(m) - tau[j] * np.outer(Y[:, j], Y[:, j]))
    assert np.allclose(np.eye(m) - Y @ T @ Y.T, P, atol=1e-14)


def test_larft_two_block_composition_rule():
    """Sec. 4.1: (I - Y1 T1 Y1^T)(I - Y2 T2 Y2^T) = I - Y T Y^T, T12 = -T1 Y1^T Y2 T2."""
    m = 30
    a = I.rng(5).standard_normal((m, 10))
    F, tau = O.qr_householder(a)
    Y = O.reflectors_of(F, 10)
    T = O.larft(Y, tau)
    T1 = O.larft(Y[:, :4], tau[:4])
    T2 = O.larft(Y[:, 4:], tau[4:])
    T12 = -T1 @ Y[:, :4].T @ Y[:, 4:] @ T2
    assert np.allclose(T[:4, :4], T1, atol=1e-14)
    assert np.allclose(T[4:, 4:], T2, atol=1e-14)
    assert np.allclose(T[:4, 4:], T12, atol=1e-13)
