"""Oracle pins over a sweep of tiny and degenerate shapes: m from 1 to 9, n
from 1 to 7, block sizes below and above n, p = 0, k = 1 and k = min(m, n),
samples with l >= m and l < m -- the edges the GPU parity cases reach.  Each
case checks what holds for any input:

* RQRCP (Alg. 4): jpvt is a permutation, A P = Q R to 1e-13 ||A||_F and Q is
  orthogonal to 1e-13;
* with an Omega of orthonormal columns (l >= m) every sample norm is exact, so
  the pivots are brute-force QRCP's (columns scaled 3^-j keep every decision
  apart);
* TRQRCP (Alg. 5) reproduces RQRCP's pivots and the first k rows of R to
  1e-12 ||A||_F;
* TUXV (Alg. 6): U and V orthonormal, ||A - U X V^T||^2 = ||A||^2 - ||X||^2,
  and its error is at most TRQRCP's, ||A||^2 - ||R||^2 (both to 1e-12 ||A||^2).
"""
import itertools

import numpy as np

import oracle as O
from paper_2008_04447_gb300 import inputs as I

SHAPES = list(itertools.product((1, 2, 3, 5, 9), (1, 2, 4, 7), (1, 2, 3, 8), (0, 2)))


def _input(m, n, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((m, n)) * 3.0 ** -np.arange(n)[g.permutation(n)]


def test_rqrcp_factorises_every_tiny_shape():
    for m, n, b, p in SHAPES:
        a = _input(m, n, 7 * m + n)
        om = np.random.default_rng(m * n + b + p).standard_normal((b + p, m))
        for k in sorted({1, min(m, n)}):
            res = O.rqrcp(a, om, b, k)
            assert np.array_equal(np.sort(res.jpvt), np.arange(n))
            Qf = O.form_q(res.F, res.tau, m)
            Rf = np.triu(res.F)
            Rf[k:, k:] = res.F[k:, k:]
            nrm = np.linalg.norm(a)
            assert np.linalg.norm(a[:, res.jpvt] - Qf @ Rf) <= 1e-13 * nrm, (m, n, b, p, k)
            assert np.linalg.norm(Qf.T @ Qf - np.eye(m)) <= 1e-13, (m, n, b, p, k)


def test_orthonormal_omega_gives_qrcp_pivots_on_tiny_shapes():
    for m, n, b, p in SHAPES:
        a = _input(m, n, 11 * m + n)
        om = I.haar(m + p + b, m, I.rng(m + 17 * n))      # l x m, orthonormal columns, l >= m
        k = min(m, n)
        res = O.rqrcp(a, om, b, k)
        _, _, jp_bf = O.qrcp(a, ncols=k)
        assert np.array_equal(res.jpvt[:k], jp_bf[:k]), (m, n, b, p)


def test_trqrcp_and_tuxv_on_tiny_shapes():
    for m, n, b, p in SHAPES:
        a = _input(m, n, 13 * m + n)
        om = np.random.default_rng(5 * m + n + b + p).standard_normal((b + p, m))
        nrm2 = float(np.sum(a * a))
        for k in sorted({1, min(m, n)}):
            full = O.rqrcp(a, om, b, k)
            tr = O.trqrcp(a, om, b, k)
            assert np.array_equal(tr.jpvt, full.jpvt), (m, n, b, p, k)
            assert np.max(np.abs(tr.R - np.triu(full.F[:k, :]))) <= 1e-12 * nrm2 ** 0.5
            t = O.tuxv(a, om, b, k)
            assert np.allclose(t.U.T @ t.U, np.eye(k), atol=1e-13)
            assert np.allclose(t.V.T @ t.V, np.eye(k), atol=1e-13)
            e2 = float(np.sum((a - t.U @ t.X @ t.V.T) ** 2))
            assert abs(e2 - (nrm2 - float(np.sum(t.X * t.X)))) <= 1e-12 * nrm2, (m, n, b, p, k)
            assert e2 <= nrm2 - float(np.sum(tr.R * tr.R)) + 1e-12 * nrm2, (m, n, b, p, k)
