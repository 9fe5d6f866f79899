"""GPU parity: rq_tuxv (Alg. 6, j_max = 1, CUDA through the C ABI) against the FP64 oracle.

U, X, V are unique given the pivots (Householder QRs with the paper's sign
rule), so they are compared entry by entry: U X V^T within 1e-12 ||A||_F,
the factors within 1e-10 (the tail columns are only as well determined as the
gap between the retained singular values); with the core SVD, sigma within
1e-12 relative to sigma_1 and U, V after the sign convention.
"""
import numpy as np
import pytest

import oracle as O
from paper_2008_04447_gb300 import inputs as I

from gpu_util import build_and_handle, first_near_tie, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    return build_and_handle()


CASES = [
    (600, 400, 64, 32, 8, "lowrank"),
    (400, 700, 100, 32, 8, "graded"),
    (1000, 800, 128, 64, 8, "lowrank"),
    (200, 150, 17, 8, 4, "graded"),
]


def _inputs(m, n, k, kind):
    if kind == "graded":
        return I.graded(m, n, 8, seed=m + n + k)
    return I.lowrank_plus_noise(m, n, 2 * k, 1e-6, seed=m + k)


@pytest.mark.parametrize("m,n,k,b,p,kind", CASES)
def test_tuxv_fp64_matches_oracle(H, m, n, k, b, p, kind):
    import torch
    a = _inputs(m, n, k, kind)
    om = I.omega(b + p, m, seed=k)
    A = to_dev(a)
    U, X, V, _, info = H.tuxv(A, to_dev(om), b, p, k)
    torch.cuda.synchronize()
    U, X, V = to_host(U), to_host(X), to_host(V)
    ref = O.tuxv(a, om, b, k)
    nrm = np.linalg.norm(a)
    assert int(info.cpu()[0]) == 0
    assert np.allclose(U.T @ U, np.eye(k), atol=1e-12)
    assert np.allclose(V.T @ V, np.eye(k), atol=1e-12)
    assert np.allclose(X, np.triu(X))
    assert np.max(np.abs(U @ X @ V.T - ref.U @ ref.X @ ref.V.T)) <= 1e-12 * nrm
    if first_near_tie(ref.tr.gaps, b, 1e-6) is None:
        assert np.max(np.abs(X - ref.X)) <= 1e-12 * nrm
        assert np.max(np.abs(V - ref.V)) <= 1e-10
    err = np.linalg.norm(a - U @ X @ V.T)
    err_ref = np.linalg.norm(a - ref.U @ ref.X @ ref.V.T)
    assert abs(err - err_ref) <= 1e-10 * nrm


def test_tuxv_core_svd_matches_oracle(H):
    import torch
    m, n, k, b, p = 700, 500, 48, 16, 8
    a = I.graded(m, n, 8, seed=7)
    om = I.omega(b + p, m, seed=8)
    U, X, V, s, info = H.tuxv(to_dev(a), to_dev(om), b, p, k, svd=True)
    torch.cuda.synchronize()
    U, X, V, s = to_host(U), to_host(X), to_host(V), to_host(s)
    ref = O.tuxv(a, om, b, k, svd=True)
    assert np.all(np.diff(s) <= 0)
    assert np.max(np.abs(s - ref.sigma)) <= 1e-12 * ref.sigma[0]
    assert np.allclose(X, np.diag(s))
    # singular vectors: equal after the sign convention, for well separated sigma
    gap = np.minimum(np.r_[np.inf, -np.diff(ref.sigma)], np.r_[-np.diff(ref.sigma), np.inf]) / ref.sigma[0]
    ok = gap > 1e-6
    assert np.max(np.abs(V[:, ok] - ref.V[:, ok])) <= 1e-9
    assert np.max(np.abs(U[:, ok] - ref.U[:, ok])) <= 1e-9
    assert np.linalg.norm(a - (U * s) @ V.T) <= np.linalg.norm(a - ref.U @ ref.X @ ref.V.T) * (1 + 1e-10)


def test_tuxv_error_bounds(H):
    """err(TUXV) <= err(TRQRCP truncation) and >= Eckart-Young (Sec. 4.2)."""
    import torch
    m, n, k, b, p = 900, 700, 96, 32, 8
    a = I.lowrank_plus_noise(m, n, 300, 1e-6, seed=11)
    om = I.omega(b + p, m, seed=12)
    U, X, V, _, info = H.tuxv(to_dev(a), to_dev(om), b, p, k)
    Y, tau, R, jpvt, info2 = H.trqrcp(to_dev(a), to_dev(om), b, p, k)
    torch.cuda.synchronize()
    U, X, V, R = to_host(U), to_host(X), to_host(V), to_host(R)
    na2 = np.linalg.norm(a) ** 2
    err = np.linalg.norm(a - U @ X @ V.T)
    assert abs(err ** 2 - (na2 - np.linalg.norm(X) ** 2)) <= 1e-10 * na2
    err_tr = np.sqrt(max(na2 - np.linalg.norm(R) ** 2, 0.0))
    s = np.linalg.svd(a, compute_uv=False)
    assert err <= err_tr * (1 + 1e-10)
    assert err >= np.sqrt(np.sum(s[k:] ** 2)) * (1 - 1e-10)


@pytest.mark.parametrize("jmax", [2, 3, 4])
def test_tuxv_iterations_match_oracle(H, jmax):
    """rq_tuxv_iter (Alg. 6 with j_max > 1) against the oracle's iterations:
    U X V^T within 1e-12 ||A||_F, X lower triangular after an even step and
    upper after an odd one, X entry by entry within 1e-12 ||A||_F when no
    sample decision is a near-tie, and the rank-k error non-increasing in j."""
    import torch
    m, n, k, b, p = 600, 400, 48, 16, 8
    a = I.graded(m, n, 3, seed=17)     # slow decay: the refinement changes the error
    om = I.omega(b + p, m, seed=18)
    A, Om = to_dev(a), to_dev(om)
    U, X, V, _, info = H.tuxv(A, Om, b, p, k, jmax=jmax)
    torch.cuda.synchronize()
    U, X, V = to_host(U), to_host(X), to_host(V)
    ref = O.tuxv(a, om, b, k, jmax=jmax)
    nrm = np.linalg.norm(a)
    assert int(info.cpu()[0]) == 0
    assert np.allclose(U.T @ U, np.eye(k), atol=1e-12)
    assert np.allclose(V.T @ V, np.eye(k), atol=1e-12)
    tri = np.tril(X) if jmax % 2 == 0 else np.triu(X)
    assert np.array_equal(X, tri)
    assert np.max(np.abs(U @ X @ V.T - ref.U @ ref.X @ ref.V.T)) <= 1e-12 * nrm
    if first_near_tie(ref.tr.gaps, b, 1e-6) is None:
        assert np.max(np.abs(X - ref.X)) <= 1e-12 * nrm
    errs = []
    for j in range(1, jmax + 1):
        Uj, Xj, Vj, _, _ = H.tuxv(A, Om, b, p, k, jmax=j)
        torch.cuda.synchronize()
        errs.append(np.linalg.norm(a - to_host(Uj) @ to_host(Xj) @ to_host(Vj).T))
    assert all(e2 <= e1 * (1 + 1e-12) for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < errs[0]


@pytest.mark.parametrize("mode", ["fp64", "mixed"])
def test_tuxv_iterations_with_core_svd(H, mode):
    import torch
    from paper_2008_04447_gb300 import RQ_MIXED
    m, n, k, b, p = 500, 700, 40, 16, 8
    a = I.graded(m, n, 3, seed=27)
    om = I.omega(b + p, m, seed=28)
    if mode == "mixed":
        a32, o32 = (np.asarray(x, np.float32).astype(np.float64) for x in (a, om))
        U, X, V, s, info = H.tuxv(to_dev(a32, torch.float32), to_dev(o32, torch.float32), b, p, k, svd=True,
                                  prec=RQ_MIXED, jmax=2)
        ref = O.tuxv(a32, o32, b, k, jmax=2, svd=True, sketch_inputs="bf16")
        tol_s, tol_o = 1e-5, 1e-5
    else:
        U, X, V, s, info = H.tuxv(to_dev(a), to_dev(om), b, p, k, svd=True, jmax=2)
        ref = O.tuxv(a, om, b, k, jmax=2, svd=True)
        tol_s, tol_o = 1e-12, 1e-12
    torch.cuda.synchronize()
    U, X, V, s = to_host(U), to_host(X), to_host(V), to_host(s)
    assert np.all(np.diff(s) <= 0)
    assert np.allclose(X, np.diag(s))
    assert np.allclose(U.T @ U, np.eye(k), atol=tol_o) and np.allclose(V.T @ V, np.eye(k), atol=tol_o)
    if first_near_tie(ref.tr.gaps, b, 1e-6 if mode == "fp64" else 1e-4) is None:
        assert np.max(np.abs(s - ref.sigma)) <= tol_s * ref.sigma[0]
    e = np.linalg.norm(a - (U * s) @ V.T)
    e_ref = np.linalg.norm(a - ref.U @ ref.X @ ref.V.T)
    assert e <= e_ref * (1 + (1e-10 if mode == "fp64" else 0.05))
