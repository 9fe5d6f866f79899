"""Plain FP64 CPU oracle for RQRCP, TRQRCP and TUXV (Duersch & Gu, arXiv 2008.04447).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this module; only the test-suite, the smoke check and the benchmark's
CPU-baseline leg use it.  It shares no code with the CUDA library.

Everything is written step by step in the order and notation of the paper, in
float64 numpy, with numpy/scipy library primitives (matrix products,
triangular solves) as single steps.  It is slow on purpose.

Conventions (readings of the paper, listed with their reasons in the design
notes):

* Matrices are numpy arrays; ``A`` is m x n.  Column permutations are index
  vectors: ``jpvt`` with ``A[:, jpvt] = Q R`` (0-based).
* Reflectors (Sec. 2): y = a - (-sign(a_1) ||a|| e_1), tau = 2 / y^T y,
  H = I - y tau y^T.  They are stored normalised, v = y / y_1 (so v_1 = 1),
  with the matching tau_v = 2 / v^T v; sign(0) is taken as +1; a zero column
  gives tau = 0, H = I and a zero diagonal.
* Pivot ties go to the lowest current (permuted) column position.
* Trailing column norms of the sample are downdated by removing the
  contribution of the row just finished (Alg. 1), in squared form, and
  recomputed from the remaining rows when the downdated value falls to
  ``sqrt(eps)`` times the value it had when last computed exactly.
* The sample update (Eq. update1) is evaluated as
  B_1 = S_12 - Omegahat_11 R_12 with Omegahat_11 = S_11 R_11^{-1} (Sec. 3.4
  obtains Omegahat_11 from S_11 and R_11); a zero diagonal of R_11
  zeroes the corresponding column of Omegahat_11.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

EPS = np.finfo(np.float64).eps
DOWNDATE_TOL = math.sqrt(EPS)

__all__ = [
    "reflector", "apply_reflector", "qr_householder", "form_q", "larft", "qrcp",
    "sample_qrcp", "SampleQRCP", "rqrcp", "RQRCPResult", "trqrcp", "TRQRCPResult",
    "tuxv", "TUXVResult", "jacobi_svd", "unpack_rqrcp", "qr_unpivoted", "reflectors_of",
    "sample_update", "round_bf16", "sketch",
]


# ----------------------------------------------------------------------------
# Householder building blocks (Sec. 2, Alg. 1; compound WY, Sec. 4.1)
# ----------------------------------------------------------------------------

def reflector(a):
    """Householder reflection of column ``a`` (Sec. 2).

    Returns (v, tau, beta): H = I - v tau v^T with v[0] = 1 maps a to beta*e_1,
    beta = -sign(a_1) ||a||_2 (sign(0) = +1).  The zero vector gives tau = 0.
    """
    a = np.asarray(a, dtype=np.float64)
    nrm = math.sqrt(float(a @ a))
    v = np.zeros_like(a)
    v[0] = 1.0
    if nrm == 0.0:
        return v, 0.0, 0.0
    sgn = 1.0 if a[0] >= 0.0 else -1.0
    beta = -sgn * nrm
    y = a.copy()
    y[0] = a[0] - beta          # y = a - beta e_1, |y_1| >= |a_1|
    v = y / y[0]                # same reflection, scaled so that v_1 = 1
    tau = 2.0 / float(v @ v)    # tau = 2 / v^T v, as tau = 2 / y^T y for y
    return v, tau, beta


def apply_reflector(v, tau, C):
    """C <- (I - v tau v^T) C, in place (C has len(v) rows)."""
    if tau == 0.0 or C.shape[1] == 0:
        return C
    w = v @ C
    C -= np.outer(tau * v, w)
    return C


def qr_householder(A, ncols=None):
    """Unblocked Householder QR (Alg. 1 without pivoting), LAPACK-style packing.

    Returns (F, tau): R on and above the diagonal of F, reflectors v (v_1 = 1
    implicit) below it; ``ncols`` reflectors (default min(m, n)).
    """
    F = np.array(A, dtype=np.float64, copy=True)
    m, n = F.shape
    kk = min(m, n) if ncols is None else ncols
    tau = np.zeros(kk)
    for j in range(kk):
        v, t, beta = reflector(F[j:, j])
        apply_reflector(v, t, F[j:, j + 1:])
        F[j, j] = beta
        F[j + 1:, j] = v[1:]
        tau[j] = t
    return F, tau


def reflectors_of(F, k):
    """Explicit m x k Y (unit diagonal, zeros above) from packed storage."""
    m = F.shape[0]
    Y = np.tril(F[:, :k], -1)
    Y[np.arange(k), np.arange(k)] = 1.0
    return Y[:m]


def form_q(F, tau, ncols):
    """First ``ncols`` columns of Q = H_1 H_2 ... H_k from packed reflectors."""
    m = F.shape[0]
    k = len(tau)
    Q = np.zeros((m, ncols))
    Q[np.arange(min(m, ncols)), np.arange(min(m, ncols))] = 1.0
    for j in range(k - 1, -1, -1):
        v = np.concatenate(([1.0], F[j + 1:, j]))
        apply_reflector(v, tau[j], Q[j:, :])
    return Q


def larft(Y, tau):
    """Upper triangular T with H_1 ... H_b = I - Y T Y^T.

    Built by composing one reflector at a time with the compound WY rule of
    Sec. 4.1: T = [[T_1, -T_1 Y_1^T Y_2 T_2], [0, T_2]] with T_2 = tau_j.
    """
    b = len(tau)
    T = np.zeros((b, b))
    for j in range(b):
        T[j, j] = tau[j]
        if j:
            T[:j, j] = -T[:j, :j] @ (Y[:, :j].T @ Y[:, j]) * tau[j]
    return T


def qr_unpivoted(A):
    """Unpivoted Householder QR of A (the performance ceiling, Table 3's QR)."""
    return qr_householder(A)


# ----------------------------------------------------------------------------
# QRCP (Alg. 1) with exactly recomputed norms: the brute-force reference
# ----------------------------------------------------------------------------

def qrcp(A, ncols=None):
    """Alg. 1, with the trailing norms recomputed exactly at every step.

    Returns (F, tau, jpvt): packed R / reflectors, A[:, jpvt] = Q R.
    """
    F = np.array(A, dtype=np.float64, copy=True)
    m, n = F.shape
    kk = min(m, n) if ncols is None else ncols
    jpvt = np.arange(n)
    tau = np.zeros(kk)
    for j in range(kk):
        norms2 = np.einsum("ij,ij->j", F[j:, j:], F[j:, j:])
        p = j + int(np.argmax(norms2))          # first maximum = lowest position
        if p != j:
            F[:, [j, p]] = F[:, [p, j]]
            jpvt[[j, p]] = jpvt[[p, j]]
        v, t, beta = reflector(F[j:, j])
        apply_reflector(v, t, F[j:, j + 1:])
        F[j, j] = beta
        F[j + 1:, j] = v[1:]
        tau[j] = t
    return F, tau, jpvt


# ----------------------------------------------------------------------------
# Partial QRCP of the sample (Sec. 3.2; the pivot step of Alg. 4)
# ----------------------------------------------------------------------------

@dataclass
class SampleQRCP:
    S: np.ndarray          # l x n_t: [S11 S12; 0 S22] after `steps` steps (permuted order)
    perm: np.ndarray       # new position -> old position (length n_t)
    swaps: np.ndarray      # swaps[i] = position exchanged with position i at step i
    V: np.ndarray          # l x steps reflectors of U (unit diagonal, zeros above)
    tau: np.ndarray        # steps
    gaps: np.ndarray       # per decision: (best - runner-up) / best in squared norm
    recomputed: int = 0    # number of exact norm recomputations


def sample_qrcp(B, steps, downdate_tol=DOWNDATE_TOL):
    """``steps`` steps of Alg. 1 on the sample B (l x n_t), norms downdated.

    Returns the partially factorised sample S = U^T B P with the pivot order.
    """
    S = np.array(B, dtype=np.float64, copy=True)
    l, nt = S.shape
    perm = np.arange(nt)
    swaps = np.zeros(steps, dtype=np.int64)
    V = np.zeros((l, steps))
    taus = np.zeros(steps)
    gaps = np.full(steps, np.inf)
    nu2 = np.einsum("ij,ij->j", S, S)      # trailing squared norms
    ref2 = nu2.copy()                       # value at the last exact computation
    recomputed = 0
    for i in range(steps):
        cand = nu2[i:]
        p = i + int(np.argmax(cand))
        if cand.size > 1:
            best = cand[p - i]
            rest = np.delete(cand, p - i)
            second = float(rest.max())
            gaps[i] = (best - second) / best if best > 0 else 0.0
        swaps[i] = p
        if p != i:
            S[:, [i, p]] = S[:, [p, i]]
            nu2[[i, p]] = nu2[[p, i]]
            ref2[[i, p]] = ref2[[p, i]]
            perm[[i, p]] = perm[[p, i]]
        if i < l:
            v, t, beta = reflector(S[i:, i])
            apply_reflector(v, t, S[i:, i + 1:])
            S[i, i] = beta
            S[i + 1:, i] = 0.0
            V[i:, i] = v
            taus[i] = t
            # remove the contribution of row i from the trailing norms (Alg. 1);
            # recompute exactly where the downdated value lost its accuracy
            nu2[i + 1:] -= S[i, i + 1:] * S[i, i + 1:]
            lost = np.nonzero(nu2[i + 1:] <= downdate_tol * ref2[i + 1:])[0] + i + 1
            if lost.size:
                nu2[lost] = np.einsum("ij,ij->j", S[i + 1:, lost], S[i + 1:, lost])
                ref2[lost] = nu2[lost]
                recomputed += lost.size
        else:
            V[:, i] = 0.0
    return SampleQRCP(S, perm, swaps, V, taus, gaps, recomputed)


def _omegahat11(S11, R11):
    """Omegahat_11 = S_11 R_11^{-1} (Sec. 3.2); zero diagonal of R_11 -> zero column."""
    b = S11.shape[0]
    X = np.zeros_like(S11)
    for j in range(b):
        rhs = S11[:, j] - X[:, :j] @ R11[:j, j]
        X[:, j] = 0.0 if R11[j, j] == 0.0 else rhs / R11[j, j]
    return X


def sample_update(S, bj, R11, R12):
    """Eq. (update1): next sample [S12 - S11 R11^{-1} R12 ; S22]."""
    S11 = np.triu(S[:bj, :bj])
    S12 = S[:bj, bj:]
    S22 = S[bj:, bj:]
    B1 = S12 - _omegahat11(S11, R11) @ R12
    return np.vstack([B1, S22])


# ----------------------------------------------------------------------------
# RQRCP (Alg. 4), optional repeated sampling (RSRQRCP) or explicit sample
# ----------------------------------------------------------------------------

@dataclass
class RQRCPResult:
    F: np.ndarray              # packed: R (k x n) on/above diag, reflectors below, trailing block
    tau: np.ndarray
    jpvt: np.ndarray
    k: int
    gaps: list = field(default_factory=list)      # per block: decision gaps
    samples: list = field(default_factory=list)   # per block: the sample used (if kept)
    omegahat: list = field(default_factory=list)  # explicit mode: (Omegahat, S, R11) per block
    sample_norms: list = field(default_factory=list)  # ||B||_F of the sample used by each block
    info: int = 0


def rqrcp(A, Omega, b, k=None, mode="update", keep_samples=False, resample=None,
          pivot=True):
    """Randomized QR with column pivoting, Alg. 4.

    mode = "update":   sample refreshed with Eq. (update1) (the paper's RQRCP);
    mode = "explicit": the same compression matrix formed explicitly,
                       Omega^[J] = (U^T Omega^[J-1] Q)(b:, b:), and applied to the
                       trailing matrix (a brute-force check of Eq. update1);
    mode = "resample": a fresh Gaussian per block, drawn by ``resample(J, l, m_t)``
                       (RSRQRCP, Sec. 3.4).
    pivot = False gives unpivoted blocked QR (same arithmetic without sampling).
    """
    F = np.array(A, dtype=np.float64, copy=True)
    m, n = F.shape
    Omega = np.asarray(Omega, dtype=np.float64)
    l = Omega.shape[0]
    if k is None:
        k = min(m, n)
    jpvt = np.arange(n)
    tau = np.zeros(k)
    res = RQRCPResult(F, tau, jpvt, k)
    Om = Omega.copy()                          # current compression matrix (explicit mode)
    B = Omega @ F if pivot else None           # Alg. 4: initial sample
    for j0 in range(0, k, b):
        bj = min(b, k - j0)
        if pivot:
            if keep_samples:
                res.samples.append(B.copy())
            sq = sample_qrcp(B, bj)
            res.gaps.append(sq.gaps)
            res.sample_norms.append(float(np.linalg.norm(B)))
            F[:, j0:] = F[:, j0:][:, sq.perm]   # permute A and completed rows of R
            jpvt[j0:] = jpvt[j0:][sq.perm]
        # b reflectors of the panel, then Q^T applied to the trailing columns
        for i in range(bj):
            c = j0 + i
            v, t, beta = reflector(F[c:, c])
            apply_reflector(v, t, F[c:, c + 1:])
            F[c, c] = beta
            F[c + 1:, c] = v[1:]
            tau[c] = t
        if not pivot or j0 + bj >= k:
            continue
        R11 = np.triu(F[j0:j0 + bj, j0:j0 + bj])
        R12 = F[j0:j0 + bj, j0 + bj:]
        if mode == "update":
            B = sample_update(sq.S, bj, R11, R12)
        elif mode == "explicit":
            # Omega^[J] = U^T Omega^[J-1] Q^[J] without its leading bj columns
            Ut_Om = Om.copy()
            for i in range(bj):
                if i < l:
                    apply_reflector(sq.V[i:, i], sq.tau[i], Ut_Om[i:, :])
            Qblk = form_q(F[j0:, j0:j0 + bj], tau[j0:j0 + bj], m - j0)
            Omh = Ut_Om @ Qblk                 # l x m_t (= U^T Omega Q)
            res.omegahat.append((Omh.copy(), sq.S.copy(), R11.copy()))
            Om = Omh[:, bj:]
            B = Om @ F[j0 + bj:, j0 + bj:]
        elif mode == "resample":
            Om = np.asarray(resample(j0 // b + 1, l, m - j0 - bj), dtype=np.float64)
            B = Om @ F[j0 + bj:, j0 + bj:]
        else:
            raise ValueError(mode)
    d = np.abs(np.diag(F[:k, :k]))
    zero = np.nonzero(d == 0.0)[0]
    res.info = int(zero[0]) + 1 if zero.size else 0
    return res


def unpack_rqrcp(res):
    """(Q_k, R_k) with A[:, jpvt] ~= Q_k R_k (Q_k m x k explicit, R_k k x n)."""
    F, k = res.F, res.k
    Q = form_q(F, res.tau, k)
    R = np.triu(F[:k, :])
    return Q, R


# ----------------------------------------------------------------------------
# Truncated RQRCP (Alg. 5)
# ----------------------------------------------------------------------------

@dataclass
class TRQRCPResult:
    Y: np.ndarray          # m x k reflectors (unit diagonal, zeros above)
    tau: np.ndarray        # k
    R: np.ndarray          # k x n, pivoted column order
    jpvt: np.ndarray       # n
    Wt: np.ndarray         # k x n accumulated inner products W^T = T^T Y^T A P
    k: int
    gaps: list = field(default_factory=list)
    sample_norms: list = field(default_factory=list)
    info: int = 0


def round_bf16(x):
    """Round to the nearest bfloat16 (ties to even), via float32; returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)


def sketch(Omega, A, inputs=None):
    """The sample B = Omega A (Alg. 4); inputs="bf16" first rounds Omega and A to
    bfloat16, the precision a reduced-precision sketch multiplies in, so that the
    pivot decisions taken from B are taken in the same precision as there."""
    if inputs == "bf16":
        return round_bf16(Omega) @ round_bf16(A)
    return Omega @ A


def trqrcp(A, Omega, b, k, sketch_inputs=None):
    """Alg. 5: RQRCP without the trailing update, through W^T = T^T Y^T A (Sec. 4.1)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    Omega = np.asarray(Omega, dtype=np.float64)
    Ap = A.copy()                  # A^[J]: the original matrix with the current column order
    jpvt = np.arange(n)
    Y = np.zeros((m, k))
    Wt = np.zeros((k, n))
    R = np.zeros((k, n))
    tau = np.zeros(k)
    gaps = []
    B = sketch(Omega, Ap, sketch_inputs)
    norms = []
    for j0 in range(0, k, b):
        bj = min(b, k - j0)
        norms.append(float(np.linalg.norm(B)))
        sq = sample_qrcp(B, bj)
        gaps.append(sq.gaps)
        # permute A^[J], W_1^T and the leading rows of R
        Ap[:, j0:] = Ap[:, j0:][:, sq.perm]
        Wt[:j0, j0:] = Wt[:j0, j0:][:, sq.perm]
        R[:j0, j0:] = R[:j0, j0:][:, sq.perm]
        jpvt[j0:] = jpvt[j0:][sq.perm]
        # selected columns of A^[J] - Y^[J-1] W_1^T
        Ahat = Ap[:, j0:j0 + bj] - Y[:, :j0] @ Wt[:j0, j0:j0 + bj]
        # reflectors Y_2 from rows j0: of the selected columns
        P, t2 = qr_householder(Ahat[j0:, :])
        Y2 = np.zeros((m, bj))
        Y2[j0:, :] = reflectors_of(P, bj)
        tau[j0:j0 + bj] = t2
        T2 = larft(Y2, t2)
        # W_2^T = T_2^T (Y_2^T A^[J] - (Y_2^T Y^[J-1]) W_1^T)
        W2t = T2.T @ (Y2.T @ Ap - (Y2.T @ Y[:, :j0]) @ Wt[:j0, :])
        Y[:, j0:j0 + bj] = Y2
        Wt[j0:j0 + bj, :] = W2t
        # new rows of R from A^[J] - Y^[J] W^[J]T (R_11 straight from the panel)
        R[j0:j0 + bj, j0:j0 + bj] = np.triu(P[:bj, :bj])
        R[j0:j0 + bj, j0 + bj:] = (Ap[j0:j0 + bj, j0 + bj:]
                                   - Y[j0:j0 + bj, :j0 + bj] @ Wt[:j0 + bj, j0 + bj:])
        if j0 + bj < k:
            B = sample_update(sq.S, bj, R[j0:j0 + bj, j0:j0 + bj], R[j0:j0 + bj, j0 + bj:])
    d = np.abs(np.diag(R[:, :k]))
    zero = np.nonzero(d == 0.0)[0]
    return TRQRCPResult(Y, tau, R, jpvt, Wt, k, gaps, norms, int(zero[0]) + 1 if zero.size else 0)


# ----------------------------------------------------------------------------
# One-sided Jacobi SVD (Hestenes 1958), for the k x k core of TUXV
# ----------------------------------------------------------------------------

def jacobi_svd(X, tol=1e-15, max_sweeps=60):
    """SVD X = U diag(s) V^T by cyclic one-sided Jacobi rotations of columns.

    Columns p < q are rotated to be orthogonal whenever
    |x_p^T x_q| > tol * ||x_p|| ||x_q||; sweeps stop when none is rotated.
    s is sorted in descending order.
    """
    W = np.array(X, dtype=np.float64, copy=True)
    nr, nc = W.shape
    V = np.eye(nc)
    for _ in range(max_sweeps):
        rotated = False
        for p in range(nc - 1):
            for q in range(p + 1, nc):
                alpha = float(W[:, p] @ W[:, p])
                beta = float(W[:, q] @ W[:, q])
                gamma = float(W[:, p] @ W[:, q])
                if gamma == 0.0 or abs(gamma) <= tol * math.sqrt(alpha * beta):
                    continue
                rotated = True
                zeta = (beta - alpha) / (2.0 * gamma)
                t = math.copysign(1.0, zeta) / (abs(zeta) + math.sqrt(1.0 + zeta * zeta))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = c * t
                wp = W[:, p].copy()
                W[:, p] = c * wp - s * W[:, q]
                W[:, q] = s * wp + c * W[:, q]
                vp = V[:, p].copy()
                V[:, p] = c * vp - s * V[:, q]
                V[:, q] = s * vp + c * V[:, q]
        if not rotated:
            break
    sv = np.sqrt(np.einsum("ij,ij->j", W, W))
    order = np.argsort(-sv, kind="stable")
    sv = sv[order]
    W = W[:, order]
    V = V[:, order]
    U = np.zeros_like(W)
    nz = sv > 0
    U[:, nz] = W[:, nz] / sv[nz]
    return U, sv, V


# ----------------------------------------------------------------------------
# TUXV (Alg. 6)
# ----------------------------------------------------------------------------

@dataclass
class TUXVResult:
    U: np.ndarray      # m x k, orthonormal columns
    X: np.ndarray      # k x k (upper triangular for odd j_max; diag(sigma) if svd)
    V: np.ndarray      # n x k, orthonormal columns
    sigma: np.ndarray | None
    tr: TRQRCPResult


def _qr_explicit(Z):
    """Householder QR of tall Z (p x k): explicit Q (p x k) and upper triangular R (k x k)."""
    F, t = qr_householder(Z)
    k = Z.shape[1]
    return form_q(F, t, k), np.triu(F[:k, :k])


def _fix_signs(U, V):
    """Make the largest-magnitude entry of each column of V positive (U follows)."""
    idx = np.argmax(np.abs(V), axis=0)
    s = np.sign(V[idx, np.arange(V.shape[1])])
    s[s == 0] = 1.0
    return U * s, V * s


def tuxv(A, Omega, b, k, jmax=1, svd=False, sketch_inputs=None):
    """Alg. 6: A ~= U X V^T with TRQRCP, an LQ of R P^T and a QR of A V_1."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    tr = trqrcp(A, Omega, b, k, sketch_inputs=sketch_inputs)
    Z = np.zeros((k, n))
    Z[:, tr.jpvt] = tr.R                     # Z^(0) = R^(0) P^(0)T
    V, Xt = _qr_explicit(Z.T)                # LQ of Z^(0) through QR of its transpose
    X = Xt.T
    U = None
    for j in range(1, jmax + 1):
        if j % 2 == 1:
            U, X = _qr_explicit(A @ V)        # Z^(j) = A V^(j)(:, 1:k)
        else:
            V, Xt = _qr_explicit((U.T @ A).T)  # Z^(j) = U^(j)(:, 1:k)^T A
            X = Xt.T
    sigma = None
    if svd:
        Uh, sigma, Vh = jacobi_svd(X)
        U = U @ Uh
        V = V @ Vh
        U, V = _fix_signs(U, V)
        X = np.diag(sigma)
    return TUXVResult(U, X, V, sigma, tr)
