"""Helpers shared by the GPU parity tests (test-side checks only)."""
import numpy as np

import oracle as O


def build_and_handle():
    from paper_2008_04447_gb300 import build, Handle
    build.build()
    return Handle()


def to_dev(a, dtype=None):
    import torch
    from paper_2008_04447_gb300 import colmajor
    t = torch.as_tensor(np.asarray(a), dtype=dtype or torch.float64)
    return colmajor(t).cuda()


def to_host(t):
    return t.detach().cpu().double().numpy()


def first_near_tie(gaps_per_block, b, thr, sample_norms=None):
    """Global pivot index of the first decision whose relative gap is below thr.

    With sample_norms, the threshold of block J grows by ||B^[0]|| / ||B^[J]||:
    the update formula cancels entries of the first sample's size, so a sample
    held in precision u is accurate to about u ||B^[0]|| / ||B^[J]|| relative.
    """
    for J, g in enumerate(gaps_per_block):
        t = thr
        if sample_norms is not None and sample_norms[J] > 0:
            t = thr * sample_norms[0] / sample_norms[J]
        idx = np.nonzero(np.asarray(g) < t)[0]
        if idx.size:
            return J * b + int(idx[0])
    return None


def factor_quality(a, F, tau, jpvt, k):
    """Residual ||A P - Q R|| / ||A|| and ||Q^T Q - I|| from packed GPU outputs (FP64 host)."""
    m, n = F.shape
    Qf = O.form_q(F, tau, m)
    Rf = np.triu(F)
    Rf[k:, k:] = F[k:, k:]
    resid = np.linalg.norm(a[:, jpvt] - Qf @ Rf) / np.linalg.norm(a)
    orth = np.linalg.norm(Qf.T @ Qf - np.eye(m))
    return resid, orth


def column_norm_mismatch(Fcols_r_norms, a_cols_norms):
    """max_j | ||R(:, j)|| - ||A(:, jpvt[j])|| | / ||A(:, jpvt[j])|| (0 / 0 taken as 0).

    An orthogonal transform preserves column norms, so the R of A P = Q R has
    ||R(:, j)|| = ||A(:, jpvt[j])|| for every j, at any size."""
    r = np.asarray(Fcols_r_norms, dtype=np.float64)
    a = np.asarray(a_cols_norms, dtype=np.float64)
    den = np.where(a > 0, a, 1.0)
    return float(np.max(np.abs(r - a) / den))


def r_column_norms(F, k):
    """||R(:, j)|| from a packed factorisation F (R on and above the diagonal in
    rows < k; rows >= k of columns >= k hold the trailing block R22)."""
    F = np.asarray(F)
    m, n = F.shape
    out = np.empty(n)
    for j in range(n):
        top = F[: min(j + 1, k), j]
        tail = F[k:, j] if j >= k else np.zeros(0)
        out[j] = np.sqrt(np.sum(top * top) + np.sum(tail * tail))
    return out


def fp64_oracle_error(a, om, b, k):
    """Rank-k error ||A - U X V^T||_F / ||A||_F of the plain FP64 oracle (Alg. 6,
    j_max = 1, FP64 sketch) on the FP64 input: the reference every
    reduced-precision TUXV result is held to (within 1.05x, per problem)."""
    a = np.asarray(a, dtype=np.float64)
    ref = O.tuxv(a, np.asarray(om, dtype=np.float64), b, k)
    return float(np.linalg.norm(a - ref.U @ ref.X @ ref.V.T) / np.linalg.norm(a)), ref


def rank_k_error(a, U, X, V):
    """||A - U X V^T||_F / ||A||_F in FP64 against the FP64 input."""
    a = np.asarray(a, dtype=np.float64)
    return float(np.linalg.norm(a - U @ X @ V.T) / np.linalg.norm(a))
