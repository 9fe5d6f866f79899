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
