"""GB300-native randomized QR with column pivoting (arXiv 2008.04447).

The compute path is the CUDA library ``librqrcp.so`` (C ABI in
``include/rqrcp.h``).  This package only marshals arguments to it:

* ``_lib``   -- one Python function per C entry point, same names;
* ``Handle`` -- convenience wrapper that allocates outputs with torch and
  raises on a non-zero status;
* ``inputs`` -- seeded synthetic matrices (no factorisation arithmetic).
"""
from __future__ import annotations

from . import _lib
from ._lib import (RQ_FP32, RQ_FP64, RQ_MIXED, RQ_OK, RQ_OP_QR, RQ_OP_RQRCP, RQ_OP_TRQRCP,  # noqa: F401
                   RQ_OP_TUXV, rq_create, rq_destroy, rq_last_error, rq_launch_count, rq_profile_enable,
                   rq_profile_read, rq_qr, rq_rqrcp, rq_set_workspace, rq_trqrcp, rq_tuxv, rq_workspace_size)

__all__ = ["Handle", "colmajor", "RQ_FP64", "RQ_FP32", "RQ_MIXED"]


def colmajor(x):
    """Column-major (Fortran-order) copy of a 2-D tensor: stride (1, rows)."""
    return x.t().contiguous().t()


def _prec_of(t):
    import torch
    if t.dtype == torch.float64:
        return RQ_FP64
    if t.dtype == torch.float32:
        return RQ_FP32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _ld(t):
    if t.dim() != 2 or t.stride(0) != 1:
        raise ValueError("column-major matrix expected (stride (1, ld)); use colmajor()")
    return max(t.stride(1), t.shape[0], 1)


class RQError(RuntimeError):
    pass


class Handle:
    """Owns one rq_handle (workspace cache) on the current CUDA device."""

    def __init__(self):
        self.h = rq_create()

    def close(self):
        if self.h is not None:
            rq_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != RQ_OK:
            raise RQError(f"{what} failed with status {rc}: {rq_last_error(self.h)}")

    @property
    def launches(self):
        return rq_launch_count(self.h)

    def profile(self, enable=True):
        self._check(rq_profile_enable(self.h, enable), "rq_profile_enable")

    def profile_read(self):
        return rq_profile_read(self.h)

    def rqrcp(self, A, Omega, b, p, k=None, prec=None, stream=None):
        """In-place RQRCP of column-major A (Alg. 4).  Returns (tau, jpvt, info)."""
        import torch
        m, n = A.shape
        k = min(m, n) if k is None else k
        prec = _prec_of(A) if prec is None else prec
        tau = torch.empty(k, dtype=A.dtype, device=A.device)
        jpvt = torch.empty(n, dtype=torch.int32, device=A.device)
        info = torch.empty(1, dtype=torch.int32, device=A.device)
        rc = rq_rqrcp(self.h, prec, m, n, A, _ld(A), b, p, k, Omega, _ld(Omega), tau, jpvt, info, stream)
        self._check(rc, "rq_rqrcp")
        return tau, jpvt, info

    def qr(self, A, b, prec=None, stream=None):
        """In-place unpivoted blocked Householder QR of column-major A."""
        import torch
        m, n = A.shape
        prec = _prec_of(A) if prec is None else prec
        tau = torch.empty(min(m, n), dtype=A.dtype, device=A.device)
        info = torch.empty(1, dtype=torch.int32, device=A.device)
        rc = rq_qr(self.h, prec, m, n, A, _ld(A), b, tau, info, stream)
        self._check(rc, "rq_qr")
        return tau, info
