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
from ._lib import (RQ_FP32, RQ_FP64, RQ_MIXED, RQ_OK, RQ_OP_QR, RQ_OP_RQRCP, RQ_OP_RSRQRCP, RQ_OP_TRQRCP,  # noqa: F401
                   RQ_OP_TUXV, rq_create, rq_destroy, rq_last_error, rq_launch_count, rq_profile_enable,
                   rq_gaussian, rq_profile_read, rq_qr, rq_rqrcp, rq_rsrqrcp, rq_set_workspace, rq_trqrcp,
                   rq_tuxv, rq_tuxv_batched, rq_tuxv_iter, rq_latent_cdf, rq_padding,
                   rq_workspace_size, rq_set_batch_tiles, rq_get_batch_tiles, rq_tiles_search, rq_tune_batched,
                   rq_gemm_bf16, rq_gemm_f64, rq_selftest_wait_timeout, rq_copy)

__all__ = ["Handle", "colmajor", "RQ_FP64", "RQ_FP32", "RQ_MIXED"]


def colmajor(x):
    """Column-major (Fortran-order) copy of a 2-D tensor: strides (1, rows).

    The copy goes into a tensor allocated as (cols, rows) and transposed, so a
    single-row matrix also gets stride 1 between rows and 1 between columns
    (``x.t().contiguous()`` would keep a 1 x N tensor's row-major strides,
    because torch does not count the stride of a size-1 dimension)."""
    import torch
    out = torch.empty((x.shape[1], x.shape[0]), dtype=x.dtype, device=x.device).t()
    out.copy_(x)
    return out


def _prec_of(t):
    import torch
    if t.dtype == torch.float64:
        return RQ_FP64
    if t.dtype == torch.float32:
        return RQ_FP32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _ld(t):
    """Leading dimension of a column-major 2-D tensor (entry (i, j) at i + j ld).

    A single-row matrix has no row stride to check: any stride(0) is accepted
    and ld is its column stride (at least 1)."""
    if t.dim() != 2:
        raise ValueError("column-major matrix expected (stride (1, ld)); use colmajor()")
    if t.shape[0] == 1:
        return max(t.stride(1), 1)
    if t.stride(0) != 1:
        raise ValueError("column-major matrix expected (stride (1, ld)); use colmajor()")
    return max(t.stride(1), t.shape[0], 1)


class RQError(RuntimeError):
    pass


def _used_on(t, stream):
    """Record that device tensor t is used by `stream` (a torch stream or a raw
    cudaStream_t), unless that is torch's current stream, on which t was
    allocated: its memory then is not reused before the stream's work is done."""
    import torch
    if stream is None:
        return
    if isinstance(stream, int):
        if stream == torch.cuda.current_stream().cuda_stream:
            return
        stream = torch.cuda.ExternalStream(stream)
    elif stream.cuda_stream == torch.cuda.current_stream().cuda_stream:
        return
    t.record_stream(stream)


class _BatchPlan:
    """Device descriptors and outputs of a batch prepared for repeated launches."""

    def __init__(self, count, outputs, info, d, bounds):
        self.count, self.outputs, self.info, self.d, self.bounds = count, outputs, info, d, bounds


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

    def rsrqrcp(self, A, seed, b, p, k=None, prec=None, stream=None):
        """In-place RQRCP with repeated sampling (Sec. 3.4): fresh Gaussian draws of
        (seed, J) sketch the trailing matrix at every block.  Returns (tau, jpvt, info)."""
        import torch
        m, n = A.shape
        k = min(m, n) if k is None else k
        prec = _prec_of(A) if prec is None else prec
        tau = torch.empty(k, dtype=A.dtype, device=A.device)
        jpvt = torch.empty(n, dtype=torch.int32, device=A.device)
        info = torch.empty(1, dtype=torch.int32, device=A.device)
        self._check(rq_rsrqrcp(self.h, prec, m, n, A, _ld(A), b, p, k, seed, tau, jpvt, info, stream), "rq_rsrqrcp")
        return tau, jpvt, info

    def trqrcp(self, A, Omega, b, p, k, prec=None, stream=None):
        """Truncated RQRCP (Alg. 5); A is read only.  Returns (Y, tau, R, jpvt, info)."""
        import torch
        m, n = A.shape
        prec = _prec_of(A) if prec is None else prec
        Y = torch.empty((k, m), dtype=A.dtype, device=A.device).t()
        R = torch.empty((n, k), dtype=A.dtype, device=A.device).t()
        tau = torch.empty(k, dtype=A.dtype, device=A.device)
        jpvt = torch.empty(n, dtype=torch.int32, device=A.device)
        info = torch.empty(1, dtype=torch.int32, device=A.device)
        rc = rq_trqrcp(self.h, prec, m, n, A, _ld(A), b, p, k, Omega, _ld(Omega), Y, m, tau, R, k, jpvt, info,
                       stream)
        self._check(rc, "rq_trqrcp")
        return Y, tau, R, jpvt, info

    def tuxv(self, A, Omega, b, p, k, svd=False, prec=None, stream=None, jmax=1):
        """TUXV (Alg. 6): A ~= U X V^T after jmax refinement steps (X upper
        triangular for odd jmax, lower for even).  Returns (U, X, V, sigma or None, info)."""
        import torch
        m, n = A.shape
        prec = _prec_of(A) if prec is None else prec
        U = torch.empty((k, m), dtype=A.dtype, device=A.device).t()
        X = torch.empty((k, k), dtype=A.dtype, device=A.device).t()
        V = torch.empty((k, n), dtype=A.dtype, device=A.device).t()
        sigma = torch.empty(k, dtype=A.dtype, device=A.device) if svd else None
        info = torch.empty(1, dtype=torch.int32, device=A.device)
        if jmax == 1:
            rc = rq_tuxv(self.h, prec, m, n, A, _ld(A), b, p, k, Omega, _ld(Omega), U, m, X, k, V, n, sigma, info,
                         stream)
        else:
            rc = rq_tuxv_iter(self.h, prec, m, n, A, _ld(A), b, p, k, jmax, Omega, _ld(Omega), U, m, X, k, V, n, sigma,
                              info, stream)
        self._check(rc, "rq_tuxv")
        return U, X, V, sigma, info

    def tuxv_batched(self, problems, prec=RQ_MIXED, stream=None, outputs=None, svd=False):
        """Batched TUXV of [(A, Omega, b, p, k), ...] (column-major FP32 device tensors).

        One persistent launch; returns [(U, X, V), ...] (with svd, the core SVD of
        every problem: [(U, X = diag(sigma), V, sigma), ...]) and the info tensor.
        The descriptors are built on the host and copied to the device.
        """
        outputs, info, d, bounds = self._batch(problems, outputs, svd)
        rc = rq_tuxv_batched(self.h, prec, len(problems), d, *bounds, stream)
        self._check(rc, "rq_tuxv_batched")
        # the descriptors must outlive the asynchronous launch: hold the latest
        # and, when the launch is on another stream than the one they were
        # allocated on, tell the caching allocator that stream uses them
        self._keep = d
        _used_on(d, stream)
        return outputs, info

    def prepare_batched(self, problems, outputs=None, svd=False):
        """Builds the device descriptors of a batch once (the per-problem Python
        work of tuxv_batched: shapes, leading dimensions, pointers), for a batch
        whose buffers are launched repeatedly (their contents may change between
        launches).  Returns a plan for launch_prepared; plan.outputs and
        plan.info hold the results of its latest launch."""
        outputs, info, d, bounds = self._batch(problems, outputs, svd)
        return _BatchPlan(len(problems), outputs, info, d, bounds)

    def launch_prepared(self, plan, prec=RQ_MIXED, stream=None):
        """One persistent launch of a prepared batch (rq_tuxv_batched on its
        descriptors); returns (outputs, info)."""
        rc = rq_tuxv_batched(self.h, prec, plan.count, plan.d, *plan.bounds, stream)
        self._check(rc, "rq_tuxv_batched")
        _used_on(plan.d, stream)
        return plan.outputs, plan.info

    def tune_batched(self, problems, prec=RQ_MIXED, reps=2, passes=2, stream=None, outputs=None, svd=False,
                     cache=None, key=None):
        """Autotunes the batched kernel's tile policy on these problems (synchronous).

        Returns ((skinny_m, skinny_n), ms, outputs, info): the policy now held by
        the handle, the batch's time under it, and the batch's result (the same
        bits under every policy).  With cache (a JSON file), a policy stored
        under the batch's key (``tuning.batch_key`` unless key is given) is
        taken without timing and the batch simply runs; a newly tuned policy
        is stored there.
        """
        from . import tuning
        if cache is not None:
            if key is None:
                import torch
                dev = problems[0][0].device
                props = torch.cuda.get_device_properties(dev)
                key = tuning.batch_key(problems, prec, props.name, props.multi_processor_count)
            hit = tuning.lookup(cache, key)
            if hit is not None:
                self.batch_tiles = hit["tiles"]
                outputs, info = self.tuxv_batched(problems, prec=prec, stream=stream, outputs=outputs, svd=svd)
                return tuple(hit["tiles"]), hit["ms"], outputs, info
        outputs, info, d, bounds = self._batch(problems, outputs, svd)
        rc, tiles, ms = _lib.rq_tune_batched(self.h, prec, len(problems), d, *bounds, reps, passes, stream)
        self._check(rc, "rq_tune_batched")
        if cache is not None:
            tuning.store(cache, key, tiles, ms)
        return tiles, ms, outputs, info

    @property
    def batch_tiles(self):
        """(skinny_m, skinny_n): the tile policy of later batched calls."""
        rc, t = _lib.rq_get_batch_tiles(self.h)
        self._check(rc, "rq_get_batch_tiles")
        return t

    @batch_tiles.setter
    def batch_tiles(self, t):
        self._check(_lib.rq_set_batch_tiles(self.h, int(t[0]), int(t[1])), "rq_set_batch_tiles")

    @staticmethod
    def _batch(problems, outputs, svd):
        """Outputs (allocated unless given), info, the device descriptor array
        and the bounds (max m, n, k, b, p) of a batched call."""
        import numpy as np
        import torch
        dev = problems[0][0].device
        if outputs is None:
            outputs = []
            for A, Om, b, p, k in problems:
                m, n = A.shape
                outputs.append((torch.empty((k, m), dtype=A.dtype, device=dev).t(),
                                torch.empty((k, k), dtype=A.dtype, device=dev).t(),
                                torch.empty((k, n), dtype=A.dtype, device=dev).t())
                               + ((torch.empty(k, dtype=A.dtype, device=dev),) if svd else ()))
        info = torch.zeros(len(problems), dtype=torch.int32, device=dev)
        desc = np.zeros(len(problems), dtype=_lib.problem_dtype())
        for i, ((A, Om, b, p, k), out) in enumerate(zip(problems, outputs)):
            m, n = A.shape
            U, X, V = out[:3]
            sg = out[3].data_ptr() if len(out) > 3 and out[3] is not None else 0
            desc[i] = (m, n, k, b, p, _ld(A), _ld(Om), _ld(U), _ld(X), _ld(V), 0, 0, A.data_ptr(), Om.data_ptr(),
                       U.data_ptr(), X.data_ptr(), V.data_ptr(), sg, info.data_ptr() + 4 * i)
        d = torch.from_numpy(desc.view(np.uint8)).to(dev)
        mm = max(int(A.shape[0]) for A, *_ in problems)
        mn = max(int(A.shape[1]) for A, *_ in problems)
        mk = max(int(t[4]) for t in problems)
        mb = max(int(t[2]) for t in problems)
        mp = max(int(t[3]) for t in problems)
        return outputs, info, d, (mm, mn, mk, mb, mp)

    def gemm_bf16(self, A, B, out=None, stream=None):
        """C = A B of column-major FP32 device matrices with both inputs rounded to
        bfloat16 and FP32 accumulation (the mixed-precision sketch's product).
        Returns (C, info)."""
        import torch
        M, K = A.shape
        K2, N = B.shape
        if K2 != K:
            raise ValueError(f"inner dimensions differ: {K} and {K2}")
        C = torch.empty((N, M), dtype=torch.float32, device=A.device).t() if out is None else out
        info = torch.zeros(1, dtype=torch.int32, device=A.device)
        rc = rq_gemm_bf16(self.h, M, N, K, A, _ld(A), B, _ld(B), C, _ld(C), info, stream)
        self._check(rc, "rq_gemm_bf16")
        return C, info

    def gemm_f64(self, A, B, out=None, stream=None):
        """C = A B of column-major FP64 device matrices on the bfloat16 tensor
        cores (sliced operands, FP64 accuracy).  Returns (C, info)."""
        import torch
        M, K = A.shape
        K2, N = B.shape
        if K2 != K:
            raise ValueError(f"inner dimensions differ: {K} and {K2}")
        C = torch.empty((N, M), dtype=torch.float64, device=A.device).t() if out is None else out
        info = torch.zeros(1, dtype=torch.int32, device=A.device)
        rc = rq_gemm_f64(self.h, M, N, K, A, _ld(A), B, _ld(B), C, _ld(C), info, stream)
        self._check(rc, "rq_gemm_f64")
        return C, info

    def gaussian(self, l, m, seed, substream=0, dtype=None, out=None, stream=None):
        """l x m column-major Gaussian draws of (seed, substream) (Sec. 3.1's Omega)."""
        import torch
        if out is None:
            out = torch.empty((m, l), dtype=dtype or torch.float64, device="cuda").t()
        prec = _prec_of(out)
        self._check(rq_gaussian(self.h, prec, seed, substream, l, m, out, _ld(out), stream), "rq_gaussian")
        return out

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
