"""ctypes binding of librqrcp.so (include/rqrcp.h): argument marshalling only.

Every exported C function is re-exported here under the same name.  Matrix
arguments may be passed as raw device addresses (int) or as CUDA tensors; a
tensor is passed by its data pointer.  Column-major matrices are tensors of
shape (rows, cols) with stride (1, ld) -- e.g. ``x.t().contiguous().t()``.

There is no fallback: if the library is missing or cannot be loaded, every
call raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librqrcp.so")

RQ_OK = 0
RQ_ENOMEM = -1000
RQ_ECUDA = -1001
RQ_ETIMEOUT = -1002
RQ_ENOTIMPL = -1003
RQ_EHANDLE = -1004
RQ_ETOOBIG = -1005
RQ_NOALLOC_SCRATCH_BYTES = 16 << 20
RQ_MAX_B, RQ_MAX_L = 256, 384

RQ_FP64, RQ_FP32, RQ_MIXED = 0, 1, 2
RQ_OP_RQRCP, RQ_OP_TRQRCP, RQ_OP_TUXV, RQ_OP_QR, RQ_OP_RSRQRCP = 0, 1, 2, 3, 4
PHASES = ["sketch", "sample_qrcp", "permute", "panel", "trailing", "sample_update", "other", "slice"]

_P = ctypes.c_void_p
_I = ctypes.c_int


class rq_batch_tiles(ctypes.Structure):
    """Tile policy of the batched kernel's block GEMMs (two int32 thresholds)."""
    _fields_ = [("skinny_m", ctypes.c_int), ("skinny_n", ctypes.c_int)]


# int (*rq_tiles_measure)(void* user, const rq_batch_tiles* tiles, double* ms)
rq_tiles_measure = ctypes.CFUNCTYPE(_I, _P, ctypes.POINTER(rq_batch_tiles), ctypes.POINTER(ctypes.c_double))
RQ_TILE_STEPS = (0, 16, 32, 64, 128, 256)
_SIGS = {
    "rq_create": ([ctypes.POINTER(_P)], _I),
    "rq_destroy": ([_P], _I),
    "rq_workspace_size": ([_P, _I, _I, _I, _I, _I, _I, _I, ctypes.POINTER(ctypes.c_size_t)], _I),
    "rq_set_workspace": ([_P, _P, ctypes.c_size_t], _I),
    "rq_last_error": ([_P, ctypes.c_char_p, ctypes.c_size_t], _I),
    "rq_launch_count": ([_P], ctypes.c_longlong),
    "rq_profile_enable": ([_P, _I], _I),
    "rq_profile_read": ([_P, _I, _P, _P, _P, _P], _I),
    "rq_rqrcp": ([_P, _I, _I, _I, _P, _I, _I, _I, _I, _P, _I, _P, _P, _P, _P], _I),
    "rq_rqrcp_noalloc": ([_I, _I, _I, _P, _I, _I, _I, _I, _P, _I, _P, _P, _P, _P], _I),
    "rq_qr": ([_P, _I, _I, _I, _P, _I, _I, _P, _P, _P], _I),
    "rq_trqrcp": ([_P, _I, _I, _I, _P, _I, _I, _I, _I, _P, _I, _P, _I, _P, _P, _I, _P, _P, _P], _I),
    "rq_tuxv": ([_P, _I, _I, _I, _P, _I, _I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P, _P, _P], _I),
    "rq_tuxv_iter": ([_P, _I, _I, _I, _P, _I, _I, _I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _I, _P, _P, _P], _I),
    "rq_tuxv_batched": ([_P, _I, _I, _P, _I, _I, _I, _I, _I, _P], _I),
    "rq_gemm_bf16": ([_P, _I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _P], _I),
    "rq_gemm_f64": ([_P, _I, _I, _I, _P, _I, _P, _I, _P, _I, _P, _P], _I),
    "rq_set_batch_tiles": ([_P, ctypes.POINTER(rq_batch_tiles)], _I),
    "rq_get_batch_tiles": ([_P, ctypes.POINTER(rq_batch_tiles)], _I),
    "rq_tiles_search": ([rq_tiles_measure, _P, ctypes.POINTER(rq_batch_tiles), _I, ctypes.POINTER(rq_batch_tiles),
                         ctypes.POINTER(ctypes.c_double)], _I),
    "rq_tune_batched": ([_P, _I, _I, _P, _I, _I, _I, _I, _I, _I, _I, _P, ctypes.POINTER(rq_batch_tiles),
                         ctypes.POINTER(ctypes.c_double)], _I),
    "rq_rsrqrcp": ([_P, _I, _I, _I, _P, _I, _I, _I, _I, ctypes.c_uint64, _P, _P, _P, _P], _I),
    "rq_latent_cdf": ([_I, ctypes.c_double, ctypes.POINTER(ctypes.c_double)], _I),
    "rq_padding": ([ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_int)], _I),
    "rq_gaussian": ([_P, _I, ctypes.c_uint64, ctypes.c_uint64, _I, _I, _P, _I, _P], _I),
    "rq_selftest_wait_timeout": ([_P, _P, _P], _I),
    "rq_copy": ([_P, _P, ctypes.c_size_t, _P], _I),
}

# rq_problem: twelve int32 then seven 64-bit device pointers (104 bytes)
PROBLEM_FIELDS = ["m", "n", "k", "b", "p", "lda", "ldo", "ldu", "ldx", "ldv", "reserved0", "reserved1",
                  "A", "Omega", "U", "X", "V", "sigma", "info"]


def problem_dtype():
    import numpy as np
    return np.dtype([(f, np.int32) for f in PROBLEM_FIELDS[:12]] + [(f, np.uint64) for f in PROBLEM_FIELDS[12:]])

_lib = None


def load(path: str = LIB_PATH):
    """Load librqrcp.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librqrcp.so not built ({path}); run paper_2008_04447_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("device tensor expected")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a device pointer")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def rq_create():
    h = _P()
    rc = load().rq_create(ctypes.byref(h))
    if rc != RQ_OK:
        raise RuntimeError(f"rq_create failed: {rc}")
    return h


def rq_destroy(h):
    return load().rq_destroy(h)


def rq_workspace_size(h, op, prec, m, n, k, b, p):
    out = ctypes.c_size_t()
    rc = load().rq_workspace_size(h, op, prec, m, n, k, b, p, ctypes.byref(out))
    return rc, out.value


def rq_set_workspace(h, dptr, nbytes):
    return load().rq_set_workspace(h, _ptr(dptr), nbytes)


def rq_last_error(h):
    buf = ctypes.create_string_buffer(256)
    load().rq_last_error(h, buf, 256)
    return buf.value.decode()


def rq_launch_count(h):
    return int(load().rq_launch_count(h))


def rq_profile_enable(h, enable):
    return load().rq_profile_enable(h, 1 if enable else 0)


def rq_profile_read(h):
    """Per-phase {name: (ms, flops, bytes, launches)} since the last read (synchronises)."""
    n = len(PHASES)
    ms = (ctypes.c_double * n)()
    fl = (ctypes.c_double * n)()
    by = (ctypes.c_double * n)()
    la = (ctypes.c_longlong * n)()
    rc = load().rq_profile_read(h, n, ctypes.cast(ms, _P), ctypes.cast(fl, _P), ctypes.cast(by, _P),
                                ctypes.cast(la, _P))
    if rc != RQ_OK:
        raise RuntimeError(f"rq_profile_read failed: {rc}")
    return {PHASES[i]: (ms[i], fl[i], by[i], la[i]) for i in range(n)}


def rq_rqrcp(h, prec, m, n, A, lda, b, p, k, Omega, ldo, tau, jpvt, info, stream=None):
    return load().rq_rqrcp(h, prec, m, n, _ptr(A), lda, b, p, k, _ptr(Omega), ldo, _ptr(tau), _ptr(jpvt),
                           _ptr(info), _stream(stream))


def rq_rqrcp_noalloc(prec, m, n, A, lda, b, p, k, Omega, ldo, tau, jpvt, info, stream=None):
    return load().rq_rqrcp_noalloc(prec, m, n, _ptr(A), lda, b, p, k, _ptr(Omega), ldo, _ptr(tau), _ptr(jpvt),
                                   _ptr(info), _stream(stream))


def _ptr_any(x):
    """Address of a CUDA tensor, a pinned CPU tensor or a raw address."""
    if x is None or isinstance(x, int):
        return x
    if not x.is_cuda and not x.is_pinned():
        raise ValueError("CUDA or pinned CPU tensor expected")
    return x.data_ptr()


def rq_copy(dst, src, nbytes, stream=None):
    """dst, src: raw addresses or tensors (CUDA, or pinned CPU)."""
    return load().rq_copy(_ptr_any(dst), _ptr_any(src), nbytes, _stream(stream))


def rq_selftest_wait_timeout(bar, info, stream=None):
    return load().rq_selftest_wait_timeout(_ptr(bar), _ptr(info), _stream(stream))


def rq_tuxv_batched(h, prec, count, problems, max_m, max_n, max_k, max_b, max_p, stream=None):
    return load().rq_tuxv_batched(h, prec, count, _ptr(problems), max_m, max_n, max_k, max_b, max_p, _stream(stream))


def rq_gemm_bf16(h, M, N, K, A, lda, B, ldb, C, ldc, info=None, stream=None):
    return load().rq_gemm_bf16(h, M, N, K, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, _ptr(info), _stream(stream))


def rq_gemm_f64(h, M, N, K, A, lda, B, ldb, C, ldc, info=None, stream=None):
    return load().rq_gemm_f64(h, M, N, K, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, _ptr(info), _stream(stream))


def rq_set_batch_tiles(h, skinny_m, skinny_n):
    return load().rq_set_batch_tiles(h, ctypes.byref(rq_batch_tiles(skinny_m, skinny_n)))


def rq_get_batch_tiles(h):
    """(status, (skinny_m, skinny_n)) of the handle's tile policy."""
    t = rq_batch_tiles()
    rc = load().rq_get_batch_tiles(h, ctypes.byref(t))
    return rc, (t.skinny_m, t.skinny_n)


def rq_tiles_search(measure, start=None, passes=2):
    """The autotuner's search with a Python cost function ``measure((m, n)) -> ms``.

    Returns (status, (skinny_m, skinny_n), ms).  An exception raised by
    ``measure`` ends the search and is re-raised here.
    """
    err = []

    def cb(_user, tiles, ms):
        try:
            ms[0] = float(measure((tiles.contents.skinny_m, tiles.contents.skinny_n)))
            return 0
        except Exception as e:  # re-raised below, after the C search has returned
            err.append(e)
            return -1001

    fn = rq_tiles_measure(cb)
    best = rq_batch_tiles()
    best_ms = ctypes.c_double()
    st = ctypes.byref(rq_batch_tiles(*start)) if start is not None else None
    rc = load().rq_tiles_search(fn, None, st, passes, ctypes.byref(best), ctypes.byref(best_ms))
    if err:
        raise err[0]
    return rc, (best.skinny_m, best.skinny_n), best_ms.value


def rq_tune_batched(h, prec, count, problems, max_m, max_n, max_k, max_b, max_p, reps=2, passes=2, stream=None):
    """(status, (skinny_m, skinny_n), ms): autotunes the handle's tile policy on a batch."""
    best = rq_batch_tiles()
    best_ms = ctypes.c_double()
    rc = load().rq_tune_batched(h, prec, count, _ptr(problems), max_m, max_n, max_k, max_b, max_p, reps, passes,
                                _stream(stream), ctypes.byref(best), ctypes.byref(best_ms))
    return rc, (best.skinny_m, best.skinny_n), best_ms.value


def rq_rsrqrcp(h, prec, m, n, A, lda, b, p, k, seed, tau, jpvt, info, stream=None):
    return load().rq_rsrqrcp(h, prec, m, n, _ptr(A), lda, b, p, k, seed & 0xFFFFFFFFFFFFFFFF, _ptr(tau), _ptr(jpvt),
                             _ptr(info), _stream(stream))


def rq_gaussian(h, prec, seed, substream, l, m, Omega, ldo, stream=None):
    return load().rq_gaussian(h, prec, seed & 0xFFFFFFFFFFFFFFFF, substream & 0xFFFFFFFFFFFFFFFF, l, m, _ptr(Omega),
                              ldo, _stream(stream))


def rq_latent_cdf(l, tau):
    """P(phi < tau | l) of the sample's posterior (Sec. 3.3), computed by the library."""
    out = ctypes.c_double()
    rc = load().rq_latent_cdf(l, tau, ctypes.byref(out))
    if rc != RQ_OK:
        raise ValueError(f"rq_latent_cdf({l}, {tau}) failed with status {rc}")
    return out.value


def rq_padding(tau, delta):
    """Smallest padding p keeping every pivot decision's P(phi < tau) <= delta."""
    out = ctypes.c_int()
    rc = load().rq_padding(tau, delta, ctypes.byref(out))
    if rc != RQ_OK:
        raise ValueError(f"rq_padding({tau}, {delta}) failed with status {rc}")
    return out.value


def rq_qr(h, prec, m, n, A, lda, b, tau, info, stream=None):
    return load().rq_qr(h, prec, m, n, _ptr(A), lda, b, _ptr(tau), _ptr(info), _stream(stream))


def rq_trqrcp(h, prec, m, n, A, lda, b, p, k, Omega, ldo, Y, ldy, tau, R, ldr, jpvt, info, stream=None):
    return load().rq_trqrcp(h, prec, m, n, _ptr(A), lda, b, p, k, _ptr(Omega), ldo, _ptr(Y), ldy, _ptr(tau),
                            _ptr(R), ldr, _ptr(jpvt), _ptr(info), _stream(stream))


def rq_tuxv_iter(h, prec, m, n, A, lda, b, p, k, jmax, Omega, ldo, U, ldu, X, ldx, V, ldv, sigma, info, stream=None):
    return load().rq_tuxv_iter(h, prec, m, n, _ptr(A), lda, b, p, k, jmax, _ptr(Omega), ldo, _ptr(U), ldu, _ptr(X),
                               ldx, _ptr(V), ldv, _ptr(sigma), _ptr(info), _stream(stream))


def rq_tuxv(h, prec, m, n, A, lda, b, p, k, Omega, ldo, U, ldu, X, ldx, V, ldv, sigma, info, stream=None):
    return load().rq_tuxv(h, prec, m, n, _ptr(A), lda, b, p, k, _ptr(Omega), ldo, _ptr(U), ldu, _ptr(X), ldx,
                          _ptr(V), ldv, _ptr(sigma), _ptr(info), _stream(stream))
