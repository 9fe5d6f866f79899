"""rq_rqrcp_noalloc through the C ABI: against the oracle and against rq_rqrcp.

rq_rqrcp_noalloc serves callers that cannot allocate device memory when they
call -- a process whose device memory is owned by another allocator, or a
latency-bound service that cannot take the device-wide synchronisation of
cudaMalloc / cudaFree in the middle of a request.  Its scratch is a fixed
array inside the library, shared by every call, so these tests run it several
times in a row (different problem sizes, so stale contents of the array would
show).  FP64: pivots equal to the oracle's (Alg. 4 in FP64) and to
rq_rqrcp's, R within 1e-12 ||A||_F of both, tau within the reflector
tolerance.  FP32: ||AP - QR|| / ||A|| and ||Q^T Q - I|| at most 1e-5, pivots
equal to the oracle's (run on the FP32-rounded input) up to the first
near-tie decision (relative gap below 1e-4, scaled by the sample's growth),
and R within 1e-5 ||A||_F of rq_rqrcp's FP32 result.  This file is collected
last.
"""
import numpy as np
import pytest

import oracle as O
from paper_2008_04447_gb300 import inputs as I

from gpu_util import factor_quality, first_near_tie

pytestmark = pytest.mark.gpu


def _dev(a, dtype):
    import torch
    from paper_2008_04447_gb300 import colmajor
    return colmajor(torch.as_tensor(a, dtype=dtype)).cuda()


def _run_noalloc(a, om, b, p, dtype):
    import torch
    from paper_2008_04447_gb300 import _lib
    m, n = a.shape
    k = min(m, n)
    prec = _lib.RQ_FP64 if dtype == torch.float64 else _lib.RQ_FP32
    A = _dev(a, dtype)
    Om = _dev(om, dtype)
    tau = torch.empty(k, dtype=dtype, device="cuda")
    jpvt = torch.empty(n, dtype=torch.int32, device="cuda")
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    rc = _lib.rq_rqrcp_noalloc(prec, m, n, A, m, b, p, k, Om, b + p, tau, jpvt, info)
    assert rc == _lib.RQ_OK, rc
    torch.cuda.synchronize()
    return (A.cpu().double().numpy(), tau.cpu().double().numpy(), jpvt.cpu().numpy().astype(np.int64),
            int(info.cpu()[0]))


def _run_alloc(a, om, b, p, dtype):
    import torch
    from paper_2008_04447_gb300 import Handle, build
    build.build()
    h = Handle()
    A = _dev(a, dtype)
    tau, jpvt, info = h.rqrcp(A, _dev(om, dtype), b, p)
    torch.cuda.synchronize()
    out = (A.cpu().double().numpy(), tau.cpu().double().numpy(), jpvt.cpu().numpy().astype(np.int64),
           int(info.cpu()[0]))
    h.close()
    return out


CASES = [(600, 450, 32, 8, 1), (257, 300, 16, 4, 2), (600, 450, 32, 8, 3)]


def test_noalloc_fp64_matches_oracle_and_rqrcp_on_consecutive_calls():
    import torch
    from paper_2008_04447_gb300 import build
    build.build()
    for (m, n, b, p, seed) in CASES:
        a = I.graded(m, n, 8, seed=seed)
        om = I.omega(b + p, m, seed=seed + 100)
        got = _run_noalloc(a, om, b, p, torch.float64)
        ref = _run_alloc(a, om, b, p, torch.float64)
        ora = O.rqrcp(a, om, b)
        nrm = np.linalg.norm(a)
        k = min(m, n)
        assert got[3] == ref[3] == ora.info
        for F, tau, jp in ((ref[0], ref[1], ref[2]), (ora.F, ora.tau, ora.jpvt)):
            assert np.array_equal(got[2], jp)
            assert np.max(np.abs(np.triu(got[0]) - np.triu(F))) <= 1e-12 * nrm
            scale = 1e-12 * nrm / np.maximum(np.abs(np.diag(F[:k, :k])), 1e-300)
            assert np.all(np.abs(got[1] - tau) <= scale)


def test_noalloc_fp32_matches_oracle_within_tolerance():
    import torch
    from paper_2008_04447_gb300 import build
    build.build()
    for (m, n, b, p, seed) in CASES:
        a = I.graded(m, n, 6, seed=seed).astype(np.float32).astype(np.float64)
        om = I.omega(b + p, m, seed=seed + 100).astype(np.float32).astype(np.float64)
        got = _run_noalloc(a, om, b, p, torch.float32)
        ref = _run_alloc(a, om, b, p, torch.float32)
        k = min(m, n)
        resid, orth = factor_quality(a, got[0], got[1], got[2], k)
        assert resid <= 1e-5 and orth <= 1e-5, (resid, orth)
        ora = O.rqrcp(a, om, b)
        tie = first_near_tie(ora.gaps, b, 1e-4, ora.sample_norms)
        upto = n if tie is None else tie
        assert upto >= b
        assert np.array_equal(got[2][:upto], ora.jpvt[:upto])
        assert got[3] == 0
        # rq_rqrcp's FP32 result: the same pivots while no decision is a near-tie
        assert np.array_equal(got[2][:upto], ref[2][:upto])
        if tie is None:
            assert np.max(np.abs(np.triu(got[0]) - np.triu(ref[0]))) <= 1e-5 * np.linalg.norm(a)


def test_noalloc_rejects_a_problem_larger_than_its_scratch():
    import torch
    from paper_2008_04447_gb300 import _lib, build
    build.build()
    m = n = 8192  # needs about 29 MiB of scratch in FP64 with b = 64, p = 8
    # full-size, valid buffers: the call must refuse on size alone
    A = torch.zeros((n, m), dtype=torch.float64, device="cuda").t()
    Om = torch.zeros((m, 72), dtype=torch.float64, device="cuda").t()
    t = torch.zeros(n, dtype=torch.float64, device="cuda")
    j = torch.zeros(n, dtype=torch.int32, device="cuda")
    i = torch.full((1,), 5, dtype=torch.int32, device="cuda")
    rc = _lib.rq_rqrcp_noalloc(_lib.RQ_FP64, m, n, A, m, 64, 8, n, Om, 72, t, j, i)
    assert rc == _lib.RQ_ETOOBIG
    torch.cuda.synchronize()
    assert int(i.cpu()[0]) == 5   # nothing was launched
