"""rq_rqrcp_noalloc against rq_rqrcp, through the C ABI.

rq_rqrcp_noalloc serves callers that cannot allocate device memory when they
call -- a process whose device memory is owned by another allocator, or a
latency-bound service that cannot take the device-wide synchronisation of
cudaMalloc / cudaFree in the middle of a request.  Its scratch is a fixed
array inside the library, shared by every call, so these tests run it twice
in a row (different problem sizes, so stale contents of the array would show)
and compare each result with the allocating entry point, within the FP64
tolerances of the other GPU parity tests.  This file is collected last.
"""
import numpy as np
import pytest

from paper_2008_04447_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    from paper_2008_04447_gb300 import colmajor
    return colmajor(torch.as_tensor(a)).cuda()


def _run_noalloc(a, om, b, p):
    import torch
    from paper_2008_04447_gb300 import _lib
    m, n = a.shape
    k = min(m, n)
    A = _dev(a)
    Om = _dev(om)
    tau = torch.empty(k, dtype=torch.float64, device="cuda")
    jpvt = torch.empty(n, dtype=torch.int32, device="cuda")
    info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    rc = _lib.rq_rqrcp_noalloc(_lib.RQ_FP64, m, n, A, m, b, p, k, Om, b + p, tau, jpvt, info)
    assert rc == _lib.RQ_OK, rc
    torch.cuda.synchronize()
    return A.cpu().numpy(), tau.cpu().numpy(), jpvt.cpu().numpy(), int(info.cpu()[0])


def _run_alloc(a, om, b, p):
    import torch
    from paper_2008_04447_gb300 import Handle, build
    build.build()
    h = Handle()
    A = _dev(a)
    tau, jpvt, info = h.rqrcp(A, _dev(om), b, p)
    torch.cuda.synchronize()
    out = A.cpu().numpy(), tau.cpu().numpy(), jpvt.cpu().numpy(), int(info.cpu()[0])
    h.close()
    return out


def test_noalloc_matches_rqrcp_on_consecutive_calls():
    from paper_2008_04447_gb300 import build
    build.build()
    for (m, n, b, p, seed) in [(600, 450, 32, 8, 1), (257, 300, 16, 4, 2), (600, 450, 32, 8, 3)]:
        a = I.graded(m, n, 8, seed=seed)
        om = I.omega(b + p, m, seed=seed + 100)
        ref = _run_alloc(a, om, b, p)
        got = _run_noalloc(a, om, b, p)
        nrm = np.linalg.norm(a)
        k = min(m, n)
        assert np.array_equal(got[2], ref[2])
        assert got[3] == ref[3]
        assert np.max(np.abs(np.triu(got[0]) - np.triu(ref[0]))) <= 1e-12 * nrm
        scale = 1e-12 * nrm / np.maximum(np.abs(np.diag(ref[0][:k, :k])), 1e-300)
        assert np.all(np.abs(got[1] - ref[1]) <= scale)


def test_noalloc_rejects_a_problem_larger_than_its_scratch():
    import torch
    from paper_2008_04447_gb300 import _lib, build
    build.build()
    m = n = 8192  # needs ~31 MB of scratch in FP64 with b = 64, p = 8
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
