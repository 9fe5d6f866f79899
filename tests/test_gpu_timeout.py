"""GPU: a device-side wait that runs out ends the kernel with RQ_ETIMEOUT.

Failure detection without a GPU fault: every wait on another CTA is bounded.
rq_selftest_wait_timeout launches two CTAs at the library's grid barrier with
a count of three, so the third arrival never comes (a flag that nothing
sets).  The kernel must return by itself within its limit (about a second or
two), leave RQ_ETIMEOUT in the info word, and leave the context usable: a
factorisation issued right after it on the same stream still matches the
oracle.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_grid_barrier_wait_runs_out_and_reports_timeout():
    import torch
    from paper_2008_04447_gb300 import _lib, build
    build.build()
    bar = torch.full((2,), 7, dtype=torch.int32, device="cuda")
    info = torch.full((1,), 5, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.time()
    assert _lib.rq_selftest_wait_timeout(bar, info) == _lib.RQ_OK
    torch.cuda.synchronize()
    dt = time.time() - t0
    assert int(info.cpu()[0]) == _lib.RQ_ETIMEOUT
    assert dt < 30.0, dt
    assert _lib.rq_selftest_wait_timeout(None, info) == -1
    assert _lib.rq_selftest_wait_timeout(bar, None) == -2


def test_context_still_usable_after_a_timeout():
    import torch
    import oracle as O
    from paper_2008_04447_gb300 import _lib, build
    from paper_2008_04447_gb300 import inputs as I
    from gpu_util import build_and_handle, to_dev
    build.build()
    bar = torch.zeros(2, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _lib.rq_selftest_wait_timeout(bar, info) == _lib.RQ_OK
    H = build_and_handle()
    a = I.graded(120, 90, 6, seed=11)
    om = I.omega(24, 120, seed=12)
    A = to_dev(a)
    tau, jpvt, inf2 = H.rqrcp(A, to_dev(om), 16, 8)
    torch.cuda.synchronize()
    assert int(info.cpu()[0]) == _lib.RQ_ETIMEOUT
    assert int(inf2.cpu()[0]) == 0
    ref = O.rqrcp(a, om, 16)
    assert np.array_equal(jpvt.cpu().numpy(), ref.jpvt)
    assert np.max(np.abs(np.triu(A.cpu().numpy()) - np.triu(ref.F))) <= 1e-12 * np.linalg.norm(a)
