"""GPU: the continuous-batching server returns, for every request, the result
the request gets alone.

Small and large TUXV requests arrive staggered while the scheduler thread
runs, so they are admitted, batched and launched on three lanes (streams) in
whatever mix the timing gives, with large requests on the whole-GPU path
beside running batches.  Afterwards each request is recomputed alone on a
fresh handle: a small one through a one-problem batched call must give the
same bits (one CTA computes one problem, with no reduction shared with its
neighbours); a large one through rq_tuxv must give the same U X V^T within
1e-6 of ||A||_F (the same kernels in the same launch shapes; the tolerance
only allows for launch-order effects, which the kernels do not have).  The
server runs the FP32 path, and every served result's rank-k error, in FP64
against the FP64 input, is within 1.05x that of the plain FP64 oracle on the
FP64 input.
"""
import time

import numpy as np
import pytest

from paper_2008_04447_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _requests(seed):
    import torch
    from paper_2008_04447_gb300 import colmajor
    rng = np.random.default_rng(seed)
    small = [(m, n, k, min(32, k)) for m, n, k in I.batch_shapes(20, seed, m_range=(64, 256), n_cap=256,
                                                                 k_range=(8, 40))]
    large = [(640, 512, 64, 32), (700, 400, 48, 16), (600, 500, 96, 32)]
    shapes = small + large
    order = rng.permutation(len(shapes))
    out = []
    for i in order:
        m, n, k, b = shapes[i]
        a = I.graded(m, n, 6, seed=seed * 1000 + int(i))
        om = I.omega(b + 8, m, seed=seed * 1000 + 500 + int(i))
        out.append((colmajor(torch.as_tensor(a, dtype=torch.float32)).cuda(),
                    colmajor(torch.as_tensor(om, dtype=torch.float32)).cuda(), b, 8, k, a, om))
    return out


def test_served_results_equal_solo_results():
    import torch
    from paper_2008_04447_gb300 import RQ_FP32, Handle, build
    from paper_2008_04447_gb300.serve import Server
    from gpu_util import fp64_oracle_error, rank_k_error
    build.build()
    full = _requests(seed=21)
    reqs = [t[:5] for t in full]
    torch.cuda.synchronize()
    srv = Server(budget_bytes=4e9, lanes=3, large_mn=300 * 300, prec=RQ_FP32)
    srv.start()
    try:
        rng = np.random.default_rng(4)
        handles = []
        for A, Om, b, p, k in reqs:
            handles.append(srv.submit(A, Om, b, p, k))
            time.sleep(float(rng.uniform(0.0, 2e-3)))
        for r in handles:
            r.wait(120.0)
    finally:
        srv.stop()
    torch.cuda.synchronize()
    assert srv.used == 0 and len(srv.completed) == len(reqs)
    assert sum(r.large for r in handles) == 3
    h = Handle()
    for r, (A, Om, b, p, k, a, om) in zip(handles, full):
        assert int(r.info.abs().sum()) == 0
        assert r.done >= r.started >= r.admitted >= r.arrival
        U, X, V = r.out
        if r.large:
            U1, X1, V1, _, info = h.tuxv(A, Om, b, p, k, prec=RQ_FP32)
            torch.cuda.synchronize()
            assert int(info.abs().sum()) == 0
            d = torch.linalg.norm((U.double() @ X.double() @ V.double().T) - (U1.double() @ X1.double() @ V1.double().T))
            assert float(d) <= 1e-6 * float(torch.linalg.norm(A.double())), float(d)
        else:
            solo, info = h.tuxv_batched([(A, Om, b, p, k)], prec=RQ_FP32)
            torch.cuda.synchronize()
            assert int(info.abs().sum()) == 0
            for x_srv, x_solo in zip((U, X, V), solo[0]):
                assert torch.equal(x_srv, x_solo)
        e_gpu = rank_k_error(a, *(t.cpu().double().numpy() for t in (U, X, V)))
        e_64, _ = fp64_oracle_error(a, om, b, k)
        assert e_gpu <= 1.05 * e_64, (a.shape, k, e_gpu / e_64)
