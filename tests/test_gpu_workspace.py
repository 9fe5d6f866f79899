"""GPU: a caller-owned workspace.

rq_workspace_size gives enough for the call it sizes: RQRCP (FP64) and TUXV
(mixed) run in exactly that many bytes of a caller buffer and give the same
bits as with the library's own workspace; one byte fewer returns RQ_ENOMEM
before any launch (A untouched), and a base that is not 256-byte aligned is
refused.
"""
import numpy as np
import pytest

from paper_2008_04447_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_caller_workspace_of_the_queried_size():
    import torch
    from paper_2008_04447_gb300 import RQ_FP64, RQ_MIXED, RQ_OP_RQRCP, RQ_OP_TUXV, Handle, RQError, _lib, build
    from gpu_util import to_dev
    build.build()
    m, n, b, p, k = 300, 200, 16, 8, 40
    a = I.graded(m, n, 8, seed=5)
    om = I.omega(b + p, m, seed=6)
    own = Handle()
    A1 = to_dev(a)
    tau1, jp1, info1 = own.rqrcp(A1, to_dev(om), b, p)
    a32, om32 = to_dev(a, torch.float32), to_dev(om, torch.float32)
    U1, X1, V1, _, _ = own.tuxv(a32, om32, b, p, k, prec=RQ_MIXED)
    torch.cuda.synchronize()

    h = Handle()
    rc, need_r = _lib.rq_workspace_size(h.h, RQ_OP_RQRCP, RQ_FP64, m, n, min(m, n), b, p)
    assert rc == 0 and need_r > 0
    rc, need_t = _lib.rq_workspace_size(h.h, RQ_OP_TUXV, RQ_MIXED, m, n, k, b, p)
    assert rc == 0 and need_t > 0
    ws = torch.empty(max(need_r, need_t) + 256, dtype=torch.uint8, device="cuda")
    assert ws.data_ptr() % 256 == 0
    assert _lib.rq_set_workspace(h.h, ws.data_ptr() + 8, need_r) == -2          # unaligned base
    assert _lib.rq_set_workspace(h.h, ws, need_r) == 0
    A2 = to_dev(a)
    tau2, jp2, info2 = h.rqrcp(A2, to_dev(om), b, p)
    assert _lib.rq_set_workspace(h.h, ws, need_t) == 0
    U2, X2, V2, _, _ = h.tuxv(a32, om32, b, p, k, prec=RQ_MIXED)
    torch.cuda.synchronize()
    for x, y in ((A1, A2), (tau1, tau2), (jp1, jp2), (U1, U2), (X1, X2), (V1, V2)):
        assert torch.equal(x, y)

    short = Handle()
    assert _lib.rq_set_workspace(short.h, ws, need_r - 1) == 0
    A3 = to_dev(a)
    with pytest.raises(RQError):
        short.rqrcp(A3, to_dev(om), b, p)
    torch.cuda.synchronize()
    assert np.array_equal(A3.cpu().numpy(), a)
