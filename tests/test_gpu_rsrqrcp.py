"""GPU parity of rq_rsrqrcp (repeated sampling, Sec. 3.4) against the oracle's
RQRCP in repeated-sampling mode fed by the oracle's own Philox draws.

The GPU draws each block's Gaussian on the device with its own implementation
of the same generator (within 1e-13 of the oracle's), so the samples agree to
rounding and the FP64 bar of the update-formula RQRCP applies: identical
pivots up to the first decision with a relative gap below 1e-6, R within
1e-12 ||A||_F, ||AP - QR||_F / ||A||_F and ||Q^T Q - I||_F <= 1e-12.  FP32:
residual and orthogonality <= 1e-5, pivots identical up to the first decision
with a relative gap below 1e-4.
"""
import numpy as np
import pytest

import oracle as O
from oracle import philox as P
from paper_2008_04447_gb300 import inputs as I

from gpu_util import build_and_handle, factor_quality, first_near_tie, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    return build_and_handle()


def oracle_rs(a, seed, b, p, k):
    m = a.shape[0]
    return O.rqrcp(a, P.gaussian(seed, b + p, m), b, k, mode="resample", resample=P.resampler(seed))


@pytest.mark.parametrize("m,n,b,p,k,seed", [
    (1000, 1000, 32, 8, None, 1),
    (517, 389, 16, 8, 200, 2 ** 63 + 5),   # truncated, ragged tiles
    (129, 97, 10, 4, None, 3),            # ragged last block
    (40, 60, 8, 0, None, 4),              # p = 0
])
def test_rsrqrcp_fp64_matches_oracle(H, m, n, b, p, k, seed):
    import torch
    a = I.graded(m, n, 8, seed=m + 5 * n)
    A = to_dev(a)
    tau, jpvt, info = H.rsrqrcp(A, seed, b, p, k)
    torch.cuda.synchronize()
    F, t, jp = to_host(A), to_host(tau), jpvt.cpu().numpy().astype(np.int64)
    ref = oracle_rs(a, seed, b, p, k)
    kk = ref.k
    resid, orth = factor_quality(a, F, t, jp, kk)
    assert resid <= 1e-12 and orth <= 1e-12, (resid, orth)
    assert int(info.cpu()[0]) == ref.info
    tie = first_near_tie(ref.gaps, b, 1e-6)
    upto = n if tie is None else tie
    assert np.array_equal(jp[:upto], ref.jpvt[:upto])
    if tie is None:
        assert np.max(np.abs(np.triu(F[:kk]) - np.triu(ref.F[:kk]))) <= 1e-12 * np.linalg.norm(a)


def test_rsrqrcp_fp32(H):
    import torch
    m, n, b, p, seed = 640, 480, 32, 8, 77
    a = np.asarray(I.graded(m, n, 6, seed=9), dtype=np.float32).astype(np.float64)
    A = to_dev(a, torch.float32)
    tau, jpvt, info = H.rsrqrcp(A, seed, b, p)
    torch.cuda.synchronize()
    F, t, jp = to_host(A), to_host(tau), jpvt.cpu().numpy().astype(np.int64)
    resid, orth = factor_quality(a, F, t, jp, min(m, n))
    assert resid <= 1e-5 and orth <= 1e-5
    ref = oracle_rs(a, seed, b, p, None)
    tie = first_near_tie(ref.gaps, b, 1e-4, ref.sample_norms)
    upto = n if tie is None else tie
    assert np.array_equal(jp[:upto], ref.jpvt[:upto])


def test_rsrqrcp_differs_from_update_but_both_valid(H):
    # the two samplings choose (in general) different pivots; both factor A
    import torch
    m, n, b, p, seed = 300, 300, 16, 8, 12
    a = I.graded(m, n, 8, seed=4)
    A1, A2 = to_dev(a), to_dev(a)
    t1, j1, _ = H.rsrqrcp(A1, seed, b, p)
    Om = H.gaussian(b + p, m, seed)
    t2, j2, _ = H.rqrcp(A2, Om, b, p)
    torch.cuda.synchronize()
    for A, t, j in ((A1, t1, j1), (A2, t2, j2)):
        resid, orth = factor_quality(a, to_host(A), to_host(t), j.cpu().numpy().astype(np.int64), min(m, n))
        assert resid <= 1e-12 and orth <= 1e-12
    # the first block uses the same draws (substream 0), so its pivots agree
    assert torch.equal(j1[:b], j2[:b])
