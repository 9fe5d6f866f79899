"""GPU parity of the reduced-precision paths (FP32 storage; tensor-core 3xTF32
products; FP64 Householder scalars and sample norms) against the FP64 oracle.

Bar (reduced precision): ||AP - QR||_F / ||A||_F <= 1e-5 and
||Q^T Q - I||_F <= 1e-5, measured in FP64 from the FP32 outputs against the
FP64 input; pivots identical to the oracle's (run on the FP32-rounded input) up
to the first near-tie decision, whose relative gap is below 1e-4 times the
growth ||B^[0]|| / ||B^[J]|| of the sample's relative error under the update
formula's cancellation: the products run as 3xTF32 on the tensor cores, whose
FP32 accumulation carries about 10 u_32 = 6e-7 relative error, so a sample is
accurate to about 6e-7 ||B^[0]|| / ||B^[J]|| and 1e-4 leaves a margin of 150;
R within 1e-5 ||A||_F entry by entry when there is no near-tie; after a
near-tie the factorisation must still reveal rank as well as the oracle's:
at every block boundary j whose trailing norm is at least 1e-3 ||A||_F (far
above the FP32 residual), ||R(j:, j:)||_F within 1.05x that of the FP64
oracle on the same input (the rank-j error of RQRCP, Sec. 3); TUXV rank-k
error, in FP64 against the FP64 input, within 1.05x that of the plain FP64
oracle on the FP64 input.
"""
import numpy as np
import pytest

import oracle as O
from paper_2008_04447_gb300 import inputs as I

from gpu_util import (build_and_handle, factor_quality, first_near_tie, fp64_oracle_error, rank_k_error,
                      to_dev, to_host)

pytestmark = pytest.mark.gpu
TIE = 1e-4


@pytest.fixture(scope="module")
def H():
    return build_and_handle()


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("m,n,b,p", [(1000, 1000, 32, 8), (640, 480, 64, 8), (517, 389, 16, 8), (300, 700, 32, 4)])
def test_rqrcp_fp32_matches_oracle(H, m, n, b, p):
    import torch
    a = f32(I.graded(m, n, 6, seed=m + 2 * n))
    om = f32(I.omega(b + p, m, seed=m + 3))
    A = to_dev(a, torch.float32)
    tau, jpvt, info = H.rqrcp(A, to_dev(om, torch.float32), b, p)
    torch.cuda.synchronize()
    F, t, jp = to_host(A), to_host(tau), jpvt.cpu().numpy().astype(np.int64)
    k = min(m, n)
    resid, orth = factor_quality(a, F, t, jp, k)
    assert resid <= 1e-5, resid
    assert orth <= 1e-5, orth
    ref = O.rqrcp(a, om, b)
    tie = first_near_tie(ref.gaps, b, TIE, ref.sample_norms)
    upto = len(jp) if tie is None else tie
    assert np.array_equal(jp[:upto], ref.jpvt[:upto])
    if tie is None:
        assert np.max(np.abs(np.triu(F[:k]) - np.triu(ref.F[:k]))) <= 1e-5 * np.linalg.norm(a)
    # rank-revealing quality at every block boundary, before and after a near-tie
    nrm = np.linalg.norm(a)
    checked = 0
    for j in range(b, k, b):
        t_ref = np.linalg.norm(np.triu(ref.F[j:, j:]))
        if t_ref < 1e-3 * nrm:
            break
        t_gpu = np.linalg.norm(np.triu(F[j:, j:]))
        assert t_gpu <= 1.05 * t_ref, (j, t_gpu / t_ref)
        checked += 1
    assert checked >= 2
    if tie is not None:
        assert tie < checked * b + b    # the check reaches past the first near-tie


@pytest.mark.parametrize("m,n,b", [(1000, 800, 64), (333, 555, 32)])
def test_unpivoted_qr_fp32(H, m, n, b):
    import torch
    a = f32(I.graded(m, n, 6, seed=m))
    A = to_dev(a, torch.float32)
    tau, info = H.qr(A, b)
    torch.cuda.synchronize()
    F, t = to_host(A), to_host(tau)
    resid, orth = factor_quality(a, F, t, np.arange(n), min(m, n))
    assert resid <= 1e-5 and orth <= 1e-5
    Fo, to = O.qr_householder(a)
    assert np.max(np.abs(np.triu(F) - np.triu(Fo))) <= 1e-5 * np.linalg.norm(a)


@pytest.mark.parametrize("mode", ["fp32", "mixed"])
def test_trqrcp_and_tuxv_fp32(H, mode):
    import torch
    from paper_2008_04447_gb300 import RQ_FP32, RQ_MIXED
    m, n, k, b, p = 1200, 900, 128, 32, 8
    a64 = I.lowrank_plus_noise(m, n, 400, 1e-6, seed=21)
    a, om = f32(a64), f32(I.omega(b + p, m, seed=22))
    prec = RQ_MIXED if mode == "mixed" else RQ_FP32
    sk = "bf16" if mode == "mixed" else None
    A, Om = to_dev(a, torch.float32), to_dev(om, torch.float32)
    Y, tau, R, jpvt, info = H.trqrcp(A, Om, b, p, k, prec=prec)
    U, X, V, _, info2 = H.tuxv(A, Om, b, p, k, prec=prec)
    torch.cuda.synchronize()
    ref = O.tuxv(a, om, b, k, sketch_inputs=sk)
    jp = jpvt.cpu().numpy().astype(np.int64)
    tie = first_near_tie(ref.tr.gaps, b, TIE, ref.tr.sample_norms)
    upto = k if tie is None else tie
    assert np.array_equal(jp[:upto], ref.tr.jpvt[:upto])
    if tie is None:
        assert np.max(np.abs(to_host(R) - ref.tr.R)) <= 1e-5 * np.linalg.norm(a)
    U, X, V = to_host(U), to_host(X), to_host(V)
    assert np.allclose(U.T @ U, np.eye(k), atol=1e-5)
    assert np.allclose(V.T @ V, np.eye(k), atol=1e-5)
    e_gpu = rank_k_error(a64, U, X, V)
    e_64, _ = fp64_oracle_error(a64, I.omega(b + p, m, seed=22), b, k)
    assert e_gpu <= 1.05 * e_64, e_gpu / e_64
