"""GPU: batched TUXV (one persistent launch over uneven problems) against the FP64 oracle.

Reduced-precision bar: per problem, the rank-k error ||A - U X V^T||_F /
||A||_F, measured in FP64 against the FP64 input, is within 1.05x that of the
plain FP64 oracle (FP64 sketch, FP64 everything) on the same input.  The FP32
mode (FP32 sketch, FP32 storage, FP64 Householder scalars, sample norms and
Omegahat_11 solve) must meet it on every problem.  The RQ_MIXED mode forms
the sketch from bfloat16-rounded Omega and A: its pivot decisions are those
of a sketch perturbed by about 2^-8 relative, which on these graded spectra
flips near-tied decisions and moves a problem's error either way (measured
0.82x to 1.18x of the FP64 oracle on 40 problems of the batch mix in a CPU
emulation), so it does not carry the per-problem bar; its test checks the
error against an oracle that takes the same bfloat16-rounded decisions
(where no decision is a near-tie) and the spread against the FP64 oracle.
U and V are orthonormal to 1e-5 and X is upper triangular.  A problem's
result is the same, bit for bit, alone and inside the batch (one CTA computes
one problem, with no reduction that depends on its neighbours).
"""
import numpy as np
import pytest

import oracle as O
from paper_2008_04447_gb300 import inputs as I

from gpu_util import first_near_tie, fp64_oracle_error, rank_k_error

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from gpu_util import build_and_handle
    return build_and_handle()


def _mix(count, seed, m_hi=640):
    shapes = I.batch_shapes(count, seed, m_range=(64, m_hi), n_cap=400, k_range=(8, 48))
    out = []
    for i, (m, n, k) in enumerate(shapes):
        b = min(32, k)
        a = I.graded(m, n, 6, seed=seed * 1000 + i)
        om = I.omega(b + 8, m, seed=seed * 1000 + 500 + i)
        out.append((a, om, b, 8, k))
    # largest problems first (the queue is processed in order)
    out.sort(key=lambda t: -(t[0].shape[0] * t[0].shape[1] * t[4]))
    return out


def _to_dev(host):
    import torch
    from paper_2008_04447_gb300 import colmajor
    return [(colmajor(torch.as_tensor(a, dtype=torch.float32)).cuda(),
             colmajor(torch.as_tensor(om, dtype=torch.float32)).cuda(), b, p, k) for a, om, b, p, k in host]


@pytest.mark.parametrize("mode", ["fp32", "mixed"])
def test_batched_tuxv_error_against_the_fp64_oracle(H, mode):
    import torch
    from paper_2008_04447_gb300 import RQ_FP32, RQ_MIXED
    host = _mix(48, seed=3)
    dev = _to_dev(host)
    outs, info = H.tuxv_batched(dev, prec=RQ_MIXED if mode == "mixed" else RQ_FP32)
    torch.cuda.synchronize()
    assert int(info.abs().sum()) == 0
    same, plain = [], []
    for (a, om, b, p, k), (U, X, V) in zip(host, outs):
        U, X, V = U.cpu().double().numpy(), X.cpu().double().numpy(), V.cpu().double().numpy()
        assert np.allclose(U.T @ U, np.eye(k), atol=1e-5)
        assert np.allclose(V.T @ V, np.eye(k), atol=1e-5)
        assert np.allclose(X, np.triu(X))
        e_gpu = rank_k_error(a, U, X, V)
        e_64, _ = fp64_oracle_error(a, om, b, k)
        plain.append(e_gpu / e_64)
        if mode == "mixed":
            a32 = a.astype(np.float32).astype(np.float64)
            o32 = om.astype(np.float32).astype(np.float64)
            ref = O.tuxv(a32, o32, b, k, sketch_inputs="bf16")
            if first_near_tie(ref.tr.gaps, b, 1e-4) is None:
                same.append(e_gpu / rank_k_error(a, ref.U, ref.X, ref.V))
    plain = np.array(plain)
    if mode == "fp32":
        assert plain.max() <= 1.05, (plain.max(), int(np.argmax(plain)))
    else:
        same = np.array(same)
        assert len(same) >= len(host) // 4
        assert same.max() <= 1.05, same.max()
        assert np.median(plain) <= 1.01
        assert plain.max() <= 1.3, plain.max()


def test_batched_result_same_alone_and_in_the_mix(H):
    import torch
    from paper_2008_04447_gb300 import RQ_MIXED
    host = _mix(24, seed=5)
    dev = _to_dev(host)
    outs, info = H.tuxv_batched(dev, prec=RQ_MIXED)
    torch.cuda.synchronize()
    for i in (0, 7, 23):
        solo, info1 = H.tuxv_batched([dev[i]], prec=RQ_MIXED)
        torch.cuda.synchronize()
        for x_mix, x_solo in zip(outs[i], solo[0]):
            assert torch.equal(x_mix, x_solo)


def test_batched_fp32_matches_single_problem_path_quality(H):
    """The batched kernel and rq_tuxv (FP32) reach the same rank-k error (within 2%)."""
    import torch
    from paper_2008_04447_gb300 import RQ_FP32
    host = _mix(6, seed=9, m_hi=400)
    dev = _to_dev(host)
    outs, info = H.tuxv_batched(dev, prec=RQ_FP32)
    torch.cuda.synchronize()
    for (A, Om, b, p, k), (U, X, V), (a, *_rest) in zip(dev, outs, host):
        U1, X1, V1, _, inf1 = H.tuxv(A, Om, b, p, k)
        torch.cuda.synchronize()
        e0 = np.linalg.norm(a - (U.double() @ X.double() @ V.double().T).cpu().numpy())
        e1 = np.linalg.norm(a - (U1.double() @ X1.double() @ V1.double().T).cpu().numpy())
        assert abs(e0 - e1) <= 0.02 * e1


def test_batched_core_svd(H):
    """sigma != NULL: the batched kernel's FP64 Jacobi SVD of each core X.

    The same problems without sigma give X bit for bit (one CTA per problem,
    the same kernel path up to the core), so sigma must equal the singular
    values of that X (numpy, FP64) to the FP32 rounding of the outputs, and
    U diag(sigma) V^T must equal U X V^T.  k = 120 keeps V outside shared
    memory and k = 170 both W and V.
    """
    import torch
    from paper_2008_04447_gb300 import RQ_MIXED
    shapes = [(300, 200, 170, 64), (260, 180, 120, 32), (200, 150, 64, 32), (120, 90, 33, 16), (50, 40, 7, 7),
              (30, 20, 1, 1)]
    host = [(I.graded(m, n, 6, seed=40 + i), I.omega(b + 8, m, seed=60 + i), b, 8, k)
            for i, (m, n, k, b) in enumerate(shapes)]
    dev = _to_dev(host)
    plain, info0 = H.tuxv_batched(dev, prec=RQ_MIXED)
    outs, info = H.tuxv_batched(dev, prec=RQ_MIXED, svd=True)
    torch.cuda.synchronize()
    assert int(info.abs().sum()) == 0 and int(info0.abs().sum()) == 0
    for (a, om, b, p, k), (U0, X0, V0), (U, X, V, s) in zip(host, plain, outs):
        U0, X0, V0 = (t.cpu().double().numpy() for t in (U0, X0, V0))
        U, X, V, s = (t.cpu().double().numpy() for t in (U, X, V, s))
        sv = np.linalg.svd(X0, compute_uv=False)
        assert np.all(np.abs(s - sv) <= 1e-6 * sv[0] + 2e-7 * sv), (k, np.max(np.abs(s - sv)) / sv[0])
        assert np.all(np.diff(s) <= 0)
        assert np.array_equal(X, np.diag(s))
        assert np.allclose(U.T @ U, np.eye(k), atol=1e-5)
        assert np.allclose(V.T @ V, np.eye(k), atol=1e-5)
        idx = np.argmax(np.abs(V), axis=0)
        assert np.all(V[idx, np.arange(k)] > 0)
        nrm = np.linalg.norm(a)
        assert np.linalg.norm((U * s) @ V.T - U0 @ X0 @ V0.T) <= 1e-5 * nrm


def test_batched_graph_capture_and_replay(H):
    """The batched call captured in a CUDA graph replays to the same bits, and
    reads its inputs at replay time (A scaled by 2 gives X scaled by 2 exactly:
    every step is homogeneous and powers of two round exactly)."""
    import torch
    from paper_2008_04447_gb300 import RQ_MIXED, rq_tuxv_batched
    host = _mix(16, seed=7)
    dev = _to_dev(host)
    outs, info = H.tuxv_batched(dev, prec=RQ_MIXED)       # sizes the workspace, uploads descriptors
    torch.cuda.synchronize()
    ref = [tuple(t.clone() for t in o) for o in outs]
    desc = H._keep
    dims = (max(int(t[0].shape[0]) for t in dev), max(int(t[0].shape[1]) for t in dev), max(t[4] for t in dev),
            max(t[2] for t in dev), max(t[3] for t in dev))
    for o in outs:
        for t in o:
            t.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rc = rq_tuxv_batched(H.h, RQ_MIXED, len(dev), desc, *dims)
    assert rc == 0
    assert all(torch.count_nonzero(t) == 0 for o in outs for t in o)   # captured, not run
    g.replay()
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        for t, u in zip(o, r):
            assert torch.equal(t, u)
    dev[0][0].mul_(2.0)
    g.replay()
    torch.cuda.synchronize()
    U, X, V = outs[0]
    assert torch.equal(U, ref[0][0]) and torch.equal(V, ref[0][2])
    assert torch.equal(X, 2.0 * ref[0][1])


def test_prepared_batch_equals_the_call(H):
    """A batch prepared once and launched twice gives the bits of tuxv_batched,
    and its second launch (the buffers unchanged) the same bits again."""
    import torch
    from paper_2008_04447_gb300 import RQ_FP32
    host = _mix(12, seed=8)
    dev = _to_dev(host)
    ref, info = H.tuxv_batched(dev, prec=RQ_FP32)
    torch.cuda.synchronize()
    ref = [tuple(t.clone() for t in o) for o in ref]
    plan = H.prepare_batched(dev)
    for _ in range(2):
        outs, info2 = H.launch_prepared(plan, prec=RQ_FP32)
        torch.cuda.synchronize()
        assert int(info2.abs().sum()) == 0
        for a, b in zip(ref, outs):
            for x, y in zip(a, b):
                assert torch.equal(x, y)
