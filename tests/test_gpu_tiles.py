"""GPU: the batched kernel's tile policy and its autotuner.

Every tile shape of the block GEMMs accumulates each output over the inner
dimension in the same order with the same FMAs, so a batch gives the same bits
under every policy (with and without the core SVD).  The tuner returns a
policy of its search grid (it starts from the default, which is on the grid),
leaves it in the handle, and its outputs are the batch's result.
"""
import pytest

from paper_2008_04447_gb300 import inputs as I

pytestmark = pytest.mark.gpu

POLICIES = [(32, 32), (0, 0), (256, 256), (0, 256), (256, 0), (16, 128), (128, 16)]


@pytest.fixture(scope="module")
def H():
    from gpu_util import build_and_handle
    return build_and_handle()


def _batch(seed):
    import torch
    from paper_2008_04447_gb300 import colmajor
    # the uneven mix plus problems whose products have 33-128 rows or columns
    shapes = list(I.batch_shapes(16, seed, m_range=(64, 640), n_cap=400, k_range=(8, 48)))
    shapes += [(400, 300, 120), (300, 260, 96), (520, 200, 64), (150, 140, 40)]
    out = []
    for i, (m, n, k) in enumerate(shapes):
        b = min(64 if k >= 96 else 32, k)
        a = I.graded(m, n, 6, seed=seed * 1000 + i)
        om = I.omega(b + 8, m, seed=seed * 1000 + 500 + i)
        out.append((colmajor(torch.as_tensor(a, dtype=torch.float32)).cuda(),
                    colmajor(torch.as_tensor(om, dtype=torch.float32)).cuda(), b, 8, k))
    out.sort(key=lambda t: -(t[0].shape[0] * t[0].shape[1] * t[4]))
    return out


def _host(outs):
    return [tuple(t.cpu() for t in o) for o in outs]


@pytest.mark.parametrize("svd", [False, True])
def test_every_tile_policy_gives_the_same_bits(H, svd):
    import torch
    from paper_2008_04447_gb300 import RQ_MIXED
    dev = _batch(seed=11)
    ref = None
    try:
        for tiles in POLICIES:
            H.batch_tiles = tiles
            assert H.batch_tiles == tiles
            outs, info = H.tuxv_batched(dev, prec=RQ_MIXED, svd=svd)
            torch.cuda.synchronize()
            assert int(info.abs().sum()) == 0
            cur = _host(outs)
            if ref is None:
                ref = cur
                continue
            for a, b in zip(ref, cur):
                for x, y in zip(a, b):
                    assert torch.equal(x, y), tiles
    finally:
        H.batch_tiles = (32, 32)


def test_tuner_keeps_a_searched_policy_and_the_result(H):
    import torch
    from paper_2008_04447_gb300 import RQ_MIXED, _lib
    dev = _batch(seed=12)
    H.batch_tiles = (32, 32)
    ref, _ = H.tuxv_batched(dev, prec=RQ_MIXED)
    torch.cuda.synchronize()
    ref = _host(ref)
    try:
        tiles, ms, outs, info = H.tune_batched(dev, prec=RQ_MIXED, reps=1, passes=1)
        torch.cuda.synchronize()
        assert tiles[0] in _lib.RQ_TILE_STEPS and tiles[1] in _lib.RQ_TILE_STEPS
        assert ms > 0.0 and H.batch_tiles == tiles
        assert int(info.abs().sum()) == 0
        for a, b in zip(ref, _host(outs)):
            for x, y in zip(a, b):
                assert torch.equal(x, y)
    finally:
        H.batch_tiles = (32, 32)


def test_tuner_argument_checks(H):
    from paper_2008_04447_gb300 import RQ_MIXED, _lib
    dev = _batch(seed=13)[:2]
    _, _, d, bounds = H._batch(dev, None, False)
    assert _lib.rq_tune_batched(H.h, RQ_MIXED, len(dev), d, *bounds, 0, 1)[0] == -10
    assert _lib.rq_tune_batched(H.h, RQ_MIXED, len(dev), d, *bounds, 1, -1)[0] == -11
    assert _lib.rq_set_batch_tiles(H.h, -1, 0) == -2
    assert H.batch_tiles == (32, 32)
