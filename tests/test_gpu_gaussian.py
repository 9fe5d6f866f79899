"""GPU parity of rq_gaussian (device Philox4x32-10 + Box-Muller) against the
oracle's own implementation of the same published generator.

Bar: FP64 draws within 1e-13 absolute of the oracle's.  Both sides take the
same 52-bit uniforms (integer work, exact); they differ only in the rounding
of log, sqrt and the angle (the oracle forms 2 pi u in FP64, the device calls
sincospi(2u)), a few ulps of values below 8.6 in magnitude, about 1e-14.
FP32 draws within one FP32 ulp of the oracle's value rounded to FP32.
"""
import numpy as np
import pytest

from oracle import philox as P

from gpu_util import build_and_handle, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    return build_and_handle()


CASES = [
    # l, m, seed, substream
    (72, 32768, 0, 0),                      # Omega of the 32768 x 16384 sketch
    (40, 1000, 123456789012345, 7),
    (9, 333, 2 ** 64 - 1, 2 ** 40 + 3),     # odd l m: the last pair is half used
    (1, 1, 3, 0),
    (1, 5, 11, 1),
]


@pytest.mark.parametrize("l,m,seed,sub", CASES)
def test_gaussian_fp64_matches_oracle(H, l, m, seed, sub):
    import torch
    G = H.gaussian(l, m, seed, sub)
    torch.cuda.synchronize()
    ref = P.gaussian(seed, l, m, sub)
    assert np.max(np.abs(to_host(G) - ref)) <= 1e-13


def test_gaussian_fp32_within_one_ulp(H):
    import torch
    l, m, seed = 72, 5000, 42
    G = H.gaussian(l, m, seed, dtype=torch.float32).cpu().numpy()
    ref = P.gaussian(seed, l, m).astype(np.float32)
    assert np.all(np.abs(G - ref) <= np.spacing(np.abs(ref)))


def test_gaussian_leading_dimension_and_prefix(H):
    import torch
    from paper_2008_04447_gb300 import colmajor
    l, m, seed = 24, 777, 9
    full = colmajor(torch.full((l + 5, m), float("nan"), dtype=torch.float64)).cuda()
    H.gaussian(l, m, seed, out=full[:l])
    wide = H.gaussian(l, m + 100, seed)
    torch.cuda.synchronize()
    f = to_host(full)
    assert np.all(np.isnan(f[l:]))                       # rows past l untouched
    assert np.array_equal(f[:l], to_host(wide)[:, :m])    # independent of ldo, prefix of a wider draw


def test_gaussian_repeatable_and_substreams_differ(H):
    import torch
    a = H.gaussian(40, 300, 5, 1)
    b = H.gaussian(40, 300, 5, 1)
    c = H.gaussian(40, 300, 5, 2)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert not torch.any(a == c)


def test_gaussian_bad_arguments(H):
    import torch
    from paper_2008_04447_gb300 import RQ_FP64, rq_gaussian
    buf = torch.empty(100, dtype=torch.float64, device="cuda")
    assert rq_gaussian(H.h, RQ_FP64, 1, 0, 0, 10, buf, 1) == -5
    assert rq_gaussian(H.h, RQ_FP64, 1, 0, 4, 0, buf, 4) == -6
    assert rq_gaussian(H.h, RQ_FP64, 1, 0, 4, 10, None, 4) == -7
    assert rq_gaussian(H.h, RQ_FP64, 1, 0, 4, 10, buf, 3) == -8
    assert rq_gaussian(H.h, 99, 1, 0, 4, 10, buf, 4) == -2
