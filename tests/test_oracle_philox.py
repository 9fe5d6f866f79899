"""Pins of the oracle's counter-based Gaussian generator (Sec. 3.1's Omega).

The Philox4x32-10 block function is pinned by its published known-answer
values; the uniform and Box-Muller stages by the distribution they must give
(moments, a Kolmogorov-Smirnov test against N(0, 1)) and by the sketch
moments of Sec. 3.1: for a fixed vector a, ||Omega a||^2 / ||a||^2 is
chi-squared with l degrees of freedom, mean l and variance 2 l.
"""
import os

import numpy as np
import pytest

from oracle import philox as P

HERE = os.path.dirname(os.path.abspath(__file__))


def _kat():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            ctr, key, out = (part.split() for part in line.split("|"))
            rows.append(([int(x, 16) for x in ctr], [int(x, 16) for x in key], [int(x, 16) for x in out]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    got = P.philox4x32_10([ctr], key)[0]
    assert [int(x) for x in got] == out


def test_uniforms_strictly_inside_unit_interval():
    w = np.array([[0, 0, 0, 0], [0xFFFFFFFF] * 4], dtype=np.uint32)
    u1, u2 = P.uniforms(w)
    assert u1[0] == 2.0 ** -53 and u2[0] == 2.0 ** -53
    assert u1[1] == 1.0 - 2.0 ** -53 and u2[1] == 1.0 - 2.0 ** -53


def test_layout_is_column_major_position():
    # entry (i, j) depends only on q = i + j l, so an l x m draw is a prefix of a wider one
    a = P.gaussian(7, 40, 33)
    b = P.gaussian(7, 40, 50)
    assert np.array_equal(a, b[:, :33])
    c = P.gaussian(7, 40, 33, substream=1)
    d = P.gaussian(8, 40, 33)
    assert not np.any(a == c) and not np.any(a == d)


def test_gaussian_distribution():
    from scipy import stats
    z = P.gaussian(12345, 1000, 1000).ravel()
    assert abs(z.mean()) < 5 / np.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # consecutive entries (the cos/sin pair of one Box-Muller draw) are uncorrelated
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 5 / np.sqrt(z.size / 2)


def test_sketch_moments_chi_squared():
    # Sec. 3.1: E ||Omega a||^2 = l ||a||^2, Var = 2 l ||a||^4
    l, m, draws = 40, 64, 3000
    a = np.linspace(-1.0, 2.0, m)
    v = np.array([np.sum((P.gaussian(99, l, m, substream=s) @ a) ** 2) for s in range(draws)]) / (a @ a)
    assert abs(v.mean() - l) < 5 * np.sqrt(2 * l / draws)
    assert abs(v.var() - 2 * l) < 5 * np.sqrt((8 * l * l + 48 * l) / draws)


def test_resampler_draws_substream_per_block():
    r = P.resampler(5)
    assert np.array_equal(r(3, 24, 100), P.gaussian(5, 24, 100, substream=3))
