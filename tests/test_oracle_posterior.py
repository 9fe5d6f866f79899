"""Pins of the posterior-CDF oracle (Sec. 3.3) and the library's host padding
helper against it (host code only; no GPU)."""
import math
import os

import numpy as np
import pytest

from oracle import posterior as Q

HERE = os.path.dirname(os.path.abspath(__file__))


def _fig1():
    rows = []
    with open(os.path.join(HERE, "golden", "latent_cdf_fig1.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                l, tau, pct = line.split()
                rows.append((int(l), float(tau), float(pct)))
    return rows


@pytest.mark.parametrize("l,tau,pct", _fig1())
def test_cdf_matches_fig1_caption(l, tau, pct):
    # the caption prints two decimals of a percentage; 0.20 % reads 0.195 % rounded up
    assert abs(100.0 * Q.latent_cdf(l, tau) - pct) <= 0.006


@pytest.mark.parametrize("l", [3, 4, 8, 9, 32, 40, 73])
def test_pdf_is_the_derivative_of_the_cdf_and_has_mean_one(l):
    from scipy.integrate import quad
    for tau in (0.1, 0.5, 1.0, 3.0):
        got, _ = quad(lambda x: Q.latent_pdf(x, l), 0.0, tau, limit=200)
        assert abs(got - Q.latent_cdf(l, tau)) <= 1e-9
    if l > 4:   # the mean exists for l > 2 and is the normalisation point phi = 1
        mean, _ = quad(lambda x: x * Q.latent_pdf(x, l), 0.0, np.inf, limit=400)
        assert abs(mean - 1.0) <= 1e-8


def test_cdf_closed_forms():
    # l = 4: Q(2, x) = e^-x (1 + x); l = 3: Q(3/2, x) = erfc(sqrt x) + 2 sqrt(x / pi) e^-x
    for tau in (0.05, 0.3, 2.0):
        x4 = 2.0 / (2.0 * tau)
        assert abs(Q.latent_cdf(4, tau) - math.exp(-x4) * (1 + x4)) <= 1e-15
        x3 = 1.0 / (2.0 * tau)
        q3 = math.erfc(math.sqrt(x3)) + 2.0 * math.sqrt(x3 / math.pi) * math.exp(-x3)
        assert abs(Q.latent_cdf(3, tau) - q3) <= 1e-15 * max(q3, 1e-300) * 10


def test_padding_reading():
    # the paper's setting p = 8: the weakest decision (rank 9) falls below 1/4 of
    # its expectation with probability under one per cent
    assert Q.latent_cdf(9, 0.25) < 0.01
    p = Q.padding(0.25, 0.01)
    assert Q.latent_cdf(p + 1, 0.25) <= 0.01 < Q.latent_cdf(p, 0.25)


def test_library_latent_cdf_matches_oracle():
    import ctypes
    from paper_2008_04447_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    out = ctypes.c_double()
    for l in list(range(3, 80)) + [128, 255, 1000]:
        for tau in (1e-3, 0.05, 0.125, 0.25, 0.5, 0.9, 1.0, 1.7, 4.0, 50.0):
            assert lib.rq_latent_cdf(l, tau, ctypes.byref(out)) == 0
            ref = Q.latent_cdf(l, tau)
            # one exp/lgamma of arguments of size ~ l fixes the largest term: ~ l eps relative
            rel = max(1e-13, 1e-15 * l)
            assert abs(out.value - ref) <= rel * max(ref, 1e-300) + 1e-300, (l, tau, out.value, ref)
    assert lib.rq_latent_cdf(2, 0.5, ctypes.byref(out)) == -1
    assert lib.rq_latent_cdf(8, 0.0, ctypes.byref(out)) == -2


def test_library_padding_matches_oracle():
    import ctypes
    from paper_2008_04447_gb300 import _lib, build
    build.build()
    lib = _lib.load()
    p = ctypes.c_int()
    for tau in (0.1, 0.125, 0.25, 0.5, 0.8):
        for delta in (1e-1, 1e-2, 3e-3, 1e-4, 1e-8):
            assert lib.rq_padding(tau, delta, ctypes.byref(p)) == 0
            assert p.value == Q.padding(tau, delta), (tau, delta)
    assert lib.rq_padding(1.5, 0.01, ctypes.byref(p)) == -1
    assert lib.rq_padding(0.5, 0.0, ctypes.byref(p)) == -2
