"""Pins of the numerical building blocks the kernels use in place of slow FP64
operations, emulated in numpy with the same steps (error bounds of the
methods; the GPU parity tests cover the kernels that use them):

* Householder scalars from one division (Sec. 2): tau = (beta - alpha) / beta
  and 1 / y1 formed from r = 1 / (beta y1) equal the paper's tau = 2 / v^T v
  (v = y / y1) and 1 / y1 to a few ulps;
* FP64 square root and reciprocal by one Newton-Raphson step from the FP32
  results (Markstein's method): at least 44 correct bits; by two steps (FP64
  data, the second residual by a fused multiply-add): within 2^-52;
* float-float (TwoSum) sums of squares of FP32 data, summed per thread and
  then by a 32-lane tree as the kernels do: relative error at most 2^-44 for
  entries of at least 2^-52 (measured about 2^-46 to 2^-48), checked against
  an exact sum; a column of entries near 2^-58, where the squares' low parts
  are subnormal, still within 2^-30.
"""
import math
from fractions import Fraction

import numpy as np

F32 = np.float32


def householder_one_division(alpha, x2):
    nrm = math.sqrt(alpha * alpha + x2)
    beta = -nrm if alpha >= 0.0 else nrm
    y1 = alpha - beta
    rr = 1.0 / (beta * y1)
    inv = beta * rr
    tau = 2.0 if x2 == 0.0 else -y1 * (y1 * rr)
    return beta, inv, tau


def test_one_division_scalars_equal_the_paper_formula():
    rng = np.random.default_rng(0)
    for _ in range(20000):
        alpha = float(rng.standard_normal() * 10.0 ** rng.uniform(-30, 30))
        x2 = float((rng.standard_normal() * 10.0 ** rng.uniform(-30, 30)) ** 2)
        beta, inv, tau = householder_one_division(alpha, x2)
        y1 = alpha - beta
        tau_paper = 2.0 / (1.0 + x2 / (y1 * y1))      # 2 / v^T v with v = y / y1
        assert abs(tau - tau_paper) <= 8e-16 * tau_paper
        assert abs(inv - 1.0 / y1) <= 6e-16 * abs(1.0 / y1)
    # a column already zero below its leading entry: tau = 2 exactly, beta = -alpha
    beta, inv, tau = householder_one_division(3.0, 0.0)
    assert tau == 2.0 and beta == -3.0


def newton_sqrt(x):
    s0 = float(np.sqrt(F32(x)))                       # FP32 hardware-like estimate
    h = float(F32(0.5) / F32(s0))
    return s0 + (x - s0 * s0) * h                     # s0^2 is exact in FP64


def newton_rcp(d):
    r0 = float(F32(1.0) / F32(d))
    return r0 + r0 * (1.0 - d * r0)


def test_newton_steps_from_fp32_seeds_give_44_bits():
    rng = np.random.default_rng(1)
    xs = np.exp2(rng.uniform(-100, 100, 50000)) * rng.uniform(1, 2, 50000)
    err_s = max(abs(newton_sqrt(x) - math.sqrt(x)) / math.sqrt(x) for x in xs)
    err_r = max(abs(newton_rcp(x) - 1.0 / x) * x for x in xs)
    assert err_s <= 2.0 ** -44, err_s
    assert err_r <= 2.0 ** -44, err_r


def two_sum_ff(h, l, bh, bl):
    s = F32(h + bh)
    bb = F32(s - h)
    err = F32(F32(h - F32(s - bb)) + F32(bh - bb))
    return s, F32(F32(l + bl) + err)


def ff_square(a):
    a = F32(a)
    p = F32(a * a)
    return p, F32(float(a) * float(a) - float(p))     # the FMA residual: exact in FP32


def ff_thread_then_tree(x, per):
    """The kernels' shape: each thread sums `per` squares in float-float, then
    the 32 lanes are combined by a pairwise (butterfly) tree; the result is
    converted to FP64 once."""
    lanes = []
    for t in range(32):
        h, l = F32(0), F32(0)
        for a in x[t * per:(t + 1) * per]:
            ph, pl = ff_square(a)
            h, l = two_sum_ff(h, l, ph, pl)
        lanes.append((h, l))
    while len(lanes) > 1:
        lanes = [two_sum_ff(*lanes[2 * i], *lanes[2 * i + 1]) for i in range(len(lanes) // 2)]
    h, l = lanes[0]
    return float(h) + float(l)


def test_float_float_sums_of_squares_are_fp64_accurate():
    """In the kernels' shape (a few rows per thread, or up to 128 for a sample
    column, then a 32-lane tree) the float-float sum of squares of FP32 entries
    of magnitude at least 2^-52 is accurate to 2^-44.  A square's rounding
    error a^2 2^-24 stays a normal float down to a = 2^-51; below, the low
    parts lose bits, and at the kernels' lower range limit (2^-60, where they
    switch to FP64) a column of such entries is accurate to about 2^-34."""
    rng = np.random.default_rng(2)
    for per in (1, 8, 128):
        for scale in (2.0 ** -45, 1e-9, 1e-3, 1.0, 1e6, 1e15):
            x = (rng.standard_normal(32 * per) * scale * np.exp(rng.uniform(-3, 3, 32 * per))).astype(np.float32)
            x = np.where(np.abs(x) >= 2.0 ** -52, x, F32(2.0 ** -52))
            exact = math.fsum(float(a) * float(a) for a in x)   # products of FP32 values are exact in FP64
            got = ff_thread_then_tree(x, per)
            assert abs(got - exact) <= 2.0 ** -44 * exact, (per, scale, abs(got - exact) / exact)
    x = (rng.standard_normal(32 * 8) * 2.0 ** -58).astype(np.float32)    # entries near 2^-58
    exact = math.fsum(float(a) * float(a) for a in x)
    assert abs(ff_thread_then_tree(x, 8) - exact) <= 2.0 ** -30 * exact


def fma(a, b, c):
    """a b + c rounded once (what the kernels' fma does)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def newton2_sqrt(x):
    s0 = float(np.sqrt(F32(x)))
    h = float(F32(0.5) / F32(s0))
    s1 = fma(fma(-s0, s0, x), h, s0)
    return fma(fma(-s1, s1, x), h, s1)


def newton2_rcp(d):
    r0 = float(F32(1.0) / F32(d))
    r1 = fma(r0, fma(-d, r0, 1.0), r0)
    return fma(r1, fma(-d, r1, 1.0), r1)


def test_two_newton_steps_give_fp64_square_roots_and_reciprocals():
    rng = np.random.default_rng(2)
    xs = np.exp2(rng.uniform(-100, 100, 4000)) * rng.uniform(1, 2, 4000)
    for x in map(float, xs):
        s = newton2_sqrt(x)
        exact_s = Fraction(x)                      # compare s^2 with x exactly: |s - sqrt(x)| / sqrt(x) ~ |s^2 - x| / 2x
        assert abs(Fraction(s) ** 2 - exact_s) / (2 * exact_s) <= Fraction(2) ** -52, x
        r = newton2_rcp(x)
        assert abs(Fraction(r) * Fraction(x) - 1) <= Fraction(2) ** -52, x
