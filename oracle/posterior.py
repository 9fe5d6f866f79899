"""Posterior of a column's latent norm given its sample (Sec. 3.3), FP64 oracle.

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product path.
It shares no code with the CUDA library's host implementation.

With a Gaussian sample B = Omega A_j of rank l and Jeffreys' prior on
||A_j||^2, the posterior of ||A_j||^2 is inverse gamma; writing
||A_j||^2 = phi ||B_j||^2 / (l - 2) (phi = 1 at the posterior mean), the
relative scaling phi has density

    p(phi | l) = ((l - 2) / 2)^(l/2) / (Gamma(l/2) phi^(l/2 + 1)) exp(-(l - 2) / (2 phi))

and distribution P(phi < tau | l) = Q(l/2, (l - 2) / (2 tau)), the regularized
upper incomplete gamma function (scipy.special.gammaincc as a library step).

Padding (a reading of Sec. 3.3): the i-th pivot decision of a block sees a
sample of effective rank l - i + 1, so the last one of a block of b sees
p + 1; P(phi < tau) grows as the rank falls, so the smallest p with
P(phi < tau | p + 1) <= delta bounds every decision of the block.
"""
from __future__ import annotations

import math

from scipy.special import gammaincc, gammaln


def latent_pdf(phi, l):
    """p(phi | l) of Sec. 3.3 (l >= 3, phi > 0)."""
    a = l / 2.0
    c = (l - 2) / 2.0
    return math.exp(a * math.log(c) - gammaln(a) - (a + 1.0) * math.log(phi) - c / phi)


def latent_cdf(l, tau):
    """P(phi < tau | l) = Gamma(l/2, (l-2)/(2 tau)) / Gamma(l/2)."""
    if tau <= 0.0:
        return 0.0
    return float(gammaincc(l / 2.0, (l - 2) / (2.0 * tau)))


def padding(tau, delta, p_max=4096):
    """Smallest p >= 2 (so that the weakest rank p + 1 >= 3 has a posterior mean) with
    P(phi < tau | p + 1) <= delta; None if none up to p_max."""
    for p in range(2, p_max + 1):
        if latent_cdf(p + 1, tau) <= delta:
            return p
    return None
