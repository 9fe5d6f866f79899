// Host helpers from the Bayesian analysis of the sample (Sec. 3.3): the
// distribution of a column's latent squared norm relative to its posterior
// expectation, and the padding p that bounds the chance that a pivot decision
// overestimates a column.
//
// With a Gaussian sample of rank l and Jeffreys' prior, ||A_j||^2 =
// phi ||B_j||^2 / (l - 2) has P(phi < tau | l) = Q(l/2, (l - 2) / (2 tau)),
// Q the regularized upper incomplete gamma function.  For a = l/2 a whole or
// half-whole number, repeated use of Q(a + 1, x) = Q(a, x) + x^a e^-x / Gamma(a + 1)
// (DLMF 8.8.6) from Q(1, x) = e^-x or Q(1/2, x) = erfc(sqrt x) gives the
// finite sums
//   Q(s, x)       = sum_{j=0}^{s-1} x^j e^-x / j!
//   Q(s + 1/2, x) = erfc(sqrt x) + sum_{j=0}^{s-1} x^(j+1/2) e^-x / Gamma(j + 3/2).
// The terms T_j are evaluated outward from the largest one (near j = x), where
// a single logarithmic evaluation fixes its value, then by the ratios
// T_{j+1} / T_j = x / (j + c + 1): no term overflows, and only terms
// negligible against the largest can underflow.  Relative error: a few units
// of roundoff times the size of the exponents in the largest term, about
// 1e-13 for l up to a few hundred.
#include <cmath>

#include "rqrcp.h"

namespace {

double q_half_whole(int l, double x) {
  const int s = l / 2;              // number of terms
  const double c = (l % 2) ? 0.5 : 0.0;
  double base = (l % 2) ? std::erfc(std::sqrt(x)) : 0.0;
  if (s == 0) return base;
  if (x == 0.0) return (l % 2) ? 1.0 : (s > 0 ? 1.0 : 0.0);
  int j0 = (int)std::floor(x - c);
  if (j0 < 0) j0 = 0;
  if (j0 > s - 1) j0 = s - 1;
  const double lx = std::log(x);
  const double t0 = std::exp((j0 + c) * lx - x - std::lgamma(j0 + c + 1.0));
  double sum = t0;
  double t = t0;
  for (int j = j0; j + 1 <= s - 1; ++j) {   // upward: T_{j+1} = T_j x / (j + c + 1)
    t *= x / (j + c + 1.0);
    if (t == 0.0) break;
    sum += t;
  }
  t = t0;
  for (int j = j0; j - 1 >= 0; --j) {       // downward: T_{j-1} = T_j (j + c) / x
    t *= (j + c) / x;
    if (t == 0.0) break;
    sum += t;
  }
  return base + sum;
}

}  // namespace

extern "C" {

int rq_latent_cdf(int l, double tau, double* prob) {
  if (l < 3) return -1;
  if (!(tau > 0.0)) return -2;
  if (!prob) return -3;
  const double x = (l - 2) / (2.0 * tau);
  double q = q_half_whole(l, x);
  *prob = q > 1.0 ? 1.0 : q;
  return RQ_OK;
}

int rq_padding(double tau, double delta, int* p) {
  if (!(tau > 0.0 && tau < 1.0)) return -1;
  if (!(delta > 0.0 && delta < 1.0)) return -2;
  if (!p) return -3;
  for (int q = 2; q <= RQ_PADDING_MAX; ++q) {
    double pr = 1.0;
    rq_latent_cdf(q + 1, tau, &pr);
    if (pr <= delta) {
      *p = q;
      return RQ_OK;
    }
  }
  return RQ_ENOTIMPL;
}

}  // extern "C"
