// Host build of the FP64-slice arithmetic (paper_2008_04447_gb300/csrc/f64_slices.cuh)
// for the CPU tests: plain C entry points over arrays.  Test infrastructure only.
#include "../../paper_2008_04447_gb300/csrc/f64_slices.cuh"

extern "C" {

void f64s_exponents(const double* m, int n, int* e) {
  for (int i = 0; i < n; ++i) e[i] = rq::f64_scale_exponent(m[i]);
}

void f64s_scaled(const double* x, const int* e, int n, unsigned long long* X) {
  for (int i = 0; i < n; ++i) X[i] = rq::f64_scaled_int(x[i], e[i]);
}

void f64s_slices(const double* x, const int* e, int n, int* s) {
  for (int i = 0; i < n; ++i) rq::f64_slices(x[i], e[i], s + static_cast<long>(i) * rq::kF64Slices);
}

int f64s_acc_unit(int K) { return rq::f64_acc_unit(K); }

// P: nchunks x levels (L = 2 .. 9 in order) exact partials; returns the accumulator.
long long f64s_combine(const float* P, int nchunks, int u) {
  int64_t acc = 0;
  for (int c = 0; c < nchunks; ++c)
    for (int l = 0; l < rq::kF64Levels; ++l) rq::f64_add_level(acc, P[c * rq::kF64Levels + l], l + 2, u);
  return acc;
}

double f64s_from_acc(long long acc, int u, int ea, int eb) { return rq::f64_from_acc(acc, u, ea, eb); }


}  // extern "C"
