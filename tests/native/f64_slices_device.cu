// Device build of the FP64-slice arithmetic for the compile check in the CPU
// tests (nvcc -c for sm_103a; nothing here is launched).  Test infrastructure only.
#include "../../paper_2008_04447_gb300/csrc/f64_slices.cuh"

__global__ void f64s_device_check(const double* x, const int* e, int n, int* s, long long* acc, const float* P,
                                  int u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  rq::f64_slices(x[i], e[i], s + rq::kF64Slices * i);
  int64_t a = 0;
  rq::f64_add_level(a, P[i], 2 + i % rq::kF64Levels, u);
  acc[i] = a + rq::f64_scale_exponent(x[i]) + static_cast<long long>(rq::f64_from_acc(a, u, 0, 0));
}
