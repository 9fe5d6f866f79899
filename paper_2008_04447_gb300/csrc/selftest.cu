// Failure-detection self-test: a grid barrier whose last arrival never comes.
//
// Every wait on another CTA in this library (grid barriers of the cooperative
// panel, sample-QRCP and Jacobi kernels; mbarrier waits of the tensor-core
// kernel) is bounded: when it runs out, the kernel writes RQ_ETIMEOUT to the
// caller's info word and returns, so a lost arrival ends a call with an error
// status instead of hanging the GPU.  rq_selftest_wait_timeout exercises that
// path on purpose with the library's own grid barrier: two CTAs wait for a
// third that is never launched.
#include <cuda_runtime.h>

#include "common.cuh"

namespace rq {
namespace {

__global__ void barrier_timeout_kernel(unsigned int* bar, int* err) {
  unsigned int epoch = 0;
  // expects gridDim.x + 1 arrivals: the wait can only end by running out
  grid_barrier(bar, gridDim.x + 1, err, epoch);
}

}  // namespace
}  // namespace rq

extern "C" int rq_selftest_wait_timeout(unsigned int* bar, int* info, rq_stream stream) {
  if (!bar) return -1;
  if (!info) return -2;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(info, 0, sizeof(int), st);
  if (e != cudaSuccess) return RQ_ECUDA;
  rq::barrier_timeout_kernel<<<2, 64, 0, st>>>(bar, info);
  return cudaGetLastError() == cudaSuccess ? RQ_OK : RQ_ECUDA;
}
