// Shared device helpers for the RQRCP library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "rqrcp.h"

namespace rq {

// Spin limit for every wait on another CTA: ~2^24 polls with a 64 ns sleep
// (about one to two seconds).  A wait that runs out sets RQ_ETIMEOUT in the
// error word and returns, so the kernel ends instead of hanging the GPU.
constexpr long long kSpinLimit = 1ll << 24;

// Grid-wide barrier for cooperative launches (all CTAs co-resident).
// bar[0] = arrival count, bar[1] = generation.  Must start at {0, g}.
// Returns false when the error word is (or becomes) set; callers then return.
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int nblocks, int* err) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vgen = bar + 1;
    volatile int* verr = err;
    if (*verr != 0) {
      ok = 0;
    } else {
      unsigned int gen = *vgen;
      __threadfence();
      unsigned int arrived = atomicAdd(bar, 1u);
      if (arrived == nblocks - 1) {
        atomicExch(bar, 0u);
        __threadfence();
        atomicAdd(bar + 1, 1u);
      } else {
        long long it = 0;
        while (*vgen == gen) {
          if (*verr != 0) { ok = 0; break; }
          if (++it > kSpinLimit) {
            atomicCAS(err, 0, RQ_ETIMEOUT);
            ok = 0;
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// (value, position) max with ties to the lowest position; pos < 0 = empty.
__device__ __forceinline__ bool better(double v1, int p1, double v2, int p2) {
  if (p2 < 0) return p1 >= 0;
  if (p1 < 0) return false;
  return (v1 > v2) || (v1 == v2 && p1 < p2);
}

__device__ __forceinline__ void warp_argmax(double& v, int& p, int& tag) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    int p2 = __shfl_xor_sync(0xffffffffu, p, o);
    int t2 = __shfl_xor_sync(0xffffffffu, tag, o);
    if (better(v2, p2, v, p)) { v = v2; p = p2; tag = t2; }
  }
}

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace rq
