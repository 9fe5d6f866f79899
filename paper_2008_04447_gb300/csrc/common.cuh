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
// Polls of a grid barrier's generation word before it gives up (each poll is
// an L2 round trip, with a 32 ns sleep after the first 256): about a second.
constexpr long long kGridWaitLimit = 1ll << 22;

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned int atom_add_acq_rel_gpu(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void st_relaxed_gpu(unsigned int* p, unsigned int v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_add_release_gpu(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for cooperative launches (all CTAs co-resident).
// bar[0] counts the arrivals since the kernel began and bar[1] the CTAs that
// have left; both are 0 when a kernel starts, and grid_exit puts them back to
// 0 when the last CTA leaves, for the next launch on the stream.  Every CTA
// counts its barriers in `epoch` (the same value in all its threads); barrier
// e is complete when bar[0] reaches (e + 1) G.  Thread 0 adds its arrival with
// release order after the CTA's bar.sync (publishing every thread's earlier
// writes) and polls with acquire loads: one L2 round trip each way.  The
// arrive and the wait are separate so that a CTA can work in between.
// Cross-CTA data written before a barrier is read after it through L2 (__ldcg).
__device__ __forceinline__ void grid_arrive(unsigned int* bar) {
  __syncthreads();
  if (threadIdx.x == 0) red_add_release_gpu(bar, 1u);
}

// Returns false when the error word is (or becomes) set or the wait runs out
// (then RQ_ETIMEOUT is recorded); callers then return.
__device__ __forceinline__ bool grid_wait(unsigned int* bar, unsigned int nblocks, int* err, unsigned int epoch) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int target = (epoch + 1u) * nblocks;
    long long it = 0;
    while (static_cast<int>(ld_acquire_gpu(bar) - target) < 0) {
      ++it;
      if ((it & 63) == 0) {
        if (*reinterpret_cast<volatile int*>(err) != 0) { ok = 0; break; }
        if (it > kGridWaitLimit) {
          atomicCAS(err, 0, RQ_ETIMEOUT);
          ok = 0;
          break;
        }
      }
      if (it > 256) __nanosleep(32);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int nblocks, int* err, unsigned int& epoch) {
  grid_arrive(bar);
  const bool ok = grid_wait(bar, nblocks, err, epoch);
  ++epoch;
  return ok;
}

// Every CTA calls this last (after its final barrier); the last one to leave
// returns both counters to 0.
__device__ __forceinline__ void grid_exit(unsigned int* bar, unsigned int nblocks) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int old = atom_add_acq_rel_gpu(bar + 1, 1u);
    if (old == nblocks - 1) {
      st_relaxed_gpu(bar, 0u);
      st_relaxed_gpu(bar + 1, 0u);
    }
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Float-float addition (Knuth's TwoSum for the high parts, the low parts
// added with the rounding error): sums of squares of FP32 values carried to
// about 2^-44 relative without FP64 arithmetic.  Commutative, so a butterfly
// leaves the same bits in every lane.
__device__ __forceinline__ void ff_add(float& h, float& l, float bh, float bl) {
  const float s = h + bh;
  const float bb = s - h;
  const float err = (h - (s - bb)) + (bh - bb);
  l = (l + bl) + err;
  h = s;
}

// Pivot argmax over squared norms, which are never negative: for non-negative
// doubles the IEEE order is the order of their bit patterns as integers, so
// the argmax compares 64-bit integers (an FP64 comparison is a long-latency
// operation on this part).  Ties go to the lowest current position; p < 0 =
// empty.
__device__ __forceinline__ bool better_key(long long k1, int p1, long long k2, int p2) {
  if (p2 < 0) return p1 >= 0;
  if (p1 < 0) return false;
  return (k1 > k2) || (k1 == k2 && p1 < p2);
}

__device__ __forceinline__ void warp_argmax_key(long long& k, int& p, int& tag) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long k2 = __shfl_xor_sync(0xffffffffu, k, o);
    const int p2 = __shfl_xor_sync(0xffffffffu, p, o);
    const int t2 = __shfl_xor_sync(0xffffffffu, tag, o);
    if (better_key(k2, p2, k, p)) { k = k2; p = p2; tag = t2; }
  }
}

// Householder scalars of a column with leading entry alpha and squared norm
// x2 below it (Sec. 2): beta = -sign(alpha) ||a|| (sign(0) = +1), y1 = alpha -
// beta, 1 / y1 and tau = (beta - alpha) / beta (= 2 / v^T v with v = y / y1),
// from one division, 1 / (beta y1); tau = 2 exactly when x2 = 0 and all three
// are 0 for a zero column.  For 2^-100 <= ||a||^2 < 2^100 the FP64 square
// root and reciprocal are Newton-Raphson steps from the FP32 hardware results
// (Markstein's method: each step doubles the correct bits) instead of an FP64
// square root and division, which cost about 650 cycles each on this part:
// one step with `fast` (data held in FP32: 24 -> about 47 bits), two for FP64
// data (the second step's residual is exact by FMA: within about one ulp).
__device__ __forceinline__ void householder_scalars(double alpha, double x2, bool fast, double& beta, double& inv,
                                                    double& tau) {
  const double nrm2 = fma(alpha, alpha, x2);
  beta = 0.0;
  inv = 0.0;
  tau = 0.0;
  const int ex = static_cast<int>((__double_as_longlong(nrm2) >> 52) & 0x7ff);
  if (ex >= 1023 - 100 && ex < 1023 + 100) {
    const float s0f = sqrtf(static_cast<float>(nrm2));
    const double s0 = s0f;
    const double h = static_cast<double>(0.5f / s0f);
    const double s1 = fma(fma(-s0, s0, nrm2), h, s0);
    const double nrm = fast ? s1 : fma(fma(-s1, s1, nrm2), h, s1);
    beta = alpha >= 0.0 ? -nrm : nrm;
    const double y1 = alpha - beta;
    const double den = beta * y1;
    const double r0 = static_cast<double>(1.0f / static_cast<float>(den));
    const double r1 = fma(r0, fma(-den, r0, 1.0), r0);
    const double rr = fast ? r1 : fma(r1, fma(-den, r1, 1.0), r1);
    inv = beta * rr;
    tau = x2 == 0.0 ? 2.0 : -y1 * (y1 * rr);
  } else if (nrm2 > 0.0) {
    const double nrm = sqrt(nrm2);
    beta = alpha >= 0.0 ? -nrm : nrm;
    const double y1 = alpha - beta;
    const double rr = 1.0 / (beta * y1);
    inv = beta * rr;
    tau = x2 == 0.0 ? 2.0 : -y1 * (y1 * rr);
  }
}

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace rq
