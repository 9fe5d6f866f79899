// Counter-based Gaussian draws on the device: the compression matrix Omega of
// Sec. 3.1 (i.i.d. N(0, 1) entries) and the fresh per-block matrices of
// repeated sampling (Sec. 3.4), as a pure function of (seed, substream,
// position).
//
// Generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the
// Box-Muller transform.  One Philox call per pair of entries:
//   key     = (seed low word, seed high word)
//   counter = (t low, t high, substream low, substream high), t = q / 2, where
//             q = i + j l is the entry's column-major position in the l x m
//             matrix (the leading dimension does not enter);
//   round   = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0) with (hi0, lo0) the
//             64-bit product 0xD2511F53 c0 and (hi1, lo1) = 0xCD9E8D57 c2;
//             ten rounds, the key advancing by (0x9E3779B9, 0xBB67AE85);
//   u1, u2  = ((x0 x1 >> 12) + 1/2) 2^-52 and ((x2 x3 >> 12) + 1/2) 2^-52,
//             both exact in FP64 and strictly inside (0, 1);
//   entries = r cos(2 pi u2) at q = 2t and r sin(2 pi u2) at q = 2t + 1,
//             r = sqrt(-2 ln u1), in FP64 with CUDA's log and sincospi; FP32
//             outputs are those values rounded to nearest.
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace rq {
namespace {

__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3, uint32_t k0,
                                             uint32_t k1) {
  const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
  const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
  c0 = hi1 ^ c1 ^ k0;
  c1 = lo1;
  c2 = hi0 ^ c3 ^ k1;
  c3 = lo0;
}

template <typename T>
__global__ void __launch_bounds__(256) gaussian_kernel(uint64_t seed, uint64_t sub, int l, long long total, T* Om,
                                                       int ldo) {
  const long long npairs = (total + 1) / 2;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < npairs; t += stride) {
    uint32_t c0 = (uint32_t)t, c1 = (uint32_t)((unsigned long long)t >> 32);
    uint32_t c2 = (uint32_t)sub, c3 = (uint32_t)(sub >> 32);
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
      philox_round(c0, c1, c2, c3, k0, k1);
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t a = ((((uint64_t)c0) << 32) | c1) >> 12;
    const uint64_t b = ((((uint64_t)c2) << 32) | c3) >> 12;
    const double u1 = ((double)a + 0.5) * 0x1p-52;
    const double u2 = ((double)b + 0.5) * 0x1p-52;
    const double r = sqrt(-2.0 * log(u1));
    double s, co;
    sincospi(2.0 * u2, &s, &co);
    const long long q = 2 * t;
    Om[(size_t)(q % l) + (size_t)(q / l) * ldo] = T(r * co);
    if (q + 1 < total) Om[(size_t)((q + 1) % l) + (size_t)((q + 1) / l) * ldo] = T(r * s);
  }
}

}  // namespace

template <typename T>
cudaError_t gaussian(const Ctx& c, uint64_t seed, uint64_t substream, int l, int m, T* Omega, int ldo) {
  const long long total = (long long)l * m;
  if (total <= 0) return cudaSuccess;
  const long long npairs = (total + 1) / 2;
  const long long cap = (long long)c.num_sms * 8;
  const long long blocks = (npairs + 255) / 256 < cap ? (npairs + 255) / 256 : cap;
  gaussian_kernel<T><<<(unsigned)blocks, 256, 0, c.stream>>>(seed, substream, l, total, Omega, ldo);
  ++*c.launches;
  return cudaGetLastError();
}

template cudaError_t gaussian<double>(const Ctx&, uint64_t, uint64_t, int, int, double*, int);
template cudaError_t gaussian<float>(const Ctx&, uint64_t, uint64_t, int, int, float*, int);

}  // namespace rq
