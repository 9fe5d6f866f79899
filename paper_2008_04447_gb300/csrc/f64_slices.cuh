// Exact FP64 products from bfloat16 tensor-core products: the integer steps.
//
// The FP64 trailing update (Alg. 4's block reflector products) is bound by
// the FP64 pipe.  These functions carry an FP64 product onto bfloat16 MMAs
// with FP32 accumulators without losing FP64 accuracy (an Ozaki-style split):
//
// * A row of the left operand (a column of the right one) is scaled by
//   2^(56 - e), e the exponent with max |x| < 2^e over that row (column), and
//   each entry truncated to the integer X = trunc(|x| 2^(56 - e)) < 2^56,
//   from the FP64 bit pattern alone (no FP64 arithmetic).
// * X is cut into eight 7-bit slices, most significant first, each carrying
//   the sign of x: X = sum_{i=1..8} |s_i| 2^(7 (8 - i)), |s_i| <= 127 (exact
//   in bfloat16).
// * A product of two slices is an integer of magnitude at most 127^2 < 2^14.
//   The pairs (i, j) with i + j = L (L = 2..9, at most eight pairs a level;
//   pairs with i + j > 9 are dropped: at most about 2^-53 2^(ea + eb) per
//   term) form level L:
//     sum_k a_k b_k ~= 2^(ea + eb - 112) sum_L P_L 2^(112 - 7 L),
//   and a level's sum over up to 128 consecutive k stays below
//   8 x 128 x 127^2 < 2^24, so an FP32 accumulator holds it exactly.
// * Each level's exact FP32 partial is drained into one int64 kept in units
//   of 2^u, u = 50 + ceil(log2 K): the sum of all terms' magnitudes is below
//   K 2^112, so no partial sum can leave the int64 range.  Levels whose unit
//   is below 2^u are shifted right with rounding to nearest (an unbiased
//   error of at most half a unit per drained partial).
// * The result returns to FP64 with one rounding, scaled by 2^(u + ea + eb -
//   112).
//
// Host and device code share these functions, so the host tests check the
// device arithmetic bit for bit.
#pragma once
#include <cstdint>
#include <cstring>
#include <cmath>

#ifdef __CUDACC__
#define RQ_HD __host__ __device__ __forceinline__
#else
#define RQ_HD inline
#endif

namespace rq {

constexpr int kF64Slices = 8;                 // slices per operand entry
constexpr int kF64SliceBits = 7;              // bits per slice (|s| <= 127)
constexpr int kF64Levels = kF64Slices;        // levels L = 2 .. kF64Slices + 1
constexpr int kF64ChunkK = 128;               // K steps per exact FP32 partial (8 pairs x 128 x 127^2 < 2^24)

RQ_HD uint64_t f64_bits(double x) {
#ifdef __CUDA_ARCH__
  return static_cast<uint64_t>(__double_as_longlong(x));
#else
  uint64_t b;
  std::memcpy(&b, &x, sizeof b);
  return b;
#endif
}

RQ_HD int clz64(uint64_t v) {
#ifdef __CUDA_ARCH__
  return __clzll(static_cast<long long>(v));
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

// e with m < 2^e for the largest magnitude m of a row or column (m >= 0
// finite; 0 for m == 0, where any e serves).
RQ_HD int f64_scale_exponent(double m) {
  const uint64_t b = f64_bits(m) & 0x7fffffffffffffffull;
  if (b == 0) return 0;
  const int E = static_cast<int>(b >> 52);
  if (E == 0) return -1074 + (64 - clz64(b));   // subnormal: m = b 2^-1074
  return E - 1022;                               // m = 1.f 2^(E - 1023) < 2^(E - 1022)
}

// trunc(|x| 2^(56 - e)) for |x| < 2^e: an integer below 2^56.
RQ_HD uint64_t f64_scaled_int(double x, int e) {
  const uint64_t b = f64_bits(x) & 0x7fffffffffffffffull;
  if (b == 0) return 0;
  const int E = static_cast<int>(b >> 52);
  uint64_t M = b & ((1ull << 52) - 1);
  int ex;                                        // |x| = M 2^ex
  if (E == 0) {
    ex = -1074;
  } else {
    M |= 1ull << 52;
    ex = E - 1075;
  }
  const int sh = ex + 56 - e;                    // |x| 2^(56 - e) = M 2^sh, sh <= 3
  if (sh >= 0) return M << sh;
  if (sh <= -64) return 0;
  return M >> (-sh);
}

// The eight signed slices of x under the exponent e, most significant first.
RQ_HD void f64_slices(double x, int e, int s[kF64Slices]) {
  const uint64_t X = f64_scaled_int(x, e);
  const bool neg = (f64_bits(x) >> 63) != 0;
#pragma unroll
  for (int i = 0; i < kF64Slices; ++i) {
    const int v = static_cast<int>((X >> (kF64SliceBits * (kF64Slices - 1 - i))) & 0x7Fu);
    s[i] = neg ? -v : v;
  }
}

// u = 50 + ceil(log2 K): the accumulator's unit exponent for a K-term product.
RQ_HD int f64_acc_unit(int K) {
  int c = 0;
  while (c < 31 && (1 << c) < K) ++c;
  return 50 + c;
}

// acc += P 2^(112 - 7 L - u): P, level L's exact partial (an integer held in
// FP32, |P| < 2^24); rounded to nearest when the level's unit is below 2^u.
RQ_HD void f64_add_level(int64_t& acc, float P, int L, int u) {
  const int64_t p = static_cast<int64_t>(P);
  const int sh = 112 - kF64SliceBits * L - u;
  if (sh >= 0)
    acc += p * (static_cast<int64_t>(1) << sh);
  else if (sh > -40)                             // |p| < 2^24: a shift of 40 or more leaves 0
    acc += (p + (static_cast<int64_t>(1) << (-sh - 1))) >> (-sh);
}

// The FP64 value of acc (units 2^u) for row and column exponents ea, eb: one
// rounding (int64 to FP64), then an exact power-of-two scaling.
RQ_HD double f64_from_acc(int64_t acc, int u, int ea, int eb) {
  return ldexp(static_cast<double>(acc), u + ea + eb - 112);
}

}  // namespace rq
