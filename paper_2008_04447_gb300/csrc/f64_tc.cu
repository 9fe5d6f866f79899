// FP64 matrix products on the bfloat16 tensor cores, to FP64 accuracy.
//
// GB300's FP64 pipe issues about two FMAs per clock per SM (1.26 TFLOP/s),
// while its tensor cores multiply bfloat16 at 2.25 PFLOP/s.  The block
// reflector products of the FP64 factorisation (Alg. 4) therefore run here as
// an Ozaki-style error-free split (Ozaki, Ogita, Oishi and Rump, 2012), with
// the integer steps of f64_slices.cuh:
//
//   D = A B^T, A M x K and B N x K (row r of an operand is its K entries).
//   Each operand row r is scaled by 2^(56 - e_r) (e_r from its largest entry)
//   and cut into eight signed 7-bit slices, stored as bfloat16 "planes"
//   (plane s holds slice s of every entry, K-major, [8][rows][Kp]).  For every
//   slice pair (i, j) with i + j <= 9 (36 pairs) the tensor cores add the
//   exact products A_i B_j^T into one FP32 TMEM accumulator per level
//   L = i + j (8 levels x 64 columns = all 512 TMEM columns).  After every
//   128 steps of K (a level's sum is then below 2^24: exact in FP32) the
//   levels are drained into int64 registers in units of 2^u, and at the end
//   the int64 sums return to FP64 with one rounding and the two exponents.
//
// Kernel: persistent, one CTA per SM; a CTA takes 128 x 64 tiles of D (and
// K ranges, for split-K) one after another.
//   warp 0     : TMA producer: per 32-step K stage the eight A planes (128 x 32)
//                and eight B planes (64 x 32), 96 KB, into a two-stage ring
//   warp 1     : TMEM allocation and the single-thread tcgen05.mma issue: per
//                16-step K slice one MMA per A plane i against B planes
//                0..7-i at once (N up to 256; pair (i, j) lands in level i + j,
//                so the B tiles and the TMEM columns are both contiguous), 12
//                MMAs instead of 36; a chunk's first MMAs wait until the drain
//                warps have read the levels they open
//   warps 2..9 : drain TMEM level by level into int64 accumulators (warp w
//                reads TMEM lane quarter w % 4, columns 32 ((w - 2) / 4) ..),
//                and after a tile's last chunk the FP64 epilogue
//                C = alpha D + beta C, while the MMAs of the next tile run
// All waits are bounded: on a timeout the kernel records RQ_ETIMEOUT, lets its
// copies land, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "common.cuh"
#include "f64_slices.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace rq {
namespace {
using namespace tc;

constexpr int OZ_BM = 128;                       // tile rows = TMEM lanes
constexpr int OZ_BN = 64;                        // tile columns
constexpr int OZ_BK = 32;                        // K per stage: 32 bf16 = one 64-byte swizzle row
constexpr int OZ_NS = 2;                         // stages in the ring
constexpr int OZ_S = kF64Slices;                 // 8 slices
constexpr int OZ_THREADS = 320;
constexpr uint32_t OZ_ABYTES = OZ_BM * OZ_BK * 2;             // one A plane tile: 8 KB
constexpr uint32_t OZ_BBYTES = OZ_BN * OZ_BK * 2;             // one B plane tile: 4 KB
constexpr uint32_t OZ_STAGE = OZ_S * (OZ_ABYTES + OZ_BBYTES); // 96 KB
constexpr uint32_t OZ_TMEM_COLS = OZ_S * OZ_BN;               // 512
constexpr int OZ_STAGES_PER_CHUNK = kF64ChunkK / OZ_BK;       // 4 stages between drains
constexpr int OZ_KPAD = 64;                                   // planes' K padding

static_assert(OZ_TMEM_COLS == 512, "one 64-column accumulator per level fills TMEM");

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups 512
// bytes apart.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(16u >> 4) << 16;    // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512u >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)4 << 61;             // 64-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major, M = 128, N = n (16 <= n <= 256, n % 16 == 0).
__host__ __device__ constexpr uint32_t bf16_idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(OZ_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dtm, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          dtm),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// acc += P 2^sh (sh >= 0) or P 2^sh rounded to nearest (sh < 0): f64_add_level's
// arithmetic with P, an exact integer below 2^24 held in FP32, converted
// through int32 (a 32-bit conversion; the 64-bit one runs on the FP64 pipe).
__device__ __forceinline__ void add_level_fast(int64_t& acc, float P, int sh) {
  const int64_t p = static_cast<int64_t>(__float2int_rz(P));
  if (sh >= 0)
    acc += p << sh;
  else if (sh > -40)
    acc += (p + (static_cast<int64_t>(1) << (-sh - 1))) >> (-sh);
}

// v 2^ex, exactly: the exponent field moves when v and the result are normal,
// else ldexp.
__device__ __forceinline__ double scale_pow2(double v, int ex) {
  const long long b = __double_as_longlong(v);
  const int E = static_cast<int>((b >> 52) & 0x7ff);
  if (E > 0 && E + ex > 0 && E + ex < 2047) return __longlong_as_double(b + (static_cast<long long>(ex) << 52));
  return v == 0.0 ? v : ldexp(v, ex);
}

struct OzArgs {
  int M, N, K;              // D = A B^T: A M x K, B N x K
  int Mp, Np;               // plane row counts (the row offset of plane s is s Mp, s Np)
  int kchunk;               // K range of one split-K part (a multiple of kF64ChunkK)
  int S;                    // split-K parts
  int u;                    // accumulator unit exponent, >= f64_acc_unit(K)
  const int* ea;            // M row exponents of A
  const int* eb;            // N row exponents of B
  double alpha, beta;
  double* C;                // element (i, j) at C[i rs + j cs] (+ z czs for split-K partials)
  long long rs, cs;
  size_t czs;
  int* err;
};

__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, OzArgs a) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  // full[2], empty[2], dfull, ldrained[8]
  __shared__ __align__(8) uint64_t bars[2 * OZ_NS + 1 + OZ_S];
  __shared__ uint32_t s_tmem;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_m = a.Mp / OZ_BM, tiles_n = a.Np / OZ_BN;
  const int items = tiles_m * tiles_n * a.S;
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (OZ_NS + s); };
  const uint32_t dfull = bar0 + 8u * (2 * OZ_NS);
  auto ldrained = [&](int L) { return bar0 + 8u * (2 * OZ_NS + 1 + L); };
  auto sA = [&](int s, int i) { return sm + (size_t)s * OZ_STAGE + (size_t)i * OZ_ABYTES; };
  auto sB = [&](int s, int j) { return sm + (size_t)s * OZ_STAGE + OZ_S * OZ_ABYTES + (size_t)j * OZ_BBYTES; };
  // item w -> tile (tm, tn) and K range z (tm fastest)
  auto item = [&](int w, int& m0, int& n0, int& kbeg, int& nk) {
    const int tm = w % tiles_m;
    const int rest = w / tiles_m;
    const int tn = rest % tiles_n, z = rest / tiles_n;
    m0 = tm * OZ_BM;
    n0 = tn * OZ_BN;
    kbeg = z * a.kchunk;
    const int kend = min(a.K, kbeg + a.kchunk);
    nk = (kend - kbeg + OZ_BK - 1) / OZ_BK;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < OZ_NS; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(dfull, 1);
    for (int L = 0; L < OZ_S; ++L) mbar_init(ldrained(L), 256);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      long long g = 0;  // stages issued so far (all items)
      bool ok = true;
      for (int w = blockIdx.x; w < items && ok; w += gridDim.x) {
        int m0, n0, kbeg, nk;
        item(w, m0, n0, kbeg, nk);
        for (int it = 0; it < nk; ++it, ++g) {
          const int s = (int)(g % OZ_NS);
          if (!mbar_wait(empty(s), (uint32_t)((g / OZ_NS) & 1) ^ 1u, a.err)) { ok = false; break; }
          mbar_expect_tx(full(s), OZ_STAGE);
          const int k = kbeg + it * OZ_BK;
#pragma unroll 1
          for (int i = 0; i < OZ_S; ++i) {
            tma_load_2d(smem_u32(sA(s, i)), &mapA, k, i * a.Mp + m0, full(s));
            tma_load_2d(smem_u32(sB(s, i)), &mapB, k, i * a.Np + n0, full(s));
          }
        }
      }
      // let the copies still in flight land before the CTA may exit
      for (long long q = (g > OZ_NS ? g - OZ_NS : 0); q < g; ++q)
        mbar_wait(full((int)(q % OZ_NS)), (uint32_t)((q / OZ_NS) & 1), a.err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      long long g = 0;   // stages consumed (all items)
      long long gc = 0;  // chunks issued (all items)
      bool ok = true;
      for (int w = blockIdx.x; w < items && ok; w += gridDim.x) {
        int m0, n0, kbeg, nk;
        item(w, m0, n0, kbeg, nk);
        for (int it = 0; it < nk && ok; ++it, ++g) {
          const int s = (int)(g % OZ_NS);
          const int st = it % OZ_STAGES_PER_CHUNK;
          if (!mbar_wait(full(s), (uint32_t)((g / OZ_NS) & 1), a.err)) { ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          // A plane i times B planes 0..7-i in one MMA (N up to 256): the B plane
          // tiles lie back to back in shared memory and pair (i, j) accumulates
          // into level i + j, TMEM columns 64 (i + j) onward, so the output
          // columns are contiguous too.
#pragma unroll 1
          for (int kk = 0; kk < OZ_BK / 16 && ok; ++kk) {
#pragma unroll 1
            for (int i = 0; i < OZ_S && ok; ++i) {
              const int ncols = (OZ_S - i) * OZ_BN;
              for (int c0 = 0; c0 < ncols; c0 += 256) {
                const int nn = ncols - c0 < 256 ? ncols - c0 : 256;
                if (st == 0 && kk == 0 && i == 0 && gc > 0) {
                  // this MMA opens levels c0/64 .. (c0+nn)/64-1: the previous chunk's must be drained
                  for (int L = c0 / OZ_BN; L < (c0 + nn) / OZ_BN; ++L)
                    if (!mbar_wait(ldrained(L), (uint32_t)((gc - 1) & 1), a.err)) { ok = false; break; }
                  if (!ok) break;
                  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                }
                const uint32_t d = tmem + (uint32_t)(i * OZ_BN + c0);
                const uint32_t ai = smem_u32(sA(s, i)) + kk * 32;
                const uint32_t bj = smem_u32(sB(s, 0)) + (uint32_t)(c0 / OZ_BN) * OZ_BBYTES + kk * 32;
                const uint32_t acc = (st == 0 && i == 0 && kk == 0) ? 0u : 1u;
                mma_bf16(d, sw64_desc(ai), sw64_desc(bj), bf16_idesc_n(nn), acc);
              }
            }
          }
          if (!ok) break;
          mma_commit(empty(s));
          if (st == OZ_STAGES_PER_CHUNK - 1 || it == nk - 1) {
            mma_commit(dfull);
            ++gc;
          }
        }
      }
    }
  } else {
    // warps 2..9: drain every chunk into int64, then the FP64 epilogue of the tile
    const int q = warp & 3;           // TMEM lane quarter this warp may read
    const int h = (warp - 2) >> 2;    // column half
    long long gc = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < items && ok; w += gridDim.x) {
      int m0, n0, kbeg, nk;
      item(w, m0, n0, kbeg, nk);
      const int nchunks = (nk + OZ_STAGES_PER_CHUNK - 1) / OZ_STAGES_PER_CHUNK;
      const int row = m0 + q * 32 + lane;
      int64_t acc[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[j] = 0;
      for (int c = 0; c < nchunks; ++c, ++gc) {
        if (!mbar_wait(dfull, (uint32_t)(gc & 1), a.err)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int L = 0; L < OZ_S; ++L) {
          uint32_t r[32];
          const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(L * OZ_BN + 32 * h);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
              "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          // level L is in registers: the next chunk's MMAs may overwrite it
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          mbar_arrive(ldrained(L));
          // level L = 2 + L of f64_add_level, unit 2^u
          const int sh = 112 - kF64SliceBits * (L + 2) - a.u;
#pragma unroll
          for (int j = 0; j < 32; ++j) add_level_fast(acc[j], __uint_as_float(r[j]), sh);
        }
      }
      if (!ok) break;
      if (row < a.M) {
        const int er = a.ea[row] + a.u - 112;
        double* C = a.C + (size_t)(w / (tiles_m * tiles_n)) * a.czs + (long long)row * a.rs;
        const int col0 = n0 + 32 * h;
        // C = alpha D + beta C with the common cases (beta 0 or 1, alpha +-1) free of FP64 multiplies;
        // every load of C is issued before any store (the stores could otherwise alias the later
        // loads, which would serialise 32 memory round trips)
        const int mode = a.beta == 0.0 ? (a.alpha == 1.0 ? 0 : 1) : (a.beta == 1.0 && a.alpha == -1.0 ? 2 : 3);
#pragma unroll
        for (int j0 = 0; j0 < 32; j0 += 16) {
          double cv[16];
          int ebv[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) ebv[j] = col0 + j0 + j < a.N ? __ldg(a.eb + col0 + j0 + j) : 0;
          if (mode >= 2) {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              cv[j] = col0 + j0 + j < a.N ? __ldcs(C + (long long)(col0 + j0 + j) * a.cs) : 0.0;
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int col = col0 + j0 + j;
            if (col < a.N) {
              const double v = scale_pow2(static_cast<double>(acc[j0 + j]), er + ebv[j]);
              double r;
              if (mode == 0)
                r = v;
              else if (mode == 1)
                r = a.alpha * v;
              else if (mode == 2)
                r = cv[j] - v;
              else
                r = fma(a.alpha, v, a.beta * cv[j]);
              __stcs(C + (long long)col * a.cs, r);
            }
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS) : "memory");
  }
}

// bfloat16 bits of a small integer (|v| <= 127: exact, the low 16 bits of the FP32 value are zero).
__device__ __forceinline__ uint32_t bf16_bits_of(int v) { return __float_as_uint(static_cast<float>(v)) >> 16; }

// Operand rows are source COLUMNS: row r's K entries are src[k + r ld] (contiguous).
// One warp per row: the largest magnitude (compared as bit patterns), its exponent,
// then the eight planes; rows r >= R and entries k >= K are zero.
__global__ void slice_cols_kernel(int R, int K, const double* __restrict__ src, long long ld, int Rp, int Kp,
                                  uint16_t* __restrict__ planes, int* __restrict__ e) {
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= Rp) return;
  const double* col = src + (long long)r * ld;
  unsigned long long mx = 0;
  if (r < R)
    for (int k = lane; k < K; k += 32) {
      const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(col[k])) & 0x7fffffffffffffffull;
      mx = b > mx ? b : mx;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  const int ex = f64_scale_exponent(__longlong_as_double(static_cast<long long>(mx)));
  if (lane == 0) e[r] = ex;
  const size_t pstride = (size_t)Rp * Kp;
  uint16_t* out = planes + (size_t)r * Kp;
  for (int k = lane; k < Kp; k += 32) {
    const double x = (r < R && k < K) ? col[k] : 0.0;
    int s[OZ_S];
    f64_slices(x, ex, s);
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) out[i * pstride + k] = static_cast<uint16_t>(bf16_bits_of(s[i]));
  }
}

// The same for long rows (K >= 1024): one 256-thread CTA per row.
__global__ void __launch_bounds__(256) slice_cols_long_kernel(int R, int K, const double* __restrict__ src,
                                                              long long ld, int Rp, int Kp,
                                                              uint16_t* __restrict__ planes, int* __restrict__ e) {
  __shared__ unsigned long long s_mx[8];
  const int r = blockIdx.x;
  const int t = threadIdx.x;
  const double* col = src + (long long)r * ld;
  unsigned long long mx = 0;
  if (r < R)
    for (int k = t; k < K; k += 256) {
      const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(col[k])) & 0x7fffffffffffffffull;
      mx = b > mx ? b : mx;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  if ((t & 31) == 0) s_mx[t >> 5] = mx;
  __syncthreads();
  mx = s_mx[0];
#pragma unroll
  for (int w = 1; w < 8; ++w) mx = s_mx[w] > mx ? s_mx[w] : mx;
  const int ex = f64_scale_exponent(__longlong_as_double(static_cast<long long>(mx)));
  if (t == 0) e[r] = ex;
  const size_t pstride = (size_t)Rp * Kp;
  uint16_t* out = planes + (size_t)r * Kp;
  for (int k = t; k < Kp; k += 256) {
    const double x = (r < R && k < K) ? col[k] : 0.0;
    int s[OZ_S];
    f64_slices(x, ex, s);
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) out[i * pstride + k] = static_cast<uint16_t>(bf16_bits_of(s[i]));
  }
}

// Operand rows are source ROWS: row r's K entries are src[r + k ld] (one thread
// per row; a warp reads 32 consecutive rows of a column at once).
__global__ void slice_rows_kernel(int R, int K, const double* __restrict__ src, long long ld, int Rp, int Kp,
                                  uint16_t* __restrict__ planes, int* __restrict__ e) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= Rp) return;
  unsigned long long mx = 0;
  if (r < R)
    for (int k = 0; k < K; ++k) {
      const unsigned long long b =
          static_cast<unsigned long long>(__double_as_longlong(src[r + (long long)k * ld])) & 0x7fffffffffffffffull;
      mx = b > mx ? b : mx;
    }
  const int ex = f64_scale_exponent(__longlong_as_double(static_cast<long long>(mx)));
  e[r] = ex;
  const size_t pstride = (size_t)Rp * Kp;
  uint16_t* out = planes + (size_t)r * Kp;
  for (int k0 = 0; k0 < Kp; k0 += 8) {
    uint32_t w[OZ_S][4];
#pragma unroll
    for (int t = 0; t < 8; t += 2) {
      int s0[OZ_S], s1[OZ_S];
      const int k = k0 + t;
      f64_slices((r < R && k < K) ? src[r + (long long)k * ld] : 0.0, ex, s0);
      f64_slices((r < R && k + 1 < K) ? src[r + (long long)(k + 1) * ld] : 0.0, ex, s1);
#pragma unroll
      for (int i = 0; i < OZ_S; ++i) w[i][t / 2] = bf16_bits_of(s0[i]) | (bf16_bits_of(s1[i]) << 16);
    }
#pragma unroll
    for (int i = 0; i < OZ_S; ++i)
      *reinterpret_cast<uint4*>(out + i * pstride + k0) = make_uint4(w[i][0], w[i][1], w[i][2], w[i][3]);
  }
}

// The same for long K (K >= 512), where one thread per row leaves the GPU
// nearly idle (Omega's 72 rows of the sketch): three passes over a 2-D grid.
// (1) per-row largest f64_scale_exponent over the nonzero entries, by
//     atomicMax into e preset to kNoExp (the function is monotone in |x|, so
//     this equals the exponent of the row's largest magnitude);
// (2) the planes from 32-row x 64-step tiles staged in shared memory, so that
//     loads run along the rows and every plane store is a 128-byte row segment;
// (3) kNoExp (an all-zero row) -> 0, the exponent of a zero row above.
constexpr int kNoExp = -2139062144;  // 0x80808080, the byte 0x80 four times

__global__ void __launch_bounds__(256) row_exp_max_kernel(int R, int K, const double* __restrict__ src, long long ld,
                                                          int* __restrict__ e) {
  __shared__ int s_ex[8][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r = blockIdx.x * 32 + lane;
  const int seg = blockIdx.y * 8 + w, nseg = gridDim.y * 8;
  unsigned long long mx = 0;
  if (r < R)
    for (int k = seg; k < K; k += nseg) {
      const unsigned long long b =
          static_cast<unsigned long long>(__double_as_longlong(src[r + (long long)k * ld])) & 0x7fffffffffffffffull;
      mx = b > mx ? b : mx;
    }
  s_ex[w][lane] = mx == 0 ? kNoExp : f64_scale_exponent(__longlong_as_double(static_cast<long long>(mx)));
  __syncthreads();
  if (w == 0 && r < R) {
    int ex = s_ex[0][lane];
#pragma unroll
    for (int q = 1; q < 8; ++q) ex = s_ex[q][lane] > ex ? s_ex[q][lane] : ex;
    if (ex != kNoExp) atomicMax(e + r, ex);
  }
}

__global__ void __launch_bounds__(256) slice_rows_tiled_kernel(int R, int K, const double* __restrict__ src,
                                                               long long ld, int Rp, int Kp,
                                                               uint16_t* __restrict__ planes,
                                                               const int* __restrict__ e) {
  __shared__ double tile[64][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 64;
  // loads: warp w takes steps k0 + w + 8 i, lane = row
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int kk = w + 8 * i, k = k0 + kk, r = r0 + lane;
    tile[kk][lane] = (r < R && k < K) ? src[r + (long long)k * ld] : 0.0;
  }
  __syncthreads();
  // thread -> (row, eight consecutive steps); a warp writes four rows' 128-byte segments per plane
  const int rr = threadIdx.x >> 3, oc = threadIdx.x & 7;
  const int r = r0 + rr;
  if (r >= Rp || k0 + 8 * oc >= Kp) return;
  int ex = __ldg(e + r);
  if (ex == kNoExp) ex = 0;
  uint32_t wds[OZ_S][4];
#pragma unroll
  for (int t = 0; t < 8; t += 2) {
    int s0[OZ_S], s1[OZ_S];
    f64_slices(tile[8 * oc + t][rr], ex, s0);
    f64_slices(tile[8 * oc + t + 1][rr], ex, s1);
#pragma unroll
    for (int i = 0; i < OZ_S; ++i) wds[i][t / 2] = bf16_bits_of(s0[i]) | (bf16_bits_of(s1[i]) << 16);
  }
  const size_t pstride = (size_t)Rp * Kp;
  uint16_t* out = planes + (size_t)r * Kp + k0 + 8 * oc;
#pragma unroll
  for (int i = 0; i < OZ_S; ++i)
    *reinterpret_cast<uint4*>(out + i * pstride) = make_uint4(wds[i][0], wds[i][1], wds[i][2], wds[i][3]);
}

__global__ void no_exp_to_zero_kernel(int Rp, int* __restrict__ e) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < Rp && e[r] == kNoExp) e[r] = 0;
}

// C = alpha sum_z P_z + beta C over the split-K partials (P_z compact, M x N
// column-major), C element (i, j) at C[i rs + j cs].
__global__ void oz_reduce_kernel(int M, int N, int S, const double* __restrict__ P, size_t pzs, double alpha,
                                 double beta, double* C, long long rs, long long cs) {
  const size_t total = (size_t)M * N;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % M), j = (int)(t / M);
    double s = 0.0;
    for (int z = 0; z < S; ++z) s += P[z * pzs + t];
    double* out = C + (long long)i * rs + (long long)j * cs;
    *out = beta != 0.0 ? fma(alpha, s, beta * *out) : alpha * s;
  }
}

// 2-D map over the planes [8][rows_per_plane][Kp] bf16: box {32, box_rows}, 64-byte swizzle.
bool make_plane_map(CUtensorMap* map, const uint16_t* base, int Kp, int rows_total, int box_rows) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows_total};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t oz_smem() { return OZ_NS * OZ_STAGE + 1024; }

}  // namespace

int oz_rows_pad(int rows, bool a_side) { return a_side ? (rows + OZ_BM - 1) / OZ_BM * OZ_BM : (rows + OZ_BN - 1) / OZ_BN * OZ_BN; }
int oz_k_pad(int K) { return (K + OZ_KPAD - 1) / OZ_KPAD * OZ_KPAD; }
size_t oz_plane_bytes(int rows_pad, int k_pad) { return (size_t)OZ_S * rows_pad * k_pad * sizeof(uint16_t); }
bool oz_supported() { return encoder() != nullptr; }

cudaError_t oz_slice(const Ctx& c, bool k_along_columns, int R, int K, const double* src, long long ld, int Rp, int Kp,
                     uint16_t* planes, int* e) {
  if (Rp <= 0) return cudaSuccess;
  if (k_along_columns && K >= 1024) {
    slice_cols_long_kernel<<<Rp, 256, 0, c.stream>>>(R, K, src, ld, Rp, Kp, planes, e);
  } else if (k_along_columns) {
    slice_cols_kernel<<<(Rp + 7) / 8, 256, 0, c.stream>>>(R, K, src, ld, Rp, Kp, planes, e);
  } else if (K >= 512) {
    cudaError_t em = cudaMemsetAsync(e, 0x80, sizeof(int) * (size_t)Rp, c.stream);
    if (em != cudaSuccess) return em;
    const int gx = (R + 31) / 32;
    int gy = (K + 8 * 64 - 1) / (8 * 64);  // at least 64 steps per warp
    if (gy > 64) gy = 64;
    row_exp_max_kernel<<<dim3(gx, gy), 256, 0, c.stream>>>(R, K, src, ld, e);
    slice_rows_tiled_kernel<<<dim3((Rp + 31) / 32, Kp / 64), 256, 0, c.stream>>>(R, K, src, ld, Rp, Kp, planes, e);
    no_exp_to_zero_kernel<<<(Rp + 255) / 256, 256, 0, c.stream>>>(Rp, e);
    *c.launches += 2;
  } else {
    slice_rows_kernel<<<(Rp + 127) / 128, 128, 0, c.stream>>>(R, K, src, ld, Rp, Kp, planes, e);
  }
  ++*c.launches;
  return cudaGetLastError();
}

cudaError_t oz_gemm(const Ctx& c, int M, int N, int K, const uint16_t* Ap, int Mp, const int* ea, const uint16_t* Bp,
                    int Np, const int* eb, int Kp, double alpha, double beta, double* C, long long rs, long long cs) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  CUtensorMap ma, mb;
  if (!make_plane_map(&ma, Ap, Kp, OZ_S * Mp, OZ_BM) || !make_plane_map(&mb, Bp, Kp, OZ_S * Np, OZ_BN))
    return cudaErrorInvalidValue;
  const int tiles = (Mp / OZ_BM) * (Np / OZ_BN);
  // Split K (chunks of whole drains, partials in FP64) by the part count S that
  // makes the launch shortest: the persistent CTAs run ceil(tiles S / SMs)
  // waves of items of kchunk / 128 drains each, plus one drain's worth per item
  // (pipeline fill and epilogue) and a small reduction per extra part.  Ties
  // keep the smaller S.
  int S = 1;
  int kchunk = Kp;
  const int nch = (K + kF64ChunkK - 1) / kF64ChunkK;
  if (c.splitk && nch > 2) {
    const size_t cap = c.splitk_bytes / (sizeof(double) * (size_t)M * N);
    const int maxS = (size_t)nch < cap ? nch : (int)cap;
    double best = (double)((tiles + c.num_sms - 1) / c.num_sms) * (nch + 1);
    for (int s = 2; s <= maxS; ++s) {
      const int kc = ((K + s - 1) / s + kF64ChunkK - 1) / kF64ChunkK * kF64ChunkK;
      const int se = (K + kc - 1) / kc;
      const long long waves = ((long long)tiles * se + c.num_sms - 1) / c.num_sms;
      const double t = (double)waves * (kc / kF64ChunkK + 1) + 0.1 * se;
      if (t < best) {
        best = t;
        S = se;
        kchunk = kc;
      }
    }
  }
  OzArgs args;
  args.S = S;
  args.M = M;
  args.N = N;
  args.K = K;
  args.Mp = Mp;
  args.Np = Np;
  args.kchunk = kchunk;
  args.u = f64_acc_unit(K);
  args.ea = ea;
  args.eb = eb;
  args.err = c.err;
  if (S == 1) {
    args.alpha = alpha;
    args.beta = beta;
    args.C = C;
    args.rs = rs;
    args.cs = cs;
    args.czs = 0;
  } else {
    args.alpha = 1.0;
    args.beta = 0.0;
    args.C = static_cast<double*>(c.splitk);
    args.rs = 1;
    args.cs = M;
    args.czs = (size_t)M * N;
  }
  const size_t smem = oz_smem();
  cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int items = tiles * S;
  const int grid = items < c.num_sms ? items : c.num_sms;
  oz_gemm_kernel<<<grid, OZ_THREADS, smem, c.stream>>>(ma, mb, args);
  ++*c.launches;
  e = cudaGetLastError();
  if (e != cudaSuccess || S == 1) return e;
  const size_t total = (size_t)M * N;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 8 * c.num_sms) blocks = 8 * c.num_sms;
  oz_reduce_kernel<<<blocks, 256, 0, c.stream>>>(M, N, S, static_cast<const double*>(c.splitk), total, alpha, beta, C,
                                                 rs, cs);
  ++*c.launches;
  return cudaGetLastError();
}

}  // namespace rq
