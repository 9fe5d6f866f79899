// FP32 GEMM on the 5th-generation tensor cores: C = alpha * A^T B + beta * C
// with 3xTF32 error compensation (or plain TF32).
//
// B is K x N column-major (K-major).  A is either K x M column-major (K-major,
// C = alpha A^T B: loaded with a 128-byte-swizzled TMA box) or M x K
// column-major (M-major, C = alpha A B: loaded with a plain TMA box and
// transposed into the K-major swizzled layout while it is split).  This covers
// the large FP32 products of the path: W^T = (YT)^T A2 and Y2^T A (K-major),
// the update A2 -= Y W^T, the sketch Omega A and Z1 = A V (M-major).
//
// Per CTA: one 128 x BN output tile, accumulated in TMEM.
//   warp 0      : TMA producer (128B-swizzled BK=32 slices of A and B)
//   warp 1      : TMEM allocation and the single-thread tcgen05.mma issue
//   warps 2..5  : split each landed slice into TF32 hi / lo parts in place
//                 (hi = x rounded to TF32, lo = x - hi rounded to TF32, so the
//                 tensor core's own TF32 truncation never bites and the split
//                 is unbiased), then the epilogue
//                 (tcgen05.ld -> registers -> C)
// For each BK slice: Ahi*Bhi + Ahi*Blo + Alo*Bhi, four K=8 MMAs per product.
// The tensor core's FP32 accumulation is not IEEE round-to-nearest: each MMA
// adds an error of about one ulp of the accumulator, all of the same sign.  So
// the Ahi*Bhi products go to one TMEM accumulator and the two correction
// products (2^-11 smaller) to a second one, and long K is cut into chunks of
// at most 1024 whose partial results are added in IEEE FP32 (split-K reduce).
// With bf16 set, both slices are instead rounded to bfloat16 in place (round
// to nearest even) and one plain TF32 MMA per K=8 step follows: bfloat16
// values are exact in TF32 and their products exact in FP32, so this is the
// BF16-input, FP32-accumulate product of the reduced-precision sketch.
// All waits are bounded; on a timeout the kernel records RQ_ETIMEOUT, lets
// its copies land, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "common.cuh"
#include "kernels.h"
#include "tc_common.cuh"

namespace rq {
namespace {
using namespace tc;

constexpr int TBM = 128;  // tile rows (M) = TMEM lanes
constexpr int TBK = 32;   // K slice: 32 FP32 = one 128-byte swizzle row
constexpr int kTcThreads = 192;

// Instruction descriptor: D f32, A and B tf32, both K-major, M = 128, N = bn.
__host__ __device__ constexpr uint32_t tf32_idesc(int bn) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(TBM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtm, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          dtm),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float4 bf16r4(float4 x) {
  x.x = bf16r(x.x);
  x.y = bf16r(x.y);
  x.z = bf16r(x.z);
  x.w = bf16r(x.w);
  return x;
}

struct TcArgs {
  int M, N, K;       // full problem
  int kchunk;        // K range of blockIdx.z
  float alpha, beta;
  float* C;
  int ldc;
  int transC;        // store C^T (C is N x M)
  size_t czs;        // blockIdx.z stride of C (split-K partials)
  int split3;        // 3xTF32 (1) or plain TF32 (0)
  int bf16;          // round both operands to bfloat16 first (plain TF32 MMA)
  int* err;
};

template <int BN, int NS, bool AMN>
__global__ void __launch_bounds__(kTcThreads)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcArgs a) {
  constexpr uint32_t ABYTES = TBM * TBK * 4;
  constexpr uint32_t BBYTES = BN * TBK * 4;
  // hi and lo copies of both slices (an M-major A slice lands in its hi area)
  constexpr uint32_t STAGE = 2 * ABYTES + 2 * BBYTES;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t bars[3 * NS + 1];
  __shared__ uint32_t s_tmem;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TBM, n0 = blockIdx.y * BN;
  const int kbeg = blockIdx.z * a.kchunk;
  const int kend = min(a.K, kbeg + a.kchunk);
  const int nk = (kend - kbeg + TBK - 1) / TBK;
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto ready = [&](int s) { return bar0 + 8u * (NS + s); };
  auto empty = [&](int s) { return bar0 + 8u * (2 * NS + s); };
  const uint32_t done = bar0 + 8u * (3 * NS);
  auto a_hi = [&](int s) { return sm + (size_t)s * STAGE; };
  auto a_lo = [&](int s) { return sm + (size_t)s * STAGE + ABYTES; };
  auto b_hi = [&](int s) { return sm + (size_t)s * STAGE + 2 * ABYTES; };
  auto b_lo = [&](int s) { return sm + (size_t)s * STAGE + 2 * ABYTES + BBYTES; };
  auto a_raw = [&](int s) { return sm + (size_t)s * STAGE; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(full(s), 1);
      mbar_init(ready(s), 128);
      mbar_init(empty(s), 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(2 * BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      bool ok = true;
      for (int it = 0; it < nk && ok; ++it) {
        const int s = it % NS;
        const uint32_t ph = (it / NS) & 1;
        if (!mbar_wait(empty(s), ph ^ 1, a.err)) { ok = false; break; }
        mbar_expect_tx(full(s), ABYTES + BBYTES);
        if (AMN)
          tma_load_2d(smem_u32(a_raw(s)), &mapA, m0, kbeg + it * TBK, full(s));
        else
          tma_load_2d(smem_u32(a_hi(s)), &mapA, kbeg + it * TBK, m0, full(s));
        tma_load_2d(smem_u32(b_hi(s)), &mapB, kbeg + it * TBK, n0, full(s));
        issued = it + 1;
      }
      // let the copies still in flight land before the CTA may exit
      for (int it = (issued > NS ? issued - NS : 0); it < issued; ++it)
        mbar_wait(full(it % NS), (it / NS) & 1, a.err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = tf32_idesc(BN);
      bool ok = true;
      for (int it = 0; it < nk && ok; ++it) {
        const int s = it % NS;
        const uint32_t ph = (it / NS) & 1;
        if (!mbar_wait(ready(s), ph, a.err)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = smem_u32(a_hi(s)), al = smem_u32(a_lo(s));
        const uint32_t bh = smem_u32(b_hi(s)), bl = smem_u32(b_lo(s));
#pragma unroll
        for (int kk = 0; kk < TBK / 8; ++kk) {
          const uint32_t off = kk * 32;
          const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
          mma_tf32(tmem, sw128_desc(ah + off), sw128_desc(bh + off), idesc, acc);
          if (a.split3) {
            mma_tf32(tmem + BN, sw128_desc(ah + off), sw128_desc(bl + off), idesc, acc);
            mma_tf32(tmem + BN, sw128_desc(al + off), sw128_desc(bh + off), idesc, 1u);
          }
        }
        mma_commit(empty(s));
      }
      mma_commit(done);
    }
  } else {
    // warps 2..5: split slices into hi / lo, then the epilogue
    const int t = threadIdx.x - 64;
    bool ok = true;
    for (int it = 0; it < nk && ok; ++it) {
      const int s = it % NS;
      const uint32_t ph = (it / NS) & 1;
      if (!mbar_wait(full(s), ph, a.err)) { ok = false; break; }
      if (AMN) {
        // the slice landed M-major as [k][m] (32 rows of 128 m) in the hi area;
        // thread t takes column m = t into registers, then (after all 128
        // threads have read) writes row t of the K-major tile, whose 16-byte
        // chunk q sits at (q ^ (t & 7)) (128-byte swizzle)
        const float* raw = reinterpret_cast<const float*>(a_raw(s));
        float xr[TBK];
#pragma unroll
        for (int k = 0; k < TBK; ++k) xr[k] = raw[k * TBM + t];
        asm volatile("bar.sync 1, 128;" ::: "memory");
        float4* ah = reinterpret_cast<float4*>(a_hi(s) + t * 128);
        float4* al = reinterpret_cast<float4*>(a_lo(s) + t * 128);
#pragma unroll
        for (int q = 0; q < TBK / 4; ++q) {
          float4 x, h, l;
          x.x = xr[4 * q + 0];
          x.y = xr[4 * q + 1];
          x.z = xr[4 * q + 2];
          x.w = xr[4 * q + 3];
          if (a.split3) {
            h.x = tf32_hi(x.x); h.y = tf32_hi(x.y); h.z = tf32_hi(x.z); h.w = tf32_hi(x.w);
            l.x = tf32_hi(x.x - h.x); l.y = tf32_hi(x.y - h.y); l.z = tf32_hi(x.z - h.z); l.w = tf32_hi(x.w - h.w);
          } else {
            h = a.bf16 ? bf16r4(x) : x;
            l = h;
          }
          ah[q ^ (t & 7)] = h;
          if (a.split3) al[q ^ (t & 7)] = l;
        }
      }
      if (a.split3 && !AMN) {
        float4* ah = reinterpret_cast<float4*>(a_hi(s));
        float4* al = reinterpret_cast<float4*>(a_lo(s));
        for (int e = t; e < (int)(ABYTES / 16); e += 128) {
          float4 x = ah[e], h, l;
          h.x = tf32_hi(x.x); h.y = tf32_hi(x.y); h.z = tf32_hi(x.z); h.w = tf32_hi(x.w);
          l.x = tf32_hi(x.x - h.x); l.y = tf32_hi(x.y - h.y); l.z = tf32_hi(x.z - h.z); l.w = tf32_hi(x.w - h.w);
          ah[e] = h;
          al[e] = l;
        }
      }
      if (a.split3) {
        float4* bh = reinterpret_cast<float4*>(b_hi(s));
        float4* bl = reinterpret_cast<float4*>(b_lo(s));
        for (int e = t; e < (int)(BBYTES / 16); e += 128) {
          float4 x = bh[e], h, l;
          h.x = tf32_hi(x.x); h.y = tf32_hi(x.y); h.z = tf32_hi(x.z); h.w = tf32_hi(x.w);
          l.x = tf32_hi(x.x - h.x); l.y = tf32_hi(x.y - h.y); l.z = tf32_hi(x.z - h.z); l.w = tf32_hi(x.w - h.w);
          bh[e] = h;
          bl[e] = l;
        }
      } else if (a.bf16) {
        if (!AMN) {
          float4* ah = reinterpret_cast<float4*>(a_hi(s));
          for (int e = t; e < (int)(ABYTES / 16); e += 128) ah[e] = bf16r4(ah[e]);
        }
        float4* bh = reinterpret_cast<float4*>(b_hi(s));
        for (int e = t; e < (int)(BBYTES / 16); e += 128) bh[e] = bf16r4(bh[e]);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(ready(s));
    }
    const bool have = ok && mbar_wait(done, 0, a.err);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (have) {
      const int q = warp & 3;  // TMEM lane quarter this warp may read
      const int row = m0 + q * 32 + lane;
      float* C = a.C + blockIdx.z * a.czs;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
        if (a.split3) {
          uint32_t q2[32];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
              "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
              : "=r"(q2[0]), "=r"(q2[1]), "=r"(q2[2]), "=r"(q2[3]), "=r"(q2[4]), "=r"(q2[5]), "=r"(q2[6]),
                "=r"(q2[7]), "=r"(q2[8]), "=r"(q2[9]), "=r"(q2[10]), "=r"(q2[11]), "=r"(q2[12]), "=r"(q2[13]),
                "=r"(q2[14]), "=r"(q2[15]), "=r"(q2[16]), "=r"(q2[17]), "=r"(q2[18]), "=r"(q2[19]), "=r"(q2[20]),
                "=r"(q2[21]), "=r"(q2[22]), "=r"(q2[23]), "=r"(q2[24]), "=r"(q2[25]), "=r"(q2[26]), "=r"(q2[27]),
                "=r"(q2[28]), "=r"(q2[29]), "=r"(q2[30]), "=r"(q2[31])
              : "r"(taddr + (uint32_t)BN));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(q2[j]));
        } else {
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        }
        if (row < a.M) {
          const size_t rs = a.transC ? (size_t)a.ldc : 1;   // step between rows
          const size_t cs = a.transC ? 1 : (size_t)a.ldc;   // step between columns
          float* base = C + (size_t)row * rs + (size_t)(n0 + c0) * cs;
          const int ncol = min(32, a.N - n0 - c0);
          float cv[32];
          if (a.beta != 0.f) {
#pragma unroll
            for (int j = 0; j < 32; ++j) cv[j] = j < ncol ? base[(size_t)j * cs] : 0.f;
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (j < ncol) {
              float v = a.alpha * __uint_as_float(r[j]);
              if (a.beta != 0.f) v = fmaf(a.beta, cv[j], v);
              base[(size_t)j * cs] = v;
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN) : "memory");
  }
}

// 2-D K-major map over a column-major (rows = K) matrix: box {32, box_rows}.
bool make_map(CUtensorMap* map, const float* base, int K, int cols, int ld, int box_rows) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)TBK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D M-major map over a column-major M x K matrix: box {128, 32}, no swizzle.
bool make_map_mn(CUtensorMap* map, const float* base, int M, int K, int ld) {
  EncodeFn enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)M, (cuuint64_t)K};
  cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)TBM, (cuuint32_t)TBK};
  cuuint32_t es[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int NS, bool AMN>
size_t tc_smem() {
  return (size_t)NS * (2 * TBM * TBK * 4 + 2 * BN * TBK * 4) + 1024;
}

template <int BN, int NS, bool AMN>
cudaError_t tc_launch(const Ctx& c, const CUtensorMap& ma, const CUtensorMap& mb, const TcArgs& args, dim3 grid) {
  const size_t smem = tc_smem<BN, NS, AMN>();
  cudaError_t e =
      cudaFuncSetAttribute(tc_gemm_kernel<BN, NS, AMN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  tc_gemm_kernel<BN, NS, AMN><<<grid, kTcThreads, smem, c.stream>>>(ma, mb, args);
  ++*c.launches;
  return cudaGetLastError();
}

template <bool AMN>
cudaError_t tc_dispatch(const Ctx& c, int bn, int K, const CUtensorMap& ma, const CUtensorMap& mb,
                        const TcArgs& args, dim3 grid) {
  if (bn == 64) {
    if (K <= 64) return tc_launch<64, 2, AMN>(c, ma, mb, args, grid);  // two CTAs per SM
    return tc_launch<64, 4, AMN>(c, ma, mb, args, grid);
  }
  return tc_launch<128, 2, AMN>(c, ma, mb, args, grid);
}

}  // namespace

bool tc_gemm_supported(const float* A, int lda, const float* B, int ldb) {
  return tc::encoder() != nullptr && (reinterpret_cast<uintptr_t>(A) % 16 == 0) &&
         (reinterpret_cast<uintptr_t>(B) % 16 == 0) && lda % 4 == 0 && ldb % 4 == 0;
}

namespace {
cudaError_t tc_gemm_any(const Ctx& c, bool amn, int M, int N, int K, float alpha, const float* A, int lda,
                        const float* B, int ldb, float beta, float* C, int ldc, bool transC, bool split3,
                        bool bf16 = false) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (!tc_gemm_supported(A, lda, B, ldb)) return cudaErrorNotSupported;
  // 64-column tiles when N is small or K is short (two CTAs per SM, so one
  // CTA's epilogue overlaps the other's loads); 128 otherwise
  const int bn = (N <= 64 || K <= 64) ? 64 : 128;
  CUtensorMap ma, mb;
  const bool okA = amn ? make_map_mn(&ma, A, M, K, lda) : make_map(&ma, A, K, M, lda, TBM);
  if (!okA || !make_map(&mb, B, K, N, ldb, bn)) return cudaErrorInvalidValue;
  const int tiles = ((M + TBM - 1) / TBM) * ((N + bn - 1) / bn);
  int S = 1;
  if (c.splitk && K > 1024) {
    // enough CTAs to fill the GPU, and (3xTF32, BF16 inputs) no chunk longer
    // than 1024: the tensor core's accumulation bias grows with the chunk
    S = tiles < 2 * c.num_sms ? (2 * c.num_sms + tiles - 1) / tiles : 1;
    if (S > K / 512) S = K / 512;
    if ((split3 || bf16) && S < (K + 1023) / 1024) S = (K + 1023) / 1024;
    const size_t cap = c.splitk_bytes / (sizeof(float) * (size_t)M * N);
    if ((size_t)S > cap) S = (int)cap;
    if (S < 2) S = 1;
  }
  int kchunk = K;
  if (S > 1) {
    kchunk = ((K + S - 1) / S + TBK - 1) / TBK * TBK;
    S = (K + kchunk - 1) / kchunk;
  }
  TcArgs args;
  args.M = M;
  args.N = N;
  args.K = K;
  args.kchunk = kchunk;
  args.split3 = split3 && !bf16 ? 1 : 0;
  args.bf16 = bf16 ? 1 : 0;
  args.err = c.err;
  if (S == 1) {
    args.alpha = alpha;
    args.beta = beta;
    args.C = C;
    args.ldc = ldc;
    args.transC = transC ? 1 : 0;
    args.czs = 0;
  } else {
    // partials: P_z (rows x cols as finally stored), reduced in z order
    args.alpha = 1.f;
    args.beta = 0.f;
    args.C = static_cast<float*>(c.splitk);
    args.transC = transC ? 1 : 0;
    args.ldc = transC ? N : M;
    args.czs = (size_t)M * N;
  }
  dim3 grid((M + TBM - 1) / TBM, (N + bn - 1) / bn, S);
  cudaError_t e = amn ? tc_dispatch<true>(c, bn, kchunk, ma, mb, args, grid)
                      : tc_dispatch<false>(c, bn, kchunk, ma, mb, args, grid);
  if (e != cudaSuccess || S == 1) return e;
  return splitk_reduce_f32(c, transC ? N : M, transC ? M : N, S, static_cast<const float*>(c.splitk),
                           (size_t)M * N, alpha, beta, C, ldc);
}
}  // namespace

cudaError_t tc_gemm_tn(const Ctx& c, int M, int N, int K, float alpha, const float* A, int lda, const float* B,
                       int ldb, float beta, float* C, int ldc, bool transC, bool split3) {
  return tc_gemm_any(c, false, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, transC, split3);
}

cudaError_t tc_gemm_nn(const Ctx& c, int M, int N, int K, float alpha, const float* A, int lda, const float* B,
                       int ldb, float beta, float* C, int ldc, bool split3) {
  return tc_gemm_any(c, true, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, false, split3);
}

cudaError_t tc_gemm_nn_bf16(const Ctx& c, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                            float* C, int ldc) {
  return tc_gemm_any(c, true, M, N, K, 1.f, A, lda, B, ldb, 0.f, C, ldc, false, false, true);
}

}  // namespace rq
