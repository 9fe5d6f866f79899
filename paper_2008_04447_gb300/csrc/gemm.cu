// Tiled SIMT GEMM, column-major, C = alpha op(A) op(B) + beta C.
//
// On GB300 the FP64 pipe issues about two DFMA per clock per SM (~1 TFLOP/s
// per GPU), so FP64 contractions are bound by the FP64 pipe, not by HBM or
// shared memory: a register-tiled SIMT kernel with enough independent
// accumulators per thread reaches that bound.  The FP32 instance serves the
// small / odd-shaped products; the large FP32 contractions use tensor cores.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace rq {
namespace {

// blockIdx.z selects a chunk of the K dimension (split-K): chunk z covers
// [z*kchunk, min(K, (z+1)*kchunk)) and writes its own C + z*czs.
template <typename T, bool BF16>
__device__ __forceinline__ T load_in(T v) {
  if constexpr (BF16) return static_cast<T>(__bfloat162float(__float2bfloat16_rn(static_cast<float>(v))));
  return v;
}

template <typename T, int BM, int BN, int BK, int TM, int TN, bool TA, bool TB, bool BF16 = false>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, T alpha,
                                                   const T* __restrict__ A, int lda,
                                                   const T* __restrict__ B, int ldb, T beta,
                                                   T* __restrict__ C, int ldc, int kchunk, size_t czs) {
  {
    const int kz = blockIdx.z * kchunk;
    A += TA ? (size_t)kz : (size_t)kz * lda;
    B += TB ? (size_t)kz * ldb : (size_t)kz;
    C += blockIdx.z * czs;
    K = min(kchunk, K - kz);
  }
  static_assert((BM / TM) * (BN / TN) == 256, "256 threads");
  constexpr int RT = BM / TM;  // threads along M
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tm = tid % RT;
  const int tn = tid / RT;
  const int i0 = blockIdx.y * BM;
  const int j0 = blockIdx.x * BN;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int e = tid; e < BM * BK; e += 256) {
      int i, k;
      if (!TA) { i = e % BM; k = e / BM; } else { k = e % BK; i = e / BK; }
      const int gi = i0 + i, gk = k0 + k;
      T v = T(0);
      if (gi < M && gk < K) v = TA ? A[gk + (size_t)gi * lda] : A[gi + (size_t)gk * lda];
      As[k][i] = load_in<T, BF16>(v);
    }
#pragma unroll
    for (int e = tid; e < BK * BN; e += 256) {
      int k, j;
      if (!TB) { k = e % BK; j = e / BK; } else { j = e % BN; k = e / BN; }
      const int gk = k0 + k, gj = j0 + j;
      T v = T(0);
      if (gk < K && gj < N) v = TB ? B[gj + (size_t)gk * ldb] : B[gk + (size_t)gj * ldb];
      Bs[k][j] = load_in<T, BF16>(v);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][tm + i * RT];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tn + j * (BN / TN)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int gj = j0 + tn + j * (BN / TN);
    if (gj >= N) continue;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int gi = i0 + tm + i * RT;
      if (gi >= M) continue;
      T* cp = C + gi + (size_t)gj * ldc;
      T v = alpha * acc[i][j];
      if (beta != T(0)) v = fma(beta, *cp, v);
      *cp = v;
    }
  }
}

// C = alpha * sum_z P_z + beta * C, summed in z order (deterministic).
template <typename T>
__global__ void splitk_reduce(int M, int N, int S, const T* __restrict__ P, size_t pzs, T alpha, T beta,
                              T* __restrict__ C, int ldc) {
  const size_t total = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    T acc = T(0);
    for (int z = 0; z < S; ++z) acc += P[z * pzs + e];
    const int i = e % M, j = e / M;
    T* cp = C + i + (size_t)j * ldc;
    T v = alpha * acc;
    if (beta != T(0)) v = fma(beta, *cp, v);
    *cp = v;
  }
}

template <typename T>
struct Tile;
template <>
struct Tile<double> {
  static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
};
template <>
struct Tile<float> {
  static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
};

template <typename T, bool TA, bool TB>
cudaError_t launch(const Ctx& c, int M, int N, int K, T alpha, const T* A, int lda, const T* B,
                   int ldb, T beta, T* C, int ldc) {
  using TL = Tile<T>;
  const int tiles = ((N + TL::BN - 1) / TL::BN) * ((M + TL::BM - 1) / TL::BM);
  // split K when the output tiles alone cannot fill the GPU (about 4 CTAs per SM)
  int S = 1;
  if (c.splitk && tiles < 4 * c.num_sms && K >= 512) {
    S = (4 * c.num_sms + tiles - 1) / tiles;
    const int smax = K / 256;
    if (S > smax) S = smax;
    const size_t cap = c.splitk_bytes / (sizeof(T) * (size_t)M * N);
    if ((size_t)S > cap) S = (int)cap;
    if (S < 2) S = 1;
  }
  if (S == 1) {
    dim3 grid((N + TL::BN - 1) / TL::BN, (M + TL::BM - 1) / TL::BM, 1);
    gemm_kernel<T, TL::BM, TL::BN, TL::BK, TL::TM, TL::TN, TA, TB>
        <<<grid, 256, 0, c.stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, K, 0);
    ++*c.launches;
    return cudaGetLastError();
  }
  int kchunk = (K + S - 1) / S;
  kchunk = (kchunk + TL::BK - 1) / TL::BK * TL::BK;
  S = (K + kchunk - 1) / kchunk;
  T* P = static_cast<T*>(c.splitk);
  const size_t pzs = (size_t)M * N;
  dim3 grid((N + TL::BN - 1) / TL::BN, (M + TL::BM - 1) / TL::BM, S);
  gemm_kernel<T, TL::BM, TL::BN, TL::BK, TL::TM, TL::TN, TA, TB>
      <<<grid, 256, 0, c.stream>>>(M, N, K, T(1), A, lda, B, ldb, T(0), P, M, kchunk, pzs);
  size_t blocks = (pzs + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  splitk_reduce<T><<<(int)blocks, 256, 0, c.stream>>>(M, N, S, P, pzs, alpha, beta, C, ldc);
  *c.launches += 2;
  return cudaGetLastError();
}

}  // namespace

cudaError_t splitk_reduce_f32(const Ctx& c, int M, int N, int S, const float* P, size_t pzs, float alpha, float beta,
                              float* C, int ldc) {
  size_t blocks = ((size_t)M * N + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  splitk_reduce<float><<<(int)blocks, 256, 0, c.stream>>>(M, N, S, P, pzs, alpha, beta, C, ldc);
  ++*c.launches;
  return cudaGetLastError();
}

cudaError_t gemm_bf16_inputs(const Ctx& c, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                             float* C, int ldc) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  using TL = Tile<float>;
  dim3 grid((N + TL::BN - 1) / TL::BN, (M + TL::BM - 1) / TL::BM, 1);
  gemm_kernel<float, TL::BM, TL::BN, TL::BK, TL::TM, TL::TN, false, false, true>
      <<<grid, 256, 0, c.stream>>>(M, N, K, 1.f, A, lda, B, ldb, 0.f, C, ldc, K, 0);
  ++*c.launches;
  return cudaGetLastError();
}

template <typename T>
cudaError_t gemm(const Ctx& c, bool ta, bool tb, int M, int N, int K, T alpha, const T* A, int lda,
                 const T* B, int ldb, T beta, T* C, int ldc) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (!ta && !tb) return launch<T, false, false>(c, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  if (ta && !tb) return launch<T, true, false>(c, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  if (!ta && tb) return launch<T, false, true>(c, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  return launch<T, true, true>(c, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

template cudaError_t gemm<double>(const Ctx&, bool, bool, int, int, int, double, const double*, int,
                                  const double*, int, double, double*, int);
template cudaError_t gemm<float>(const Ctx&, bool, bool, int, int, int, float, const float*, int,
                                 const float*, int, float, float*, int);

}  // namespace rq
