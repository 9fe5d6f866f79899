// Tiled SIMT GEMM, column-major, C = alpha op(A) op(B) + beta C.
//
// On GB300 the FP64 pipe issues about two DFMA per clock per SM (~1 TFLOP/s
// per GPU), so FP64 contractions are bound by the FP64 pipe, not by HBM or
// shared memory: a register-tiled SIMT kernel with enough independent
// accumulators per thread reaches that bound.  The FP32 instance serves the
// small / odd-shaped products; the large FP32 contractions use tensor cores.
#include "common.cuh"
#include "kernels.h"

namespace rq {
namespace {

template <typename T, int BM, int BN, int BK, int TM, int TN, bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, T alpha,
                                                   const T* __restrict__ A, int lda,
                                                   const T* __restrict__ B, int ldb, T beta,
                                                   T* __restrict__ C, int ldc) {
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
      As[k][i] = v;
    }
#pragma unroll
    for (int e = tid; e < BK * BN; e += 256) {
      int k, j;
      if (!TB) { k = e % BK; j = e / BK; } else { j = e % BN; k = e / BN; }
      const int gk = k0 + k, gj = j0 + j;
      T v = T(0);
      if (gk < K && gj < N) v = TB ? B[gj + (size_t)gk * ldb] : B[gk + (size_t)gj * ldb];
      Bs[k][j] = v;
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
  dim3 grid((N + TL::BN - 1) / TL::BN, (M + TL::BM - 1) / TL::BM);
  gemm_kernel<T, TL::BM, TL::BN, TL::BK, TL::TM, TL::TN, TA, TB>
      <<<grid, 256, 0, c.stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  ++*c.launches;
  return cudaGetLastError();
}

}  // namespace

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
