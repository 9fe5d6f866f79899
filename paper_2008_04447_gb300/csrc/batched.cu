// Batched truncated RQRCP + TUXV (Alg. 5 and Alg. 6, j_max = 1) for many
// small, uneven problems in ONE persistent launch.
//
// Each CTA pulls problem indices from an atomic queue and runs the whole
// factorisation of that problem: sketch, per block the sample QRCP, the panel,
// the accumulated inner products W^T and the new rows of R, the sample update,
// then the LQ / QR tail with explicit U and V.  Problems never wait for each
// other, so uneven sizes balance dynamically (list the largest first).  The
// per-problem scratch lives in one slot per CTA of a workspace sized for the
// largest problem.  Storage and the contractions are FP32 (the sketch's inputs
// rounded to BF16 in RQ_MIXED); Householder scalars (norms, beta, tau), the
// downdated sample norms, T and the Omegahat_11 solve are FP64.
#include <cmath>
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace rq {
namespace {

constexpr int NT = 256;
constexpr int NW = NT / 32;
constexpr int kMaxBB = 64;   // largest block size of the batched path
constexpr int kMaxLB = 128;  // largest sample rank of the batched path
// Dynamic shared memory per CTA: the block GEMM's tiles, or (at other times)
// the live sample or the current panel when they fit, so that the serial
// pivot / reflector steps run out of shared memory instead of L2.
constexpr int kStageFloats = 27 * 1024;  // 108 KB: two CTAs per SM
constexpr int kMaxDevices = 64;

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// C (M x N) = alpha op(A) op(B) + beta C, FP32, block-level (all NT threads).
// Double-buffered: the next K slice is loaded into registers while the current
// one is multiplied out of shared memory, so global latency is hidden.
// Shared scratch: 2 * 32 * (BM + BN + 2) floats.
template <bool TA, bool TB, int BM, int BN, bool BF16>
__device__ void bgemm(int M, int N, int K, float alpha, const float* A, int lda, const float* B, int ldb, float beta,
                      float* C, int ldc, float* sm) {
  constexpr int BK = 32;
  constexpr int RT = 16, CT = 16;  // thread grid
  constexpr int TM = BM / RT, TN = BN / CT;
  constexpr int AE = BM * BK / NT, BE = BK * BN / NT;
  float* As0 = sm;
  float* As1 = sm + BK * (BM + 1);
  float* Bs0 = sm + 2 * BK * (BM + 1);
  float* Bs1 = Bs0 + BK * (BN + 1);
  const int tid = threadIdx.x;
  const int tm = tid % RT, tn = tid / RT;
  for (int i0 = 0; i0 < M; i0 += BM) {
    for (int j0 = 0; j0 < N; j0 += BN) {
      float acc[TM][TN];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
      float ra[AE], rb[BE];
      auto gload = [&](int k0) {
#pragma unroll
        for (int q = 0; q < AE; ++q) {
          const int e = tid + q * NT;
          int i, kk;
          if (!TA) { i = e % BM; kk = e / BM; } else { kk = e % BK; i = e / BK; }
          const int gi = i0 + i, gk = k0 + kk;
          ra[q] = (gi < M && gk < K) ? (TA ? A[gk + (size_t)gi * lda] : A[gi + (size_t)gk * lda]) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < BE; ++q) {
          const int e = tid + q * NT;
          int kk, j;
          if (!TB) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
          const int gk = k0 + kk, gj = j0 + j;
          rb[q] = (gk < K && gj < N) ? (TB ? B[gj + (size_t)gk * ldb] : B[gk + (size_t)gj * ldb]) : 0.f;
        }
      };
      auto sstore = [&](float* As, float* Bs) {
#pragma unroll
        for (int q = 0; q < AE; ++q) {
          const int e = tid + q * NT;
          int i, kk;
          if (!TA) { i = e % BM; kk = e / BM; } else { kk = e % BK; i = e / BK; }
          As[kk * (BM + 1) + i] = BF16 ? bf16_round(ra[q]) : ra[q];
        }
#pragma unroll
        for (int q = 0; q < BE; ++q) {
          const int e = tid + q * NT;
          int kk, j;
          if (!TB) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
          Bs[kk * (BN + 1) + j] = BF16 ? bf16_round(rb[q]) : rb[q];
        }
      };
      gload(0);
      sstore(As0, Bs0);
      __syncthreads();
      int buf = 0;
      for (int k0 = 0; k0 < K; k0 += BK) {
        const bool more = k0 + BK < K;
        if (more) gload(k0 + BK);
        const float* As = buf ? As1 : As0;
        const float* Bs = buf ? Bs1 : Bs0;
#pragma unroll 8
        for (int kk = 0; kk < BK; ++kk) {
          float av[TM], bv[TN];
#pragma unroll
          for (int i = 0; i < TM; ++i) av[i] = As[kk * (BM + 1) + tm + i * RT];
#pragma unroll
          for (int j = 0; j < TN; ++j) bv[j] = Bs[kk * (BN + 1) + tn + j * CT];
#pragma unroll
          for (int i = 0; i < TM; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (more) sstore(buf ? As0 : As1, buf ? Bs0 : Bs1);
        __syncthreads();
        buf ^= 1;
      }
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int gj = j0 + tn + j * CT;
        if (gj >= N) continue;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
          const int gi = i0 + tm + i * RT;
          if (gi >= M) continue;
          float* cp = C + gi + (size_t)gj * ldc;
          float v = alpha * acc[i][j];
          if (beta != 0.f) v = fmaf(beta, *cp, v);
          *cp = v;
        }
      }
    }
  }
  __syncthreads();
}

// The launch's tile policy, copied into shared memory by the kernel's first
// threads (every CTA reads the same two values, so the dispatch is uniform).
__shared__ int s_skinny_m, s_skinny_n;

// Dispatch on the output shape and the tile policy: 32 x 128 tiles when
// M <= skinny_m, else 128 x 32 tiles when N <= skinny_n, else 64 x 64.  Every
// tile shape accumulates each output over K in the same order with the same
// FMAs, so the policy changes the speed, never a bit of C.
template <bool TA, bool TB, bool BF16 = false>
__device__ void gemm_b(int M, int N, int K, float alpha, const float* A, int lda, const float* B, int ldb, float beta,
                       float* C, int ldc, float* sm) {
  if (M <= 0 || N <= 0) return;
  if (M <= s_skinny_m)
    bgemm<TA, TB, 32, 128, BF16>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sm);
  else if (N <= s_skinny_n)
    bgemm<TA, TB, 128, 32, BF16>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sm);
  else
    bgemm<TA, TB, 64, 64, BF16>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sm);
}

struct Shm {
  double redd[NW];
  long long redk[NW];
  float redf[NW];
  double sc[4];
  float scf[4];
  float vf[kMaxLB];
  int si[4];
  int wp[NW];
  float dots[NW][kMaxBB];
  float tw[kMaxBB];
  double tvec[kMaxBB];
};

// Householder QR of the mt x bj panel P (column-major, ld ldp) in place; v below
// the diagonal, R above; explicit Y (zeros above, unit diagonal) into Yout
// (ld ldy); tau; T (bj x bj, ld ldt, FP64) by the compound WY rule.
__device__ void panel_b(float* P, int ldp, int mt, int bj, float* Yout, int ldy, float* tau, double* T, int ldt,
                        Shm& s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < bj * bj; e += NT) T[(e % bj) + (size_t)(e / bj) * ldt] = 0.0;
  for (int j = 0; j < bj; ++j) {
    float* aj = P + (size_t)j * ldp;
    // squared norm below row j: float-float per thread and warp (FP64 for a
    // warp holding an entry outside [2^-60, 2^55]; about 2^-46 relative while
    // the column's largest entries are at least 2^-52, falling toward 2^-34
    // for a column of entries near 2^-60), combined
    // in FP64 by thread 0, which forms the reflector's scalars (FP64 is slow
    // on this part, so it stays off the all-thread path)
    {
      float xh = 0.f, xl = 0.f;
      bool oor = false;
      for (int g = j + 1 + tid; g < mt; g += NT) {
        const float a = aj[g], fa = fabsf(a);
        oor |= a != 0.f && (fa > 0x1p55f || fa < 0x1p-60f);
        const float pp = a * a;
        ff_add(xh, xl, pp, fmaf(a, a, -pp));
      }
      double xd = 0.0;
      if (__any_sync(0xffffffffu, oor)) {
        for (int g = j + 1 + tid; g < mt; g += NT) xd = fma((double)aj[g], (double)aj[g], xd);
        xd = warp_sum(xd);
      } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float bh = __shfl_xor_sync(0xffffffffu, xh, o);
          const float bl = __shfl_xor_sync(0xffffffffu, xl, o);
          ff_add(xh, xl, bh, bl);
        }
        if (lane == 0) xd = (double)xh + (double)xl;
      }
      if (lane == 0) s.redd[warp] = xd;
    }
    __syncthreads();
    if (tid == 0) {
      const double x2 = ((s.redd[0] + s.redd[1]) + (s.redd[2] + s.redd[3])) + ((s.redd[4] + s.redd[5]) + (s.redd[6] + s.redd[7]));
      double beta, inv, tu;
      householder_scalars((double)aj[j], x2, true, beta, inv, tu);
      s.sc[0] = tu;
      s.sc[2] = beta;
      s.scf[0] = (float)tu;
      s.scf[1] = (float)inv;
      tau[j] = (float)tu;
    }
    __syncthreads();
    const double tu = s.sc[0];
    {
      const float invf = s.scf[1];
      for (int g = j + 1 + tid; g < mt; g += NT) aj[g] *= invf;
    }
    __syncthreads();
    // d_c = sum_{g > j} v_g P(g, c) for every other column c of the panel,
    // sixteen columns at a time
    for (int cb = 0; cb < bj; cb += 16) {
      float d[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) d[c] = 0.f;
      for (int g = j + 1 + tid; g < mt; g += NT) {
        const float v = aj[g];
#pragma unroll
        for (int c = 0; c < 16; ++c)
          if (cb + c < bj && cb + c != j) d[c] = fmaf(v, P[g + (size_t)(cb + c) * ldp], d[c]);
      }
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        if (cb + c >= bj) break;
        const float t = warp_sum(d[c]);
        if (lane == 0) s.dots[warp][cb + c] = t;
      }
    }
    __syncthreads();
    if (tid < bj) {
      float t = 0.f;
#pragma unroll
      for (int w = 0; w < NW; ++w) t += s.dots[w][tid];
      s.dots[0][tid] = t;
    }
    __syncthreads();
    // w_c = P(j, c) + d_c for c > j; (Y^T v)_i = y_i(j) + d_i for i < j
    if (tid > j && tid < bj) s.tw[tid] = s.scf[0] * (P[j + (size_t)tid * ldp] + s.dots[0][tid]);
    if (tid < j) s.tvec[tid] = (double)P[j + (size_t)tid * ldp] + (double)s.dots[0][tid];
    __syncthreads();
    // columns c > j: P(:, c) -= tau w_c v
    for (int c = j + 1; c < bj; ++c) {
      const float tw = s.tw[c];
      float* ac = P + (size_t)c * ldp;
      for (int g = j + tid; g < mt; g += NT) ac[g] = fmaf(-tw, g == j ? 1.f : aj[g], ac[g]);
    }
    // T(0:j, j) = -tau T(0:j, 0:j) (Y^T v): four threads per entry, two
    // independent chains each (short FP64 dependency chains)
    {
      const int ti = tid >> 2, sub = tid & 3;
      double a0 = 0.0, a1 = 0.0;
      if (ti < j) {
        int q = ti + sub;
        for (; q + 4 < j; q += 8) {
          a0 = fma(T[ti + (size_t)q * ldt], s.tvec[q], a0);
          a1 = fma(T[ti + (size_t)(q + 4) * ldt], s.tvec[q + 4], a1);
        }
        if (q < j) a0 = fma(T[ti + (size_t)q * ldt], s.tvec[q], a0);
      }
      double acc = a0 + a1;
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (sub == 0 && ti < j) T[ti + (size_t)j * ldt] = -tu * acc;
    }
    if (tid == 0) {
      T[j + (size_t)j * ldt] = tu;
      aj[j] = (float)s.sc[2];
    }
    __syncthreads();
  }
  for (int e = tid; e < mt * bj; e += NT) {
    const int g = e % mt, c = e / mt;
    Yout[g + (size_t)c * ldy] = g < c ? 0.f : (g == c ? 1.f : P[g + (size_t)c * ldp]);
  }
  __syncthreads();
}

// `steps` pivots from the l x nt sample B (ld l), exchanging columns in place
// (B, jp, norms), downdating FP64 squared norms; S11 (FP64, ld lds) out.
__device__ void sample_qrcp_b(float* B, int l, int nt, int steps, int* jp, double* nu2, double* ref2, double* S11,
                              int lds, Shm& s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double tol = 3.4526698300124393e-04;  // sqrt(FLT_EPSILON): the sample is held in FP32
  for (int c = tid; c < nt; c += NT) {
    // squared column norm in float-float arithmetic (FP64 when an entry lies
    // outside [2^-60, 2^55]; about 2^-46 relative while the column's largest
    // entries are at least 2^-52, falling toward 2^-34 near 2^-60)
    const float* bc = B + (size_t)c * l;
    float h = 0.f, lo = 0.f;
    bool oor = false;
    for (int r = 0; r < l; ++r) {
      const float a = bc[r], fa = fabsf(a);
      oor |= a != 0.f && (fa > 0x1p55f || fa < 0x1p-60f);
      const float pp = a * a;
      ff_add(h, lo, pp, fmaf(a, a, -pp));
    }
    double acc = (double)h + (double)lo;
    if (oor) {
      acc = 0.0;
      for (int r = 0; r < l; ++r) acc = fma((double)bc[r], (double)bc[r], acc);
    }
    nu2[c] = acc;
    ref2[c] = acc;
  }
  __syncthreads();
  for (int i = 0; i < steps; ++i) {
    // argmax on the squared norms' bit patterns (non-negative doubles)
    long long bv = 0;
    int bp = -1, dummy = 0;
    for (int c = i + tid; c < nt; c += NT) {
      const long long kc = __double_as_longlong(nu2[c]);
      if (better_key(kc, c, bv, bp)) { bv = kc; bp = c; }
    }
    warp_argmax_key(bv, bp, dummy);
    if (lane == 0) { s.redk[warp] = bv; s.wp[warp] = bp; }
    __syncthreads();
    if (tid == 0) {
      long long gv = 0;
      int gp = -1;
      for (int w = 0; w < NW; ++w)
        if (better_key(s.redk[w], s.wp[w], gv, gp)) { gv = s.redk[w]; gp = s.wp[w]; }
      s.si[1] = gp;
    }
    __syncthreads();
    const int p = s.si[1];
    if (p != i) {
      for (int r = tid; r < l; r += NT) {
        const float t = B[r + (size_t)i * l];
        B[r + (size_t)i * l] = B[r + (size_t)p * l];
        B[r + (size_t)p * l] = t;
      }
      if (tid == 0) {
        double t = nu2[i]; nu2[i] = nu2[p]; nu2[p] = t;
        t = ref2[i]; ref2[i] = ref2[p]; ref2[p] = t;
        const int ti = jp[i]; jp[i] = jp[p]; jp[p] = ti;
      }
    }
    __syncthreads();
    float* bi = B + (size_t)i * l;
    if (warp == 0) {
      double x2 = 0.0;
      for (int r = i + 1 + lane; r < l; r += 32) x2 = fma((double)bi[r], (double)bi[r], x2);
      x2 = warp_sum(x2);
      double beta, inv, tau;
      householder_scalars((double)bi[i], x2, true, beta, inv, tau);
      for (int r = lane; r < steps; r += 32) S11[r + (size_t)i * lds] = r < i ? (double)bi[r] : (r == i ? beta : 0.0);
      const float invf = (float)inv;
      for (int r = lane; r < l; r += 32) s.vf[r] = r < i ? 0.f : (r == i ? 1.f : bi[r] * invf);
      if (lane == 0) { s.sc[0] = tau; s.sc[2] = beta; }
    }
    __syncthreads();
    const float tu = (float)s.sc[0];
    for (int c = i + 1 + tid; c < nt; c += NT) {
      float* bc = B + (size_t)c * l;
      if (tu != 0.f) {
        float w0 = bc[i], w1 = 0.f;
        int r = i + 1;
        for (; r + 1 < l; r += 2) {
          w0 = fmaf(s.vf[r], bc[r], w0);
          w1 = fmaf(s.vf[r + 1], bc[r + 1], w1);
        }
        if (r < l) w0 = fmaf(s.vf[r], bc[r], w0);
        const float tw = tu * (w0 + w1);
        bc[i] -= tw;
        for (int r2 = i + 1; r2 < l; ++r2) bc[r2] = fmaf(-tw, s.vf[r2], bc[r2]);
      }
      const double x = bc[i];
      double nn = nu2[c] - x * x;
      if (nn <= tol * ref2[c]) {
        nn = 0.0;
        for (int r = i + 1; r < l; ++r) nn = fma((double)bc[r], (double)bc[r], nn);
        ref2[c] = nn;
      }
      nu2[c] = nn;
    }
    __syncthreads();
    for (int r = tid; r < l; r += NT) bi[r] = r < i ? bi[r] : (r == i ? (float)s.sc[2] : 0.f);
    __syncthreads();
  }
}

struct Slot {
  float *B, *Wt, *Z, *Y, *P, *Xt, *G, *Wsel, *taus, *Tf, *Zt, *Z1, *Yq, *YTq, *Wq, *tauq, *Uh, *Vh;
  double *nu2, *ref2, *S11, *Oh, *T, *Tq, *jac;
  int* jp;
  size_t bytes;
};

__host__ __device__ inline Slot carve_slot(char* base, int m, int n, int k, int b, int l) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    off = (off + 255) / 256 * 256;
    char* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  const int rmax = m > n ? m : n;
  const int nb = (k + b - 1) / b;
  Slot s;
  s.B = (float*)take(sizeof(float) * (size_t)l * n);
  s.Wt = (float*)take(sizeof(float) * (size_t)k * n);
  s.Z = (float*)take(sizeof(float) * (size_t)k * n);
  s.Y = (float*)take(sizeof(float) * (size_t)m * k);
  s.P = (float*)take(sizeof(float) * (size_t)m * b);
  s.Xt = (float*)take(sizeof(float) * (size_t)b * n);
  s.G = (float*)take(sizeof(float) * (size_t)b * k);
  s.Wsel = (float*)take(sizeof(float) * (size_t)k * b);
  s.taus = (float*)take(sizeof(float) * (size_t)k);
  s.Tf = (float*)take(sizeof(float) * (size_t)b * b);
  s.Zt = (float*)take(sizeof(float) * (size_t)n * k);
  s.Z1 = (float*)take(sizeof(float) * (size_t)m * k);
  s.Yq = (float*)take(sizeof(float) * (size_t)rmax * k);
  s.YTq = (float*)take(sizeof(float) * (size_t)rmax * b);
  s.Wq = (float*)take(sizeof(float) * (size_t)b * k);
  s.tauq = (float*)take(sizeof(float) * (size_t)k);
  s.nu2 = (double*)take(sizeof(double) * (size_t)n);
  s.ref2 = (double*)take(sizeof(double) * (size_t)n);
  s.S11 = (double*)take(sizeof(double) * (size_t)b * b);
  s.Oh = (double*)take(sizeof(double) * (size_t)b * b);
  s.T = (double*)take(sizeof(double) * (size_t)b * b);
  s.Tq = (double*)take(sizeof(double) * (size_t)nb * b * b);
  s.jp = (int*)take(sizeof(int) * (size_t)n);
  // core SVD (problems that ask for sigma): FP64 W, V and norms when they do
  // not fit in shared memory; the FP32 rotations Uh, Vh
  s.jac = (double*)take(sizeof(double) * (2 * (size_t)k * k + k));
  s.Uh = (float*)take(sizeof(float) * (size_t)k * k);
  s.Vh = (float*)take(sizeof(float) * (size_t)k * k);
  s.bytes = (off + 255) / 256 * 256;
  return s;
}

__device__ void copy_T(const double* T, int ldt, int bj, float* Tf, int ldf) {
  for (int e = threadIdx.x; e < bj * bj; e += NT) Tf[(e % bj) + (size_t)(e / bj) * ldf] = (float)T[(e % bj) + (size_t)(e / bj) * ldt];
  __syncthreads();
}

__device__ void copy_mat(const float* src, int lds, int rows, int cols, float* dst, int ldd) {
  for (int e = threadIdx.x; e < rows * cols; e += NT) {
    const int i = e % rows, j = e / rows;
    dst[i + (size_t)j * ldd] = src[i + (size_t)j * lds];
  }
  __syncthreads();
}

// Panel factorisation, staged through shared memory when the panel fits.
__device__ void panel_staged(float* P, int ldp, int mt, int bj, float* Yout, int ldy, float* tau, double* T, int ldt,
                             Shm& s, float* sm) {
  if ((size_t)mt * bj <= (size_t)kStageFloats) {
    copy_mat(P, ldp, mt, bj, sm, mt);
    panel_b(sm, mt, mt, bj, Yout, ldy, tau, T, ldt, s);
    copy_mat(sm, mt, mt, bj, P, ldp);
  } else {
    panel_b(P, ldp, mt, bj, Yout, ldy, tau, T, ldt, s);
  }
}

// Sample QRCP, staged through shared memory when the live sample fits.
__device__ void sample_staged(float* B, int l, int nt, int steps, int* jp, double* nu2, double* ref2, double* S11,
                              int lds, Shm& s, float* sm) {
  if ((size_t)l * nt <= (size_t)kStageFloats) {
    copy_mat(B, l, l, nt, sm, l);
    sample_qrcp_b(sm, l, nt, steps, jp, nu2, ref2, S11, lds, s);
    copy_mat(sm, l, l, nt, B, l);
  } else {
    sample_qrcp_b(B, l, nt, steps, jp, nu2, ref2, S11, lds, s);
  }
}

// QR of the rows x k matrix M in place (block size b) with explicit Q(:, 1:k)
// into Q (ld ldq) and, if Rout, R (k x k, upper) into Rout.
__device__ void qr_explicit_b(float* M, int ldm, int rows, int k, int b, Slot& w, float* Q, int ldq, float* Rout,
                              int ldr, Shm& s, float* sm) {
  const int nb = (k + b - 1) / b;
  for (int e = threadIdx.x; e < rows * k; e += NT) w.Yq[e] = 0.f;
  __syncthreads();
  for (int J = 0; J < nb; ++J) {
    const int j0 = J * b, bj = min(b, k - j0), mt = rows - j0, n2 = k - j0 - bj;
    float* Yj = w.Yq + j0 + (size_t)j0 * rows;
    double* Tj = w.Tq + (size_t)J * b * b;
    panel_staged(M + j0 + (size_t)j0 * ldm, ldm, mt, bj, Yj, rows, w.tauq + j0, Tj, b, s, sm);
    if (n2 > 0) {
      copy_T(Tj, b, bj, w.Tf, b);
      float* M2 = M + j0 + (size_t)(j0 + bj) * ldm;
      gemm_b<false, false>(mt, bj, bj, 1.f, Yj, rows, w.Tf, b, 0.f, w.YTq, mt, sm);
      gemm_b<true, false>(bj, n2, mt, 1.f, w.YTq, mt, M2, ldm, 0.f, w.Wq, b, sm);
      gemm_b<false, false>(mt, n2, bj, -1.f, Yj, rows, w.Wq, b, 1.f, M2, ldm, sm);
    }
  }
  if (Rout) {
    for (int e = threadIdx.x; e < k * k; e += NT) {
      const int i = e % k, j = e / k;
      Rout[i + (size_t)j * ldr] = i <= j ? M[i + (size_t)j * ldm] : 0.f;
    }
  }
  for (int e = threadIdx.x; e < rows * k; e += NT) {
    const int i = e % rows, j = e / rows;
    Q[i + (size_t)j * ldq] = i == j ? 1.f : 0.f;
  }
  __syncthreads();
  for (int J = nb - 1; J >= 0; --J) {
    const int j0 = J * b, bj = min(b, k - j0), mt = rows - j0, nc = k - j0;
    const float* Yj = w.Yq + j0 + (size_t)j0 * rows;
    copy_T(w.Tq + (size_t)J * b * b, b, bj, w.Tf, b);
    float* Qs = Q + j0 + (size_t)j0 * ldq;
    gemm_b<true, false>(bj, nc, mt, 1.f, Yj, rows, Qs, ldq, 0.f, w.Wq, b, sm);
    gemm_b<false, false>(bj, nc, bj, 1.f, w.Tf, b, w.Wq, b, 0.f, w.YTq, b, sm);
    gemm_b<false, false>(mt, nc, bj, -1.f, Yj, rows, w.YTq, b, 1.f, Qs, ldq, sm);
  }
}

struct BatchArgs {
  const rq_problem* problems;
  int count;
  char* ws;
  size_t slot_bytes;
  int* counter;
  int mixed;
  int skinny_m, skinny_n;  // tile policy of the block GEMMs (gemm_b)
};

__device__ void solve_one(const rq_problem& pr, Slot& w, Shm& s, float* sm, bool mixed) {
  const int m = pr.m, n = pr.n, k = pr.k, b = pr.b, l = pr.b + pr.p;
  const float* A = static_cast<const float*>(pr.A);
  const float* Om = static_cast<const float*>(pr.Omega);
  const int lda = pr.lda;
  const int tid = threadIdx.x;
  for (int c = tid; c < n; c += NT) w.jp[c] = c;
  for (int e = tid; e < m * k; e += NT) w.Y[e] = 0.f;
  __syncthreads();
  // sketch B = Omega A (BF16 inputs in the mixed precision mode)
  if (mixed)
    gemm_b<false, false, true>(l, n, m, 1.f, Om, pr.ldo, A, lda, 0.f, w.B, l, sm);
  else
    gemm_b<false, false, false>(l, n, m, 1.f, Om, pr.ldo, A, lda, 0.f, w.B, l, sm);
  for (int j0 = 0; j0 < k; j0 += b) {
    const int bj = min(b, k - j0), nt = n - j0, mt = m - j0, n2 = nt - bj;
    float* BJ = w.B + (size_t)j0 * l;  // the live sample: columns j0.. (exchanged in place)
    sample_staged(BJ, l, nt, bj, w.jp + j0, w.nu2 + j0, w.ref2 + j0, w.S11, b, s, sm);
    // selected columns of A - Y W^T
    for (int e = tid; e < m * bj; e += NT) {
      const int g = e % m, c = e / m;
      w.P[g + (size_t)c * m] = A[g + (size_t)w.jp[j0 + c] * lda];
    }
    if (j0 > 0)
      for (int e = tid; e < j0 * bj; e += NT) {
        const int r = e % j0, c = e / j0;
        w.Wsel[r + (size_t)c * k] = w.Wt[r + (size_t)w.jp[j0 + c] * k];
      }
    __syncthreads();
    if (j0 > 0) gemm_b<false, false>(m, bj, j0, -1.f, w.Y, m, w.Wsel, k, 1.f, w.P, m, sm);
    float* Y2 = w.Y + j0 + (size_t)j0 * m;
    panel_staged(w.P + j0, m, mt, bj, Y2, m, w.taus + j0, w.T, b, s, sm);
    copy_T(w.T, b, bj, w.Tf, b);
    // W_2^T = T_2^T (Y_2^T A - (Y_2^T Y_1) W_1^T)
    gemm_b<true, false>(bj, n, mt, 1.f, Y2, m, A + j0, lda, 0.f, w.Xt, b, sm);
    if (j0 > 0) {
      gemm_b<true, false>(bj, j0, mt, 1.f, Y2, m, w.Y + j0, m, 0.f, w.G, b, sm);
      gemm_b<false, false>(bj, n, j0, -1.f, w.G, b, w.Wt, k, 1.f, w.Xt, b, sm);
    }
    gemm_b<true, false>(bj, n, bj, 1.f, w.Tf, b, w.Xt, b, 0.f, w.Wt + j0, k, sm);
    // new rows of R (original column order)
    for (int e = tid; e < bj * n; e += NT) {
      const int r = e % bj, c = e / bj;
      w.Z[j0 + r + (size_t)c * k] = A[j0 + r + (size_t)c * lda];
    }
    __syncthreads();
    gemm_b<false, false>(bj, n, j0 + bj, -1.f, w.Y + j0, m, w.Wt, k, 1.f, w.Z + j0, k, sm);
    for (int e = tid; e < bj * (j0 + bj); e += NT) {
      const int r = e % bj, pos = e / bj;
      float v = 0.f;
      if (pos >= j0) {
        const int c = pos - j0;
        v = r <= c ? w.P[j0 + r + (size_t)c * m] : 0.f;
      }
      w.Z[j0 + r + (size_t)w.jp[pos] * k] = v;
    }
    __syncthreads();
    if (j0 + bj < k) {
      // Eq. (update1): Omegahat11 = S11 R11^{-1} by forward substitution along
      // each row in FP64 (four threads per row, the diagonal's reciprocals
      // first: FP64 division and long FP64 chains are slow on this part), then
      // B1 = S12 - Omegahat11 R12 accumulated in FP32 like the sample itself
      if (tid < bj) {
        const double d = w.P[j0 + tid + (size_t)tid * m];
        s.tvec[tid] = d != 0.0 ? 1.0 / d : 0.0;
      }
      __syncthreads();
      {
        const int r = tid >> 2, sub = tid & 3;
        for (int j = 0; j < bj; ++j) {
          double acc = 0.0;
          if (r < bj)
            for (int i = r + sub; i < j; i += 4)
              acc = fma(w.Oh[r + (size_t)i * b], (double)w.P[j0 + i + (size_t)j * m], acc);
          acc += __shfl_xor_sync(0xffffffffu, acc, 1);
          acc += __shfl_xor_sync(0xffffffffu, acc, 2);
          if (r < bj && sub == 0) w.Oh[r + (size_t)j * b] = j < r ? 0.0 : (w.S11[r + (size_t)j * b] - acc) * s.tvec[j];
          __syncwarp();
        }
      }
      __syncthreads();
      float* sO = sm;  // Omegahat11 rounded to FP32 (the staging area is free here)
      for (int e = tid; e < bj * bj; e += NT) sO[e] = (float)w.Oh[(e % bj) + (size_t)(e / bj) * b];
      __syncthreads();
      float* B1 = BJ + (size_t)bj * l;
      for (int e = tid; e < bj * n2; e += NT) {
        const int r = e % bj, t = e / bj;
        const float* zc = w.Z + j0 + (size_t)w.jp[j0 + bj + t] * k;
        float acc = 0.f;
        for (int i = r; i < bj; ++i) acc = fmaf(sO[r + i * bj], zc[i], acc);
        B1[r + (size_t)t * l] -= acc;
      }
      __syncthreads();
    }
  }
  // TUXV tail: V from the LQ of Z0 = R P^T, Z1 = A V, QR of Z1 -> U, X
  float* U = static_cast<float*>(pr.U);
  float* X = static_cast<float*>(pr.X);
  float* V = static_cast<float*>(pr.V);
  for (int e = tid; e < k * n; e += NT) {
    const int r = e % k, c = e / k;
    w.Zt[c + (size_t)r * n] = w.Z[r + (size_t)c * k];
  }
  __syncthreads();
  qr_explicit_b(w.Zt, n, n, k, b, w, V, pr.ldv, nullptr, 0, s, sm);
  gemm_b<false, false>(m, k, n, 1.f, A, lda, V, pr.ldv, 0.f, w.Z1, m, sm);
  qr_explicit_b(w.Z1, m, m, k, b, w, U, pr.ldu, X, pr.ldx, s, sm);
  if (tid == 0 && pr.info) *pr.info = 0;
  __syncthreads();
}

constexpr int kMaxSweepsB = 40;

// Core SVD of the k x k upper triangular X (Sec. 4.2; FP64 one-sided Jacobi,
// Hestenes' method): X Vh = Uh diag(sigma), then U <- U Uh, V <- V Vh and
// X <- diag(sigma), sigma descending (ties to the lower column), and each
// column of V with its largest-magnitude entry (lowest row on ties) positive,
// U's column following.  A round rotates kk/2 disjoint column pairs (circle
// method), one warp per pair; a sweep is kk - 1 rounds; sweeps stop when one
// rotates nothing.  W and V live in the staging area when they fit.
__device__ void core_svd_b(const rq_problem& pr, Slot& w, float* sm) {
  const int m = pr.m, n = pr.n, k = pr.k;
  float* U = static_cast<float*>(pr.U);
  float* X = static_cast<float*>(pr.X);
  float* V = static_cast<float*>(pr.V);
  float* sig = static_cast<float*>(pr.sigma);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t k2 = (size_t)k * k;
  const size_t cap = (size_t)kStageFloats * sizeof(float) / sizeof(double);
  double* dsm = reinterpret_cast<double*>(sm);
  double* W = k2 <= cap ? dsm : w.jac;
  double* Vr = 2 * k2 <= cap ? dsm + k2 : w.jac + k2;
  double* nrm = w.jac + 2 * k2;
  for (size_t e = tid; e < k2; e += NT) {
    const int i = e % k, j = e / k;
    W[e] = (double)X[i + (size_t)j * pr.ldx];
    Vr[e] = i == j ? 1.0 : 0.0;
  }
  __shared__ int s_rot;
  const int kk = (k + 1) / 2 * 2, npairs = kk / 2;
  const double tol = (k > 1 ? (double)k : 2.0) * 2.220446049250313e-16;
  __syncthreads();
  for (int sweep = 0; sweep < kMaxSweepsB; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < kk - 1; ++r) {
      for (int pi = warp; pi < npairs; pi += NW) {
        // circle method: position 0 fixed, positions 1..kk-1 rotate by r
        int p = pi == 0 ? 0 : 1 + (pi - 1 + r) % (kk - 1);
        const int pos = kk - 1 - pi;
        int q = 1 + (pos - 1 + r) % (kk - 1);
        if (p >= k || q >= k) continue;
        if (p > q) { const int t = p; p = q; q = t; }
        double* wp = W + (size_t)p * k;
        double* wq = W + (size_t)q * k;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < k; i += 32) {
          const double x = wp[i], y = wq[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        // butterfly sums: every lane holds the same bits, so all take the same branch
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga != 0.0 && fabs(ga) > tol * sqrt(al * be)) {
          const double zeta = (be - al) / (2.0 * ga);
          const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
          double* vp = Vr + (size_t)p * k;
          double* vq = Vr + (size_t)q * k;
          for (int i = lane; i < k; i += 32) {
            const double x = wp[i], y = wq[i];
            wp[i] = c * x - sn * y;
            wq[i] = sn * x + c * y;
            const double u = vp[i], v = vq[i];
            vp[i] = c * u - sn * v;
            vq[i] = sn * u + c * v;
          }
          if (lane == 0) atomicAdd(&s_rot, 1);
        }
      }
      __syncthreads();
    }
    const int rotated = s_rot;
    __syncthreads();
    if (rotated == 0) break;
  }
  for (int j = warp; j < k; j += NW) {
    double a2 = 0.0;
    for (int i = lane; i < k; i += 32) a2 = fma(W[i + (size_t)j * k], W[i + (size_t)j * k], a2);
    a2 = warp_sum(a2);
    if (lane == 0) nrm[j] = sqrt(a2);
  }
  __syncthreads();
  for (int j = warp; j < k; j += NW) {
    const double sj = nrm[j];
    int cnt = 0;
    for (int i = lane; i < k; i += 32) {
      const double si = nrm[i];
      cnt += (si > sj || (si == sj && i < j)) ? 1 : 0;
    }
    const int rk = warp_sum(cnt);
    const double inv = sj > 0.0 ? 1.0 / sj : 0.0;
    for (int i = lane; i < k; i += 32) {
      w.Uh[i + (size_t)rk * k] = (float)(W[i + (size_t)j * k] * inv);
      w.Vh[i + (size_t)rk * k] = (float)Vr[i + (size_t)j * k];
    }
    if (lane == 0) sig[rk] = (float)sj;
  }
  __syncthreads();
  // U <- U Uh and V <- V Vh through the (now free) Z1 (m x k) and Zt (n x k)
  gemm_b<false, false>(m, k, k, 1.f, U, pr.ldu, w.Uh, k, 0.f, w.Z1, m, sm);
  gemm_b<false, false>(n, k, k, 1.f, V, pr.ldv, w.Vh, k, 0.f, w.Zt, n, sm);
  __syncthreads();
  for (size_t e = tid; e < (size_t)m * k; e += NT) U[(e % m) + (e / m) * pr.ldu] = w.Z1[e];
  for (size_t e = tid; e < (size_t)n * k; e += NT) V[(e % n) + (e / n) * pr.ldv] = w.Zt[e];
  __syncthreads();
  for (int j = warp; j < k; j += NW) {
    float* v = V + (size_t)j * pr.ldv;
    float best = -1.f;
    int bi = 0x7fffffff;
    for (int i = lane; i < n; i += 32) {
      const float x = fabsf(v[i]);
      if (x > best || (x == best && i < bi)) { best = x; bi = i; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const float b2 = __shfl_xor_sync(0xffffffffu, best, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
      if (b2 > best || (b2 == best && i2 < bi)) { best = b2; bi = i2; }
    }
    if (bi < n && v[bi] < 0.f) {
      for (int i = lane; i < n; i += 32) v[i] = -v[i];
      float* u = U + (size_t)j * pr.ldu;
      for (int i = lane; i < m; i += 32) u[i] = -u[i];
    }
  }
  for (size_t e = tid; e < k2; e += NT) {
    const int i = e % k, j = e / k;
    X[i + (size_t)j * pr.ldx] = i == j ? sig[i] : 0.f;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(NT, 2) tuxv_batched_kernel(BatchArgs a) {
  extern __shared__ float sm[];
  __shared__ Shm s;
  __shared__ int s_idx;
  char* base = a.ws + (size_t)blockIdx.x * a.slot_bytes;
  if (threadIdx.x == 0) {
    s_skinny_m = a.skinny_m;
    s_skinny_n = a.skinny_n;
  }
  while (true) {
    if (threadIdx.x == 0) s_idx = atomicAdd(a.counter, 1);
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= a.count) break;
    const rq_problem pr = a.problems[idx];
    Slot w = carve_slot(base, pr.m, pr.n, pr.k, pr.b, pr.b + pr.p);
    solve_one(pr, w, s, sm, a.mixed != 0);
    if (pr.sigma != nullptr) core_svd_b(pr, w, sm);
  }
}

}  // namespace

size_t batched_slot_bytes(int max_m, int max_n, int max_k, int max_b, int max_p) {
  return carve_slot(nullptr, max_m, max_n, max_k, max_b, max_b + max_p).bytes;
}

int batched_limits_ok(int max_b, int max_p) { return max_b >= 1 && max_b <= kMaxBB && max_b + max_p <= kMaxLB; }

constexpr size_t kBatchSmem = (size_t)kStageFloats * sizeof(float);
static_assert(kStageFloats >= 2 * 32 * (128 + 32 + 2), "the GEMM tiles share the staging area");

// Per device, once: raise the kernel's dynamic shared memory limit and record
// how many CTAs fit on an SM.  Later calls make no CUDA runtime call here, so a
// call captured into a CUDA graph issues only the memset and the launch.
int batched_ctas_per_sm() {
  static std::mutex mu;
  static int per_sm_of[kMaxDevices] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return -1;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (per_sm_of[dev] == 0) {
    const size_t smem = kBatchSmem;
    int per_sm = 0;
    if (cudaFuncSetAttribute(tuxv_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tuxv_batched_kernel, NT, smem) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      return -1;
    }
    per_sm_of[dev] = per_sm;
  }
  return per_sm_of[dev];
}

cudaError_t tuxv_batched(const Ctx& c, int count, const rq_problem* problems, char* ws, size_t slot_bytes, int slots,
                         int* counter, bool mixed, int skinny_m, int skinny_n) {
  const size_t smem = kBatchSmem;
  if (batched_ctas_per_sm() < 1) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), c.stream);
  if (e != cudaSuccess) return e;
  BatchArgs a{problems, count, ws, slot_bytes, counter, mixed ? 1 : 0, skinny_m, skinny_n};
  tuxv_batched_kernel<<<slots, NT, smem, c.stream>>>(a);
  ++*c.launches;
  return cudaGetLastError();
}

int batched_slots(int num_sms) {
  const int per_sm = batched_ctas_per_sm();
  return (per_sm < 1 ? 1 : per_sm) * num_sms;
}

}  // namespace rq
