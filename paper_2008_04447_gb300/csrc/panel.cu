// Householder QR of one m_t x b panel (the b reflectors of Alg. 4), with
// the compact-WY factor T of Sec. 4.1 built alongside.
//
// One cooperative launch per panel.  CTA c keeps rows [c*rpc, (c+1)*rpc) of
// the panel in shared memory (storage precision, column-major inside the slab)
// for all b reflectors.  The reflector scalars (norms, beta, tau) and T are
// FP64; the dot products and updates run in the storage precision.  Reflector j needs only global sums over the rows below j:
//   x2 = sum a_j^2, e'_c = sum a_j a_c (c > j), e_i = sum y_i a_j (i < j),
// plus row j itself.  Each CTA writes its partial sums, one grid barrier
// follows, and every CTA adds the partials in the same order, so all CTAs
// hold bit-identical reflector data.  From them:
//   beta = -sign(alpha) sqrt(alpha^2 + x2), y1 = alpha - beta, v = a / y1,
//   tau = 2 / (1 + x2 / y1^2), w_c = v^T a_c = a_c(j) + e'_c / y1,
// and the update a_c -= tau w_c v is applied lazily, fused with the next
// reflector's partial sums.  T grows by the compound WY rule:
//   T(0:j, j) = -tau_j T(0:j, 0:j) (Y^T v_j),  (Y^T v_j)_i = y_i(j) + e_i / y1.
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace rq {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxB = 256;
static_assert(RQ_MAX_B <= kMaxB, "the panel kernels hold the largest block");
constexpr int kMaxRec = 20;  // partial records summed per thread: G <= kMaxRec * kWarps = 160

template <typename TS>
struct PanelArgs {
  TS* P;
  int ldp, mt, bj;
  TS* tau;
  TS* Y;
  int ldy;
  double* T;
  int ldt;
  double* part;    // 2 * G * (bj + 1)
  double* rowbuf;  // 2 * (2 * bj)
  unsigned int* bar;
  int* err;
  int rpc;
};

template <typename TS>
__global__ void __launch_bounds__(kThreads) panel_kernel(PanelArgs<TS> a) {
  extern __shared__ double sm[];
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int bj = a.bj, rpc = a.rpc;
  const int r0 = cta * rpc;
  const int nr = max(0, min(rpc, a.mt - r0));
  double* tw = sm;                    // bj
  double* sums = tw + bj;             // bj
  double* redw = sums + bj;           // kWarps * bj
  double* Tm = redw + kWarps * bj;    // bj * bj (CTA 0)
  double* tv = Tm + (size_t)bj * bj;  // bj
  double* tv2 = tv + bj;              // 2 * bj: row j of the panel, this step
  TS* p = reinterpret_cast<TS*>(tv2 + 2 * bj);  // p[c * rpc + r]
  __shared__ double s_tau, s_y1, s_beta;
  const int recn = bj + 1;

  for (int e = tid; e < nr * bj; e += kThreads) {
    const int r = e % nr, c = e / nr;
    p[(size_t)c * rpc + r] = a.P[(size_t)(r0 + r) + (size_t)c * a.ldp];
  }
  for (int e = tid; e < bj * bj; e += kThreads) Tm[e] = 0.0;
  __syncthreads();

  unsigned int epoch = 0;
  for (int j = 0; j < bj; ++j) {
    const int par = j & 1;
    double* part = a.part + (size_t)par * G * recn;
    double* rowb = a.rowbuf + (size_t)par * 2 * bj;
    // column j receives reflector j-1
    if (j > 0) {
      const TS t = static_cast<TS>(tw[j]);
      for (int r = tid; r < nr; r += kThreads) {
        const int g = r0 + r;
        if (g >= j - 1) {
          const TS v = (g == j - 1) ? TS(1) : p[(size_t)(j - 1) * rpc + r];
          p[(size_t)j * rpc + r] = fma(-t, v, p[(size_t)j * rpc + r]);
        }
      }
      __syncthreads();
    }
    // partial sums over rows g > j; columns c > j first receive reflector j-1
    for (int task = warp; task < bj; task += kWarps) {
      double acc = 0.0;
      const TS* aj = p + (size_t)j * rpc;
      if (task == 0) {
        // the squared norm feeds beta and tau: accumulated in FP64
        for (int r = lane; r < nr; r += 32)
          if (r0 + r > j) {
            const double x = static_cast<double>(aj[r]);
            acc = fma(x, x, acc);
          }
      } else if (task < bj - j) {
        const int c = j + task;
        TS* ac = p + (size_t)c * rpc;
        const TS t = (j > 0) ? static_cast<TS>(tw[c]) : TS(0);
        TS dot = TS(0);
        for (int r = lane; r < nr; r += 32) {
          const int g = r0 + r;
          if (j > 0 && g >= j - 1) {
            const TS v = (g == j - 1) ? TS(1) : p[(size_t)(j - 1) * rpc + r];
            ac[r] = fma(-t, v, ac[r]);
          }
          if (g > j) dot = fma(aj[r], ac[r], dot);
        }
        acc = static_cast<double>(dot);
      } else {
        const int i = task - (bj - j);
        const TS* yi = p + (size_t)i * rpc;
        TS dot = TS(0);
        for (int r = lane; r < nr; r += 32)
          if (r0 + r > j) dot = fma(yi[r], aj[r], dot);
        acc = static_cast<double>(dot);
      }
      acc = warp_sum(acc);
      if (lane == 0) part[(size_t)cta * recn + task] = acc;
    }
    __syncthreads();
    if (r0 <= j && j < r0 + nr) {
      const int jl = j - r0;
      for (int c = tid; c < bj; c += kThreads) {
        rowb[c] = (c >= j) ? static_cast<double>(p[(size_t)c * rpc + jl]) : 0.0;
        rowb[bj + c] = (c < j) ? static_cast<double>(p[(size_t)c * rpc + jl]) : 0.0;
      }
    }
    if (!grid_barrier(a.bar, G, a.err, epoch)) return;
    // reduce the partials in a fixed order (CTA 0 also needs the e_i)
    const int need = (cta == 0) ? bj : (bj - j);
    for (int t = lane; t < need; t += 32) {
      // independent loads first (all in flight together), then a fixed-order sum
      double v[kMaxRec];
#pragma unroll
      for (int u = 0; u < kMaxRec; ++u) {
        const int q = warp + u * kWarps;
        v[u] = q < G ? __ldcg(part + (size_t)q * recn + t) : 0.0;
      }
      double acc = 0.0;
#pragma unroll
      for (int u = 0; u < kMaxRec; ++u) acc += v[u];
      redw[warp * bj + t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < need; t += kThreads) {
      double acc = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) acc += redw[w * bj + t];
      sums[t] = acc;
    }
    __syncthreads();
    for (int t = tid; t < 2 * bj; t += kThreads) tv2[t] = __ldcg(rowb + t);
    __syncthreads();
    if (tid == 0) {
      const double alpha = tv2[j];
      const double x2 = sums[0];
      const double nrm2 = fma(alpha, alpha, x2);
      double tau = 0.0, beta = 0.0, y1 = 1.0;
      if (nrm2 > 0.0) {
        const double nrm = sqrt(nrm2);
        beta = alpha >= 0.0 ? -nrm : nrm;
        y1 = alpha - beta;
        tau = 2.0 / (1.0 + x2 / (y1 * y1));
      }
      s_tau = tau;
      s_y1 = y1;
      s_beta = beta;
      if (cta == 0) a.tau[j] = static_cast<TS>(tau);
    }
    __syncthreads();
    const double tau = s_tau, y1 = s_y1, beta = s_beta;
    for (int c = j + 1 + tid; c < bj; c += kThreads) tw[c] = tau * (tv2[c] + sums[c - j] / y1);
    for (int r = tid; r < nr; r += kThreads) {
      const int g = r0 + r;
      if (g > j)
        p[(size_t)j * rpc + r] = tau != 0.0 ? static_cast<TS>(static_cast<double>(p[(size_t)j * rpc + r]) / y1) : TS(0);
      else if (g == j)
        p[(size_t)j * rpc + r] = static_cast<TS>(beta);
    }
    if (cta == 0) {
      // T(0:j, j) = -tau T(0:j, 0:j) (Y^T v_j)
      for (int i = tid; i < j; i += kThreads) tv[i] = tv2[bj + i] + sums[bj - j + i] / y1;
      __syncthreads();
      for (int i = tid; i < j; i += kThreads) {
        double acc = 0.0;
        for (int q = i; q < j; ++q) acc = fma(Tm[(size_t)q * bj + i], tv[q], acc);
        Tm[(size_t)j * bj + i] = -tau * acc;
      }
      if (tid == 0) Tm[(size_t)j * bj + j] = tau;
    }
    __syncthreads();
  }

  grid_exit(a.bar, G);
  for (int e = tid; e < nr * bj; e += kThreads) {
    const int r = e % nr, c = e / nr;
    const int g = r0 + r;
    const TS x = p[(size_t)c * rpc + r];
    a.P[(size_t)g + (size_t)c * a.ldp] = x;
    a.Y[(size_t)g + (size_t)c * a.ldy] = g < c ? TS(0) : (g == c ? TS(1) : x);
  }
  if (cta == 0)
    for (int e = tid; e < bj * bj; e += kThreads) a.T[(size_t)(e / bj) * a.ldt + (e % bj)] = Tm[e];
}

// ---------------------------------------------------------------------------
// Latency-oriented variant for b <= 64 (the common case): the per-column step
// is a chain of waits (a grid barrier, reductions, one FP64 square root and
// division), so it is shaped to keep that chain short.
//   * Each thread owns one row of the panel (two threads split a row's 64
//     columns in FP64) and keeps it in registers; reflector j-1 is applied to
//     the row's columns >= j with no barrier inside the CTA.
//   * Finished columns stay unscaled in the registers: y_c(g) = a_c(g) / y1_c,
//     and every use (the e_i sums, T, the outputs) applies 1 / y1_c.
//   * The row's products a_c(g) a_j(g) for all c are reduced over the warp at
//     once by a reduce-scatter butterfly (62 shuffles for 64 sums), then over
//     the warps through shared memory; the squared norm is summed in FP64.
//   * CTA 0 forms T's previous column between its arrival at the grid barrier
//     and its wait, off the critical path.
//   * tau = (beta - alpha) / beta and 1 / y1 come from one FP64 division,
//     1 / (beta y1); tau = 2 exactly when the column is zero below row j.
//   * FP64 instructions are slow on this part (a dependent FP64 step costs
//     about 64 cycles, a division or square root about 650, and the pipe
//     executes about two lanes per clock per SM), so FP64 work is kept off
//     the all-thread code: for FP32 rows each warp carries the squared norm
//     in float-float arithmetic (FP64 when an entry is out of its safe
//     range) and the sums across warps and CTAs are FP64; tau, 1 / y1 and
//     beta come from the FP64 norm with the square root and reciprocal
//     refined from FP32 estimates (a few dependent FP64 steps rather than
//     an FP64 square root and division); the lazy update's coefficients
//     and the reflector entries are FP32 as stored.
// The global squared norm, beta, tau, 1 / y1 and T are FP64; the lazy update,
// the products and their reductions run in the storage precision, like the
// general kernel above.
constexpr int kFB = 64;
constexpr int kMaxG4 = 40;  // partial records per thread in the sums: G <= 160

template <typename TS>
struct FastArgs {
  TS* P;
  int ldp, mt, bj;
  TS* tau;
  TS* Y;
  int ldy;
  double* T;
  int ldt;
  TS* part;        // 2 * G * bj partial sums
  double* x2part;  // 2 * G partial squared norms
  TS* rowb;        // 2 * bj: row j of the panel
  unsigned int* bar;
  int* err;
  int rpc;   // rows of CTAs 1.. (CTA c > 0 keeps rows [rpc0 + (c - 1) rpc, rpc0 + c rpc))
  int rpc0;  // rows of CTA 0, which also forms T
};

// v[0..N) per lane, LPG lanes per group (N = 2 LPG): afterwards lane l of the
// group holds in v[0], v[1] the group sums of values 2l and 2l + 1.
template <typename T, int N, int LPG>
__device__ __forceinline__ void reduce_scatter(T (&v)[N]) {
  static_assert(N == 2 * LPG, "two sums per lane");
#pragma unroll
  for (int lev = 0; (LPG >> (lev + 1)) >= 1; ++lev) {
    const int off = LPG >> (lev + 1);
    const int n = N >> lev;
    const bool up = (threadIdx.x & off) != 0;
#pragma unroll
    for (int i = 0; i < n / 2; ++i) {
      const T send = up ? v[i] : v[i + n / 2];
      const T keep = up ? v[i + n / 2] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
}

// T(0:jc, jc) = -tau T(0:jc, 0:jc) tv, T(jc, jc) = tau (compound WY, Sec. 4.1);
// four threads per entry, fixed order.
__device__ __forceinline__ void t_column(int jc, double tau, double* sT, const double* tv) {
  const int i = threadIdx.x >> 2, sub = threadIdx.x & 3;
  // only the needed products, in two independent chains (a dependent FP64
  // step costs about 64 cycles here, and the FP64 pipe is narrow)
  double a0 = 0.0, a1 = 0.0;
  if (i < jc) {
    int q = i + sub;
    for (; q + 4 < jc; q += 8) {
      a0 = fma(sT[(size_t)q * kFB + i], tv[q], a0);
      a1 = fma(sT[(size_t)(q + 4) * kFB + i], tv[q + 4], a1);
    }
    if (q < jc) a0 = fma(sT[(size_t)q * kFB + i], tv[q], a0);
  }
  double acc = a0 + a1;
  acc += __shfl_xor_sync(0xffffffffu, acc, 1);
  acc += __shfl_xor_sync(0xffffffffu, acc, 2);
  if (sub == 0 && i < jc) sT[(size_t)jc * kFB + i] = -tau * acc;
  if (threadIdx.x == 0) sT[(size_t)jc * kFB + jc] = tau;
}

template <typename TS, int TPR>
__global__ void __launch_bounds__(kThreads, 1) panel_fast_kernel(FastArgs<TS> a) {
  constexpr int CPT = kFB / TPR;  // columns per thread
  constexpr int LPG = 32 / TPR;   // lanes (rows) per group of a warp
  constexpr bool kF32 = sizeof(TS) == sizeof(float);
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int bj = a.bj;
  const int half = lane / LPG;
  const int lp = lane % LPG;
  const int nrows = cta == 0 ? a.rpc0 : a.rpc;
  const int rbase = cta == 0 ? 0 : a.rpc0 + (cta - 1) * a.rpc;
  const int r = warp * LPG + lp;
  const int g = rbase + r;
  const bool live = r < nrows && g < a.mt;
  // a warp with no row of the panel skips the per-row FP64 work (warp-uniform)
  const bool wlive = warp * LPG < nrows && rbase + warp * LPG < a.mt;
  const int cbase = half * CPT;
  __shared__ TS s_tw[kFB];     // tau_j w_c, the lazy update's coefficients
  __shared__ TS s_sumT[kFB];   // global dot sums of this column
  __shared__ TS s_rowT[kFB];   // row j
  __shared__ TS s_invT[kFB];   // 1 / y1 per finished column, storage precision
  __shared__ double s_inv[kFB];
  __shared__ double s_beta[kFB];
  __shared__ double s_tv[kFB];
  __shared__ double s_T[kFB * kFB];
  __shared__ TS s_red[kWarps][kFB];
  __shared__ double s_redx[kWarps];
  __shared__ double s_sc[4];  // tau, 1 / y1, -, tau of the column T is completing
  __shared__ TS s_scT[2];     // tau, 1 / y1 in the storage precision

  TS row[CPT];
#pragma unroll
  for (int q = 0; q < CPT; ++q) {
    const int c = cbase + q;
    row[q] = (live && c < bj) ? a.P[(size_t)g + (size_t)c * a.ldp] : TS(0);
  }
  if (cta == 0)
    for (int e = tid; e < kFB * kFB; e += kThreads) s_T[e] = 0.0;
  TS vprev = TS(0);

  for (int j = 0; j < bj; ++j) {
    const int par = j & 1;
    TS* part = a.part + (size_t)par * G * bj;
    double* x2p = a.x2part + (size_t)par * G;
    TS* rowb = a.rowb + (size_t)par * bj;
    // (1) reflector j-1 on this row's columns >= j; pick up a_j(g)
    TS aj = TS(0);
    if (wlive) {
      const bool upd = j > 0 && live && g >= j - 1;
      // finished columns (c < j) never change again: chunks of 16 columns that
      // lie wholly below j are skipped
  #pragma unroll
      for (int q0 = 0; q0 < CPT; q0 += 16) {
        if (cbase + q0 + 16 > j) {
  #pragma unroll
          for (int q = q0; q < q0 + 16; ++q) {
            const int c = cbase + q;
            if (upd && c >= j && c < bj) row[q] = fma(-s_tw[c], vprev, row[q]);
            if (c == j) aj = row[q];
          }
        }
      }
      if (TPR == 2) {
        const TS o = __shfl_xor_sync(0xffffffffu, aj, 16);
        if (half != j / CPT) aj = o;
      }
      if (live && g == j) {
  #pragma unroll
        for (int q = 0; q < CPT; ++q)
          if (cbase + q < bj) rowb[cbase + q] = row[q];
      }
      // (2) this row's share of the sums over rows g > j, reduced over the CTA;
      // the squared norm in FP64 (float-float for FP32 rows)
      const bool below = live && g > j;
      const bool mine = below && half == j / CPT;
      // (the products with finished columns, c < j, feed T's sums, which need
      // every CTA's rows)
      TS prod[CPT];
  #pragma unroll
      for (int q = 0; q < CPT; ++q) {
        const int c = cbase + q;
        prod[q] = (below && c != j && c < bj) ? row[q] * aj : TS(0);
      }
      double x2d = 0.0;
      if constexpr (kF32) {
        // float-float squares while every |a_j(g)| of the warp lies in
        // [2^-60, 2^55] (no overflow for up to 2^17 rows; about 2^-46 relative
        // while the column's largest entries are at least 2^-52, falling toward
        // 2^-34 for a column of entries near 2^-60, where the squares' low parts
        // become subnormal); otherwise this warp sums in FP64
        const float fa = fabsf(aj);
        const bool out_of_range = mine && aj != 0.f && (fa > 0x1p55f || fa < 0x1p-60f);
        if (__any_sync(0xffffffffu, out_of_range)) {
          x2d = mine ? static_cast<double>(aj) * static_cast<double>(aj) : 0.0;
          x2d = warp_sum(x2d);
        } else {
          float x2h = 0.f, x2l = 0.f;
          if (mine) {
            x2h = aj * aj;
            x2l = fmaf(aj, aj, -x2h);
          }
  #pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float bh = __shfl_xor_sync(0xffffffffu, x2h, o);
            const float bl = __shfl_xor_sync(0xffffffffu, x2l, o);
            ff_add(x2h, x2l, bh, bl);
          }
          if (lane == 0) x2d = static_cast<double>(x2h) + static_cast<double>(x2l);
        }
      } else {
        x2d = mine ? static_cast<double>(aj) * static_cast<double>(aj) : 0.0;
        x2d = warp_sum(x2d);
      }
      reduce_scatter<TS, CPT, LPG>(prod);
      s_red[warp][cbase + 2 * lp] = prod[0];
      s_red[warp][cbase + 2 * lp + 1] = prod[1];
      if (lane == 0) s_redx[warp] = x2d;
    } else {
      s_red[warp][cbase + 2 * lp] = TS(0);
      s_red[warp][cbase + 2 * lp + 1] = TS(0);
      if (lane == 0) s_redx[warp] = 0.0;
    }
    __syncthreads();
    if (tid < bj) {
      TS acc = TS(0);
#pragma unroll
      for (int w = 0; w < kWarps; ++w) acc += s_red[w][tid];
      part[(size_t)cta * bj + tid] = acc;
    } else if (tid == kFB) {
      x2p[cta] = ((s_redx[0] + s_redx[1]) + (s_redx[2] + s_redx[3])) + ((s_redx[4] + s_redx[5]) + (s_redx[6] + s_redx[7]));
    }
    // (3) grid barrier; CTA 0 completes T's previous column meanwhile
    grid_arrive(a.bar);
    if (cta == 0 && j > 0) t_column(j - 1, s_sc[3], s_T, s_tv);
    if (!grid_wait(a.bar, G, a.err, static_cast<unsigned int>(j))) return;
    // (4) global sums in a fixed order (identical on every CTA), four threads
    // per value, every load in flight at once; CTA 0 also needs the columns < j
    // for T.  The squared norm (FP64) is summed by group j alone, which then
    // goes straight on to reflector j's FP64 scalars.
    {
      const int v = tid >> 2, sub = tid & 3;
      const bool want = v < bj && (v >= j || cta == 0);
      TS t = TS(0);
      double d = 0.0, alpha = 0.0;
      if (want && v != j) {
        TS x[kMaxG4];
#pragma unroll
        for (int u = 0; u < kMaxG4; ++u) {
          const int q = sub + 4 * u;
          x[u] = q < G ? __ldcg(part + (size_t)q * bj + v) : TS(0);
        }
#pragma unroll
        for (int u = 0; u < kMaxG4; ++u) t += x[u];
      } else if (want) {
        alpha = static_cast<double>(__ldcg(rowb + j));
        double x[kMaxG4];
#pragma unroll
        for (int u = 0; u < kMaxG4; ++u) {
          const int q = sub + 4 * u;
          x[u] = q < G ? __ldcg(x2p + q) : 0.0;
        }
        // pairwise tree over the 40 slots (fixed shape: deterministic)
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] += x[u + 32];
#pragma unroll
        for (int w = 16; w >= 1; w >>= 1)
#pragma unroll
          for (int u = 0; u < w; ++u) x[u] += x[u + w];
        d = x[0];
      }
      t += __shfl_xor_sync(0xffffffffu, t, 1);
      t += __shfl_xor_sync(0xffffffffu, t, 2);
      if (warp == (j >> 3)) {  // the warp holding group j
        d += __shfl_xor_sync(0xffffffffu, d, 1);
        d += __shfl_xor_sync(0xffffffffu, d, 2);
      }
      if (sub == 0 && want && v != j) s_sumT[v] = t;
      if (sub == 0 && v == j) {
        // (5) reflector j (FP64): beta = -sign(alpha) ||a||, y1 = alpha - beta,
        // 1 / y1 and tau = (beta - alpha) / beta from one division
        double tau, beta, inv;
        householder_scalars(alpha, d, kF32, beta, inv, tau);
        s_sc[0] = tau;
        s_sc[1] = inv;
        s_scT[0] = static_cast<TS>(tau);
        s_scT[1] = static_cast<TS>(inv);
        s_inv[j] = inv;
        s_invT[j] = static_cast<TS>(inv);
        s_beta[j] = beta;
        if (cta == 0) a.tau[j] = static_cast<TS>(tau);
      }
    }
    if (tid < bj) s_rowT[tid] = __ldcg(rowb + tid);
    __syncthreads();
    // (6) the lazy update's coefficients and this row's entry of reflector j,
    // in the storage precision; CTA 0 also forms (Y^T v_j) for T in FP64
    {
      const TS tauT = s_scT[0], invT = s_scT[1];
      if (tid > j && tid < bj) s_tw[tid] = tauT * fma(s_sumT[tid], invT, s_rowT[tid]);
      vprev = !live ? TS(0) : (g > j ? aj * invT : (g == j ? TS(1) : TS(0)));
    }
    if (cta == 0 && tid < j)
      s_tv[tid] = s_inv[tid] * fma(static_cast<double>(s_sumT[tid]), s_sc[1], static_cast<double>(s_rowT[tid]));
    if (cta == 0 && tid == 0) s_sc[3] = s_sc[0];
    __syncthreads();
  }
  grid_exit(a.bar, G);
  if (cta == 0) {
    t_column(bj - 1, s_sc[3], s_T, s_tv);
    __syncthreads();
  }
  if (live) {
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const int c = cbase + q;
      if (c >= bj) continue;
      TS op, oy;
      if (g > c) {
        op = row[q] * s_invT[c];
        oy = op;
      } else if (g == c) {
        op = static_cast<TS>(s_beta[c]);
        oy = TS(1);
      } else {
        op = row[q];
        oy = TS(0);
      }
      a.P[(size_t)g + (size_t)c * a.ldp] = op;
      a.Y[(size_t)g + (size_t)c * a.ldy] = oy;
    }
  }
  if (cta == 0)
    for (int e = tid; e < bj * bj; e += kThreads)
      a.T[(size_t)(e / bj) * a.ldt + (e % bj)] = s_T[(size_t)(e / bj) * kFB + (e % bj)];
}

template <typename TS>
size_t smem_bytes(int bj, int rpc) {
  return (bj + bj + (size_t)kWarps * bj + (size_t)bj * bj + 3 * (size_t)bj) * sizeof(double) +
         (size_t)bj * rpc * sizeof(TS);
}

}  // namespace

size_t panel_scratch_doubles(int bj, int num_sms) {
  return 2 * (size_t)num_sms * (bj + 1) + 4 * (size_t)bj;
}

template <typename TS>
cudaError_t panel_qr(const Ctx& c, TS* P, int ldp, int mt, int bj, TS* tau, TS* Y, int ldy,
                     double* T, int ldt, double* scratch) {
  if (bj > kMaxB || bj > mt || bj < 1) return cudaErrorInvalidValue;
  {
    // the thread-per-row kernel when the panel fits one row per thread
    constexpr int TPR = sizeof(TS) == sizeof(double) ? 2 : 1;
    constexpr int RPP = kThreads / TPR;
    // FP32 rows: as few CTAs as hold the panel (the step is latency-bound and
    // fewer CTAs make cheaper reductions); FP64 rows: the FP64 pipe bounds the
    // step, so spread the rows over every SM (below, in whole warps of rows)
    int Gf = (mt + RPP - 1) / RPP;
    if (sizeof(TS) == sizeof(double)) {
      const int g64 = (mt + 63) / 64;
      Gf = g64 < c.num_sms ? (g64 > Gf ? g64 : Gf) : (c.num_sms > Gf ? c.num_sms : Gf);
    }
    if (bj <= kFB && Gf <= c.num_sms && Gf <= 4 * kMaxG4) {
      static int per_sm_fast = -1;
      if (per_sm_fast < 0) {
        cudaError_t eo = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_fast, panel_fast_kernel<TS, TPR>,
                                                                       kThreads, 0);
        if (eo != cudaSuccess) return eo;
      }
      int rpc = (mt + Gf - 1) / Gf, rpc0 = rpc;
      if (sizeof(TS) == sizeof(double)) {
        // FP64 rows in whole warps (RPP / kWarps rows each): as few warps per CTA as the SMs
        // allow (a warp without rows skips the per-row FP64 work), at least two, and CTA 0,
        // which also forms T in FP64, one warp lighter when the grid still fits
        const int wr = RPP / kWarps;
        const int units = (mt + wr - 1) / wr;
        const int gmax = c.num_sms < 4 * kMaxG4 ? c.num_sms : 4 * kMaxG4;
        int k = (units + gmax - 1) / gmax;
        if (k < 2) k = 2;
        if (k > kWarps) k = kWarps;
        int k0 = k - 1;
        int g = units > k0 ? 1 + (units - k0 + k - 1) / k : 1;
        if (g > gmax) {
          k0 = k;
          g = (units + k - 1) / k;
        }
        if (g <= gmax) {
          Gf = g;
          rpc = k * wr;
          rpc0 = k0 * wr;
        }
      }
      if (per_sm_fast * c.num_sms >= Gf) {
        TS* part = reinterpret_cast<TS*>(scratch);
        double* x2part = scratch + 2 * (size_t)Gf * bj;
        TS* rowb = reinterpret_cast<TS*>(x2part + 2 * (size_t)Gf);
        FastArgs<TS> fa{P, ldp, mt, bj, tau, Y, ldy, T, ldt, part, x2part, rowb, c.bar, c.err, rpc, rpc0};
        void* fargs[] = {&fa};
        cudaError_t ef = cudaLaunchCooperativeKernel((const void*)panel_fast_kernel<TS, TPR>, dim3(Gf),
                                                     dim3(kThreads), fargs, 0, c.stream);
        ++*c.launches;
        return ef;
      }
    }
  }
  int G = (mt + 31) / 32;
  if (G > c.num_sms) G = c.num_sms;
  if (G > kMaxRec * kWarps) G = kMaxRec * kWarps;
  if (G < 1) G = 1;
  const int rpc = (mt + G - 1) / G;
  const size_t smem = smem_bytes<TS>(bj, rpc);
  static int max_optin = -1;
  if (max_optin < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  if (smem > (size_t)max_optin - 2048) return cudaErrorInvalidConfiguration;
  cudaError_t e =
      cudaFuncSetAttribute(panel_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, panel_kernel<TS>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm * c.num_sms < G) return cudaErrorCooperativeLaunchTooLarge;
  double* part = scratch;
  double* rowbuf = scratch + 2 * (size_t)c.num_sms * (bj + 1);
  PanelArgs<TS> a{P, ldp, mt, bj, tau, Y, ldy, T, ldt, part, rowbuf, c.bar, c.err, rpc};
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)panel_kernel<TS>, dim3(G), dim3(kThreads), args, smem,
                                  c.stream);
  ++*c.launches;
  return e;
}

template cudaError_t panel_qr<double>(const Ctx&, double*, int, int, int, double*, double*, int, double*,
                                      int, double*);
template cudaError_t panel_qr<float>(const Ctx&, float*, int, int, int, float*, float*, int, double*, int,
                                     double*);

}  // namespace rq
