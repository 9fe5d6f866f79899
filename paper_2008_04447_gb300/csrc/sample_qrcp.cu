// Partial QRCP of the sample matrix B (Sec. 3.2; the pivot step of Alg. 4).
//
// One cooperative launch per block of pivots.  Each CTA holds a slab of the
// sample's columns in shared memory (in the storage precision, row-major inside
// the slab so that consecutive threads touch consecutive columns) for all
// `steps` decisions,
// so B is read from HBM once and written once per block.  Per decision:
//   1. every CTA finds its best alive column (max downdated squared norm,
//      ties -> lowest current position) and publishes (norm^2, position,
//      column values) to a double-buffered candidate table;
//   2. one grid barrier;
//   3. every CTA reduces the table in the same order (so all agree bit for
//      bit), rebuilds the Householder vector of the winner in FP64 (tau =
//      (beta - alpha) / beta, with 1 / y1 from the same division), applies
//      it (rounded to the storage precision) to its alive columns in the storage
//      precision and downdates their FP64 squared norms (removing the
//      contribution of the finished row, Alg. 1), recomputing a norm from
//      the remaining rows when the downdated value has fallen to sqrt(eps)
//      of its last exactly computed value (eps of the sample's precision:
//      the downdate's relative error is about eps / (that ratio)).
// Column exchanges are never moved in memory: each CTA tracks the current
// position of its columns (only the column at position i moves per swap), so
// ties resolve exactly as with physical swaps.
#include <cfloat>
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace rq {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxSteps = 256;
static_assert(RQ_MAX_B <= kMaxSteps && RQ_MAX_L <= kMaxSteps + 128, "the sample kernel holds the largest sample");
constexpr int kMaxRecS = 8;  // candidate records per lane: G <= 256

template <typename TS>
struct SqArgs {
  const TS* B;
  int ldb, l, nt, steps;
  TS* Bn;
  int ldbn;
  double* S11;
  int lds;
  int* swaps;
  int* src;
  int* chg;      // 2*steps: positions whose column changes (-1 = none)
  double* cand;  // 2 * G * (l + 2)
  unsigned int* bar;
  int* err;
  int cpc;  // columns per CTA
};

template <typename TS>
__global__ void __launch_bounds__(kThreads) sample_qrcp_kernel(SqArgs<TS> a) {
  extern __shared__ double sm[];
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int l = a.l, cpc = a.cpc, steps = a.steps;
  const int c0 = cta * cpc;
  const int nc = max(0, min(cpc, a.nt - c0));
  // recompute a downdated norm once it has fallen to sqrt(eps) of its last exact
  // value, eps being the precision the sample is held in
  const double tol = sizeof(TS) == sizeof(double) ? 1.4901161193847656e-08 : 3.4526698300124393e-04;
  double* nu2 = sm;                           // cpc
  double* ref2 = nu2 + cpc;                   // cpc
  TS* s = reinterpret_cast<TS*>(ref2 + cpc);  // s[r * cpc + c]
  TS* vv = s + (size_t)l * cpc;               // l
  int* pos = reinterpret_cast<int*>(vv + l + 1);
  int* alive = pos + cpc;
  __shared__ long long red_v[kWarps];
  __shared__ int red_p[kWarps], red_t[kWarps];
  __shared__ int s_best_lc, s_win_cta, s_win_pos;
  __shared__ double s_tau;
  __shared__ int s_swaps[kMaxSteps];
  const int rec = l + 2;

  for (int e = tid; e < l * nc; e += kThreads) {
    const int r = e % l, c = e / l;
    s[(size_t)r * cpc + c] = a.B[(size_t)(c0 + c) * a.ldb + r];
  }
  __syncthreads();
  for (int c = tid; c < nc; c += kThreads) {
    double acc = 0.0;
    for (int r = 0; r < l; ++r) {
      const double x = static_cast<double>(s[(size_t)r * cpc + c]);
      acc = fma(x, x, acc);
    }
    nu2[c] = acc;
    ref2[c] = acc;
    pos[c] = c0 + c;
    alive[c] = 1;
  }
  __syncthreads();

  unsigned int epoch = 0;
  for (int i = 0; i < steps; ++i) {
    const int par = i & 1;
    double* tab = a.cand + (size_t)par * G * rec;
    // (1) local best alive column
    long long bv = 0;
    int bp = -1, bt = -1;
    for (int c = tid; c < nc; c += kThreads) {
      const long long kc = __double_as_longlong(nu2[c]);
      if (alive[c] && better_key(kc, pos[c], bv, bp)) { bv = kc; bp = pos[c]; bt = c; }
    }
    warp_argmax_key(bv, bp, bt);
    if (lane == 0) { red_v[warp] = bv; red_p[warp] = bp; red_t[warp] = bt; }
    __syncthreads();
    if (warp == 0) {
      bv = lane < kWarps ? red_v[lane] : 0;
      bp = lane < kWarps ? red_p[lane] : -1;
      bt = lane < kWarps ? red_t[lane] : -1;
      warp_argmax_key(bv, bp, bt);
      if (lane == 0) {
        s_best_lc = bt;
        tab[(size_t)cta * rec + 0] = __longlong_as_double(bv);
        tab[(size_t)cta * rec + 1] = static_cast<double>(bp);
      }
    }
    __syncthreads();
    {
      const int lc = s_best_lc;
      if (lc >= 0)
        for (int r = tid; r < l; r += kThreads) tab[(size_t)cta * rec + 2 + r] = static_cast<double>(s[(size_t)r * cpc + lc]);
    }
    // (2)
    if (!grid_barrier(a.bar, G, a.err, epoch)) return;
    // (3) global winner: same reduction order on every CTA
    if (warp == 0) {
      long long gv = 0;
      int gp = -1, gt = -1;
      long long vs[kMaxRecS];
      int ps[kMaxRecS];
#pragma unroll
      for (int u = 0; u < kMaxRecS; ++u) {
        const int q = lane + 32 * u;
        vs[u] = q < G ? __double_as_longlong(__ldcg(tab + (size_t)q * rec + 0)) : 0;
        ps[u] = q < G ? static_cast<int>(__ldcg(tab + (size_t)q * rec + 1)) : -1;
      }
#pragma unroll
      for (int u = 0; u < kMaxRecS; ++u) {
        const int q = lane + 32 * u;
        if (q < G && better_key(vs[u], ps[u], gv, gp)) { gv = vs[u]; gp = ps[u]; gt = q; }
      }
      warp_argmax_key(gv, gp, gt);
      if (lane == 0) { s_win_cta = gt; s_win_pos = gp; }
    }
    __syncthreads();
    const int wc = s_win_cta, q = s_win_pos;
    __shared__ double wcol[kMaxSteps + 128];
    for (int r = tid; r < l; r += kThreads) wcol[r] = __ldcg(tab + (size_t)wc * rec + 2 + r);
    if (tid == 0) {
      if (wc == cta) { alive[s_best_lc] = 0; pos[s_best_lc] = i; }
      if (cta == 0) { a.swaps[i] = q; s_swaps[i] = q; }
    }
    __syncthreads();
    for (int c = tid; c < nc; c += kThreads)
      if (alive[c] && pos[c] == i) pos[c] = q;
    // reflector of the winner, rows i..l-1 (Sec. 2 formula, v_i = 1)
    if (warp == 0) {
      double x2 = 0.0;
      for (int r = i + 1 + lane; r < l; r += 32) x2 = fma(wcol[r], wcol[r], x2);
      x2 = warp_sum(x2);
      const double alpha = wcol[i];
      double beta, inv, tau;
      householder_scalars(alpha, x2, sizeof(TS) == sizeof(float), beta, inv, tau);
      if (cta == 0) {
        double* col = a.S11 + (size_t)i * a.lds;
        for (int r = lane; r < steps; r += 32) col[r] = r < i ? wcol[r] : (r == i ? beta : 0.0);
      }
      __syncwarp();
      for (int r = lane; r < l; r += 32) {
        TS v;
        if (r < i) v = TS(0);
        else if (r == i) v = TS(1);
        else v = static_cast<TS>(wcol[r] * inv);
        vv[r] = v;
      }
      if (lane == 0) s_tau = tau;
    }
    __syncthreads();
    const TS tau = static_cast<TS>(s_tau);
    for (int c = tid; c < nc; c += kThreads) {
      if (!alive[c]) continue;
      if (tau != TS(0)) {
        // w = v^T s_c with four partial sums (a short dependency chain)
        TS w0 = s[(size_t)i * cpc + c], w1 = TS(0), w2 = TS(0), w3 = TS(0);
        int r = i + 1;
        for (; r + 3 < l; r += 4) {
          w0 = fma(vv[r], s[(size_t)r * cpc + c], w0);
          w1 = fma(vv[r + 1], s[(size_t)(r + 1) * cpc + c], w1);
          w2 = fma(vv[r + 2], s[(size_t)(r + 2) * cpc + c], w2);
          w3 = fma(vv[r + 3], s[(size_t)(r + 3) * cpc + c], w3);
        }
        for (; r < l; ++r) w0 = fma(vv[r], s[(size_t)r * cpc + c], w0);
        const TS w = (w0 + w1) + (w2 + w3);
        const TS tw = tau * w;
        s[(size_t)i * cpc + c] -= tw;
        for (int r = i + 1; r < l; ++r) s[(size_t)r * cpc + c] = fma(-tw, vv[r], s[(size_t)r * cpc + c]);
      }
      const double x = static_cast<double>(s[(size_t)i * cpc + c]);
      double nn = nu2[c] - x * x;
      if (nn <= tol * ref2[c]) {
        double n0 = 0.0, n1 = 0.0;
        int r = i + 1;
        for (; r + 1 < l; r += 2) {
          const double y0 = static_cast<double>(s[(size_t)r * cpc + c]);
          const double y1 = static_cast<double>(s[(size_t)(r + 1) * cpc + c]);
          n0 = fma(y0, y0, n0);
          n1 = fma(y1, y1, n1);
        }
        if (r < l) {
          const double y0 = static_cast<double>(s[(size_t)r * cpc + c]);
          n0 = fma(y0, y0, n0);
        }
        nn = n0 + n1;
        ref2[c] = nn;
      }
      nu2[c] = nn;
    }
    __syncthreads();
  }

  grid_exit(a.bar, G);
  // outputs: new order of the columns, the reordered trailing sample
  for (int c = tid; c < nc; c += kThreads) a.src[pos[c]] = c0 + c;
  for (int e = tid; e < l * nc; e += kThreads) {
    const int r = e % l, c = e / l;
    if (alive[c]) a.Bn[(size_t)(pos[c] - steps) * a.ldbn + r] = s[(size_t)r * cpc + c];
  }
  if (cta == 0) {
    for (int i = tid; i < steps; i += kThreads) {
      a.chg[i] = i;
      const int qq = s_swaps[i];
      bool keep = qq >= steps;
      for (int j = 0; j < i && keep; ++j) keep = s_swaps[j] != qq;
      a.chg[steps + i] = keep ? qq : -1;
    }
  }
}

template <typename TS>
size_t smem_bytes(int l, int cpc) {
  return 2 * (size_t)cpc * sizeof(double) + ((size_t)l * cpc + l + 1) * sizeof(TS) + 2 * (size_t)cpc * sizeof(int) +
         16;
}

}  // namespace

size_t sample_qrcp_scratch_doubles(int l, int num_sms) { return 2 * (size_t)num_sms * (l + 2); }

template <typename TS>
cudaError_t sample_qrcp(const Ctx& c, const TS* B, int ldb, int l, int nt, int steps, TS* Bn,
                        int ldbn, double* S11, int lds, int* swaps, int* src, int* chg,
                        double* cand) {
  if (steps > kMaxSteps || steps > nt || steps > l || l > kMaxSteps + 128) return cudaErrorInvalidValue;
  int G = (nt + 31) / 32;
  if (G > c.num_sms) G = c.num_sms;
  if (G > 32 * kMaxRecS) G = 32 * kMaxRecS;
  if (G < 1) G = 1;
  int cpc = (nt + G - 1) / G;
  size_t smem = smem_bytes<TS>(l, cpc);
  static int max_optin = -1;
  if (max_optin < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  if (smem > (size_t)max_optin - 2048) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaFuncSetAttribute(sample_qrcp_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sample_qrcp_kernel<TS>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm * c.num_sms < G) return cudaErrorCooperativeLaunchTooLarge;
  SqArgs<TS> a{B, ldb, l, nt, steps, Bn, ldbn, S11, lds, swaps, src, chg, cand, c.bar, c.err, cpc};
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)sample_qrcp_kernel<TS>, dim3(G), dim3(kThreads), args, smem,
                                  c.stream);
  ++*c.launches;
  return e;
}

template cudaError_t sample_qrcp<double>(const Ctx&, const double*, int, int, int, int, double*, int,
                                         double*, int, int*, int*, int*, double*);
template cudaError_t sample_qrcp<float>(const Ctx&, const float*, int, int, int, int, float*, int,
                                        double*, int, int*, int*, int*, double*);

}  // namespace rq
