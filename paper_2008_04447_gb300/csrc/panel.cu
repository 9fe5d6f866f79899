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
    if (!grid_barrier(a.bar, G, a.err)) return;
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
