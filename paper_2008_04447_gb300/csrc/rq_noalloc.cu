// rq_rqrcp_noalloc: RQRCP (FP64 or FP32) whose scratch lives in a fixed
// device array compiled into the library, for callers that cannot allocate
// device memory at call time.
//
// Such callers include services that have handed all device memory to another
// allocator (a framework's caching pool), latency-sensitive code for which a
// cudaMalloc / cudaFree would add a device-wide synchronisation in the middle
// of a request, and code that must not fail for lack of memory once it runs.
//
// The scratch array is RQ_NOALLOC_SCRATCH_BYTES large and every GPU that
// loads this library holds it until the process exits.  All calls share it:
// calls that overlap on the GPU (different streams, or different host
// threads) race on it and give wrong results; serialise them.  The first call
// on a device looks up the array's device address (cudaGetSymbolAddress) with
// that device current; make that first call before any stream capture.
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace rq {
namespace {

static __device__ __align__(256) unsigned char g_scratch[RQ_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};
int g_sms[kMaxDevices] = {0};
long long g_launches = 0;

struct Carve {
  char* base;
  size_t off;
  template <typename T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

template <typename TS>
struct Ws {
  unsigned int* bar;
  int* err;
  TS *B0, *B1, *Ybuf, *YT, *Wt, *ptmp, *Tts;
  double *S11, *Oh, *T, *cand, *pscr;
  int *jtmp, *chg, *swaps, *src;
  size_t bytes;
};

template <typename TS>
Ws<TS> carve(void* base, int m, int n, int b, int l, int sms) {
  Carve c{static_cast<char*>(base), 0};
  Ws<TS> w;
  w.bar = c.take<unsigned int>(4);
  w.err = reinterpret_cast<int*>(w.bar + 2);
  w.B0 = c.take<TS>((size_t)l * n);
  w.B1 = c.take<TS>((size_t)l * n);
  w.S11 = c.take<double>((size_t)b * b);
  w.Oh = c.take<double>((size_t)b * b);
  w.T = c.take<double>((size_t)b * b);
  w.Tts = c.take<TS>((size_t)b * b);
  w.Ybuf = c.take<TS>((size_t)m * b);
  w.YT = c.take<TS>((size_t)m * b);
  w.Wt = c.take<TS>((size_t)b * n);
  w.ptmp = c.take<TS>((size_t)2 * b * m);
  w.jtmp = c.take<int>((size_t)2 * b);
  w.chg = c.take<int>((size_t)2 * b);
  w.swaps = c.take<int>((size_t)b);
  w.src = c.take<int>((size_t)n);
  w.cand = c.take<double>(sample_qrcp_scratch_doubles(l, sms));
  w.pscr = c.take<double>(panel_scratch_doubles(b, sms));
  w.bytes = align_up(c.off, 256);
  return w;
}

// Device address of the static array and SM count of the current device,
// looked up once per device (the set-up the file header describes).
int setup(void** addr, int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RQ_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return RQ_ECUDA;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RQ_ECUDA;
    g_addr[dev] = p;
    g_sms[dev] = n;
  }
  *addr = g_addr[dev];
  *sms = g_sms[dev];
  return RQ_OK;
}

template <typename TS>
int run(int m, int n, TS* A, int lda, int b, int p, int k, const TS* Omega, int ldo, TS* tau, int* jpvt,
        int* info, cudaStream_t st) {
  void* base = nullptr;
  int sms = 0;
  int rc = setup(&base, &sms);
  if (rc) return rc;
  const int l = b + p;
  Ws<TS> w = carve<TS>(nullptr, m, n, b, l, sms);
  if (w.bytes > (size_t)RQ_NOALLOC_SCRATCH_BYTES) return RQ_ETOOBIG;
  w = carve<TS>(base, m, n, b, l, sms);
  Ctx c{st, sms, &g_launches, w.err, w.bar};
  // the array keeps the previous call's contents: the barrier words must start at zero
  if (cudaMemsetAsync(w.bar, 0, 16, st) != cudaSuccess) return RQ_ECUDA;
  if (iota(c, jpvt, n) != cudaSuccess) return RQ_ECUDA;
  TS* Bc = w.B0;
  TS* Bn = w.B1;
  if (gemm<TS>(c, false, false, l, n, m, TS(1), Omega, ldo, A, lda, TS(0), Bc, l) != cudaSuccess) return RQ_ECUDA;
  for (int j0 = 0; j0 < k; j0 += b) {
    const int bj = (k - j0) < b ? (k - j0) : b;
    const int nt = n - j0, mt = m - j0, n2 = nt - bj;
    TS* Aj = A + j0 + (size_t)j0 * lda;
    cudaError_t e = sample_qrcp<TS>(c, Bc, l, l, nt, bj, Bn, l, w.S11, b, w.swaps, w.src, w.chg, w.cand);
    if (e == cudaSuccess)
      e = permute_columns<TS>(c, A + (size_t)j0 * lda, lda, m, bj, w.chg, w.src, jpvt + j0, w.ptmp, w.jtmp);
    if (e == cudaSuccess) e = panel_qr<TS>(c, Aj, lda, mt, bj, tau + j0, w.Ybuf, mt, w.T, b, w.pscr);
    if (e == cudaSuccess && n2 > 0) {
      TS* A2 = A + j0 + (size_t)(j0 + bj) * lda;
      const TS* Tm = reinterpret_cast<const TS*>(w.T);
      if (sizeof(TS) != sizeof(double)) {
        e = convert<TS, double>(c, bj, bj, w.T, b, w.Tts, b);
        Tm = w.Tts;
      }
      if (e == cudaSuccess) e = gemm<TS>(c, false, false, mt, bj, bj, TS(1), w.Ybuf, mt, Tm, b, TS(0), w.YT, mt);
      if (e == cudaSuccess) e = gemm<TS>(c, true, false, bj, n2, mt, TS(1), w.YT, mt, A2, lda, TS(0), w.Wt, b);
      if (e == cudaSuccess)
        e = gemm<TS>(c, false, false, mt, n2, bj, TS(-1), w.Ybuf, mt, w.Wt, b, TS(1), A2, lda);
      if (e == cudaSuccess && j0 + bj < k) {
        e = omegahat11<TS>(c, w.S11, b, Aj, lda, bj, w.Oh, b);
        if (e == cudaSuccess) e = sample_update<TS>(c, bj, n2, w.Oh, b, A2, lda, Bn, l);
      }
    }
    if (e != cudaSuccess) {
      return (e == cudaErrorInvalidConfiguration || e == cudaErrorCooperativeLaunchTooLarge) ? RQ_ENOTIMPL
                                                                                              : RQ_ECUDA;
    }
    TS* t = Bc;
    Bc = Bn;
    Bn = t;
  }
  if (finish_info<TS>(c, A, lda, k, info) != cudaSuccess) return RQ_ECUDA;
  return RQ_OK;
}

}  // namespace
}  // namespace rq

extern "C" int rq_rqrcp_noalloc(int prec, int m, int n, void* A, int lda, int b, int p, int k, const void* Omega,
                                int ldo, void* tau, int* jpvt, int* info, rq_stream stream) {
  if (prec != RQ_FP64 && prec != RQ_FP32) return -1;
  if (m < 1) return -2;
  if (n < 1) return -3;
  if (!A) return -4;
  if (lda < m) return -5;
  if (b < 1 || b > RQ_MAX_B) return -6;
  if (p < 0 || b + p > RQ_MAX_L) return -7;
  if (k < 1 || k > (m < n ? m : n)) return -8;
  if (!Omega) return -9;
  if (ldo < b + p) return -10;
  if (!tau) return -11;
  if (!jpvt) return -12;
  if (!info) return -13;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == RQ_FP64)
    return rq::run<double>(m, n, static_cast<double*>(A), lda, b, p, k, static_cast<const double*>(Omega), ldo,
                           static_cast<double*>(tau), jpvt, info, st);
  return rq::run<float>(m, n, static_cast<float*>(A), lda, b, p, k, static_cast<const float*>(Omega), ldo,
                        static_cast<float*>(tau), jpvt, info, st);
}
