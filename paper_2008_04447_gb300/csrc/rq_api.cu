// C ABI and host orchestration of the RQRCP library (include/rqrcp.h).
//
// Everything a call does is issued asynchronously on the caller's stream; the
// host never waits on the device inside rqrcp/qr (pivots, the sample and the
// reflectors stay on the GPU between blocks).
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.h"

struct rq_prof_rec {
  int phase;
  int ev0, ev1;
  long long launches;
};

struct rq_handle_s {
  int magic;
  int device;
  int num_sms;
  void* ws;
  size_t ws_bytes;
  bool ws_owned;
  long long launches;
  char last_error[256];
  // per-phase timing (rq_profile_enable)
  bool prof_on;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used;
  std::vector<rq_prof_rec> prof;
  double prof_flops[RQ_NUM_PHASES];
  double prof_bytes[RQ_NUM_PHASES];
};

namespace rq {
namespace {

constexpr int kMagic = 0x52515243;

struct Carver {
  char* base;
  size_t off;
  explicit Carver(void* b) : base(static_cast<char*>(b)), off(0) {}
  template <typename T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

int fail(rq_handle h, int code, const char* msg) {
  if (h) snprintf(h->last_error, sizeof(h->last_error), "%s", msg);
  return code;
}

int cuda_fail(rq_handle h, cudaError_t e, const char* where) {
  if (h) snprintf(h->last_error, sizeof(h->last_error), "%s: %s", where, cudaGetErrorString(e));
  if (e == cudaErrorInvalidConfiguration || e == cudaErrorCooperativeLaunchTooLarge) return RQ_ENOTIMPL;
  return RQ_ECUDA;
}

bool valid(rq_handle h) { return h != nullptr && h->magic == kMagic; }

int next_event(rq_handle h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    h->ev_pool.push_back(e);
  }
  return (int)h->ev_used++;
}

// Records CUDA events around one phase on the call's stream (when profiling),
// and accounts the phase's algorithmic flops / bytes.
struct Phase {
  rq_handle h;
  cudaStream_t st;
  int phase, ev0;
  long long l0;
  Phase(rq_handle h_, cudaStream_t st_, int ph, double flops, double bytes)
      : h(h_), st(st_), phase(ph), ev0(-1), l0(h_->launches) {
    if (!h->prof_on) return;
    ev0 = next_event(h);
    if (ev0 >= 0) cudaEventRecord(h->ev_pool[ev0], st);
    h->prof_flops[ph] += flops;
    h->prof_bytes[ph] += bytes;
  }
  ~Phase() {
    if (!h->prof_on || ev0 < 0) return;
    int ev1 = next_event(h);
    if (ev1 < 0) return;
    cudaEventRecord(h->ev_pool[ev1], st);
    h->prof.push_back({phase, ev0, ev1, h->launches - l0});
  }
};

// Workspace of the full / unpivoted factorisation (RQRCP and QR).
template <typename TS>
struct FactorWs {
  unsigned int* bar;
  int* err;
  TS *B0, *B1, *Ybuf, *YT, *Wt, *ptmp, *Tts;
  double *S11, *Oh, *T, *cand, *pscr;
  int *jtmp, *chg, *swaps, *src;
  size_t bytes;
};

template <typename TS>
FactorWs<TS> carve_factor(void* base, int m, int n, int b, int l, int num_sms) {
  Carver c(base);
  FactorWs<TS> w;
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
  w.cand = c.take<double>(sample_qrcp_scratch_doubles(l, num_sms));
  w.pscr = c.take<double>(panel_scratch_doubles(b, num_sms));
  w.bytes = align_up(c.off, 256);
  return w;
}

int ensure_ws(rq_handle h, size_t bytes) {
  if (h->ws && h->ws_bytes >= bytes) return RQ_OK;
  if (h->ws && !h->ws_owned) return fail(h, RQ_ENOMEM, "caller workspace too small");
  if (h->ws) {
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(h, RQ_ENOMEM, "cudaMalloc of the workspace failed");
  }
  h->ws = p;
  h->ws_bytes = bytes;
  h->ws_owned = true;
  return RQ_OK;
}

// Blocked Householder QR, pivoted by the sample (Alg. 4) or unpivoted.
template <typename TS>
int run_factor(rq_handle h, bool pivot, int m, int n, TS* A, int lda, int b, int p, int k, const TS* Omega,
               int ldo, TS* tau, int* jpvt, int* info, cudaStream_t st) {
  const int l = pivot ? b + p : 1;
  FactorWs<TS> w = carve_factor<TS>(nullptr, m, n, b, l, h->num_sms);
  int rc = ensure_ws(h, w.bytes);
  if (rc) return rc;
  w = carve_factor<TS>(h->ws, m, n, b, l, h->num_sms);
  Ctx c{st, h->num_sms, &h->launches, w.err, w.bar};
  cudaError_t e = cudaMemsetAsync(w.bar, 0, 16, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "memset");
  if (jpvt && (e = iota(c, jpvt, n)) != cudaSuccess) return cuda_fail(h, e, "iota");
  TS* Bc = w.B0;
  TS* Bn = w.B1;
  const double sz = sizeof(TS);
  if (pivot) {
    // Alg. 4: B = Omega A
    Phase ph(h, st, RQ_PHASE_SKETCH, 2.0 * l * (double)m * n, sz * ((double)m * n + (double)l * m + (double)l * n));
    e = gemm<TS>(c, false, false, l, n, m, TS(1), Omega, ldo, A, lda, TS(0), Bc, l);
    if (e != cudaSuccess) return cuda_fail(h, e, "sketch");
  }
  for (int j0 = 0; j0 < k; j0 += b) {
    const int bj = (k - j0) < b ? (k - j0) : b;
    const int nt = n - j0, mt = m - j0, n2 = nt - bj;
    TS* Aj = A + j0 + (size_t)j0 * lda;
    if (pivot) {
      {
        Phase ph(h, st, RQ_PHASE_SAMPLE_QRCP, 4.0 * l * (double)nt * bj, 2.0 * sz * l * (double)nt);
        e = sample_qrcp<TS>(c, Bc, l, l, nt, bj, Bn, l, w.S11, b, w.swaps, w.src, w.chg, w.cand);
        if (e != cudaSuccess) return cuda_fail(h, e, "sample_qrcp");
      }
      Phase ph(h, st, RQ_PHASE_PERMUTE, 0.0, 4.0 * sz * bj * (double)m);
      e = permute_columns<TS>(c, A + (size_t)j0 * lda, lda, m, bj, w.chg, w.src, jpvt + j0, w.ptmp, w.jtmp);
      if (e != cudaSuccess) return cuda_fail(h, e, "permute");
    }
    {
      Phase ph(h, st, RQ_PHASE_PANEL, 2.0 * (double)mt * bj * bj, 2.0 * sz * (double)mt * bj);
      e = panel_qr<TS>(c, Aj, lda, mt, bj, tau + j0, w.Ybuf, mt, w.T, b, w.pscr);
      if (e != cudaSuccess) return cuda_fail(h, e, "panel");
    }
    if (n2 > 0) {
      TS* A2 = A + j0 + (size_t)(j0 + bj) * lda;
      const TS* Tm;
      if (sizeof(TS) == sizeof(double)) {
        Tm = reinterpret_cast<const TS*>(w.T);
      } else {
        Phase ph(h, st, RQ_PHASE_OTHER, 0.0, 12.0 * bj * bj);
        e = convert<TS, double>(c, bj, bj, w.T, b, w.Tts, b);
        if (e != cudaSuccess) return cuda_fail(h, e, "convert T");
        Tm = w.Tts;
      }
      {
        // W^T = (Y T)^T A2 ; A2 -= Y W^T  (block reflector, Alg. 4 "finish b rows", "update")
        Phase ph(h, st, RQ_PHASE_TRAILING, 4.0 * mt * (double)n2 * bj + 2.0 * mt * (double)bj * bj,
                 sz * (3.0 * mt * (double)n2 + 2.0 * bj * (double)n2 + 3.0 * mt * (double)bj));
        e = gemm<TS>(c, false, false, mt, bj, bj, TS(1), w.Ybuf, mt, Tm, b, TS(0), w.YT, mt);
        if (e == cudaSuccess) e = gemm<TS>(c, true, false, bj, n2, mt, TS(1), w.YT, mt, A2, lda, TS(0), w.Wt, b);
        if (e == cudaSuccess)
          e = gemm<TS>(c, false, false, mt, n2, bj, TS(-1), w.Ybuf, mt, w.Wt, b, TS(1), A2, lda);
        if (e != cudaSuccess) return cuda_fail(h, e, "trailing update");
      }
      if (pivot && j0 + bj < k) {
        // Eq. (update1): B1 = S12 - (S11 R11^{-1}) R12, B2 = S22
        Phase ph(h, st, RQ_PHASE_SAMPLE_UPDATE, (double)bj * bj * bj / 3.0 + (double)bj * bj * n2,
                 sz * 3.0 * bj * (double)n2);
        e = omegahat11<TS>(c, w.S11, b, Aj, lda, bj, w.Oh, b);
        if (e == cudaSuccess) e = sample_update<TS>(c, bj, n2, w.Oh, b, A2, lda, Bn, l);
        if (e != cudaSuccess) return cuda_fail(h, e, "sample update");
      }
    }
    TS* t = Bc;
    Bc = Bn;
    Bn = t;
  }
  {
    Phase ph(h, st, RQ_PHASE_OTHER, 0.0, 0.0);
    e = finish_info<TS>(c, A, lda, k, info);
    if (e != cudaSuccess) return cuda_fail(h, e, "info");
  }
  return RQ_OK;
}

int check_common(rq_handle h, int prec) {
  if (!valid(h)) return RQ_EHANDLE;
  if (prec != RQ_FP64 && prec != RQ_FP32 && prec != RQ_MIXED) return -2;
  return RQ_OK;
}

}  // namespace
}  // namespace rq

using namespace rq;

extern "C" {

int rq_create(rq_handle* out) {
  if (!out) return -1;
  rq_handle h = new (std::nothrow) rq_handle_s();
  if (!h) return RQ_ENOMEM;
  h->magic = kMagic;
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return RQ_ECUDA;
  }
  h->ws = nullptr;
  h->ws_bytes = 0;
  h->ws_owned = false;
  h->launches = 0;
  h->last_error[0] = 0;
  h->prof_on = false;
  h->ev_used = 0;
  for (int i = 0; i < RQ_NUM_PHASES; ++i) h->prof_flops[i] = h->prof_bytes[i] = 0.0;
  *out = h;
  return RQ_OK;
}

int rq_destroy(rq_handle h) {
  if (!valid(h)) return RQ_EHANDLE;
  if (h->ws && h->ws_owned) cudaFree(h->ws);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  h->magic = 0;
  delete h;
  return RQ_OK;
}

int rq_workspace_size(rq_handle h, int op, int prec, int m, int n, int k, int b, int p, size_t* bytes) {
  int rc = check_common(h, prec);
  if (rc) return rc == -2 ? -3 : rc;
  if (m < 1) return -4;
  if (n < 1) return -5;
  if (b < 1) return -7;
  if (p < 0) return -8;
  if (!bytes) return -9;
  const int l = (op == RQ_OP_QR) ? 1 : b + p;
  if (op == RQ_OP_RQRCP || op == RQ_OP_QR) {
    *bytes = prec == RQ_FP64 ? carve_factor<double>(nullptr, m, n, b, l, h->num_sms).bytes
                             : carve_factor<float>(nullptr, m, n, b, l, h->num_sms).bytes;
    return RQ_OK;
  }
  (void)k;
  return RQ_ENOTIMPL;
}

int rq_set_workspace(rq_handle h, void* dptr, size_t bytes) {
  if (!valid(h)) return RQ_EHANDLE;
  if (h->ws && h->ws_owned) cudaFree(h->ws);
  h->ws = dptr;
  h->ws_bytes = dptr ? bytes : 0;
  h->ws_owned = false;
  return RQ_OK;
}

int rq_last_error(rq_handle h, char* buf, size_t len) {
  if (!valid(h)) return RQ_EHANDLE;
  if (!buf || len == 0) return -2;
  snprintf(buf, len, "%s", h->last_error);
  return RQ_OK;
}

long long rq_launch_count(rq_handle h) { return valid(h) ? h->launches : -1; }

int rq_profile_enable(rq_handle h, int enable) {
  if (!valid(h)) return RQ_EHANDLE;
  h->prof_on = enable != 0;
  return RQ_OK;
}

int rq_profile_read(rq_handle h, int nphases, double* ms, double* flops, double* bytes, long long* launches) {
  if (!valid(h)) return RQ_EHANDLE;
  if (nphases < 0) return -2;
  const int np = nphases < RQ_NUM_PHASES ? nphases : RQ_NUM_PHASES;
  for (int i = 0; i < np; ++i) {
    if (ms) ms[i] = 0.0;
    if (launches) launches[i] = 0;
    if (flops) flops[i] = h->prof_flops[i];
    if (bytes) bytes[i] = h->prof_bytes[i];
  }
  int rc = RQ_OK;
  if (!h->prof.empty()) {
    cudaError_t e = cudaEventSynchronize(h->ev_pool[h->prof.back().ev1]);
    if (e != cudaSuccess) rc = cuda_fail(h, e, "rq_profile_read");
    for (const rq_prof_rec& r : h->prof) {
      float t = 0.f;
      if (rc == RQ_OK && cudaEventElapsedTime(&t, h->ev_pool[r.ev0], h->ev_pool[r.ev1]) != cudaSuccess) {
        cudaGetLastError();
        t = 0.f;
      }
      if (r.phase < np) {
        if (ms) ms[r.phase] += t;
        if (launches) launches[r.phase] += r.launches;
      }
    }
  }
  h->prof.clear();
  h->ev_used = 0;
  for (int i = 0; i < RQ_NUM_PHASES; ++i) h->prof_flops[i] = h->prof_bytes[i] = 0.0;
  return rc;
}

int rq_rqrcp(rq_handle h, int prec, int m, int n, void* A, int lda, int b, int p, int k, const void* Omega,
             int ldo, void* tau, int* jpvt, int* info, rq_stream stream) {
  int rc = check_common(h, prec);
  if (rc) return rc;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (!A) return -5;
  if (lda < m) return -6;
  if (b < 1) return -7;
  if (p < 0) return -8;
  if (k < 1 || k > (m < n ? m : n)) return -9;
  if (!Omega) return -10;
  if (ldo < b + p) return -11;
  if (!tau) return -12;
  if (!jpvt) return -13;
  if (!info) return -14;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == RQ_FP64)
    return run_factor<double>(h, true, m, n, static_cast<double*>(A), lda, b, p, k,
                              static_cast<const double*>(Omega), ldo, static_cast<double*>(tau), jpvt, info, st);
  if (prec == RQ_FP32)
    return run_factor<float>(h, true, m, n, static_cast<float*>(A), lda, b, p, k, static_cast<const float*>(Omega),
                             ldo, static_cast<float*>(tau), jpvt, info, st);
  return fail(h, RQ_ENOTIMPL, "rq_rqrcp: RQ_MIXED is not provided for the full factorisation");
}

int rq_qr(rq_handle h, int prec, int m, int n, void* A, int lda, int b, void* tau, int* info, rq_stream stream) {
  int rc = check_common(h, prec);
  if (rc) return rc;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (!A) return -5;
  if (lda < m) return -6;
  if (b < 1) return -7;
  if (!tau) return -8;
  if (!info) return -9;
  const int k = m < n ? m : n;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == RQ_FP64)
    return run_factor<double>(h, false, m, n, static_cast<double*>(A), lda, b, 0, k, nullptr, 1,
                              static_cast<double*>(tau), nullptr, info, st);
  if (prec == RQ_FP32)
    return run_factor<float>(h, false, m, n, static_cast<float*>(A), lda, b, 0, k, nullptr, 1,
                             static_cast<float*>(tau), nullptr, info, st);
  return fail(h, RQ_ENOTIMPL, "rq_qr: RQ_MIXED is not provided");
}

int rq_trqrcp(rq_handle h, int prec, int m, int n, const void* A, int lda, int b, int p, int k, const void* Omega,
              int ldo, void* Y, int ldy, void* tau, void* R, int ldr, int* jpvt, int* info, rq_stream stream) {
  (void)prec; (void)m; (void)n; (void)A; (void)lda; (void)b; (void)p; (void)k; (void)Omega; (void)ldo;
  (void)Y; (void)ldy; (void)tau; (void)R; (void)ldr; (void)jpvt; (void)info; (void)stream;
  if (!valid(h)) return RQ_EHANDLE;
  return fail(h, RQ_ENOTIMPL, "rq_trqrcp: not built yet");
}

int rq_tuxv(rq_handle h, int prec, int m, int n, const void* A, int lda, int b, int p, int k, const void* Omega,
            int ldo, void* U, int ldu, void* X, int ldx, void* V, int ldv, void* sigma, int* info,
            rq_stream stream) {
  (void)prec; (void)m; (void)n; (void)A; (void)lda; (void)b; (void)p; (void)k; (void)Omega; (void)ldo;
  (void)U; (void)ldu; (void)X; (void)ldx; (void)V; (void)ldv; (void)sigma; (void)info; (void)stream;
  if (!valid(h)) return RQ_EHANDLE;
  return fail(h, RQ_ENOTIMPL, "rq_tuxv: not built yet");
}

}  // extern "C"
