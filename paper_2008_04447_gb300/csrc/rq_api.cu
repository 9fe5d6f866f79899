// C ABI and host orchestration of the RQRCP library (include/rqrcp.h).
//
// Everything a call does is issued asynchronously on the caller's stream; the
// host never waits on the device inside rqrcp/qr (pivots, the sample and the
// reflectors stay on the GPU between blocks).
#include <nvtx3/nvToolsExt.h>
#include <cmath>
#include <cstdio>
#include <cstdlib>
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
  // tile policy of the batched kernel's block GEMMs (rq_batch_tiles)
  int tile_m, tile_n;
  // FP64 block reflector products on the bfloat16 tensor cores: 0 off (FP64
  // pipe), 1 the update A2 -= Y W^T only, 2 also W^T = (Y T)^T A2
  int f64_tc;
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
constexpr int kDefaultTile = 32;  // rq_batch_tiles of a new handle

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
// Each phase is also an NVTX range (header-only NVTX v3: a no-op unless a
// profiling tool is attached), so timeline tools show the path's phases.
const char* const kPhaseNames[RQ_NUM_PHASES] = {"rq sketch",         "rq sample QRCP",    "rq permute",
                                                "rq panel",          "rq trailing update", "rq sample update",
                                                "rq other",          "rq FP64 slices"};

struct Phase {
  rq_handle h;
  cudaStream_t st;
  int phase, ev0;
  long long l0;
  Phase(rq_handle h_, cudaStream_t st_, int ph, double flops, double bytes)
      : h(h_), st(st_), phase(ph), ev0(-1), l0(h_ ? h_->launches : 0) {
    nvtxRangePushA(kPhaseNames[ph]);
    if (!h || !h->prof_on) return;
    ev0 = next_event(h);
    if (ev0 >= 0) cudaEventRecord(h->ev_pool[ev0], st);
    h->prof_flops[ph] += flops;
    h->prof_bytes[ph] += bytes;
  }
  ~Phase() {
    nvtxRangePop();
    if (!h || !h->prof_on || ev0 < 0) return;
    int ev1 = next_event(h);
    if (ev1 < 0) return;
    cudaEventRecord(h->ev_pool[ev1], st);
    h->prof.push_back({phase, ev0, ev1, h->launches - l0});
  }
};

// Scratch of one FP64 tensor-core product: barrier / error words, the two
// operands' slice planes and exponents, and FP64 split-K partials.
struct OzWs {
  unsigned int* bar;
  int* err;
  uint16_t *Ap, *Bp;
  int *ea, *eb;
  char* split;
  size_t split_bytes;
};

OzWs carve_oz(Carver& cv, int Mp, int Np, int Kp, size_t mn) {
  OzWs z;
  z.bar = cv.take<unsigned int>(4);
  z.err = reinterpret_cast<int*>(z.bar + 2);
  z.Ap = cv.take<uint16_t>(oz_plane_bytes(Mp, Kp) / 2);
  z.Bp = cv.take<uint16_t>(oz_plane_bytes(Np, Kp) / 2);
  z.ea = cv.take<int>(Mp);
  z.eb = cv.take<int>(Np);
  const int chunks = (Kp + 127) / 128;
  z.split_bytes = (size_t)(chunks < 16 ? chunks : 16) * sizeof(double) * mn;
  z.split = cv.take<char>(z.split_bytes);
  return z;
}

// Workspace of the full / unpivoted factorisation (RQRCP and QR).
template <typename TS>
struct FactorWs {
  unsigned int* bar;
  int* err;
  TS *B0, *B1, *Ybuf, *YT, *Wt, *ptmp, *Tts;
  TS* Om;  // l x m Gaussian draws (repeated sampling only)
  double *S11, *Oh, *T, *cand, *pscr;
  int *jtmp, *chg, *swaps, *src;
  char* splitk;
  size_t splitk_bytes;
  // slice planes and exponents of the FP64 tensor-core products (FP64 only):
  // 1 = W^T = (Y T)^T A2 (A2's columns, Y T's columns), 2 = A2 -= Y W^T (Y's
  // rows, W^T's columns)
  uint16_t *Ap1, *Bp1, *Ap2, *Bp2;
  int *ea1, *eb1, *ea2, *eb2;
  uint16_t* Osl;  // slices of Omega for the FP64 sketch on the tensor cores (B = Omega A)
  int* eo;
  size_t bytes;
};

inline int pad4(int x) { return (x + 3) / 4 * 4; }

// Split-K partials of the b x n W^T product: up to `copies` partial copies.
inline size_t splitk_bytes_for(int b, int n, size_t elem, int copies = 16) {
  return (size_t)copies * b * n * elem;
}

template <typename TS>
FactorWs<TS> carve_factor(void* base, int m, int n, int b, int l, int num_sms, bool resample = false,
                          int splitk_copies = 16, int f64tc = 0) {
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
  w.Ybuf = c.take<TS>((size_t)pad4(m) * b);
  w.YT = c.take<TS>((size_t)pad4(m) * b);
  w.Wt = c.take<TS>((size_t)b * n);
  w.ptmp = c.take<TS>((size_t)2 * b * m);
  w.jtmp = c.take<int>((size_t)2 * b);
  w.chg = c.take<int>((size_t)2 * b);
  w.swaps = c.take<int>((size_t)b);
  w.src = c.take<int>((size_t)n);
  w.cand = c.take<double>(sample_qrcp_scratch_doubles(l, num_sms));
  w.pscr = c.take<double>(panel_scratch_doubles(b, num_sms));
  w.splitk_bytes = splitk_bytes_for(b, n, sizeof(TS), splitk_copies);
  w.splitk = splitk_copies > 0 ? c.take<char>(w.splitk_bytes) : nullptr;
  w.Om = resample ? c.take<TS>((size_t)l * m) : nullptr;
  w.Ap1 = w.Bp1 = w.Ap2 = w.Bp2 = w.Osl = nullptr;
  w.ea1 = w.eb1 = w.ea2 = w.eb2 = w.eo = nullptr;
  if (sizeof(TS) == sizeof(double) && f64tc > 0) {
    const int kb = oz_k_pad(b);
    w.Ap2 = c.take<uint16_t>(oz_plane_bytes(oz_rows_pad(m, true), kb) / 2);
    w.ea2 = c.take<int>(oz_rows_pad(m, true));
    w.Bp2 = c.take<uint16_t>(oz_plane_bytes(oz_rows_pad(n, false), kb) / 2);
    w.eb2 = c.take<int>(oz_rows_pad(n, false));
    if (f64tc > 1) {
      const int km = oz_k_pad(m);
      w.Ap1 = c.take<uint16_t>(oz_plane_bytes(oz_rows_pad(n, true), km) / 2);
      w.ea1 = c.take<int>(oz_rows_pad(n, true));
      w.Bp1 = c.take<uint16_t>(oz_plane_bytes(oz_rows_pad(b, false), km) / 2);
      w.eb1 = c.take<int>(oz_rows_pad(b, false));
      if (l > 1) {
        w.Osl = c.take<uint16_t>(oz_plane_bytes(oz_rows_pad(l, true), km) / 2);
        w.eo = c.take<int>(oz_rows_pad(l, true));
      }
    }
  }
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

// C (bj x n2, ld ldc) = P^T Q with P (K x bj) and Q (K x n2) column-major: the
// skinny products W^T = (Y T)^T A2 and Y2^T A.  FP32 runs on the tensor cores
// (3xTF32, computed as (Q^T P)^T); FP64 and unaligned operands use the SIMT kernel.
template <typename TS>
cudaError_t prod_tn_skinny(const Ctx& c, int bj, int n2, int K, const TS* P, int ldp, const TS* Q, int ldq, TS* C,
                           int ldc) {
  if constexpr (sizeof(TS) == sizeof(float)) {
    if (tc_gemm_supported(Q, ldq, P, ldp))
      return tc_gemm_tn(c, n2, bj, K, 1.f, Q, ldq, P, ldp, 0.f, C, ldc, true, true);
  }
  return gemm<TS>(c, true, false, bj, n2, K, TS(1), P, ldp, Q, ldq, TS(0), C, ldc);
}

// C (M x N) = alpha A B + beta C, A M x K and B K x N column-major: the block
// update A2 -= Y W^T, the sketch Omega A and Z1 = A V.  FP32 on the tensor cores
// (3xTF32), else SIMT.
template <typename TS>
cudaError_t prod_nn(const Ctx& c, int M, int N, int K, TS alpha, const TS* A, int lda, const TS* B, int ldb, TS beta,
                    TS* C, int ldc) {
  if constexpr (sizeof(TS) == sizeof(float)) {
    if (tc_gemm_supported(A, lda, B, ldb)) return tc_gemm_nn(c, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, true);
  }
  return gemm<TS>(c, false, false, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

}  // namespace

// Blocked Householder QR, pivoted by the sample (Alg. 4) or unpivoted, over a
// workspace `ws` of factor_ws_bytes bytes that the caller provides (the
// handle's, or the fixed array of rq_rqrcp_noalloc).  With rs_seed (repeated
// sampling, Sec. 3.4) Omega is drawn from (seed, 0) and each block's sample is
// a fresh sketch of the trailing matrix by the draws of (seed, J) instead of
// the update of Eq. (update1).  h may be NULL (no profiling, no message).
template <typename TS>
int factor_blocks(rq_handle h, void* ws, int num_sms, long long* launches, bool pivot, int m, int n, TS* A, int lda,
                  int b, int p, int k, const TS* Omega, int ldo, TS* tau, int* jpvt, int* info, cudaStream_t st,
                  const uint64_t* rs_seed, int splitk_copies, int f64tc) {
  const int l = pivot ? b + p : 1;
  const bool rs = pivot && rs_seed != nullptr;
  FactorWs<TS> w = carve_factor<TS>(ws, m, n, b, l, num_sms, rs, splitk_copies, f64tc);
  Ctx c{st, num_sms, launches, w.err, w.bar, w.splitk, w.splitk_bytes};
  cudaError_t e = cudaMemsetAsync(w.bar, 0, 16, st);
  if (e != cudaSuccess) return cuda_fail(h, e, "memset");
  if (jpvt && (e = iota(c, jpvt, n)) != cudaSuccess) return cuda_fail(h, e, "iota");
  TS* Bc = w.B0;
  TS* Bn = w.B1;
  const double sz = sizeof(TS);
  if (rs) {
    Phase ph(h, st, RQ_PHASE_OTHER, 0.0, sz * l * (double)m);
    e = gaussian<TS>(c, *rs_seed, 0, l, m, w.Om, l);
    if (e != cudaSuccess) return cuda_fail(h, e, "gaussian");
    Omega = w.Om;
    ldo = l;
  }
  if (pivot) {
    // Alg. 4: B = Omega A
    Phase ph(h, st, RQ_PHASE_SKETCH, 2.0 * l * (double)m * n, sz * ((double)m * n + (double)l * m + (double)l * n));
    if (w.Osl) {
      // FP64 B = Omega A on the tensor cores: operand rows are Omega's rows and A's columns, K = m
      const int Mp = oz_rows_pad(l, true), Np = oz_rows_pad(n, false), Kp = oz_k_pad(m);
      e = oz_slice(c, false, l, m, reinterpret_cast<const double*>(Omega), ldo, Mp, Kp, w.Osl, w.eo);
      if (e == cudaSuccess)
        e = oz_slice(c, true, n, m, reinterpret_cast<const double*>(A), lda, Np, Kp, w.Ap1, w.ea1);
      if (e == cudaSuccess)
        e = oz_gemm(c, l, n, m, w.Osl, Mp, w.eo, w.Ap1, Np, w.ea1, Kp, 1.0, 0.0, reinterpret_cast<double*>(Bc), 1, l);
    } else {
      e = prod_nn<TS>(c, l, n, m, TS(1), Omega, ldo, A, lda, TS(0), Bc, l);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "sketch");
  }
  const int ldy = pad4(m);
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
      e = panel_qr<TS>(c, Aj, lda, mt, bj, tau + j0, w.Ybuf, ldy, w.T, b, w.pscr);
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
        // W^T = (Y T)^T A2 ; A2 -= Y W^T  (block reflector: the new R rows and the trailing update of Alg. 4).
        // On the FP64 tensor-core path the operand slicing is timed as its own phase.
        {
          Phase ph(h, st, RQ_PHASE_TRAILING, 4.0 * mt * (double)n2 * bj + 2.0 * mt * (double)bj * bj,
                   sz * (3.0 * mt * (double)n2 + 2.0 * bj * (double)n2 + 3.0 * mt * (double)bj));
          e = gemm<TS>(c, false, false, mt, bj, bj, TS(1), w.Ybuf, ldy, Tm, b, TS(0), w.YT, ldy);
          if (e == cudaSuccess && !w.Ap1) e = prod_tn_skinny<TS>(c, bj, n2, mt, w.YT, ldy, A2, lda, w.Wt, b);
        }
        if (e == cudaSuccess && w.Ap1) {
          // W = A2^T (Y T) on the tensor cores (FP64 through slices), stored as W^T (bj x n2, ld b)
          const int Mp = oz_rows_pad(n2, true), Np = oz_rows_pad(bj, false), Kp = oz_k_pad(mt);
          {
            Phase ph(h, st, RQ_PHASE_SLICE, 0.0, 8.0 * ((double)mt * n2 + (double)mt * bj));
            e = oz_slice(c, true, n2, mt, reinterpret_cast<const double*>(A2), lda, Mp, Kp, w.Ap1, w.ea1);
            if (e == cudaSuccess)
              e = oz_slice(c, true, bj, mt, reinterpret_cast<const double*>(w.YT), ldy, Np, Kp, w.Bp1, w.eb1);
          }
          Phase ph(h, st, RQ_PHASE_TRAILING, 0.0, 0.0);
          if (e == cudaSuccess)
            e = oz_gemm(c, n2, bj, mt, w.Ap1, Mp, w.ea1, w.Bp1, Np, w.eb1, Kp, 1.0, 0.0,
                        reinterpret_cast<double*>(w.Wt), b, 1);
        }
        if (e == cudaSuccess && w.Ap2) {
          // A2 -= Y W^T on the tensor cores: operand rows are Y's rows and W^T's columns, K = bj
          const int Mp = oz_rows_pad(mt, true), Np = oz_rows_pad(n2, false), Kp = oz_k_pad(bj);
          {
            Phase ph(h, st, RQ_PHASE_SLICE, 0.0, 8.0 * ((double)mt * bj + (double)bj * n2));
            e = oz_slice(c, false, mt, bj, reinterpret_cast<const double*>(w.Ybuf), ldy, Mp, Kp, w.Ap2, w.ea2);
            if (e == cudaSuccess)
              e = oz_slice(c, true, n2, bj, reinterpret_cast<const double*>(w.Wt), b, Np, Kp, w.Bp2, w.eb2);
          }
          Phase ph(h, st, RQ_PHASE_TRAILING, 0.0, 0.0);
          if (e == cudaSuccess)
            e = oz_gemm(c, mt, n2, bj, w.Ap2, Mp, w.ea2, w.Bp2, Np, w.eb2, Kp, -1.0, 1.0,
                        reinterpret_cast<double*>(A2), 1, lda);
        } else if (e == cudaSuccess) {
          Phase ph(h, st, RQ_PHASE_TRAILING, 0.0, 0.0);
          e = prod_nn<TS>(c, mt, n2, bj, TS(-1), w.Ybuf, ldy, w.Wt, b, TS(1), A2, lda);
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "trailing update");
      }
      if (rs && j0 + bj < k) {
        // Sec. 3.4, repeated sampling: B = Omega^(J) A(j0+bj:, j0+bj:), fresh draws of (seed, J)
        const int m2 = mt - bj;
        Phase ph(h, st, RQ_PHASE_SAMPLE_UPDATE, 2.0 * l * (double)m2 * n2,
                 sz * ((double)m2 * n2 + 2.0 * l * (double)m2 + (double)l * n2));
        e = gaussian<TS>(c, *rs_seed, (uint64_t)(j0 / b + 1), l, m2, w.Om, l);
        if (w.Osl && m2 > 0) {
          // FP64 on the tensor cores: operand rows are the draws' rows and the trailing columns, K = m2
          const int Mp = oz_rows_pad(l, true), Np = oz_rows_pad(n2, false), Kp = oz_k_pad(m2);
          if (e == cudaSuccess)
            e = oz_slice(c, false, l, m2, reinterpret_cast<const double*>(w.Om), l, Mp, Kp, w.Osl, w.eo);
          if (e == cudaSuccess)
            e = oz_slice(c, true, n2, m2, reinterpret_cast<const double*>(A2 + bj), lda, Np, Kp, w.Ap1, w.ea1);
          if (e == cudaSuccess)
            e = oz_gemm(c, l, n2, m2, w.Osl, Mp, w.eo, w.Ap1, Np, w.ea1, Kp, 1.0, 0.0, reinterpret_cast<double*>(Bn),
                        1, l);
        } else if (e == cudaSuccess) {
          e = prod_nn<TS>(c, l, n2, m2, TS(1), w.Om, l, A2 + bj, lda, TS(0), Bn, l);
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "resample");
      } else if (pivot && j0 + bj < k) {
        // Eq. (update1): B1 = S12 - (S11 R11^{-1}) R12, B2 = S22
        Phase ph(h, st, RQ_PHASE_SAMPLE_UPDATE, (double)bj * bj * bj / 3.0 + (double)bj * bj * n2,
                 sz * 3.0 * bj * (double)n2);
        e = omegahat11<TS>(c, w.S11, b, Aj, lda, bj, w.Oh, b);
        // B1 -= Omegahat11 R12 with R12 the top bj rows of the updated A2
        if (e == cudaSuccess) {
          if constexpr (sizeof(TS) == sizeof(double)) {
            if (w.Ap2) {
              // on the tensor cores: operand rows are Omegahat11's rows and R12's columns, K = bj
              const int Mp = oz_rows_pad(bj, true), Np = oz_rows_pad(n2, false), Kp = oz_k_pad(bj);
              e = oz_slice(c, false, bj, bj, w.Oh, b, Mp, Kp, w.Ap2, w.ea2);
              if (e == cudaSuccess)
                e = oz_slice(c, true, n2, bj, reinterpret_cast<const double*>(A2), lda, Np, Kp, w.Bp2, w.eb2);
              if (e == cudaSuccess)
                e = oz_gemm(c, bj, n2, bj, w.Ap2, Mp, w.ea2, w.Bp2, Np, w.eb2, Kp, -1.0, 1.0,
                            reinterpret_cast<double*>(Bn), 1, l);
            } else {
              e = gemm<TS>(c, false, false, bj, n2, bj, TS(-1), reinterpret_cast<const TS*>(w.Oh), b, A2, lda, TS(1),
                           Bn, l);
            }
          } else {
            e = convert<TS, double>(c, bj, bj, w.Oh, b, w.Tts, b);
            if (e == cudaSuccess) e = prod_nn<TS>(c, bj, n2, bj, TS(-1), w.Tts, b, A2, lda, TS(1), Bn, l);
          }
        }
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

template <typename TS>
size_t factor_ws_bytes(int m, int n, int b, int p, int num_sms, bool pivot, bool resample, int splitk_copies,
                       int f64tc) {
  return carve_factor<TS>(nullptr, m, n, b, pivot ? b + p : 1, num_sms, pivot && resample, splitk_copies, f64tc)
      .bytes;
}

template int factor_blocks<float>(rq_handle, void*, int, long long*, bool, int, int, float*, int, int, int, int,
                                  const float*, int, float*, int*, int*, cudaStream_t, const uint64_t*, int, int);
template int factor_blocks<double>(rq_handle, void*, int, long long*, bool, int, int, double*, int, int, int, int,
                                   const double*, int, double*, int*, int*, cudaStream_t, const uint64_t*, int, int);
template size_t factor_ws_bytes<float>(int, int, int, int, int, bool, bool, int, int);
template size_t factor_ws_bytes<double>(int, int, int, int, int, bool, bool, int, int);

namespace {

// The FP64 tensor-core mode of the handle's factorisations (0 when the driver
// has no tensor-map encoder).
int f64_tc_mode(rq_handle h) { return oz_supported() ? h->f64_tc : 0; }

// The handle's factorisation: grows the handle's workspace, then the block loop.
template <typename TS>
int run_factor(rq_handle h, bool pivot, int m, int n, TS* A, int lda, int b, int p, int k, const TS* Omega,
               int ldo, TS* tau, int* jpvt, int* info, cudaStream_t st, const uint64_t* rs_seed = nullptr) {
  const int f64tc = f64_tc_mode(h);
  int rc = ensure_ws(h, factor_ws_bytes<TS>(m, n, b, p, h->num_sms, pivot, rs_seed != nullptr, 16, f64tc));
  if (rc) return rc;
  return factor_blocks<TS>(h, h->ws, h->num_sms, &h->launches, pivot, m, n, A, lda, b, p, k, Omega, ldo, tau, jpvt,
                           info, st, rs_seed, 16, f64tc);
}

// Workspace of truncated RQRCP (Alg. 5).
template <typename TS>
struct TruncWs {
  unsigned int* bar;
  int* err;
  TS *B0, *B1, *Tts, *Wt, *Z, *P, *Wsel, *G, *X;
  double *S11, *Oh, *T, *cand, *pscr;
  int *jtmp, *chg, *swaps, *src;
  char* splitk;
  size_t splitk_bytes;
  size_t bytes;
};

template <typename TS>
TruncWs<TS> carve_trunc(void* base, int m, int n, int k, int b, int l, int num_sms) {
  Carver c(base);
  TruncWs<TS> w;
  w.bar = c.take<unsigned int>(4);
  w.err = reinterpret_cast<int*>(w.bar + 2);
  w.B0 = c.take<TS>((size_t)l * n);
  w.B1 = c.take<TS>((size_t)l * n);
  w.S11 = c.take<double>((size_t)b * b);
  w.Oh = c.take<double>((size_t)b * b);
  w.T = c.take<double>((size_t)b * b);
  w.Tts = c.take<TS>((size_t)b * b);
  w.Wt = c.take<TS>((size_t)k * n);
  w.Z = c.take<TS>((size_t)k * n);
  w.P = c.take<TS>((size_t)m * b);
  w.Wsel = c.take<TS>((size_t)k * b);
  w.G = c.take<TS>((size_t)b * k);
  w.X = c.take<TS>((size_t)b * n);
  w.jtmp = c.take<int>((size_t)2 * b);
  w.chg = c.take<int>((size_t)2 * b);
  w.swaps = c.take<int>((size_t)b);
  w.src = c.take<int>((size_t)n);
  w.cand = c.take<double>(sample_qrcp_scratch_doubles(l, num_sms));
  w.pscr = c.take<double>(panel_scratch_doubles(b, num_sms));
  w.splitk_bytes = splitk_bytes_for(b > k ? b : k, n, sizeof(TS));
  w.splitk = c.take<char>(w.splitk_bytes);
  w.bytes = align_up(c.off, 256);
  return w;
}

// Truncated RQRCP without trailing update, Alg. 5.  A is never written.  The
// accumulated inner products W^T = T^T Y^T A and the finished rows of R are
// kept in A's ORIGINAL column order (Z = R P^T), so no large array is ever
// permuted: the selected columns are gathered through jpvt, and the pivoted R
// is gathered once at the end.
template <typename TS>
cudaError_t sketch_gemm(const Ctx& c, bool mixed, int l, int n, int m, const TS* Omega, int ldo, const TS* A, int lda,
                        TS* B) {
  if constexpr (sizeof(TS) == sizeof(float)) {
    if (mixed) {
      if (tc_gemm_supported(Omega, ldo, A, lda)) return tc_gemm_nn_bf16(c, l, n, m, Omega, ldo, A, lda, B, l);
      return gemm_bf16_inputs(c, l, n, m, Omega, ldo, A, lda, B, l);
    }
  }
  return prod_nn<TS>(c, l, n, m, TS(1), Omega, ldo, A, lda, TS(0), B, l);
}

template <typename TS>
int run_trqrcp(rq_handle h, int m, int n, const TS* A, int lda, int b, int p, int k, const TS* Omega, int ldo,
               TS* Y, int ldy, TS* tau, TS* R, int ldr, int* jpvt, int* info, cudaStream_t st, TS** Z_out,
               TruncWs<TS>* ws_out, bool mixed = false) {
  const int l = b + p;
  TruncWs<TS> w = carve_trunc<TS>(nullptr, m, n, k, b, l, h->num_sms);
  int rc = ensure_ws(h, w.bytes);
  if (rc) return rc;
  w = carve_trunc<TS>(h->ws, m, n, k, b, l, h->num_sms);
  Ctx c{st, h->num_sms, &h->launches, w.err, w.bar, w.splitk, w.splitk_bytes};
  const double sz = sizeof(TS);
  cudaError_t e = cudaMemsetAsync(w.bar, 0, 16, st);
  if (e == cudaSuccess) e = cudaMemset2DAsync(Y, (size_t)ldy * sizeof(TS), 0, (size_t)m * sizeof(TS), k, st);
  if (e == cudaSuccess) e = iota(c, jpvt, n);
  if (e != cudaSuccess) return cuda_fail(h, e, "trqrcp setup");
  TS* Bc = w.B0;
  TS* Bn = w.B1;
  {
    Phase ph(h, st, RQ_PHASE_SKETCH, 2.0 * l * (double)m * n, sz * ((double)m * n + (double)l * m + (double)l * n));
    e = sketch_gemm<TS>(c, mixed, l, n, m, Omega, ldo, A, lda, Bc);
    if (e != cudaSuccess) return cuda_fail(h, e, "sketch");
  }
  for (int j0 = 0; j0 < k; j0 += b) {
    const int bj = (k - j0) < b ? (k - j0) : b;
    const int nt = n - j0, mt = m - j0, n2 = nt - bj;
    {
      Phase ph(h, st, RQ_PHASE_SAMPLE_QRCP, 4.0 * l * (double)nt * bj, 2.0 * sz * l * (double)nt);
      e = sample_qrcp<TS>(c, Bc, l, l, nt, bj, Bn, l, w.S11, b, w.swaps, w.src, w.chg, w.cand);
      if (e != cudaSuccess) return cuda_fail(h, e, "sample_qrcp");
    }
    {
      Phase ph(h, st, RQ_PHASE_PERMUTE, 0.0, 2.0 * sz * bj * (double)m);
      e = permute_index(c, bj, w.chg, w.src, jpvt + j0, w.jtmp);
      // selected columns of A - Y^[J-1] W_1^T (Alg. 5)
      if (e == cudaSuccess) e = gather_columns<TS>(c, A, lda, m, jpvt + j0, bj, w.P, m);
      if (e != cudaSuccess) return cuda_fail(h, e, "gather");
    }
    if (j0 > 0) {
      Phase ph(h, st, RQ_PHASE_OTHER, 2.0 * m * (double)j0 * bj, sz * ((double)m * j0 + 2.0 * m * bj));
      e = gather_columns<TS>(c, w.Wt, k, j0, jpvt + j0, bj, w.Wsel, k);
      if (e == cudaSuccess) e = gemm<TS>(c, false, false, m, bj, j0, TS(-1), Y, ldy, w.Wsel, k, TS(1), w.P, m);
      if (e != cudaSuccess) return cuda_fail(h, e, "selected columns");
    }
    {
      Phase ph(h, st, RQ_PHASE_PANEL, 2.0 * (double)mt * bj * bj, 2.0 * sz * (double)mt * bj);
      e = panel_qr<TS>(c, w.P + j0, m, mt, bj, tau + j0, Y + j0 + (size_t)j0 * ldy, ldy, w.T, b, w.pscr);
      if (e != cudaSuccess) return cuda_fail(h, e, "panel");
    }
    const TS* Tm;
    if (sizeof(TS) == sizeof(double)) {
      Tm = reinterpret_cast<const TS*>(w.T);
    } else {
      e = convert<TS, double>(c, bj, bj, w.T, b, w.Tts, b);
      if (e != cudaSuccess) return cuda_fail(h, e, "convert T");
      Tm = w.Tts;
    }
    const TS* Y2 = Y + j0 + (size_t)j0 * ldy;  // rows j0.. of the block's reflectors
    {
      // W_2^T = T_2^T (Y_2^T A - (Y_2^T Y_1) W_1^T)  (Alg. 5)
      Phase ph(h, st, RQ_PHASE_TRAILING,
               2.0 * bj * (double)mt * n + 2.0 * bj * (double)mt * j0 + 2.0 * bj * (double)j0 * n +
                   2.0 * bj * (double)bj * n,
               sz * ((double)mt * n + (double)mt * (bj + j0) + (double)(j0 + 2 * bj) * n));
      e = prod_tn_skinny<TS>(c, bj, n, mt, Y2, ldy, A + j0, lda, w.X, b);
      if (e == cudaSuccess && j0 > 0) {
        e = gemm<TS>(c, true, false, bj, j0, mt, TS(1), Y2, ldy, Y + j0, ldy, TS(0), w.G, b);
        if (e == cudaSuccess) e = gemm<TS>(c, false, false, bj, n, j0, TS(-1), w.G, b, w.Wt, k, TS(1), w.X, b);
      }
      if (e == cudaSuccess) e = gemm<TS>(c, true, false, bj, n, bj, TS(1), Tm, b, w.X, b, TS(0), w.Wt + j0, k);
      if (e != cudaSuccess) return cuda_fail(h, e, "inner products");
    }
    {
      // new rows of R from A - Y W^T (original column order)
      Phase ph(h, st, RQ_PHASE_OTHER, 2.0 * bj * (double)(j0 + bj) * n,
               sz * (2.0 * bj * (double)n + (double)(j0 + bj) * n + (double)bj * (j0 + bj)));
      e = convert<TS, TS>(c, bj, n, A + j0, lda, w.Z + j0, k);
      if (e == cudaSuccess)
        e = gemm<TS>(c, false, false, bj, n, j0 + bj, TS(-1), Y + j0, ldy, w.Wt, k, TS(1), w.Z + j0, k);
      if (e == cudaSuccess) e = trq_fix_new_rows<TS>(c, w.Z + j0, k, bj, j0, jpvt, w.P + j0, m);
      if (e != cudaSuccess) return cuda_fail(h, e, "R rows");
    }
    if (j0 + bj < k) {
      Phase ph(h, st, RQ_PHASE_SAMPLE_UPDATE, (double)bj * bj * bj / 3.0 + (double)bj * bj * n2,
               sz * 3.0 * bj * (double)n2);
      e = omegahat11<TS>(c, w.S11, b, w.P + j0, m, bj, w.Oh, b);
      if (e == cudaSuccess) e = sample_update_idx<TS>(c, bj, n2, w.Oh, b, w.Z + j0, k, jpvt + j0 + bj, Bn, l);
      if (e != cudaSuccess) return cuda_fail(h, e, "sample update");
    }
    TS* t = Bc;
    Bc = Bn;
    Bn = t;
  }
  {
    Phase ph(h, st, RQ_PHASE_OTHER, 0.0, 2.0 * sz * k * (double)n);
    if (R) {
      e = gather_columns<TS>(c, w.Z, k, k, jpvt, n, R, ldr);
      if (e == cudaSuccess) e = finish_info<TS>(c, R, ldr, k, info);
    } else {
      e = finish_info<TS>(c, w.P, m, 0, info);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "R gather");
  }
  if (Z_out) *Z_out = w.Z;
  if (ws_out) *ws_out = w;
  return RQ_OK;
}

// Blocked Householder QR of a tall rows x k matrix M (in place) with the
// explicit Q(:, 1:k) formed by applying the block reflectors backwards to
// [I; 0] and the upper triangular R copied out (Alg. 6's QR / LQ steps).
template <typename TS>
struct QrScratch {
  TS *Yall, *YT, *Wt, *Tts, *tau;
  double *Tall, *pscr;
};

template <typename TS>
cudaError_t qr_explicit(const Ctx& c, TS* M, int ldm, int rows, int k, int b, const QrScratch<TS>& s, TS* Q, int ldq,
                        TS* Rout, int ldr) {
  cudaError_t e = cudaMemset2DAsync(s.Yall, (size_t)rows * sizeof(TS), 0, (size_t)rows * sizeof(TS), k, c.stream);
  const int nb = (k + b - 1) / b;
  for (int J = 0; J < nb && e == cudaSuccess; ++J) {
    const int j0 = J * b, bj = (k - j0) < b ? (k - j0) : b, mt = rows - j0, n2 = k - j0 - bj;
    TS* Yj = s.Yall + j0 + (size_t)j0 * rows;
    double* Tj = s.Tall + (size_t)J * b * b;
    e = panel_qr<TS>(c, M + j0 + (size_t)j0 * ldm, ldm, mt, bj, s.tau + j0, Yj, rows, Tj, b, s.pscr);
    if (e != cudaSuccess || n2 <= 0) continue;
    const TS* Tm = reinterpret_cast<const TS*>(Tj);
    if (sizeof(TS) != sizeof(double)) {
      e = convert<TS, double>(c, bj, bj, Tj, b, s.Tts, b);
      Tm = s.Tts;
    }
    TS* M2 = M + j0 + (size_t)(j0 + bj) * ldm;
    if (e == cudaSuccess) e = gemm<TS>(c, false, false, mt, bj, bj, TS(1), Yj, rows, Tm, b, TS(0), s.YT, mt);
    if (e == cudaSuccess) e = prod_tn_skinny<TS>(c, bj, n2, mt, s.YT, mt, M2, ldm, s.Wt, b);
    if (e == cudaSuccess) e = prod_nn<TS>(c, mt, n2, bj, TS(-1), Yj, rows, s.Wt, b, TS(1), M2, ldm);
  }
  if (e == cudaSuccess && Rout) e = copy_upper<TS>(c, k, M, ldm, Rout, ldr);
  if (e == cudaSuccess) e = set_eye<TS>(c, rows, k, Q, ldq);
  for (int J = nb - 1; J >= 0 && e == cudaSuccess; --J) {
    const int j0 = J * b, bj = (k - j0) < b ? (k - j0) : b, mt = rows - j0, nc = k - j0;
    const TS* Yj = s.Yall + j0 + (size_t)j0 * rows;
    const double* Tj = s.Tall + (size_t)J * b * b;
    const TS* Tm = reinterpret_cast<const TS*>(Tj);
    if (sizeof(TS) != sizeof(double)) {
      e = convert<TS, double>(c, bj, bj, Tj, b, s.Tts, b);
      Tm = s.Tts;
    }
    TS* Qs = Q + j0 + (size_t)j0 * ldq;
    // Qs <- (I - Y T Y^T) Qs
    if (e == cudaSuccess) e = prod_tn_skinny<TS>(c, bj, nc, mt, Yj, rows, Qs, ldq, s.Wt, b);
    if (e == cudaSuccess) e = gemm<TS>(c, false, false, bj, nc, bj, TS(1), Tm, b, s.Wt, b, TS(0), s.YT, b);
    if (e == cudaSuccess) e = prod_nn<TS>(c, mt, nc, bj, TS(-1), Yj, rows, s.YT, b, TS(1), Qs, ldq);
  }
  return e;
}

// TUXV workspace: the TRQRCP workspace followed by the tail's buffers.
template <typename TS>
struct TuxvWs {
  TruncWs<TS> tr;
  TS *Ytr, *taut, *Zt, *Z1, *Uh, *Vh, *Tmp;
  QrScratch<TS> qs;
  double* jac;
  int *rot, *jp;
  size_t bytes;
};

constexpr int kMaxSweeps = 40;

template <typename TS>
TuxvWs<TS> carve_tuxv(void* base, int m, int n, int k, int b, int l, int num_sms) {
  TuxvWs<TS> w;
  w.tr = carve_trunc<TS>(base, m, n, k, b, l, num_sms);
  Carver c(base);
  c.off = w.tr.bytes;
  const int rows = m > n ? m : n;
  const int nb = (k + b - 1) / b;
  w.Ytr = c.take<TS>((size_t)m * k);
  w.taut = c.take<TS>((size_t)k);
  w.Zt = c.take<TS>((size_t)n * k);
  w.Z1 = c.take<TS>((size_t)m * k);
  w.Uh = c.take<TS>((size_t)k * k);
  w.Vh = c.take<TS>((size_t)k * k);
  w.Tmp = c.take<TS>((size_t)rows * k);
  w.qs.Yall = c.take<TS>((size_t)rows * k);
  w.qs.YT = c.take<TS>((size_t)rows * b);
  w.qs.Wt = c.take<TS>((size_t)b * k);
  w.qs.Tts = c.take<TS>((size_t)b * b);
  w.qs.tau = c.take<TS>((size_t)k);
  w.qs.Tall = c.take<double>((size_t)nb * b * b);
  w.qs.pscr = c.take<double>(panel_scratch_doubles(b, num_sms));
  w.jac = c.take<double>(jacobi_scratch_doubles(k));
  w.rot = c.take<int>(kMaxSweeps);
  w.jp = c.take<int>((size_t)n);
  w.bytes = align_up(c.off, 256);
  return w;
}

// TUXV, Alg. 6: TRQRCP -> Z0 = R P^T -> LQ of Z0 (QR of Z0^T, V explicit) ->
// Z1 = A V -> QR of Z1 (U explicit, X = R); for j = 2..jmax the refinement
// alternates (even j: Z = U^T A, LQ through the QR of A^T U, V explicit and
// X = R^T lower triangular; odd j: Z = A V, QR as for j = 1) -> optional core SVD.
template <typename TS>
int run_tuxv(rq_handle h, int m, int n, const TS* A, int lda, int b, int p, int k, const TS* Omega, int ldo, TS* U,
             int ldu, TS* X, int ldx, TS* V, int ldv, TS* sigma, int* info, cudaStream_t st, bool mixed = false,
             int jmax = 1) {
  const int l = b + p;
  TuxvWs<TS> w = carve_tuxv<TS>(nullptr, m, n, k, b, l, h->num_sms);
  int rc = ensure_ws(h, w.bytes);
  if (rc) return rc;
  w = carve_tuxv<TS>(h->ws, m, n, k, b, l, h->num_sms);
  // the TRQRCP part carves the same prefix of the workspace and leaves Z = R P^T there
  int* jp = w.jp;  // the column permutation P0 of TRQRCP (absorbed into V, not an output)
  TS* Z = nullptr;
  rc = run_trqrcp<TS>(h, m, n, A, lda, b, p, k, Omega, ldo, w.Ytr, m, w.taut, nullptr, k, jp, info, st, &Z, nullptr,
                      mixed);
  if (rc) return rc;
  Ctx c{st, h->num_sms, &h->launches, w.tr.err, w.tr.bar, w.tr.splitk, w.tr.splitk_bytes};
  const double sz = sizeof(TS);
  cudaError_t e;
  {
    // LQ of Z0 = R P^T through the QR of its transpose: V = Q(:, 1:k)
    Phase ph(h, st, RQ_PHASE_OTHER, 4.0 * n * (double)k * k, sz * 6.0 * n * (double)k);
    e = transpose<TS>(c, k, n, Z, k, w.Zt, n);
    if (e == cudaSuccess) e = qr_explicit<TS>(c, w.Zt, n, n, k, b, w.qs, V, ldv, nullptr, 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "LQ of Z0");
  }
  {
    // Z1 = A V(:, 1:k): one more pass over A (Alg. 6)
    Phase ph(h, st, RQ_PHASE_TRAILING, 2.0 * m * (double)n * k, sz * ((double)m * n + (double)n * k + (double)m * k));
    e = prod_nn<TS>(c, m, k, n, TS(1), A, lda, V, ldv, TS(0), w.Z1, m);
    if (e != cudaSuccess) return cuda_fail(h, e, "Z1 = A V");
  }
  {
    Phase ph(h, st, RQ_PHASE_OTHER, 4.0 * m * (double)k * k, sz * 6.0 * m * (double)k);
    e = qr_explicit<TS>(c, w.Z1, m, m, k, b, w.qs, U, ldu, X, ldx);
    if (e != cudaSuccess) return cuda_fail(h, e, "QR of Z1");
  }
  for (int j = 2; j <= jmax; ++j) {
    if (j % 2 == 0) {
      // Z^(j) = U^T A: its LQ through the QR of Z^T = A^T U (n x k); X = R^T
      Phase ph(h, st, RQ_PHASE_TRAILING, 2.0 * m * (double)n * k + 4.0 * n * (double)k * k,
               sz * ((double)m * n + (double)m * k + 6.0 * (double)n * k));
      e = prod_tn_skinny<TS>(c, n, k, m, A, lda, U, ldu, w.Zt, n);
      if (e == cudaSuccess) e = qr_explicit<TS>(c, w.Zt, n, n, k, b, w.qs, V, ldv, w.Vh, k);
      if (e == cudaSuccess) e = transpose<TS>(c, k, k, w.Vh, k, X, ldx);
      if (e != cudaSuccess) return cuda_fail(h, e, "LQ of U^T A");
    } else {
      // Z^(j) = A V and its QR, as for j = 1
      Phase ph(h, st, RQ_PHASE_TRAILING, 2.0 * m * (double)n * k + 4.0 * m * (double)k * k,
               sz * ((double)m * n + (double)n * k + 6.0 * (double)m * k));
      e = prod_nn<TS>(c, m, k, n, TS(1), A, lda, V, ldv, TS(0), w.Z1, m);
      if (e == cudaSuccess) e = qr_explicit<TS>(c, w.Z1, m, m, k, b, w.qs, U, ldu, X, ldx);
      if (e != cudaSuccess) return cuda_fail(h, e, "QR of A V");
    }
  }
  if (sigma) {
    // core SVD of X: U <- U Uh, V <- V Vh, X <- diag(sigma)
    Phase ph(h, st, RQ_PHASE_OTHER, 2.0 * (double)(m + n) * k * k, sz * 2.0 * (double)(m + n) * k);
    e = jacobi_svd<TS>(c, k, X, ldx, w.Uh, k, w.Vh, k, sigma, w.jac, w.rot, kMaxSweeps);
    if (e == cudaSuccess) e = gemm<TS>(c, false, false, m, k, k, TS(1), U, ldu, w.Uh, k, TS(0), w.Tmp, m);
    if (e == cudaSuccess) e = convert<TS, TS>(c, m, k, w.Tmp, m, U, ldu);
    if (e == cudaSuccess) e = gemm<TS>(c, false, false, n, k, k, TS(1), V, ldv, w.Vh, k, TS(0), w.Tmp, n);
    if (e == cudaSuccess) e = convert<TS, TS>(c, n, k, w.Tmp, n, V, ldv);
    if (e == cudaSuccess) e = fix_signs<TS>(c, m, n, k, U, ldu, V, ldv);
    if (e == cudaSuccess) e = set_diag<TS>(c, k, sigma, X, ldx);
    if (e != cudaSuccess) return cuda_fail(h, e, "core SVD");
  }
  e = finish_info<TS>(c, X, ldx, 0, info);
  if (e != cudaSuccess) return cuda_fail(h, e, "info");
  return RQ_OK;
}

int check_common(rq_handle h, int prec) {
  if (!valid(h)) return RQ_EHANDLE;
  if (prec != RQ_FP64 && prec != RQ_FP32 && prec != RQ_MIXED) return -2;
  return RQ_OK;
}

// ---- tile autotuner of the batched kernel ---------------------------------

constexpr int kTileSteps[RQ_TILE_STEPS] = {0, 16, 32, 64, 128, 256};
constexpr double kTileMargin = 0.99;  // a candidate must beat the incumbent by 1 %

struct TilePoint {
  int m, n;
  double ms;
};

// Time of the policy (m, n): from the memo, else from the caller's measure.
int tile_cost(rq_tiles_measure measure, void* user, std::vector<TilePoint>& memo, int m, int n, double* ms) {
  for (const TilePoint& p : memo)
    if (p.m == m && p.n == n) {
      *ms = p.ms;
      return RQ_OK;
    }
  const rq_batch_tiles t{m, n};
  double v = -1.0;
  const int rc = measure(user, &t, &v);
  if (rc != 0) return rc;
  if (!std::isfinite(v) || v < 0.0) return -1;
  memo.push_back({m, n, v});
  *ms = v;
  return RQ_OK;
}

// rq_tune_batched's measure: the fastest of `reps` launches of the batch
// under the policy, by CUDA events on the call's stream.
struct TuneCtx {
  rq_handle h;
  int prec, count;
  const rq_problem* problems;
  int max_m, max_n, max_k, max_b, max_p, reps;
  rq_stream stream;
  cudaEvent_t e0, e1;
};

int tune_measure(void* user, const rq_batch_tiles* t, double* ms) {
  TuneCtx& c = *static_cast<TuneCtx*>(user);
  c.h->tile_m = t->skinny_m;
  c.h->tile_n = t->skinny_n;
  const cudaStream_t st = static_cast<cudaStream_t>(c.stream);
  double fastest = -1.0;
  for (int r = 0; r < c.reps; ++r) {
    cudaError_t e = cudaEventRecord(c.e0, st);
    if (e != cudaSuccess) return cuda_fail(c.h, e, "rq_tune_batched: event");
    const int rc = rq_tuxv_batched(c.h, c.prec, c.count, c.problems, c.max_m, c.max_n, c.max_k, c.max_b, c.max_p,
                                   c.stream);
    if (rc != RQ_OK) return rc;
    float v = 0.f;
    e = cudaEventRecord(c.e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(c.e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&v, c.e0, c.e1);
    if (e != cudaSuccess) return cuda_fail(c.h, e, "rq_tune_batched: timing");
    if (fastest < 0.0 || v < fastest) fastest = v;
  }
  *ms = fastest;
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
  h->tile_m = kDefaultTile;
  h->tile_n = kDefaultTile;
  {
    // RQ_F64_TC: "0" keeps the FP64 block reflector products on the FP64 pipe,
    // "1" moves the update A2 -= Y W^T to the tensor cores; default: both products
    const char* v = getenv("RQ_F64_TC");
    h->f64_tc = (v && v[0] == '0') ? 0 : (v && v[0] == '1') ? 1 : 2;
  }
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
  if (b < 1 || b > RQ_MAX_B) return -7;
  if (p < 0 || b + p > RQ_MAX_L) return -8;
  if (!bytes) return -9;
  const int l = (op == RQ_OP_QR) ? 1 : b + p;
  if (op == RQ_OP_RQRCP || op == RQ_OP_QR || op == RQ_OP_RSRQRCP) {
    const bool rs = op == RQ_OP_RSRQRCP;
    *bytes = prec == RQ_FP64 ? carve_factor<double>(nullptr, m, n, b, l, h->num_sms, rs, 16, f64_tc_mode(h)).bytes
                             : carve_factor<float>(nullptr, m, n, b, l, h->num_sms, rs).bytes;
    return RQ_OK;
  }
  if (op == RQ_OP_TUXV) {
    if (k < 1) return -6;
    *bytes = prec == RQ_FP64 ? carve_tuxv<double>(nullptr, m, n, k, b, l, h->num_sms).bytes
                             : carve_tuxv<float>(nullptr, m, n, k, b, l, h->num_sms).bytes;
    return RQ_OK;
  }
  if (op == RQ_OP_TRQRCP) {
    if (k < 1) return -6;
    *bytes = prec == RQ_FP64 ? carve_trunc<double>(nullptr, m, n, k, b, l, h->num_sms).bytes
                             : carve_trunc<float>(nullptr, m, n, k, b, l, h->num_sms).bytes;
    return RQ_OK;
  }
  return RQ_ENOTIMPL;
}

int rq_set_workspace(rq_handle h, void* dptr, size_t bytes) {
  if (!valid(h)) return RQ_EHANDLE;
  if (dptr && reinterpret_cast<uintptr_t>(dptr) % 256 != 0) return fail(h, -2, "workspace not 256-byte aligned");
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
  if (b < 1 || b > RQ_MAX_B) return -7;
  if (p < 0 || b + p > RQ_MAX_L) return -8;
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

int rq_rsrqrcp(rq_handle h, int prec, int m, int n, void* A, int lda, int b, int p, int k, uint64_t seed, void* tau,
               int* jpvt, int* info, rq_stream stream) {
  int rc = check_common(h, prec);
  if (rc) return rc;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (!A) return -5;
  if (lda < m) return -6;
  if (b < 1 || b > RQ_MAX_B) return -7;
  if (p < 0 || b + p > RQ_MAX_L) return -8;
  if (k < 1 || k > (m < n ? m : n)) return -9;
  if (!tau) return -11;
  if (!jpvt) return -12;
  if (!info) return -13;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == RQ_FP64)
    return run_factor<double>(h, true, m, n, static_cast<double*>(A), lda, b, p, k, nullptr, 0,
                              static_cast<double*>(tau), jpvt, info, st, &seed);
  if (prec == RQ_FP32)
    return run_factor<float>(h, true, m, n, static_cast<float*>(A), lda, b, p, k, nullptr, 0,
                             static_cast<float*>(tau), jpvt, info, st, &seed);
  return fail(h, RQ_ENOTIMPL, "rq_rsrqrcp: RQ_MIXED is not provided for the full factorisation");
}

int rq_qr(rq_handle h, int prec, int m, int n, void* A, int lda, int b, void* tau, int* info, rq_stream stream) {
  int rc = check_common(h, prec);
  if (rc) return rc;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (!A) return -5;
  if (lda < m) return -6;
  if (b < 1 || b > RQ_MAX_B) return -7;
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
  int rc = check_common(h, prec);
  if (rc) return rc;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (!A) return -5;
  if (lda < m) return -6;
  if (b < 1 || b > RQ_MAX_B) return -7;
  if (p < 0 || b + p > RQ_MAX_L) return -8;
  if (k < 1 || k > (m < n ? m : n)) return -9;
  if (!Omega) return -10;
  if (ldo < b + p) return -11;
  if (!Y) return -12;
  if (ldy < m) return -13;
  if (!tau) return -14;
  if (!R) return -15;
  if (ldr < k) return -16;
  if (!jpvt) return -17;
  if (!info) return -18;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == RQ_FP64)
    return run_trqrcp<double>(h, m, n, static_cast<const double*>(A), lda, b, p, k,
                              static_cast<const double*>(Omega), ldo, static_cast<double*>(Y), ldy,
                              static_cast<double*>(tau), static_cast<double*>(R), ldr, jpvt, info, st, nullptr,
                              nullptr);
  return run_trqrcp<float>(h, m, n, static_cast<const float*>(A), lda, b, p, k, static_cast<const float*>(Omega), ldo,
                           static_cast<float*>(Y), ldy, static_cast<float*>(tau), static_cast<float*>(R), ldr, jpvt,
                           info, st, nullptr, nullptr, prec == RQ_MIXED);
}

int rq_tuxv(rq_handle h, int prec, int m, int n, const void* A, int lda, int b, int p, int k, const void* Omega,
            int ldo, void* U, int ldu, void* X, int ldx, void* V, int ldv, void* sigma, int* info,
            rq_stream stream) {
  int rc = check_common(h, prec);
  if (rc) return rc;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (!A) return -5;
  if (lda < m) return -6;
  if (b < 1 || b > RQ_MAX_B) return -7;
  if (p < 0 || b + p > RQ_MAX_L) return -8;
  if (k < 1 || k > (m < n ? m : n)) return -9;
  if (!Omega) return -10;
  if (ldo < b + p) return -11;
  if (!U) return -12;
  if (ldu < m) return -13;
  if (!X) return -14;
  if (ldx < k) return -15;
  if (!V) return -16;
  if (ldv < n) return -17;
  if (!info) return -19;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == RQ_FP64)
    return run_tuxv<double>(h, m, n, static_cast<const double*>(A), lda, b, p, k, static_cast<const double*>(Omega),
                            ldo, static_cast<double*>(U), ldu, static_cast<double*>(X), ldx, static_cast<double*>(V),
                            ldv, static_cast<double*>(sigma), info, st);
  return run_tuxv<float>(h, m, n, static_cast<const float*>(A), lda, b, p, k, static_cast<const float*>(Omega), ldo,
                         static_cast<float*>(U), ldu, static_cast<float*>(X), ldx, static_cast<float*>(V), ldv,
                         static_cast<float*>(sigma), info, st, prec == RQ_MIXED);
}

int rq_tuxv_iter(rq_handle h, int prec, int m, int n, const void* A, int lda, int b, int p, int k, int jmax,
                 const void* Omega, int ldo, void* U, int ldu, void* X, int ldx, void* V, int ldv, void* sigma,
                 int* info, rq_stream stream) {
  int rc = check_common(h, prec);
  if (rc) return rc;
  if (m < 1) return -3;
  if (n < 1) return -4;
  if (!A) return -5;
  if (lda < m) return -6;
  if (b < 1 || b > RQ_MAX_B) return -7;
  if (p < 0 || b + p > RQ_MAX_L) return -8;
  if (k < 1 || k > (m < n ? m : n)) return -9;
  if (jmax < 1) return -10;
  if (!Omega) return -11;
  if (ldo < b + p) return -12;
  if (!U) return -13;
  if (ldu < m) return -14;
  if (!X) return -15;
  if (ldx < k) return -16;
  if (!V) return -17;
  if (ldv < n) return -18;
  if (!info) return -20;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == RQ_FP64)
    return run_tuxv<double>(h, m, n, static_cast<const double*>(A), lda, b, p, k, static_cast<const double*>(Omega),
                            ldo, static_cast<double*>(U), ldu, static_cast<double*>(X), ldx, static_cast<double*>(V),
                            ldv, static_cast<double*>(sigma), info, st, false, jmax);
  return run_tuxv<float>(h, m, n, static_cast<const float*>(A), lda, b, p, k, static_cast<const float*>(Omega), ldo,
                         static_cast<float*>(U), ldu, static_cast<float*>(X), ldx, static_cast<float*>(V), ldv,
                         static_cast<float*>(sigma), info, st, prec == RQ_MIXED, jmax);
}

int rq_gaussian(rq_handle h, int prec, uint64_t seed, uint64_t substream, int l, int m, void* Omega, int ldo,
                rq_stream stream) {
  int rc = check_common(h, prec);
  if (rc) return rc;
  if (l < 1) return -5;
  if (m < 1) return -6;
  if (!Omega) return -7;
  if (ldo < l) return -8;
  Ctx c{static_cast<cudaStream_t>(stream), h->num_sms, &h->launches, nullptr, nullptr};
  cudaError_t e;
  {
    const double bytes = (double)l * m * (prec == RQ_FP64 ? 8.0 : 4.0);
    Phase ph(h, c.stream, RQ_PHASE_OTHER, 0.0, bytes);
    e = prec == RQ_FP64 ? gaussian<double>(c, seed, substream, l, m, static_cast<double*>(Omega), ldo)
                        : gaussian<float>(c, seed, substream, l, m, static_cast<float*>(Omega), ldo);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "rq_gaussian");
  return RQ_OK;
}

int rq_tuxv_batched(rq_handle h, int prec, int count, const rq_problem* problems, int max_m, int max_n, int max_k,
                    int max_b, int max_p, rq_stream stream) {
  if (!valid(h)) return RQ_EHANDLE;
  if (prec != RQ_FP32 && prec != RQ_MIXED) return prec == RQ_FP64 ? fail(h, RQ_ENOTIMPL, "batched FP64") : -2;
  if (count < 0) return -3;
  if (count > 0 && !problems) return -4;
  if (max_m < 1) return -5;
  if (max_n < 1) return -6;
  if (max_k < 1 || max_k > (max_m < max_n ? max_m : max_n)) return -7;
  if (!batched_limits_ok(max_b, 0)) return -8;
  if (max_p < 0 || !batched_limits_ok(max_b, max_p)) return -9;
  if (count == 0) return RQ_OK;
  const int slots = batched_slots(h->num_sms);
  const size_t slot = batched_slot_bytes(max_m, max_n, max_k, max_b, max_p);
  const size_t need = 256 + (size_t)slots * slot;
  int rc = ensure_ws(h, need);
  if (rc) return rc;
  char* base = static_cast<char*>(h->ws);
  int* counter = reinterpret_cast<int*>(base);
  unsigned int* bar = reinterpret_cast<unsigned int*>(base + 16);
  Ctx c{static_cast<cudaStream_t>(stream), h->num_sms, &h->launches, reinterpret_cast<int*>(base + 32), bar};
  cudaError_t e;
  {
    Phase ph(h, c.stream, RQ_PHASE_OTHER, 0.0, 0.0);
    e = tuxv_batched(c, count, problems, base + 256, slot, slots, counter, prec == RQ_MIXED, h->tile_m, h->tile_n);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "rq_tuxv_batched");
  return RQ_OK;
}

int rq_gemm_bf16(rq_handle h, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
                 int ldc, int* info, rq_stream stream) {
  if (!valid(h)) return RQ_EHANDLE;
  if (M < 1) return -2;
  if (N < 1) return -3;
  if (K < 1) return -4;
  if (!A) return -5;
  if (lda < M) return -6;
  if (!B) return -7;
  if (ldb < K) return -8;
  if (!C) return -9;
  if (ldc < M) return -10;
  {
    // C may not overlap A or B (their column-major extents, in bytes)
    const auto lo = [](const float* x) { return reinterpret_cast<uintptr_t>(x); };
    const auto hi = [](const float* x, int ld, int rows, int cols) {
      return reinterpret_cast<uintptr_t>(x) + sizeof(float) * ((size_t)ld * (cols - 1) + rows);
    };
    const uintptr_t c0 = lo(C), c1 = hi(C, ldc, M, N);
    if ((c0 < hi(A, lda, M, K) && lo(A) < c1) || (c0 < hi(B, ldb, K, N) && lo(B) < c1)) return -9;
  }
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool tc = tc_gemm_supported(A, lda, B, ldb);
  // split-K scratch on the tensor cores: one FP32 partial of C per chunk of
  // at most 1024 K steps (the chunk rule of the tensor-core product)
  const size_t chunks = (tc && K > 1024) ? (size_t)(K + 1023) / 1024 : 0;
  const size_t split = chunks * sizeof(float) * (size_t)M * (size_t)N;
  const int rc = ensure_ws(h, 256 + split);
  if (rc) return rc;
  char* base = static_cast<char*>(h->ws);
  unsigned int* bar = reinterpret_cast<unsigned int*>(base);
  int* err = reinterpret_cast<int*>(bar + 2);
  Ctx c{st, h->num_sms, &h->launches, err, bar, chunks ? base + 256 : nullptr, split};
  cudaError_t e;
  {
    Phase ph(h, st, RQ_PHASE_SKETCH, 2.0 * M * N * (double)K,
             4.0 * ((double)M * K + (double)K * N + (double)M * N));
    e = cudaMemsetAsync(bar, 0, 16, st);
    if (e == cudaSuccess)
      e = tc ? tc_gemm_nn_bf16(c, M, N, K, A, lda, B, ldb, C, ldc)
             : gemm_bf16_inputs(c, M, N, K, A, lda, B, ldb, C, ldc);
    if (e == cudaSuccess && info) e = cudaMemcpyAsync(info, err, sizeof(int), cudaMemcpyDeviceToDevice, st);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "rq_gemm_bf16");
  return RQ_OK;
}

int rq_gemm_f64(rq_handle h, int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
                int ldc, int* info, rq_stream stream) {
  if (!valid(h)) return RQ_EHANDLE;
  if (M < 1) return -2;
  if (N < 1) return -3;
  if (K < 1) return -4;
  if (!A) return -5;
  if (lda < M) return -6;
  if (!B) return -7;
  if (ldb < K) return -8;
  if (!C) return -9;
  if (ldc < M) return -10;
  {
    const auto lo = [](const double* x) { return reinterpret_cast<uintptr_t>(x); };
    const auto hi = [](const double* x, int ld, int rows, int cols) {
      return reinterpret_cast<uintptr_t>(x) + sizeof(double) * ((size_t)ld * (cols - 1) + rows);
    };
    const uintptr_t c0 = lo(C), c1 = hi(C, ldc, M, N);
    if ((c0 < hi(A, lda, M, K) && lo(A) < c1) || (c0 < hi(B, ldb, K, N) && lo(B) < c1)) return -9;
  }
  if (!oz_supported()) return fail(h, RQ_ENOTIMPL, "rq_gemm_f64: no tensor-map encoder in this driver");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int Mp = oz_rows_pad(M, true), Np = oz_rows_pad(N, false), Kp = oz_k_pad(K);
  Carver cv(nullptr);
  OzWs z = carve_oz(cv, Mp, Np, Kp, (size_t)M * N);
  const int rc = ensure_ws(h, align_up(cv.off, 256));
  if (rc) return rc;
  Carver cw(h->ws);
  z = carve_oz(cw, Mp, Np, Kp, (size_t)M * N);
  Ctx c{st, h->num_sms, &h->launches, z.err, z.bar, z.split, z.split_bytes};
  cudaError_t e;
  {
    Phase ph(h, st, RQ_PHASE_OTHER, 2.0 * M * N * (double)K, 8.0 * ((double)M * K + (double)K * N + (double)M * N));
    e = cudaMemsetAsync(z.bar, 0, 16, st);
    if (e == cudaSuccess) e = oz_slice(c, false, M, K, A, lda, Mp, Kp, z.Ap, z.ea);
    if (e == cudaSuccess) e = oz_slice(c, true, N, K, B, ldb, Np, Kp, z.Bp, z.eb);
    if (e == cudaSuccess) e = oz_gemm(c, M, N, K, z.Ap, Mp, z.ea, z.Bp, Np, z.eb, Kp, 1.0, 0.0, C, 1, ldc);
    if (e == cudaSuccess && info) e = cudaMemcpyAsync(info, z.err, sizeof(int), cudaMemcpyDeviceToDevice, st);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "rq_gemm_f64");
  return RQ_OK;
}

int rq_set_batch_tiles(rq_handle h, const rq_batch_tiles* t) {
  if (!valid(h)) return RQ_EHANDLE;
  if (!t || t->skinny_m < 0 || t->skinny_n < 0) return -2;
  h->tile_m = t->skinny_m;
  h->tile_n = t->skinny_n;
  return RQ_OK;
}

int rq_get_batch_tiles(rq_handle h, rq_batch_tiles* t) {
  if (!valid(h)) return RQ_EHANDLE;
  if (!t) return -2;
  t->skinny_m = h->tile_m;
  t->skinny_n = h->tile_n;
  return RQ_OK;
}

int rq_tiles_search(rq_tiles_measure measure, void* user, const rq_batch_tiles* start, int passes,
                    rq_batch_tiles* best, double* best_ms) {
  if (!measure) return -1;
  if (start && (start->skinny_m < 0 || start->skinny_n < 0)) return -3;
  if (passes < 0) return -4;
  if (!best) return -5;
  std::vector<TilePoint> memo;
  int cur[2] = {start ? start->skinny_m : kDefaultTile, start ? start->skinny_n : kDefaultTile};
  double cur_ms = 0.0;
  int rc = tile_cost(measure, user, memo, cur[0], cur[1], &cur_ms);
  if (rc != RQ_OK) return rc;
  for (int pass = 0; pass < passes; ++pass) {
    bool moved = false;
    for (int axis = 0; axis < 2; ++axis) {
      for (int v : kTileSteps) {
        if (v == cur[axis]) continue;
        int cand[2] = {cur[0], cur[1]};
        cand[axis] = v;
        double ms = 0.0;
        rc = tile_cost(measure, user, memo, cand[0], cand[1], &ms);
        if (rc != RQ_OK) return rc;
        if (ms < kTileMargin * cur_ms) {
          cur[0] = cand[0];
          cur[1] = cand[1];
          cur_ms = ms;
          moved = true;
        }
      }
    }
    if (!moved) break;
  }
  best->skinny_m = cur[0];
  best->skinny_n = cur[1];
  if (best_ms) *best_ms = cur_ms;
  return RQ_OK;
}

int rq_tune_batched(rq_handle h, int prec, int count, const rq_problem* problems, int max_m, int max_n, int max_k,
                    int max_b, int max_p, int reps, int passes, rq_stream stream, rq_batch_tiles* best,
                    double* best_ms) {
  if (!valid(h)) return RQ_EHANDLE;
  if (reps < 1) return -10;
  if (passes < 0) return -11;
  // validates arguments 2-9, sizes the workspace and warms up
  int rc = rq_tuxv_batched(h, prec, count, problems, max_m, max_n, max_k, max_b, max_p, stream);
  if (rc != RQ_OK) return rc;
  const rq_batch_tiles old{h->tile_m, h->tile_n};
  rq_batch_tiles chosen = old;
  double ms = 0.0;
  if (count > 0) {
    TuneCtx c{h, prec, count, problems, max_m, max_n, max_k, max_b, max_p, reps, stream, nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&c.e0);
    if (e == cudaSuccess) {
      e = cudaEventCreate(&c.e1);
      if (e != cudaSuccess) cudaEventDestroy(c.e0);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "rq_tune_batched: event");
    rc = rq_tiles_search(tune_measure, &c, &old, passes, &chosen, &ms);
    cudaEventDestroy(c.e0);
    cudaEventDestroy(c.e1);
    if (rc != RQ_OK) {
      h->tile_m = old.skinny_m;
      h->tile_n = old.skinny_n;
      return rc;
    }
  }
  h->tile_m = chosen.skinny_m;
  h->tile_n = chosen.skinny_n;
  if (best) *best = chosen;
  if (best_ms) *best_ms = ms;
  return RQ_OK;
}

}  // extern "C"
