// Internal launcher declarations (host side) for the RQRCP library kernels.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>

namespace rq {

struct Ctx {
  cudaStream_t stream;
  int num_sms;
  long long* launches;  // launch counter of the handle
  int* err;             // device error word (RQ_ETIMEOUT from bounded waits)
  unsigned int* bar;    // device grid barrier {count, generation}
};

// C = alpha * op(A) * op(B) + beta * C, column-major (SIMT tiles).
template <typename T>
cudaError_t gemm(const Ctx& c, bool ta, bool tb, int M, int N, int K, T alpha, const T* A, int lda,
                 const T* B, int ldb, T beta, T* C, int ldc);

// Partial QRCP of the sample (l x nt): `steps` pivots, norms downdated.
// Writes S11 (steps x steps, FP64, ld lds), swaps[steps], src[nt] (old position
// of the column now at each new position) and the reordered trailing sample
// Bn (l x (nt - steps), ld ldbn): rows 0..steps-1 = S12, the rest = S22.
// `cand` is scratch of sample_qrcp_scratch(l) * (2 * num_sms) doubles.
// chg (2*steps): the positions whose column changes (-1 entries are unused).
template <typename TS>
cudaError_t sample_qrcp(const Ctx& c, const TS* B, int ldb, int l, int nt, int steps, TS* Bn,
                        int ldbn, double* S11, int lds, int* swaps, int* src, int* chg, double* cand);
size_t sample_qrcp_scratch_doubles(int l, int num_sms);

// Householder QR of the mt x bj panel P (in place: R above, v below), tau,
// explicit Y (mt x bj, ld ldy) and the compact-WY T (bj x bj, FP64, ld ldt).
template <typename TS>
cudaError_t panel_qr(const Ctx& c, TS* P, int ldp, int mt, int bj, TS* tau, TS* Y, int ldy,
                     double* T, int ldt, double* scratch);
size_t panel_scratch_doubles(int bj, int num_sms);

// Apply the block's column permutation to the columns of A (m rows) and to
// jpvt: for every listed position e (chg), column e <- old column src[e].
// tmp holds 2*steps columns of m entries, jtmp 2*steps ints.
template <typename TS>
cudaError_t permute_columns(const Ctx& c, TS* A, int lda, int m, int steps, const int* chg,
                            const int* src, int* jpvt, TS* tmp, int* jtmp);

// Omegahat11 = S11 * R11^{-1} (bj x bj upper triangular), FP64.
template <typename TS>
cudaError_t omegahat11(const Ctx& c, const double* S11, int lds, const TS* R11, int ldr, int bj,
                       double* Oh, int ldo);

// B1 (bj x n2, ld ldb) -= Oh (bj x bj, FP64) * R12 (bj x n2, ld ldr).
template <typename TS>
cudaError_t sample_update(const Ctx& c, int bj, int n2, const double* Oh, int ldo, const TS* R12,
                          int ldr, TS* B1, int ldb);

cudaError_t iota(const Ctx& c, int* v, int n);
// info = RQ_ETIMEOUT if the device error word is set, else the first j with
// A(j-1, j-1) == 0 (1-based), else 0.
template <typename TS>
cudaError_t finish_info(const Ctx& c, const TS* A, int lda, int k, int* info);
template <typename TD, typename TS>
cudaError_t convert(const Ctx& c, int rows, int cols, const TS* src, int lds, TD* dst, int ldd);

}  // namespace rq
