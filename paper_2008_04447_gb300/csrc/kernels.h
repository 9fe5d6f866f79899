// Internal launcher declarations (host side) for the RQRCP library kernels.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "rqrcp.h"

namespace rq {

struct Ctx {
  cudaStream_t stream;
  int num_sms;
  long long* launches;  // launch counter of the handle
  int* err;             // device error word (RQ_ETIMEOUT from bounded waits)
  unsigned int* bar;    // device grid barrier {count, generation}
  void* splitk = nullptr;       // scratch for split-K partial products (nullptr: no split)
  size_t splitk_bytes = 0;
};

// C = alpha * op(A) * op(B) + beta * C, column-major (SIMT tiles).
template <typename T>
cudaError_t gemm(const Ctx& c, bool ta, bool tb, int M, int N, int K, T alpha, const T* A, int lda,
                 const T* B, int ldb, T beta, T* C, int ldc);

// C = A B with both inputs rounded to BF16 (products exact in FP32), FP32
// accumulation: the reduced-precision sketch.
cudaError_t gemm_bf16_inputs(const Ctx& c, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                             float* C, int ldc);

// C (M x N) = alpha * sum_z P_z + beta * C, z in order (P_z: M x N, stride pzs).
cudaError_t splitk_reduce_f32(const Ctx& c, int M, int N, int S, const float* P, size_t pzs, float alpha, float beta,
                              float* C, int ldc);

// Tensor-core FP32 GEMM, C = alpha A^T B + beta C (A: K x M, B: K x N, column-major,
// i.e. both K-major), 3xTF32 when split3; C^T stored when transC.  Needs
// 16-byte aligned bases and leading dimensions that are multiples of 4
// (tc_gemm_supported); splits K through c.splitk when the tiles are few.
bool tc_gemm_supported(const float* A, int lda, const float* B, int ldb);
cudaError_t tc_gemm_tn(const Ctx& c, int M, int N, int K, float alpha, const float* A, int lda, const float* B,
                       int ldb, float beta, float* C, int ldc, bool transC, bool split3);
// Same with A M-major (M x K column-major): C = alpha A B + beta C.
cudaError_t tc_gemm_nn(const Ctx& c, int M, int N, int K, float alpha, const float* A, int lda, const float* B,
                       int ldb, float beta, float* C, int ldc, bool split3);
// C = A B (A M x K, M-major; B K x N, K-major) with both inputs rounded to
// bfloat16 and FP32 accumulation on the tensor cores (K chunks of at most 1024).
cudaError_t tc_gemm_nn_bf16(const Ctx& c, int M, int N, int K, const float* A, int lda, const float* B, int ldb,
                            float* C, int ldc);

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

// dst(:, i) = src(:, idx[i]), i < count (rows entries per column).
template <typename TS>
cudaError_t gather_columns(const Ctx& c, const TS* src, int lds, int rows, const int* idx, int count, TS* dst,
                           int ldd);

// The permutation of permute_columns applied to an index vector only.
cudaError_t permute_index(const Ctx& c, int steps, const int* chg, const int* src, int* v, int* tmp);

// TRQRCP: in the new rows Zb (bj x n, original column order) set the columns
// chosen in earlier blocks (positions < j0) to zero and the block's own
// columns (positions j0..j0+bj-1) to R11 (upper triangle of R11, ld ldr).
template <typename TS>
cudaError_t trq_fix_new_rows(const Ctx& c, TS* Zb, int ldz, int bj, int j0, const int* jpvt, const TS* R11,
                             int ldr);

// B1 (bj x n2) -= Oh * R12 with R12(:, t) = Zb(:, idx[t]).
template <typename TS>
cudaError_t sample_update_idx(const Ctx& c, int bj, int n2, const double* Oh, int ldo, const TS* Zb, int ldz,
                              const int* idx, TS* B1, int ldb);

// TUXV tail helpers.
template <typename TS>
cudaError_t transpose(const Ctx& c, int rows, int cols, const TS* s, int lds, TS* d, int ldd);
template <typename TS>
cudaError_t set_eye(const Ctx& c, int rows, int cols, TS* d, int ldd);
template <typename TS>
cudaError_t copy_upper(const Ctx& c, int k, const TS* s, int lds, TS* d, int ldd);
// One-sided Jacobi SVD of the k x k X: X = Uh diag(sigma) Vh^T, sigma descending.
// scratch: jacobi_scratch_doubles(k); rot: max_sweeps ints.
size_t jacobi_scratch_doubles(int k);
template <typename TS>
cudaError_t jacobi_svd(const Ctx& c, int k, const TS* X, int ldx, TS* Uh, int ldu, TS* Vh, int ldv, TS* sigma,
                       double* scratch, int* rot, int max_sweeps);
// Make the largest-magnitude entry of each column of V positive (U follows).
template <typename TS>
cudaError_t fix_signs(const Ctx& c, int m, int n, int k, TS* U, int ldu, TS* V, int ldv);
template <typename TS>
cudaError_t set_diag(const Ctx& c, int k, const TS* s, TS* X, int ldx);

// Batched TRQRCP + TUXV (persistent, one CTA per problem at a time).
size_t batched_slot_bytes(int max_m, int max_n, int max_k, int max_b, int max_p);
int batched_limits_ok(int max_b, int max_p);
int batched_slots(int num_sms);
// skinny_m, skinny_n: the block GEMMs' tile policy (rq_batch_tiles).
cudaError_t tuxv_batched(const Ctx& c, int count, const rq_problem* problems, char* ws, size_t slot_bytes, int slots,
                         int* counter, bool mixed, int skinny_m, int skinny_n);

cudaError_t iota(const Ctx& c, int* v, int n);

// Omega (l x m, leading dimension ldo) = the Gaussian draws of (seed,
// substream): Philox4x32-10 counters keyed by the seed, Box-Muller in FP64.
template <typename T>
cudaError_t gaussian(const Ctx& c, uint64_t seed, uint64_t substream, int l, int m, T* Omega, int ldo);
// info = RQ_ETIMEOUT if the device error word is set, else the first j with
// A(j-1, j-1) == 0 (1-based), else 0.
template <typename TS>
cudaError_t finish_info(const Ctx& c, const TS* A, int lda, int k, int* info);
template <typename TD, typename TS>
cudaError_t convert(const Ctx& c, int rows, int cols, const TS* src, int lds, TD* dst, int ldd);

// FP64 products on the bfloat16 tensor cores (f64_tc.cu).  An operand is held
// as eight bfloat16 slice planes [8][rows_pad][k_pad] plus one exponent per
// row; oz_slice makes them from an FP64 matrix whose operand rows are its
// columns (k_along_columns: row r's entries at src[k + r ld]) or its rows
// (src[r + k ld]).  oz_gemm: C = alpha A B^T + beta C, C element (i, j) at
// C[i rs + j cs]; A M x K (rows padded to 128), B N x K (rows padded to 64).
int oz_rows_pad(int rows, bool a_side);
int oz_k_pad(int K);
size_t oz_plane_bytes(int rows_pad, int k_pad);
bool oz_supported();
cudaError_t oz_slice(const Ctx& c, bool k_along_columns, int R, int K, const double* src, long long ld, int Rp, int Kp,
                     uint16_t* planes, int* e);
cudaError_t oz_gemm(const Ctx& c, int M, int N, int K, const uint16_t* Ap, int Mp, const int* ea, const uint16_t* Bp,
                    int Np, const int* eb, int Kp, double alpha, double beta, double* C, long long rs, long long cs);

// Blocked Householder QR (Alg. 4 with pivot, unpivoted without) over a
// caller-provided workspace of factor_ws_bytes bytes; h may be NULL.  Shared by
// rq_rqrcp / rq_qr / rq_rsrqrcp (the handle's workspace) and rq_rqrcp_noalloc
// (a fixed device array), so both run the same block loop.
// f64tc (FP64 only): 0 block reflector products on the FP64 pipe, 1 the update
// A2 -= Y W^T on the bfloat16 tensor cores (oz_gemm), 2 also W^T = (Y T)^T A2.
template <typename TS>
int factor_blocks(rq_handle h, void* ws, int num_sms, long long* launches, bool pivot, int m, int n, TS* A, int lda,
                  int b, int p, int k, const TS* Omega, int ldo, TS* tau, int* jpvt, int* info, cudaStream_t st,
                  const uint64_t* rs_seed, int splitk_copies, int f64tc);
template <typename TS>
size_t factor_ws_bytes(int m, int n, int b, int p, int num_sms, bool pivot, bool resample, int splitk_copies,
                       int f64tc);

}  // namespace rq
