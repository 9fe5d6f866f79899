/*
 * rqrcp.h -- C ABI of the GB300 (sm_103a) RQRCP / TRQRCP / TUXV library.
 *
 * Randomized QR with column pivoting and its truncated low-rank forms,
 * after Duersch & Gu, "Randomized Projection for Rank-Revealing Matrix
 * Factorizations and Low-Rank Approximations" (arXiv 2008.04447).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Matrices are column-major with LAPACK leading dimensions (element (i, j)
 *   of an m x n matrix X with leading dimension ldx is X[i + j*ldx],
 *   ldx >= max(1, rows)).
 * - Every matrix / vector pointer is a DEVICE pointer owned by the caller;
 *   the library never frees or retains it beyond the call's stream work.
 * - Element type follows `prec`: RQ_FP64 -> double, RQ_FP32 and RQ_MIXED ->
 *   float (A, Omega, tau, R, Y, U, X, V, sigma).  Index vectors are int32.
 * - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *   stream); rq_profile_read and rq_tune_batched synchronise, as their
 *   comments say.  The return value reports argument / launch problems found
 *   on the host; numerical status is written to the caller's device `info`
 *   word.
 * - The library owns only its workspace, held in the handle (see
 *   rq_workspace_size / rq_set_workspace).  No exception crosses the ABI.
 * - A handle serves one host thread at a time (its workspace is not locked);
 *   separate handles may be used from separate threads on separate streams at
 *   once, as the continuous-batching server's lanes are.  Kernel launch
 *   settings (shared-memory limits, occupancy) are taken once per process for
 *   the device current at the first call: one GPU per process.
 *
 * Return codes: RQ_OK (0); -i when argument i (1-based, counting the handle
 * as argument 1) is invalid; or one of the named negative codes below.
 */
#ifndef RQRCP_H
#define RQRCP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RQ_OK 0
#define RQ_ENOMEM (-1000)   /* workspace allocation failed / caller workspace too small */
#define RQ_ECUDA (-1001)    /* a CUDA launch or runtime call failed (see rq_last_error) */
#define RQ_ETIMEOUT (-1002) /* a bounded device-side wait ran out (kernel returned early) */
#define RQ_ENOTIMPL (-1003) /* combination of arguments not supported by this build */
#define RQ_EHANDLE (-1004)  /* NULL or destroyed handle */
#define RQ_ETOOBIG (-1005)  /* rq_rqrcp_noalloc: the problem needs more scratch than the fixed array */

/* Arithmetic / storage precision of a call. */
#define RQ_FP64 0  /* everything FP64 */
#define RQ_FP32 1  /* FP32 storage and updates (3xTF32 tensor-core products); the Householder
                      scalars, T and squared norms carried with FP64 accuracy */
#define RQ_MIXED 2 /* as RQ_FP32, with the sketch formed from bfloat16-rounded Omega and A
                      (FP32 accumulation); core SVD in FP64 */

/* Operations, for rq_workspace_size. */
#define RQ_OP_RQRCP 0
#define RQ_OP_TRQRCP 1
#define RQ_OP_TUXV 2
#define RQ_OP_QR 3
#define RQ_OP_RSRQRCP 4

typedef struct rq_handle_s* rq_handle;
typedef void* rq_stream; /* cudaStream_t */

/* Create a handle bound to the current CUDA device.  Ownership of *h passes
 * to the caller, who releases it with rq_destroy. */
int rq_create(rq_handle* h);

/* Release the handle and any workspace the library allocated for it.  The
 * caller must make sure no work that uses the handle is still running. */
int rq_destroy(rq_handle h);

/* Bytes of device workspace that operation `op` needs for these sizes:
 * RQ_OP_RQRCP (rq_rqrcp), RQ_OP_RSRQRCP, RQ_OP_QR (k ignored), RQ_OP_TRQRCP
 * and RQ_OP_TUXV (rq_tuxv and rq_tuxv_iter).  The batched call sizes its
 * slots from its max_* bounds, rq_gemm_bf16 needs 256 bytes plus, on the
 * tensor cores with K > 1024, 4 M N ceil(K / 1024) bytes, and
 * rq_rqrcp_noalloc uses no handle. */
int rq_workspace_size(rq_handle h, int op, int prec, int m, int n, int k, int b, int p,
                      size_t* bytes);

/* Give the handle a caller-owned device workspace (NULL / 0 to go back to
 * library-managed workspace).  dptr must be 256-byte aligned, as cudaMalloc's
 * are (the workspace holds FP64 arrays and tensor-map operands at 256-byte
 * offsets from it): another address returns -2.  The caller keeps ownership
 * and must keep it alive while work issued through the handle runs.  A call
 * whose need exceeds a caller workspace returns RQ_ENOMEM before launching
 * anything.  Without a caller workspace the library grows its own with
 * cudaMalloc (synchronising the device). */
int rq_set_workspace(rq_handle h, void* dptr, size_t bytes);

/* Copy the last host-side error message of this handle into buf. */
int rq_last_error(rq_handle h, char* buf, size_t len);

/* Number of this library's kernel launches issued through the handle so far. */
long long rq_launch_count(rq_handle h);

/* Phases of the factorisations, for per-phase timing. */
#define RQ_PHASE_SKETCH 0        /* B = Omega A, the initial sample (Alg. 4) */
#define RQ_PHASE_SAMPLE_QRCP 1   /* block pivots from the sample (Sec. 3.2) */
#define RQ_PHASE_PERMUTE 2       /* column permutation of A and jpvt */
#define RQ_PHASE_PANEL 3         /* Householder panel + compact-WY T */
#define RQ_PHASE_TRAILING 4      /* W^T = T^T Y^T A2, A2 -= Y W^T (block reflector) */
#define RQ_PHASE_SAMPLE_UPDATE 5 /* Eq. (update1) */
#define RQ_PHASE_OTHER 6         /* TRQRCP / TUXV products, small kernels */
#define RQ_PHASE_SLICE 7         /* FP64 operands cut into bfloat16 slices for the tensor cores */
#define RQ_NUM_PHASES 8

/* Enable (1) or disable (0) per-phase timing: CUDA events are recorded on the
 * call's stream around each phase.  Adds two event records per phase. */
int rq_profile_enable(rq_handle h, int enable);

/* Synchronise on the recorded events and return, per phase (arrays of
 * `nphases` entries, any may be NULL): elapsed milliseconds, algorithmic
 * floating-point operations, algorithmic HBM bytes and kernel launches,
 * summed since the last read.  Clears the accumulated records. */
int rq_profile_read(rq_handle h, int nphases, double* ms, double* flops, double* bytes,
                    long long* launches);

/* Largest block size b and sample rank l = b + p of the single-problem
 * calls (larger values return the argument's index).  Blocks of up to 64
 * columns run on the register-resident panel kernel; larger ones on the
 * general panel kernel, whose shared-memory tile (b^2 + b ceil(m / SMs)
 * values) must fit one CTA: about b <= 110 for FP64 at m = 16384.  A panel
 * that does not fit returns RQ_ENOTIMPL when the factorisation reaches it,
 * with A partly updated. */
#define RQ_MAX_B 256
#define RQ_MAX_L 384

/*
 * rq_rqrcp -- Randomized QR with column pivoting, Alg. 4 (Sec. 3.4), with the
 * sample update formula Eq. (update1).
 *
 *   A      [in/out] m x n, lda >= m.  On exit: rows 0..k-1 on and above the
 *          diagonal hold R (k x n upper trapezoidal, pivoted column order);
 *          below the diagonal of columns 0..k-1 the Householder vectors v
 *          (v_1 = 1 implicit, H = I - v tau v^T); the block A[k:m, k:n] holds
 *          the trailing matrix (R22) left by the last block update.
 *   b      block size (pivots per sample), 1 <= b <= RQ_MAX_B.
 *   p      oversampling; the sample has l = b + p rows, p >= 0, l <= RQ_MAX_L.
 *   k      factorisation rank, 1 <= k <= min(m, n).
 *   Omega  l x m Gaussian compression matrix (ldo >= l), read only; the same
 *          Omega serves every block through the update formula.
 *   tau    k reflector coefficients (out).
 *   jpvt   n int32 (out): 0-based column permutation, A_in[:, jpvt] = Q R.
 *   info   device int32 (out): 0, or j > 0 when R(j-1, j-1) is exactly zero
 *          (first such j; the factorisation still completes).
 * Precisions: RQ_FP64 and RQ_FP32 (RQ_MIXED returns RQ_ENOTIMPL: the BF16
 * sketch serves the truncated paths).  In FP64 the two block reflector
 * products of every block (W^T = (Y T)^T A2 and A2 -= Y W^T), the sketch
 * B = Omega A and the sample update's product run on the bfloat16 tensor
 * cores through the exact slice split of rq_gemm_f64, which keeps FP64
 * accuracy; the handle's workspace then also holds the slices of A2, about
 * 16 m n bytes (the environment variable RQ_F64_TC, read when the handle is
 * created, selects "0": every product on the FP64 pipe, "1": only the update
 * and the sample update on the tensor cores).  rq_qr and rq_rsrqrcp do the
 * same.
 */
int rq_rqrcp(rq_handle h, int prec, int m, int n, void* A, int lda, int b, int p, int k,
             const void* Omega, int ldo, void* tau, int* jpvt, int* info, rq_stream stream);

/*
 * rq_rqrcp_noalloc -- the same factorisation as rq_rqrcp (same arguments
 * without the handle, same outputs), for callers that cannot allocate device
 * memory when they call: a process whose device memory is all owned by
 * another allocator, or a latency-bound service that cannot afford the
 * device-wide synchronisation of cudaMalloc / cudaFree mid-request.  The
 * paper has no counterpart; this is a deployment variant.
 *
 * It runs rq_rqrcp's block loop over a fixed device array of
 * RQ_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU that
 * loads the library holds until the process exits.  It keeps fewer split-K
 * partial copies of the W^T product than a handle (none in FP64, four in
 * FP32) and runs the FP64 products on the FP64 pipe (rq_rqrcp's tensor-core
 * slices would not fit the array), so FP64 results equal rq_rqrcp's to
 * rounding and FP32 results agree within the FP32 path's tolerances (the
 * products may be cut into different inner-dimension chunks), not bit for
 * bit.  Its scratch, with s the element
 * size (8 FP64, 4 FP32), G the device's SM count and every term rounded up to
 * 256 bytes, is
 *   s (2 l n + b^2 + 2 ceil4(m) b + b n + 2 b m + c b n)
 *   + 8 (3 b^2 + 2 G (l + 2) + 2 G (b + 1) + 4 b) + 4 (5 b + n) + 16
 * bytes, c = 0 (FP64) or 4 (FP32), ceil4(m) = m rounded up to a multiple of
 * 4: about 3.7 KB x n for FP64 at m = n, b = 64, p = 8 (n up to about 4400),
 * 2.9 KB x n for FP32 (n up to about 5700).  A problem needing more returns
 * RQ_ETOOBIG before any launch.  All calls share the array, so calls that overlap on the GPU race:
 * serialise them.  Each call looks up the array's address with the current
 * device; the first call on a device also loads the library there, so make
 * it before any stream capture.  prec is RQ_FP64 or RQ_FP32; argument errors
 * return -(index), counting prec as argument 1.
 */
#define RQ_NOALLOC_SCRATCH_BYTES (16u << 20)
int rq_rqrcp_noalloc(int prec, int m, int n, void* A, int lda, int b, int p, int k, const void* Omega,
                     int ldo, void* tau, int* jpvt, int* info, rq_stream stream);

/*
 * rq_gaussian -- fills Omega (l x m, column-major, leading dimension ldo)
 * with i.i.d. standard normal draws, the Gaussian compression matrix of
 * Sec. 3.1 (and, with substream J, the fresh l x m_t matrix that repeated
 * sampling draws for block J + 1, Sec. 3.4).  The draws are a pure function
 * of (seed, substream, i + j l): Philox4x32-10 (Salmon et al., SC'11) keyed by
 * the 64-bit seed, counter (t, substream) with t = (i + j l) / 2, two 52-bit
 * uniforms per call, Box-Muller in FP64.  They do not depend on ldo, the
 * stream or the GPU, and an l x m draw is the first m columns of an l x m'
 * draw for m' > m.
 *   prec   RQ_FP64 writes double; RQ_FP32 and RQ_MIXED write float (the FP64
 *          value rounded to nearest).
 *   Omega  device buffer of ldo * m elements, owned by the caller; entries
 *          with row index >= l are left untouched.
 * Errors: -(argument index) for l < 1, m < 1, Omega == NULL or ldo < l;
 * RQ_ECUDA if the launch fails.  Asynchronous on stream.
 */
int rq_gaussian(rq_handle h, int prec, uint64_t seed, uint64_t substream, int l, int m, void* Omega, int ldo,
                rq_stream stream);

/*
 * rq_rsrqrcp -- RQRCP with repeated sampling (RSRQRCP, Sec. 3.4): the
 * ablation of the sample update.  Instead of refreshing the sample with
 * Eq. (update1), every block after the first draws a fresh l x m_t Gaussian
 * Omega^(J) and sketches the updated trailing matrix again, B = Omega^(J)
 * A(j0+b:m, j0+b:n), at an extra 2 l m_t n_t flops and one more pass over the
 * trailing matrix per block; the paper's update formula exists to avoid it.
 * The draws come from rq_gaussian's generator: the first sample uses
 * (seed, substream 0) at l x m, block J's fresh draws (seed, substream J) at
 * l x (m - J b).  Outputs, precisions and errors as rq_rqrcp (argument
 * indices follow this signature: seed is 10, tau 11, jpvt 12, info 13).
 */
int rq_rsrqrcp(rq_handle h, int prec, int m, int n, void* A, int lda, int b, int p, int k, uint64_t seed,
               void* tau, int* jpvt, int* info, rq_stream stream);

/*
 * rq_latent_cdf -- host function (no GPU work).  The Bayesian analysis of the
 * sample (Sec. 3.3): with a Gaussian sample of rank l and Jeffreys' prior, a
 * column's latent squared norm is phi ||B_j||^2 / (l - 2), and this returns
 * P(phi < tau | l) = Q(l/2, (l - 2) / (2 tau)) (the regularized upper
 * incomplete gamma function; e.g. 0.30 % for l = 4, tau = 1/8) in *prob.
 * Errors: -1 for l < 3, -2 for tau <= 0, -3 for prob == NULL.
 *
 * rq_padding -- host function.  The smallest padding p >= 2 such that every
 * pivot decision of a block keeps P(phi < tau) <= delta: the i-th decision
 * of a block sees a sample of effective rank l - i + 1, so the weakest is the
 * last, at rank p + 1 (the paper's p = 8, b = 32 gives ranks 9 to 40).
 * Errors: -1 unless 0 < tau < 1, -2 unless 0 < delta < 1, -3 for p == NULL,
 * RQ_ENOTIMPL if no p <= RQ_PADDING_MAX is enough.
 */
#define RQ_PADDING_MAX 4096
int rq_latent_cdf(int l, double tau, double* prob);
int rq_padding(double tau, double delta, int* p);

/*
 * rq_qr -- unpivoted blocked Householder QR with the same panel and block
 * reflector kernels as rq_rqrcp but no sampling or pivoting: the QR the paper
 * compares RQRCP against, which is RQRCP with the sampling and pivoting
 * steps removed (Sec. 5.2, Table 3).  A is overwritten as in
 * rq_rqrcp with k = min(m, n); tau has min(m, n) entries.  Precisions and
 * errors as rq_rqrcp (argument indices follow this signature).
 */
int rq_qr(rq_handle h, int prec, int m, int n, void* A, int lda, int b, void* tau, int* info,
          rq_stream stream);

/*
 * rq_trqrcp -- truncated RQRCP without trailing update, Alg. 5 (Sec. 4.1),
 * through the accumulated inner products W^T = T^T Y^T A.
 *   A   m x n, READ ONLY.
 *   Y   m x k (ldy >= m, out): reflectors, unit diagonal, zeros above.
 *   tau k (out).
 *   R   k x n (ldr >= k, out): upper trapezoidal, pivoted column order.
 *   b, p, k, Omega, jpvt, info as for rq_rqrcp.
 * Precisions: RQ_FP64, RQ_FP32 and RQ_MIXED (the sketch from bfloat16-rounded
 * Omega and A, FP32 accumulation).
 */
int rq_trqrcp(rq_handle h, int prec, int m, int n, const void* A, int lda, int b, int p, int k,
              const void* Omega, int ldo, void* Y, int ldy, void* tau, void* R, int ldr, int* jpvt,
              int* info, rq_stream stream);

/*
 * rq_tuxv -- TUXV approximation of the truncated SVD, Alg. 6 with j_max = 1
 * (Sec. 4.2, Eq. TUXV): A ~= U X V^T.
 *   U     m x k (ldu >= m, out), orthonormal columns.
 *   X     k x k (ldx >= k, out), upper triangular; diag(sigma) when sigma != NULL.
 *   V     n x k (ldv >= n, out), orthonormal columns.
 *   sigma NULL, or k entries (out): the singular values of X from a one-sided
 *         Jacobi SVD (descending); U and V are then rotated by the core
 *         singular vectors and X is returned as diag(sigma).
 *   b, p, k, Omega, info as for rq_trqrcp; precisions as rq_trqrcp (the core
 *   SVD in FP64 in every mode).
 */
int rq_tuxv(rq_handle h, int prec, int m, int n, const void* A, int lda, int b, int p, int k,
            const void* Omega, int ldo, void* U, int ldu, void* X, int ldx, void* V, int ldv,
            void* sigma, int* info, rq_stream stream);

/*
 * rq_tuxv_iter -- rq_tuxv with j_max >= 1 refinement steps (Alg. 6; Sec. 4.2
 * on iterating the flip between row and column bases).  Step 1 is rq_tuxv's;
 * an even step j forms Z = U^T A and takes its LQ (the QR of A^T U, one pass
 * over A), giving a new V and X = R^T, LOWER triangular; an odd step j > 1
 * forms Z = A V and takes its QR, giving a new U and an upper triangular X.
 * Each step after the first costs 2 m n k flops and one pass over A, and the
 * rank-k error never increases.  Arguments as rq_tuxv with jmax inserted
 * after k (argument 10; jmax < 1 returns -10); sigma, if set, is the SVD of the
 * final X.
 */
int rq_tuxv_iter(rq_handle h, int prec, int m, int n, const void* A, int lda, int b, int p, int k, int jmax,
                 const void* Omega, int ldo, void* U, int ldu, void* X, int ldx, void* V, int ldv, void* sigma,
                 int* info, rq_stream stream);

/*
 * One problem of a batched TUXV call.  All pointers are device pointers owned
 * by the caller; sizes and leading dimensions as for rq_tuxv.  Layout: twelve
 * int32 then seven 64-bit pointers (104 bytes).
 */
typedef struct rq_problem {
  int m, n, k, b, p;          /* 1 <= k <= min(m, n); 1 <= b <= 64; b + p <= 128 */
  int lda, ldo, ldu, ldx, ldv;
  int reserved0, reserved1;   /* set to 0 */
  const void* A;              /* m x n, read only */
  const void* Omega;          /* (b + p) x m */
  void* U;                    /* m x k (out) */
  void* X;                    /* k x k (out), upper triangular; diag(sigma) when sigma != NULL */
  void* V;                    /* n x k (out) */
  void* sigma;                /* NULL, or k entries (out): the core SVD as in rq_tuxv (FP64 Jacobi) */
  int* info;                  /* 1 int32 (out): 0 */
} rq_problem;

/*
 * rq_tuxv_batched -- TUXV (Alg. 6, j_max = 1, on truncated RQRCP, Alg. 5) of
 * `count` independent problems of different sizes in one persistent kernel
 * launch: each CTA takes the next problem from a device queue, so uneven
 * problems balance on their own; list the largest problems first.
 *   problems  device array of `count` rq_problem descriptors.
 *   max_*     upper bounds of m, n, k, b, p over the batch (they size the
 *             per-CTA scratch slots; a problem beyond them is undefined).
 *   prec      RQ_FP32 (FP32 sketch) or RQ_MIXED (sketch inputs rounded to
 *             BF16, FP32 accumulation); contractions FP32, Householder scalars,
 *             sample norms, T and the Omegahat_11 solve FP64.
 * A problem with sigma != NULL also gets the core SVD of X (Sec. 4.2) with
 * rq_tuxv's conventions: an FP64 one-sided Jacobi SVD of X inside the
 * problem's CTA, U <- U Uh, V <- V Vh, X <- diag(sigma), sigma descending,
 * each column of V with its largest-magnitude entry positive.
 * The call issues one memset and one kernel; it does not synchronise, so it
 * can be captured in a CUDA graph once the handle's workspace is large enough
 * (make one call, or rq_set_workspace, before capturing).
 */
int rq_tuxv_batched(rq_handle h, int prec, int count, const rq_problem* problems, int max_m, int max_n, int max_k,
                    int max_b, int max_p, rq_stream stream);

/*
 * rq_gemm_bf16 -- C = A B with both inputs rounded to bfloat16 (to nearest
 * even) and FP32 accumulation: the product the RQ_MIXED sketch B = Omega A
 * uses (Sec. 3.1), for sketching other matrices the same way.
 *   A     M x K (lda >= M), B  K x N (ldb >= K), C  M x N (ldc >= M, out):
 *         FP32, column-major, device arrays owned by the caller; C must not
 *         overlap A or B (an overlap returns -9).
 *   info  nullable device int32 (out): 0, or RQ_ETIMEOUT if a bounded wait of
 *         the tensor-core kernel ran out.
 * Products of bfloat16 values are exact in FP32.  On the tensor cores
 * (tcgen05; A and B 16-byte aligned with lda, ldb multiples of 4) K is cut
 * into chunks of at most 1024 whose results are added in IEEE FP32, since
 * the tensor core's own accumulation is not round-to-nearest; otherwise CUDA
 * cores accumulate each output in FP32 in K order.
 * Errors: -(argument index) for M, N or K < 1, a NULL array or a short
 * leading dimension (h is argument 1).  Asynchronous on stream.
 */
int rq_gemm_bf16(rq_handle h, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
                 int ldc, int* info, rq_stream stream);

/*
 * rq_gemm_f64 -- C = A B in FP64 on the bfloat16 tensor cores: the product the
 * FP64 factorisations' block reflector updates use (Alg. 4's trailing update
 * W^T = (Y T)^T A2, A2 -= Y W^T), for other FP64 matrices.
 *   A  M x K (lda >= M), B  K x N (ldb >= K), C  M x N (ldc >= M, out):
 *      FP64, column-major, device arrays owned by the caller; C must not
 *      overlap A or B (an overlap returns -9).
 *   info  nullable device int32 (out): 0, or RQ_ETIMEOUT if a bounded wait of
 *         the tensor-core kernel ran out.
 * Each row of A and each column of B is scaled by a power of two from its
 * largest entry and cut into eight signed 7-bit slices (exact in bfloat16);
 * the 36 slice pairs whose weights reach 2^-63 of the leading pair are
 * multiplied on the tensor cores, summed per weight in FP32 over at most 128
 * steps of K (exact: every partial sum stays below 2^24), gathered in int64
 * and returned to FP64 with one rounding (one per part when K is split over
 * several CTAs, at most one part per 128 steps of K, whose FP64 partials are
 * then summed).  The error is about that of an FP64 GEMM: below
 * (3 K 2^-53 + 2^-52) 2^(ea_i + eb_j) per entry, with 2^ea_i and 2^eb_j the
 * powers of two just above the largest magnitude of row i of A and column j
 * of B, plus, for a result in the subnormal range, one unit 2^-1074 per part
 * and one for their sum (entries of 2^-1000 or less relative to their row's
 * largest lose accuracy to underflow).  The handle's workspace holds the slices:
 * 16 (ceil128(M) + ceil64(N)) ceil64(K) bytes, plus FP64 split-K partials.
 * Errors: -(argument index) for M, N or K < 1, a NULL array or a short
 * leading dimension (h is argument 1); RQ_ENOTIMPL without a tensor-map
 * encoder in the driver.  Asynchronous on stream.
 */
int rq_gemm_f64(rq_handle h, int M, int N, int K, const double* A, int lda, const double* B, int ldb, double* C,
                int ldc, int* info, rq_stream stream);

/*
 * Tile policy of rq_tuxv_batched's block-level FP32 products.  A product with
 * M output rows and N output columns runs on 32 x 128 tiles when
 * M <= skinny_m, else on 128 x 32 tiles when N <= skinny_n, else on 64 x 64
 * tiles.  Every tile shape accumulates each output over the inner dimension
 * in the same order with the same operations, so the policy changes the speed
 * only: the results are the same bit for bit under every policy.  A new handle
 * holds {32, 32}.
 */
typedef struct rq_batch_tiles {
  int skinny_m; /* >= 0 */
  int skinny_n; /* >= 0 */
} rq_batch_tiles;

/*
 * rq_set_batch_tiles / rq_get_batch_tiles -- the handle's policy, used by its
 * later rq_tuxv_batched calls (a call captured in a CUDA graph keeps the
 * policy it was captured with).  t NULL or a negative threshold -> -2.
 */
int rq_set_batch_tiles(rq_handle h, const rq_batch_tiles* t);
int rq_get_batch_tiles(rq_handle h, rq_batch_tiles* t);

/*
 * Cost of one policy for rq_tiles_search: writes a time (any unit; finite and
 * >= 0) to *ms and returns 0.  A non-zero return ends the search with that
 * status.
 */
typedef int (*rq_tiles_measure)(void* user, const rq_batch_tiles* tiles, double* ms);

/* The values each threshold takes in the search. */
#define RQ_TILE_STEPS 6 /* 0, 16, 32, 64, 128, 256 */

/*
 * rq_tiles_search -- the autotuner's search; host only, no CUDA call.
 * Coordinate descent over the two thresholds: from `start` (NULL: {32, 32}),
 * a pass tries every other value of skinny_m, then every other value of
 * skinny_n, and moves to a candidate only when its time is below 0.99 x the
 * incumbent's (so timing noise does not move it).  The search stops after a
 * pass that moves nothing, or after `passes` passes; no policy is measured
 * twice.
 *   measure, user  the cost function and its context pointer.
 *   start          nullable; thresholds >= 0.
 *   passes         >= 0; 0 measures `start` alone.
 *   best           out: the chosen policy.  best_ms (nullable): its time.
 * Returns 0; -1 if measure is NULL or gives a time that is not finite and
 * >= 0; -3 for a negative threshold in start; -4 for passes < 0; -5 if best
 * is NULL; else the measure's own non-zero status.
 */
int rq_tiles_search(rq_tiles_measure measure, void* user, const rq_batch_tiles* start, int passes,
                    rq_batch_tiles* best, double* best_ms);

/*
 * rq_tune_batched -- autotunes the handle's tile policy on a batch.  Arguments
 * 1-9 as rq_tuxv_batched.  It runs the batch once to warm up, then
 * rq_tiles_search from the handle's current policy, measuring a policy as the
 * fastest of `reps` launches (CUDA events on `stream`), and stores the chosen
 * policy in the handle.  It synchronises the stream, so it cannot be captured
 * in a CUDA graph.  The outputs hold the batch's result afterwards (every
 * policy gives the same bits).
 *   reps    >= 1 (argument 10).      passes  >= 0 (argument 11).
 *   best    nullable: the chosen policy.  best_ms (nullable): its time in ms.
 * On an error the handle's policy is left as it was.
 */
int rq_tune_batched(rq_handle h, int prec, int count, const rq_problem* problems, int max_m, int max_n, int max_k,
                    int max_b, int max_p, int reps, int passes, rq_stream stream, rq_batch_tiles* best,
                    double* best_ms);

/*
 * rq_copy -- copies `bytes` bytes from src to dst with the GPU's SMs (loads and
 * stores through the device's view of each buffer) instead of its copy
 * engines; the paper has no counterpart.  src and dst may each be device
 * memory, managed memory or pinned (page-locked, registered or
 * cudaHostAlloc'ed) host memory; the ranges must not overlap.  On a GB300
 * node the first large copy-engine transfer after heavy GPU work took about
 * 215 ms for 2.1 GB against 10 ms repeated; this copy took about 40 ms after
 * the same work.  Errors: -1 for a NULL or unreachable (pageable host)
 * destination or overlapping ranges, -2 for a NULL or unreachable source,
 * RQ_ECUDA if a launch fails.  Asynchronous on stream.
 */
int rq_copy(void* dst, const void* src, size_t bytes, rq_stream stream);

/*
 * rq_selftest_wait_timeout -- failure-detection self-test (the paper has no
 * counterpart).  Every wait on another CTA in this library is bounded: when
 * an arrival does not come within about a second or two, the kernel writes
 * RQ_ETIMEOUT to the call's info word and returns, leaving the CUDA context
 * usable.  This call launches two CTAs at the library's grid barrier with a
 * count of three, so their wait can only run out; once the stream reaches it,
 * *info == RQ_ETIMEOUT.
 *   bar   device array of 2 uint32 owned by the caller (zeroed by the call).
 *   info  device int32 (out): zeroed, then RQ_ETIMEOUT.
 * Errors: -1 / -2 for a NULL bar / info; RQ_ECUDA if the launch fails.
 * Asynchronous on stream.
 */
int rq_selftest_wait_timeout(unsigned int* bar, int* info, rq_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* RQRCP_H */
