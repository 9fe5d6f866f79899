// Small kernels of the RQRCP path: column permutation, the sample update
// (Eq. update1), index initialisation, the LAPACK-style info word.
#include "common.cuh"
#include "kernels.h"

namespace rq {
namespace {

// Gather the changed columns (new position e <- old position src[e]) to tmp.
template <typename TS>
__global__ void perm_gather(const TS* __restrict__ A, int lda, int m, const int* __restrict__ chg,
                            const int* __restrict__ src, const int* __restrict__ jpvt, TS* __restrict__ tmp,
                            int* __restrict__ jtmp) {
  const int slot = blockIdx.y;
  const int e = chg[slot];
  if (e < 0) return;
  const int s = src[e];
  const TS* col = A + (size_t)s * lda;
  TS* out = tmp + (size_t)slot * m;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) out[r] = col[r];
  if (blockIdx.x == 0 && threadIdx.x == 0) jtmp[slot] = jpvt[s];
}

template <typename TS>
__global__ void perm_scatter(TS* __restrict__ A, int lda, int m, const int* __restrict__ chg,
                             const TS* __restrict__ tmp, const int* __restrict__ jtmp, int* __restrict__ jpvt) {
  const int slot = blockIdx.y;
  const int e = chg[slot];
  if (e < 0) return;
  TS* col = A + (size_t)e * lda;
  const TS* in = tmp + (size_t)slot * m;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) col[r] = in[r];
  if (blockIdx.x == 0 && threadIdx.x == 0) jpvt[e] = jtmp[slot];
}

// Omegahat11 = S11 R11^{-1}: row r solves x R11 = S11(r, :) (both upper
// triangular, so x(r, j) = 0 for j < r).  One thread per row, R11 in shared memory.
template <typename TS>
__global__ void omegahat_kernel(const double* __restrict__ S11, int lds, const TS* __restrict__ R11, int ldr,
                                int bj, double* __restrict__ Oh, int ldo) {
  extern __shared__ double sR[];  // bj x bj, column-major
  for (int e = threadIdx.x; e < bj * bj; e += blockDim.x) {
    const int i = e % bj, j = e / bj;
    sR[e] = i <= j ? static_cast<double>(R11[i + (size_t)j * ldr]) : 0.0;
  }
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= bj) return;
  double* x = Oh + r;  // row r of Oh, stride ldo
  for (int j = 0; j < r; ++j) x[(size_t)j * ldo] = 0.0;
  for (int j = r; j < bj; ++j) {
    double acc = S11[r + (size_t)j * lds];
    for (int i = r; i < j; ++i) acc = fma(-x[(size_t)i * ldo], sR[i + j * bj], acc);
    const double d = sR[j + j * bj];
    x[(size_t)j * ldo] = d != 0.0 ? acc / d : 0.0;
  }
}

// B1 -= Oh * R12 (K = bj), one thread per output entry.  Omegahat_11 comes
// from an FP64 solve; the product accumulates in the storage precision.
template <typename TS>
__global__ void sample_update_kernel(int bj, int n2, const double* __restrict__ Oh, int ldo,
                                     const TS* __restrict__ R12, int ldr, TS* __restrict__ B1, int ldb) {
  extern __shared__ __align__(8) unsigned char so_raw[];
  TS* sO = reinterpret_cast<TS*>(so_raw);  // bj x bj
  for (int e = threadIdx.x; e < bj * bj; e += blockDim.x)
    sO[e] = static_cast<TS>(Oh[(e % bj) + (size_t)(e / bj) * ldo]);
  __syncthreads();
  const int col = blockIdx.x;
  if (col >= n2) return;
  const TS* rc = R12 + (size_t)col * ldr;
  TS* bc = B1 + (size_t)col * ldb;
  for (int r = threadIdx.x; r < bj; r += blockDim.x) {
    TS acc = TS(0);
    for (int i = r; i < bj; ++i) acc = fma(sO[r + i * bj], rc[i], acc);
    bc[r] -= acc;
  }
}

// dst(:, i) = src(:, idx[i]) for i < count (rows x count, column-major).
template <typename TS>
__global__ void gather_cols_kernel(const TS* __restrict__ src, int lds, int rows, const int* __restrict__ idx,
                                   int count, TS* __restrict__ dst, int ldd) {
  const int i = blockIdx.y;
  if (i >= count) return;
  const TS* s = src + (size_t)idx[i] * lds;
  TS* d = dst + (size_t)i * ldd;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) d[r] = s[r];
}

__global__ void index_gather(const int* __restrict__ chg, const int* __restrict__ src, const int* __restrict__ v,
                             int* __restrict__ tmp, int slots) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= slots) return;
  const int e = chg[t];
  if (e >= 0) tmp[t] = v[src[e]];
}

__global__ void index_scatter(const int* __restrict__ chg, const int* __restrict__ tmp, int* __restrict__ v,
                              int slots) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= slots) return;
  const int e = chg[t];
  if (e >= 0) v[e] = tmp[t];
}

// New rows j0..j0+bj-1 of Z = R P^T (original column order): the columns chosen
// in earlier blocks are zero there; the block's own columns take R11 from the panel.
template <typename TS>
__global__ void trq_fix_rows(TS* __restrict__ Zb, int ldz, int bj, int j0, const int* __restrict__ jpvt,
                             const TS* __restrict__ R11, int ldr) {
  const int pos = blockIdx.x;  // < j0 + bj
  const int col = jpvt[pos];
  for (int r = threadIdx.x; r < bj; r += blockDim.x) {
    TS v = TS(0);
    if (pos >= j0) {
      const int c = pos - j0;
      v = r <= c ? R11[r + (size_t)c * ldr] : TS(0);
    }
    Zb[r + (size_t)col * ldz] = v;
  }
}

// B1(:, t) -= Oh * Z(:, idx[t]) (K = bj), storage-precision accumulation.
template <typename TS>
__global__ void sample_update_idx_kernel(int bj, int n2, const double* __restrict__ Oh, int ldo,
                                         const TS* __restrict__ Zb, int ldz, const int* __restrict__ idx,
                                         TS* __restrict__ B1, int ldb) {
  extern __shared__ __align__(8) unsigned char so_raw[];
  TS* sO = reinterpret_cast<TS*>(so_raw);
  for (int e = threadIdx.x; e < bj * bj; e += blockDim.x)
    sO[e] = static_cast<TS>(Oh[(e % bj) + (size_t)(e / bj) * ldo]);
  __syncthreads();
  const int col = blockIdx.x;
  if (col >= n2) return;
  const TS* rc = Zb + (size_t)idx[col] * ldz;
  TS* bc = B1 + (size_t)col * ldb;
  for (int r = threadIdx.x; r < bj; r += blockDim.x) {
    TS acc = TS(0);
    for (int i = r; i < bj; ++i) acc = fma(sO[r + i * bj], rc[i], acc);
    bc[r] -= acc;
  }
}

// Omegahat_11 = S11 R11^{-1} for b <= 64 by forward substitution along each
// row, Oh(r, j) = (S11(r, j) - sum_{i<j} Oh(r, i) R11(i, j)) / R11(j, j), all
// rows at once, four threads per row (partial sums over i = sub mod 4, in a
// fixed order), the rows kept in shared memory.
template <typename TS>
// Oh = S11 R11^{-1} for b <= 64, right-looking: at step j the rows' entries of
// column j are final (X(r, j) = W(r, j) / R(j, j)), and every later column of
// the working copy W of S11 drops X(r, j) R(j, j') at once.  Each step is one
// independent FP64 FMA per entry instead of a dependent dot product (an FP64
// FMA waits about 64 cycles here), and the rows are split over CTAs of 16 rows
// so that the FP64 work is spread over SMs.  Oh is upper triangular (S11 and
// R11 are): rows r > j of column j are 0 and are skipped.
__global__ void __launch_bounds__(256) omegahat_fast_kernel(const double* __restrict__ S11, int lds,
                                                            const TS* __restrict__ R11, int ldr, int bj,
                                                            double* __restrict__ Oh, int ldo) {
  __shared__ double sR[64 * 64];   // sR[i * 64 + j] = R11(i, j), upper
  __shared__ double sW[16 * 65];   // this CTA's rows of S11, then of Oh
  __shared__ double sInv[64];
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * 16;
  for (int e = tid; e < bj * bj; e += 256) {
    const int i = e % bj, j = e / bj;
    sR[i * 64 + j] = i <= j ? static_cast<double>(R11[i + (size_t)j * ldr]) : 0.0;
  }
  for (int e = tid; e < 16 * bj; e += 256) {
    const int rr = e % 16, j = e / 16, r = r0 + rr;
    sW[rr * 65 + j] = r < bj && r <= j ? S11[r + (size_t)j * lds] : 0.0;
  }
  __syncthreads();
  if (tid < bj) {
    const double d = sR[tid * 64 + tid];
    sInv[tid] = d != 0.0 ? 1.0 / d : 0.0;
  }
  __syncthreads();
  const int rr = tid >> 4, cg = tid & 15, r = r0 + rr;
  for (int j = 0; j < bj; ++j) {
    // X(r, j) for this CTA's rows r <= j (sixteen threads)
    if (tid < 16 && r0 + tid < bj && r0 + tid <= j) sW[tid * 65 + j] *= sInv[j];
    __syncthreads();
    if (r < bj && r <= j) {
      const double x = sW[rr * 65 + j];
      for (int jj = j + 1 + cg; jj < bj; jj += 16) sW[rr * 65 + jj] = fma(-x, sR[j * 64 + jj], sW[rr * 65 + jj]);
    }
    __syncthreads();
  }
  for (int e = tid; e < 16 * bj; e += 256) {
    const int q = e % 16, j = e / 16, rw = r0 + q;
    if (rw < bj) Oh[rw + (size_t)j * ldo] = sW[q * 65 + j];
  }
}

// B1(:, t) -= Oh R12(:, t), R12(:, t) = Zb(:, idx[t]), for b <= 64: one CTA per
// 64 columns, Oh and the gathered R12 tile in shared memory; each entry
// accumulates over i = r .. b-1 in order, in the storage precision.
template <typename TS>
__global__ void __launch_bounds__(256) sample_update_tile_kernel(int bj, int n2, const double* __restrict__ Oh,
                                                                 int ldo, const TS* __restrict__ Zb, int ldz,
                                                                 const int* __restrict__ idx, TS* __restrict__ B1,
                                                                 int ldb) {
  extern __shared__ __align__(16) unsigned char su_raw[];
  TS* sO = reinterpret_cast<TS*>(su_raw);  // sO[r * 64 + i]
  TS* sZ = sO + 64 * 64;                   // sZ[i * 65 + cc]
  const int tid = threadIdx.x, col0 = blockIdx.x * 64;
  for (int e = tid; e < bj * bj; e += 256) {
    const int r = e % bj, i = e / bj;
    sO[r * 64 + i] = static_cast<TS>(Oh[r + (size_t)i * ldo]);
  }
  for (int e = tid; e < bj * 64; e += 256) {
    const int i = e % bj, cc = e / bj, col = col0 + cc;
    sZ[i * 65 + cc] = col < n2 ? Zb[i + (size_t)idx[col] * ldz] : TS(0);
  }
  __syncthreads();
  const int cc = tid & 63, rg = tid >> 6, col = col0 + cc;
  if (col >= n2) return;
  for (int rr = 0; rr < 16; ++rr) {
    const int r = rg * 16 + rr;
    if (r >= bj) break;
    TS acc = TS(0);
    for (int i = r; i < bj; ++i) acc = fma(sO[r * 64 + i], sZ[i * 65 + cc], acc);
    B1[r + (size_t)col * ldb] -= acc;
  }
}

__global__ void iota_kernel(int* v, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = i;
}

// info = first j (1-based) with A(j-1, j-1) == 0, or RQ_ETIMEOUT if a bounded
// wait gave up somewhere in the call.
template <typename TS>
__global__ void info_kernel(const TS* __restrict__ A, int lda, int k, const int* __restrict__ err,
                            int* __restrict__ info) {
  __shared__ int first;
  if (threadIdx.x == 0) first = k;
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x)
    if (A[(size_t)i * lda + i] == TS(0)) atomicMin(&first, i);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int e = *reinterpret_cast<const volatile int*>(err);
    *info = e != 0 ? e : (first < k ? first + 1 : 0);
  }
}

template <typename TD, typename TS>
__global__ void convert_kernel(int rows, int cols, const TS* __restrict__ s, int lds, TD* __restrict__ d, int ldd) {
  const size_t total = (size_t)rows * cols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = e % rows, j = e / rows;
    d[i + (size_t)j * ldd] = static_cast<TD>(s[i + (size_t)j * lds]);
  }
}

}  // namespace

template <typename TS>
cudaError_t permute_columns(const Ctx& c, TS* A, int lda, int m, int steps, const int* chg, const int* src,
                            int* jpvt, TS* tmp, int* jtmp) {
  if (steps <= 0) return cudaSuccess;
  int bx = (m + 255) / 256;
  if (bx > 64) bx = 64;
  dim3 grid(bx, 2 * steps);
  perm_gather<TS><<<grid, 256, 0, c.stream>>>(A, lda, m, chg, src, jpvt, tmp, jtmp);
  perm_scatter<TS><<<grid, 256, 0, c.stream>>>(A, lda, m, chg, tmp, jtmp, jpvt);
  *c.launches += 2;
  return cudaGetLastError();
}

template <typename TS>
cudaError_t omegahat11(const Ctx& c, const double* S11, int lds, const TS* R11, int ldr, int bj, double* Oh,
                       int ldo) {
  if (bj <= 64) {
    omegahat_fast_kernel<TS><<<(bj + 15) / 16, 256, 0, c.stream>>>(S11, lds, R11, ldr, bj, Oh, ldo);
  } else {
    const int threads = bj <= 128 ? 128 : 256;
    omegahat_kernel<TS><<<(bj + threads - 1) / threads, threads, (size_t)bj * bj * sizeof(double), c.stream>>>(
        S11, lds, R11, ldr, bj, Oh, ldo);
  }
  ++*c.launches;
  return cudaGetLastError();
}

template <typename TS>
cudaError_t sample_update(const Ctx& c, int bj, int n2, const double* Oh, int ldo, const TS* R12, int ldr,
                          TS* B1, int ldb) {
  if (n2 <= 0) return cudaSuccess;
  const int threads = bj <= 32 ? 32 : (bj <= 64 ? 64 : (bj <= 128 ? 128 : 256));
  sample_update_kernel<TS><<<n2, threads, (size_t)bj * bj * sizeof(double), c.stream>>>(bj, n2, Oh, ldo, R12,
                                                                                         ldr, B1, ldb);
  ++*c.launches;
  return cudaGetLastError();
}

template <typename TS>
cudaError_t gather_columns(const Ctx& c, const TS* src, int lds, int rows, const int* idx, int count, TS* dst,
                           int ldd) {
  if (rows <= 0 || count <= 0) return cudaSuccess;
  int bx = (rows + 255) / 256;
  if (bx > 64) bx = 64;
  gather_cols_kernel<TS><<<dim3(bx, count), 256, 0, c.stream>>>(src, lds, rows, idx, count, dst, ldd);
  ++*c.launches;
  return cudaGetLastError();
}

cudaError_t permute_index(const Ctx& c, int steps, const int* chg, const int* src, int* v, int* tmp) {
  if (steps <= 0) return cudaSuccess;
  const int slots = 2 * steps;
  index_gather<<<(slots + 127) / 128, 128, 0, c.stream>>>(chg, src, v, tmp, slots);
  index_scatter<<<(slots + 127) / 128, 128, 0, c.stream>>>(chg, tmp, v, slots);
  *c.launches += 2;
  return cudaGetLastError();
}

template <typename TS>
cudaError_t trq_fix_new_rows(const Ctx& c, TS* Zb, int ldz, int bj, int j0, const int* jpvt, const TS* R11,
                             int ldr) {
  trq_fix_rows<TS><<<j0 + bj, 64, 0, c.stream>>>(Zb, ldz, bj, j0, jpvt, R11, ldr);
  ++*c.launches;
  return cudaGetLastError();
}

template <typename TS>
cudaError_t sample_update_idx(const Ctx& c, int bj, int n2, const double* Oh, int ldo, const TS* Zb, int ldz,
                              const int* idx, TS* B1, int ldb) {
  if (n2 <= 0) return cudaSuccess;
  if (bj <= 64) {
    const size_t smem = (64 * 64 + 64 * 65) * sizeof(TS);
    static bool attr = false;
    if (!attr) {
      cudaError_t ea =
          cudaFuncSetAttribute(sample_update_tile_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (ea != cudaSuccess) return ea;
      attr = true;
    }
    sample_update_tile_kernel<TS><<<(n2 + 63) / 64, 256, smem, c.stream>>>(bj, n2, Oh, ldo, Zb, ldz, idx, B1, ldb);
  } else {
    const int threads = bj <= 128 ? 128 : 256;
    sample_update_idx_kernel<TS><<<n2, threads, (size_t)bj * bj * sizeof(double), c.stream>>>(bj, n2, Oh, ldo, Zb,
                                                                                               ldz, idx, B1, ldb);
  }
  ++*c.launches;
  return cudaGetLastError();
}

cudaError_t iota(const Ctx& c, int* v, int n) {
  iota_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, c.stream>>>(v, n);
  ++*c.launches;
  return cudaGetLastError();
}

template <typename TS>
cudaError_t finish_info(const Ctx& c, const TS* A, int lda, int k, int* info) {
  info_kernel<TS><<<1, 256, 0, c.stream>>>(A, lda, k, c.err, info);
  ++*c.launches;
  return cudaGetLastError();
}

template <typename TD, typename TS>
cudaError_t convert(const Ctx& c, int rows, int cols, const TS* src, int lds, TD* dst, int ldd) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  size_t total = (size_t)rows * cols;
  int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
  convert_kernel<TD, TS><<<blocks, 256, 0, c.stream>>>(rows, cols, src, lds, dst, ldd);
  ++*c.launches;
  return cudaGetLastError();
}

#define RQ_INST(TS)                                                                                          \
  template cudaError_t permute_columns<TS>(const Ctx&, TS*, int, int, int, const int*, const int*, int*, TS*, \
                                           int*);                                                            \
  template cudaError_t omegahat11<TS>(const Ctx&, const double*, int, const TS*, int, int, double*, int);    \
  template cudaError_t sample_update<TS>(const Ctx&, int, int, const double*, int, const TS*, int, TS*, int); \
  template cudaError_t finish_info<TS>(const Ctx&, const TS*, int, int, int*);                              \
  template cudaError_t gather_columns<TS>(const Ctx&, const TS*, int, int, const int*, int, TS*, int);       \
  template cudaError_t trq_fix_new_rows<TS>(const Ctx&, TS*, int, int, int, const int*, const TS*, int);      \
  template cudaError_t sample_update_idx<TS>(const Ctx&, int, int, const double*, int, const TS*, int,        \
                                             const int*, TS*, int);
RQ_INST(double)
RQ_INST(float)
template cudaError_t convert<float, double>(const Ctx&, int, int, const double*, int, float*, int);
template cudaError_t convert<double, float>(const Ctx&, int, int, const float*, int, double*, int);
template cudaError_t convert<float, float>(const Ctx&, int, int, const float*, int, float*, int);
template cudaError_t convert<double, double>(const Ctx&, int, int, const double*, int, double*, int);

}  // namespace rq
