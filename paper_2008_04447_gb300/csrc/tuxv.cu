// Kernels of the TUXV tail (Alg. 6, Sec. 4.2): transposes and identity fills
// for the explicit-Q QR factorisations, and the one-sided Jacobi SVD of the
// k x k core X (Hestenes' method, cyclic round-robin ordering of column pairs).
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace rq {
namespace {

template <typename TS>
__global__ void transpose_kernel(int rows, int cols, const TS* __restrict__ s, int lds, TS* __restrict__ d,
                                 int ldd) {
  __shared__ TS tile[32][33];
  const int bi = blockIdx.x * 32, bj = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int i = bi + threadIdx.x, j = bj + dy;
    if (i < rows && j < cols) tile[dy][threadIdx.x] = s[i + (size_t)j * lds];
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int j = bj + threadIdx.x, i = bi + dy;  // d(j, i) = s(i, j)
    if (i < rows && j < cols) d[j + (size_t)i * ldd] = tile[threadIdx.x][dy];
  }
}

template <typename TS>
__global__ void eye_kernel(int rows, int cols, TS* __restrict__ d, int ldd) {
  const size_t total = (size_t)rows * cols;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = e % rows, j = e / rows;
    d[i + (size_t)j * ldd] = i == j ? TS(1) : TS(0);
  }
}

template <typename TS>
__global__ void upper_kernel(int k, const TS* __restrict__ s, int lds, TS* __restrict__ d, int ldd) {
  const size_t total = (size_t)k * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = e % k, j = e / k;
    d[i + (size_t)j * ldd] = i <= j ? s[i + (size_t)j * lds] : TS(0);
  }
}

constexpr int kJThreads = 256;

struct JacArgs {
  double* W;  // k x k, ld k: X rotated in place (columns become U * sigma)
  double* V;  // k x k, ld k: accumulated right rotations
  int k, kk;  // kk = k rounded up to even (a dummy column pairs with the odd one out)
  unsigned int* bar;
  int* err;
  int* rot;  // max_sweeps counters of rotations, zeroed by the host
  int max_sweeps;
  double tol;
};

__device__ __forceinline__ void pair_of(int r, int i, int kk, int& p, int& q) {
  // circle method: position 0 fixed, positions 1..kk-1 rotate by r
  auto at = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + r) % (kk - 1); };
  p = at(i);
  q = at(kk - 1 - i);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (kJThreads / 32) ? red[threadIdx.x] : 0.0;
    t = warp_sum(t);
  }
  if (threadIdx.x == 0) red[kJThreads / 32] = t;
  __syncthreads();
  return red[kJThreads / 32];
}

// One cooperative launch runs all sweeps; one grid barrier per round of
// kk/2 disjoint pairs.  Every CTA reads the same rotation count at the end of a
// sweep, so all stop together when a sweep rotated nothing.
__global__ void __launch_bounds__(kJThreads) jacobi_kernel(JacArgs a) {
  __shared__ double red[kJThreads / 32 + 1];
  __shared__ double s_c, s_s;
  __shared__ int s_go;
  const int G = gridDim.x, k = a.k, kk = a.kk, npairs = kk / 2;
  unsigned int epoch = 0;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    for (int r = 0; r < kk - 1; ++r) {
      for (int pi = blockIdx.x; pi < npairs; pi += G) {
        int p, q;
        pair_of(r, pi, kk, p, q);
        if (p >= k || q >= k) continue;
        if (p > q) { const int t = p; p = q; q = t; }
        double* wp = a.W + (size_t)p * k;
        double* wq = a.W + (size_t)q * k;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = threadIdx.x; i < k; i += kJThreads) {
          const double x = wp[i], y = wq[i];
          al = fma(x, x, al);
          be = fma(y, y, be);
          ga = fma(x, y, ga);
        }
        al = block_sum(al, red);
        be = block_sum(be, red);
        ga = block_sum(ga, red);
        if (threadIdx.x == 0) {
          int go = 0;
          if (ga != 0.0 && fabs(ga) > a.tol * sqrt(al * be)) {
            const double zeta = (be - al) / (2.0 * ga);
            const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double c = 1.0 / sqrt(1.0 + t * t);
            s_c = c;
            s_s = c * t;
            go = 1;
            atomicAdd(a.rot + sweep, 1);
          }
          s_go = go;
        }
        __syncthreads();
        if (s_go) {
          const double c = s_c, s = s_s;
          double* vp = a.V + (size_t)p * k;
          double* vq = a.V + (size_t)q * k;
          for (int i = threadIdx.x; i < k; i += kJThreads) {
            const double x = wp[i], y = wq[i];
            wp[i] = c * x - s * y;
            wq[i] = s * x + c * y;
            const double u = vp[i], v = vq[i];
            vp[i] = c * u - s * v;
            vq[i] = s * u + c * v;
          }
        }
        __syncthreads();
      }
      if (!grid_barrier(a.bar, G, a.err, epoch)) return;
    }
    __shared__ int s_count;
    if (threadIdx.x == 0) s_count = __ldcg(a.rot + sweep);
    __syncthreads();
    if (s_count == 0) break;
  }
  grid_exit(a.bar, G);
}

// nrm_j = ||W(:, j)||
__global__ void jacobi_norms(int k, const double* __restrict__ W, double* __restrict__ nrm) {
  __shared__ double red[kJThreads / 32 + 1];
  const int j = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) acc = fma(W[i + (size_t)j * k], W[i + (size_t)j * k], acc);
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) nrm[j] = sqrt(acc);
}

// sigma sorted descending (ties by column index); Uh = W(:, order) / sigma,
// Vh = V(:, order).
template <typename TS>
__global__ void jacobi_finish(int k, const double* __restrict__ W, const double* __restrict__ V,
                              const double* __restrict__ nrm, TS* __restrict__ Uh, int ldu, TS* __restrict__ Vh,
                              int ldv, TS* __restrict__ sigma) {
  __shared__ double red[kJThreads / 32 + 1];
  const int j = blockIdx.x;
  const double sj = nrm[j];
  double cnt = 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double si = nrm[i];
    if (si > sj || (si == sj && i < j)) cnt += 1.0;
  }
  const int rk = (int)block_sum(cnt, red);
  const double inv = sj > 0.0 ? 1.0 / sj : 0.0;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    Uh[i + (size_t)rk * ldu] = static_cast<TS>(W[i + (size_t)j * k] * inv);
    Vh[i + (size_t)rk * ldv] = static_cast<TS>(V[i + (size_t)j * k]);
  }
  if (threadIdx.x == 0) sigma[rk] = static_cast<TS>(sj);
}

// Column j of V: the entry of largest magnitude (lowest row on ties) is made
// positive; column j of U follows.
template <typename TS>
__global__ void sign_fix(int m, int n, TS* __restrict__ U, int ldu, TS* __restrict__ V, int ldv) {
  const int j = blockIdx.x;
  TS* v = V + (size_t)j * ldv;
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = fabs(static_cast<double>(v[i]));
    if (x > best || (x == best && i < bi)) { best = x; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double b2 = __shfl_xor_sync(0xffffffffu, best, o);
    const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
    if (b2 > best || (b2 == best && i2 < bi)) { best = b2; bi = i2; }
  }
  __shared__ double sb[8];
  __shared__ int si[8];
  __shared__ double s_sign;
  if ((threadIdx.x & 31) == 0) { sb[threadIdx.x >> 5] = best; si[threadIdx.x >> 5] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (sb[w] > best || (sb[w] == best && si[w] < bi)) { best = sb[w]; bi = si[w]; }
    bi = bi < n ? bi : 0;
    s_sign = static_cast<double>(v[bi]) < 0.0 ? -1.0 : 1.0;
  }
  __syncthreads();
  if (s_sign < 0.0) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = -v[i];
    TS* u = U + (size_t)j * ldu;
    for (int i = threadIdx.x; i < m; i += blockDim.x) u[i] = -u[i];
  }
}

template <typename TS>
__global__ void diag_kernel(int k, const TS* __restrict__ s, TS* __restrict__ X, int ldx) {
  const size_t total = (size_t)k * k;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int i = e % k, j = e / k;
    X[i + (size_t)j * ldx] = i == j ? s[i] : TS(0);
  }
}

int grid_for(size_t total) {
  size_t b = (total + 255) / 256;
  return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

}  // namespace

template <typename TS>
cudaError_t transpose(const Ctx& c, int rows, int cols, const TS* s, int lds, TS* d, int ldd) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  transpose_kernel<TS><<<dim3((rows + 31) / 32, (cols + 31) / 32), dim3(32, 8), 0, c.stream>>>(rows, cols, s, lds,
                                                                                                d, ldd);
  ++*c.launches;
  return cudaGetLastError();
}

template <typename TS>
cudaError_t set_eye(const Ctx& c, int rows, int cols, TS* d, int ldd) {
  eye_kernel<TS><<<grid_for((size_t)rows * cols), 256, 0, c.stream>>>(rows, cols, d, ldd);
  ++*c.launches;
  return cudaGetLastError();
}

template <typename TS>
cudaError_t copy_upper(const Ctx& c, int k, const TS* s, int lds, TS* d, int ldd) {
  upper_kernel<TS><<<grid_for((size_t)k * k), 256, 0, c.stream>>>(k, s, lds, d, ldd);
  ++*c.launches;
  return cudaGetLastError();
}

size_t jacobi_scratch_doubles(int k) { return 2 * (size_t)k * k + k + 64; }

template <typename TS>
cudaError_t jacobi_svd(const Ctx& c, int k, const TS* X, int ldx, TS* Uh, int ldu, TS* Vh, int ldv, TS* sigma,
                       double* scratch, int* rot, int max_sweeps) {
  double* W = scratch;
  double* V = W + (size_t)k * k;
  double* sv = V + (size_t)k * k;
  cudaError_t e = convert<double, TS>(c, k, k, X, ldx, W, k);
  if (e != cudaSuccess) return e;
  e = set_eye<double>(c, k, k, V, k);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(rot, 0, sizeof(int) * max_sweeps, c.stream);
  if (e != cudaSuccess) return e;
  const int kk = (k + 1) / 2 * 2;
  int G = kk / 2;
  if (G > c.num_sms) G = c.num_sms;
  if (G < 1) G = 1;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, kJThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm * c.num_sms < G) return cudaErrorCooperativeLaunchTooLarge;
  const double tol = (k > 1 ? (double)k : 2.0) * 2.220446049250313e-16;
  JacArgs a{W, V, k, kk, c.bar, c.err, rot, max_sweeps, tol};
  void* args[] = {&a};
  e = cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(G), dim3(kJThreads), args, 0, c.stream);
  ++*c.launches;
  if (e != cudaSuccess) return e;
  jacobi_norms<<<k, kJThreads, 0, c.stream>>>(k, W, sv);
  jacobi_finish<TS><<<k, kJThreads, 0, c.stream>>>(k, W, V, sv, Uh, ldu, Vh, ldv, sigma);
  *c.launches += 2;
  return cudaGetLastError();
}

template <typename TS>
cudaError_t fix_signs(const Ctx& c, int m, int n, int k, TS* U, int ldu, TS* V, int ldv) {
  sign_fix<TS><<<k, 256, 0, c.stream>>>(m, n, U, ldu, V, ldv);
  ++*c.launches;
  return cudaGetLastError();
}

template <typename TS>
cudaError_t set_diag(const Ctx& c, int k, const TS* s, TS* X, int ldx) {
  diag_kernel<TS><<<grid_for((size_t)k * k), 256, 0, c.stream>>>(k, s, X, ldx);
  ++*c.launches;
  return cudaGetLastError();
}

#define RQ_TUXV_INST(TS)                                                                                      \
  template cudaError_t transpose<TS>(const Ctx&, int, int, const TS*, int, TS*, int);                        \
  template cudaError_t set_eye<TS>(const Ctx&, int, int, TS*, int);                                          \
  template cudaError_t copy_upper<TS>(const Ctx&, int, const TS*, int, TS*, int);                            \
  template cudaError_t jacobi_svd<TS>(const Ctx&, int, const TS*, int, TS*, int, TS*, int, TS*, double*, int*, \
                                      int);                                                                  \
  template cudaError_t fix_signs<TS>(const Ctx&, int, int, int, TS*, int, TS*, int);                         \
  template cudaError_t set_diag<TS>(const Ctx&, int, const TS*, TS*, int);
RQ_TUXV_INST(double)
RQ_TUXV_INST(float)

}  // namespace rq
