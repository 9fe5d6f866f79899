// rq_rqrcp_noalloc: RQRCP (FP64 or FP32) whose scratch lives in a fixed
// device array compiled into the library, for callers that cannot allocate
// device memory at call time.
//
// Such callers include services that have handed all device memory to another
// allocator (a framework's caching pool), latency-sensitive code for which a
// cudaMalloc / cudaFree would add a device-wide synchronisation in the middle
// of a request, and code that must not fail for lack of memory once it runs.
//
// The factorisation is the one rq_rqrcp runs (the same block loop,
// factor_blocks), over the fixed array instead of a handle's workspace, with
// fewer split-K partial copies (none in FP64) and, in FP64, the block
// reflector products on the FP64 pipe (the tensor-core path's slice planes
// would not fit), to keep the array modest.
//
// The scratch array is RQ_NOALLOC_SCRATCH_BYTES large and every GPU that
// loads this library holds it until the process exits.  All calls share it:
// calls that overlap on the GPU (different streams, or different host
// threads) race on it and give wrong results; serialise them.  Each call
// looks up the array's device address (cudaGetSymbolAddress) with the
// caller's device current, so the address is never stale after a device
// reset; the first call on a device also loads the library's kernels there,
// so make it before any stream capture.
#include "common.cuh"
#include "kernels.h"

namespace rq {
namespace {

static __device__ __align__(256) unsigned char g_scratch[RQ_NOALLOC_SCRATCH_BYTES];

long long g_launches = 0;

// Split-K partial copies of the skinny W^T product: FP32 keeps four so the
// tensor-core products can still cut long inner dimensions into chunks of at
// most 1024; FP64 runs without.
template <typename TS>
constexpr int kSplitCopies = sizeof(TS) == sizeof(float) ? 4 : 0;

// Device address of the static array and SM count of the current device.
int setup(void** addr, int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RQ_ECUDA;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return RQ_ECUDA;
  }
  if (cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RQ_ECUDA;
  *addr = p;
  return RQ_OK;
}

template <typename TS>
int run(int m, int n, TS* A, int lda, int b, int p, int k, const TS* Omega, int ldo, TS* tau, int* jpvt,
        int* info, cudaStream_t st) {
  void* base = nullptr;
  int sms = 0;
  int rc = setup(&base, &sms);
  if (rc) return rc;
  if (factor_ws_bytes<TS>(m, n, b, p, sms, true, false, kSplitCopies<TS>, 0) > (size_t)RQ_NOALLOC_SCRATCH_BYTES)
    return RQ_ETOOBIG;
  // factor_blocks clears the barrier words first: the array keeps the previous call's contents
  return factor_blocks<TS>(nullptr, base, sms, &g_launches, true, m, n, A, lda, b, p, k, Omega, ldo, tau, jpvt, info,
                           st, nullptr, kSplitCopies<TS>, 0);
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
