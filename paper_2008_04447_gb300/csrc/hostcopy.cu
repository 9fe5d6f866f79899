// rq_copy: a copy between pinned host memory and device memory (or within
// either) done by the SMs instead of the copy engines.
//
// On a GB300 node (Grace CPU, NVLink-C2C) the first large copy-engine transfer
// after heavy GPU work was measured at about 215 ms for 2.1 GB, against 10 ms
// when repeated; the same transfer by SM loads and stores through the pinned
// buffer's device mapping took about 40 ms after the same work and 10 ms
// repeated.  The end-to-end factorisations (input in, result out every step)
// use it for their large transfers.
#include <cuda_runtime.h>
#include <cstdint>

#include "rqrcp.h"

namespace {

__global__ void copy16_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst, size_t n16) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __ldcs(src + i);
}

__global__ void copy1_kernel(const unsigned char* __restrict__ src, unsigned char* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// The device address of p: itself for device or managed memory, the device
// mapping for pinned host memory; nullptr for memory the device cannot reach
// through a mapping (pageable host memory).
const void* device_view(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return p;
  if (at.type == cudaMemoryTypeHost) return at.devicePointer;
  return nullptr;
}

}  // namespace

extern "C" int rq_copy(void* dst, const void* src, size_t bytes, rq_stream stream) {
  if (!dst) return -1;
  if (!src) return -2;
  if (bytes == 0) return RQ_OK;
  unsigned char* d = static_cast<unsigned char*>(const_cast<void*>(device_view(dst)));
  const unsigned char* s = static_cast<const unsigned char*>(device_view(src));
  if (!d) return -1;
  if (!s) return -2;
  // the copied ranges may not overlap
  const uintptr_t d0 = reinterpret_cast<uintptr_t>(d), s0 = reinterpret_cast<uintptr_t>(s);
  if (d0 < s0 + bytes && s0 < d0 + bytes) return -1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return RQ_ECUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int grid = 8 * sms;
  size_t done = 0;
  if ((d0 % 16) == (s0 % 16)) {
    // bytes up to the first 16-byte boundary, then 16-byte words, then the tail
    const size_t head = ((16 - d0 % 16) % 16) < bytes ? (16 - d0 % 16) % 16 : bytes;
    if (head) copy1_kernel<<<1, 32, 0, st>>>(s, d, head);
    const size_t n16 = (bytes - head) / 16;
    if (n16) copy16_kernel<<<grid, 512, 0, st>>>(reinterpret_cast<const uint4*>(s + head),
                                                  reinterpret_cast<uint4*>(d + head), n16);
    done = head + 16 * n16;
  }
  if (done < bytes) copy1_kernel<<<grid, 512, 0, st>>>(s + done, d + done, bytes - done);
  return cudaGetLastError() == cudaSuccess ? RQ_OK : RQ_ECUDA;
}
