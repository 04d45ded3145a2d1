// Parameter-block uploads of small host tables (see upload.cuh).
#include "upload.cuh"

#include <string.h>

#include "timing.cuh"

namespace psf {

namespace {

constexpr unsigned kChunk = 16384;

struct Chunk {
  uint4 w[kChunk / 16];
};

__global__ void k_upload(const __grid_constant__ Chunk c, unsigned n, unsigned char* dst) {
  const unsigned char* src = reinterpret_cast<const unsigned char*>(c.w);
  if (((uintptr_t)dst & 15) == 0) {
    uint4* d = reinterpret_cast<uint4*>(dst);
    for (unsigned i = threadIdx.x; i < n / 16; i += blockDim.x) d[i] = c.w[i];
    for (unsigned i = (n / 16) * 16 + threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
  } else {
    for (unsigned i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
  }
}

}  // namespace

cudaError_t upload_async(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  // beyond 16 launches one plain copy is cheaper than the launches
  if (bytes > 16 * (size_t)kChunk) {
    cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    return cudaPeekAtLastError();
  }
  const unsigned char* h = static_cast<const unsigned char*>(src);
  unsigned char* d = static_cast<unsigned char*>(dst);
  for (size_t o = 0; o < bytes; o += kChunk) {
    TimingScope ts(kTimeSetup, s);
    const unsigned n = (unsigned)(bytes - o < kChunk ? bytes - o : kChunk);
    Chunk c;
    memcpy(c.w, h + o, n);
    k_upload<<<1, 256, 0, s>>>(c, n, d + o);
  }
  return cudaPeekAtLastError();
}

}  // namespace psf
