// Host -> device copies of small per-call tables without a host
// synchronisation.  cudaMemcpyAsync from pageable host memory synchronises
// the stream before the copy, so every such copy drains the GPU while the
// host waits, and the launches behind it reach an idle device.  Here the
// bytes travel in a kernel's parameter block (16 KB per launch; the copy is
// taken when the launch is issued, so the host buffer may be freed at once)
// and one CTA writes them to the destination in stream order.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace psf {

// Copies `bytes` from host `src` to device `dst` on `s` (through parameter
// blocks up to 256 KB, by cudaMemcpyAsync above); returns the launch error
// state (cudaSuccess).
cudaError_t upload_async(void* dst, const void* src, size_t bytes, cudaStream_t s);

}  // namespace psf
