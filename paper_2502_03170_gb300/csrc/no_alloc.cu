// psf_fourier_vectorial_noalloc: the Fourier forward for callers that cannot
// allocate device memory themselves.
//
// Some hosts own every byte of device memory through their own allocator (a
// deep-learning framework's caching allocator, an imaging application that
// hands plug-ins a fixed memory budget), and some latency-critical loops must
// not call cudaMalloc at all because it can synchronise the whole device.
// Such callers still own their inputs and outputs, but cannot provide the
// scratch workspace psf_fourier_vectorial() needs.  This entry point takes
// that scratch from one fixed-size array in device memory that belongs to the
// library instead, and otherwise runs the same kernels.
//
// The array is a file-scope __device__ variable, so every GPU on which the
// library is loaded holds PSF_NOALLOC_SCRATCH_BYTES of it until the process
// exits.  Host code cannot use the array's name as a device address: each
// call looks its address up in the current context with
// cudaGetSymbolAddress.
#include <stdio.h>

#include "psf_common.cuh"

namespace psf {
// psf_api.cu: workspace of the Fourier forward at one plane per z-chunk
size_t fourier_min_workspace_size(const psf_optics* opt, int n_pupil, const psf_grid* grid,
                                  int precision);
}  // namespace psf

namespace psf {
void set_last_error(const char* msg);
}

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[PSF_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array in the current context.  It is looked
// up on every call (a host-side lookup) rather than cached, so a call after
// a device reset, which reloads the module, sees the new address.
int scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) {
    psf::set_last_error("noalloc: cudaGetSymbolAddress of the scratch array failed");
    return PSF_ERR_CUDA;
  }
  *out = p;
  return PSF_OK;
}

}  // namespace

extern "C" int psf_fourier_vectorial_noalloc(const psf_optics* opt, int n_pupil,
                                             const psf_grid* grid,
                                             const double* zernike, int n_zern,
                                             const float* phase_map,
                                             float* intensity, void* fields,
                                             void* stream) {
  // the forward shortens its z-chunks to the array; reject what one plane
  // per chunk does not fit
  const size_t need = psf::fourier_min_workspace_size(opt, n_pupil, grid, PSF_PREC_FP32);
  if (need == 0) return PSF_ERR_ARG;   // message set by the size check
  if (need > (size_t)PSF_NOALLOC_SCRATCH_BYTES) {
    char msg[200];
    snprintf(msg, sizeof(msg),
             "noalloc: these sizes need %zu bytes of scratch even one plane at a "
             "time; the fixed array holds %zu (use psf_fourier_vectorial with a workspace)",
             need, (size_t)PSF_NOALLOC_SCRATCH_BYTES);
    psf::set_last_error(msg);
    return PSF_ERR_WORKSPACE;
  }
  void* scratch = nullptr;
  const int r = scratch_address(&scratch);
  if (r != PSF_OK) return r;
  return psf_fourier_vectorial(opt, n_pupil, grid, zernike, n_zern, phase_map,
                               PSF_PREC_FP32, intensity, fields, scratch,
                               (size_t)PSF_NOALLOC_SCRATCH_BYTES, stream);
}
