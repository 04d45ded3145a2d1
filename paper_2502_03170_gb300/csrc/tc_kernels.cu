#include "tc_kernels.cuh"

namespace psf {

const char* tc_fourier_supported(int, int, int) {
  return "tensor-core kernels are not part of this build";
}

void tc_fourier_carve(char*, size_t*, int, int, int, int, TcOperands* out) {
  out->Ax = out->Ay = out->P = out->U = nullptr;
}

int tc_fourier_forward(const TcOperands&, NodeTable, const float2*, int, int,
                       int, double, double, int, int, double, float, int,
                       float*, float2*, int*, cudaStream_t) {
  return PSF_ERR_PRECISION;
}

}  // namespace psf
