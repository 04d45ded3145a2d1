// Split-precision tensor-core (tcgen05 / TMEM / TMA) path of the Fourier
// strategy.
#pragma once

#include "fourier_kernels.cuh"

namespace psf {

struct TcOperands {
  void* Ax;   // zoom-matrix operands (split hi/lo)
  void* Ay;
  void* P;    // pupil operands for one z-chunk
  void* U;    // stage-1 output operands for one z-chunk
};

// nullptr if (N, nx, ny) can run on the split-precision path, else a reason.
const char* tc_fourier_supported(int N, int nx, int ny);

// Carves the split-precision buffers from the workspace at *off.
void tc_fourier_carve(char* base, size_t* off, int N, int nx, int ny, int zc,
                      TcOperands* out);

int tc_fourier_forward(const TcOperands& ops, NodeTable nodes, const float2* zz,
                       int N, int nx, int ny, double dx, double dy, int nz,
                       int zc, double na_over_lambda, float scale,
                       int precision, float* intensity, float2* fields,
                       int* status, cudaStream_t s);

}  // namespace psf
