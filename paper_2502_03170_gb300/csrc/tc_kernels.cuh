// Split-precision tensor-core (tcgen05 / TMEM / TMA) path of the Fourier
// strategy.
//
// Each complex contraction D = A X^T (A a zoom matrix, X pupil fields or the
// stage-1 result) runs as one real GEMM on 16-bit operands:
//   * complex -> real: the zoom matrix is stored as 2x2 real blocks, row
//     (i, re) = [Re A_i | -Im A_i], row (i, im) = [Im A_i | Re A_i], and the
//     data as [Re X | Im X] along K, so D rows alternate Re / Im of the output;
//   * precision: every operand is split x = hi + lo (fp16 or bf16, power-of-two
//     pre-scaled so fp16 never leaves its normal range) and the three products
//     hi.hi + lo.hi + hi.lo accumulate in FP32 in TMEM.
#pragma once

#include "fourier_kernels.cuh"

namespace psf {

struct TcOperands {
  uint16_t *Ax_hi, *Ax_lo;   // [2 nx][2 N] zoom-matrix blocks
  uint16_t *Ay_hi, *Ay_lo;   // [2 ny][2 N]
  uint16_t *P_hi, *P_lo;     // [zc][3][N][2 N] pupil fields of one z-chunk
  uint16_t *U_hi, *U_lo;     // [zc][3][ny][2 N] stage-1 output
};

// nullptr if (N, nx, ny) can run on the split-precision path, else a reason.
const char* tc_fourier_supported(int N, int nx, int ny);

// Planes per z-chunk of the split path.
int tc_fourier_zchunk(int N, int nx, int ny, int nz);

// Carves the split-precision buffers from the workspace at *off.
void tc_fourier_carve(char* base, size_t* off, int N, int nx, int ny, int zc,
                      TcOperands* out);

// Upper bound of |P_c| over the pupil (for the power-of-two operand scales).
double tc_pupil_amplitude_bound(const NodeParams& np);

int tc_fourier_forward(const TcOperands& ops, NodeTable nodes, const float2* zz,
                       int N, int nx, int ny, double dx, double dy, int nz,
                       int zc, double na_over_lambda, float scale,
                       double amp_bound, int precision, float* intensity,
                       float2* fields, int* status, cudaStream_t s);

}  // namespace psf
