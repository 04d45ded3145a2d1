// BF16 kernels of the learned surrogate: an MLP 23 -> 256 x 4 (SiLU) -> 1536
// mapping a query (21 Noll Zernike coefficients, emitter depth, defocus z)
// to the complex radial profiles I_0, I_1, I_2 at 256 radii, plus an error
// head 256 -> 1 that predicts log10 of the relative L2 error of the output.
#pragma once

#include "psf_common.cuh"

namespace psf {
namespace mlp {

constexpr int IN = 23;           // query: c_1..c_21, depth, z
constexpr int NFREQ = 24;        // Fourier features per coordinate (depth, z)
constexpr int IN_FEAT = IN + 4 * NFREQ;   // 21 + 2 normalised values + sin/cos features
constexpr int IN_PAD = 120;      // network input width padded to a multiple of 8
constexpr int HID = 256;
constexpr int NHID = 4;          // hidden layers
constexpr int OUT = 1536;        // 3 profiles x 256 radii x (re, im)
constexpr int NLAYER = 5;

// layer l: W_l [out][in_pad] (row-major), b_l [out]
__host__ __device__ constexpr int layer_in(int l) { return l == 0 ? IN_PAD : HID; }
__host__ __device__ constexpr int layer_out(int l) { return l == NLAYER - 1 ? OUT : HID; }

// Packed FP32 parameter vector: W_0, b_0, ..., W_4, b_4, We [HID], be [1].
struct ParamLayout {
  size_t W[NLAYER], b[NLAYER], We, be, total;
};
ParamLayout param_layout();

// Generic BF16 GEMM on tcgen05: C[m][n] = sum_k A[m][k] B[n][k] (both K-major
// bf16 in global memory), FP32 accumulation, one of the epilogues below.
enum Epilogue {
  EPI_HIDDEN = 0,   // z = C + bias; Y = z sigmoid(z) -> Y, Y^T, Z (bf16)
  EPI_LINEAR = 1,   // out = C + bias (fp32)
  EPI_DSILU = 2,    // dZ = C * SiLU'(Z) -> dZ, dZ^T (bf16)
  EPI_STORE = 3     // out = C (fp32)
};

struct GemmArgs {
  const uint16_t* A;  int lda;   // [M][K]
  const uint16_t* B;  int ldb;   // [N][K]
  int M, N, K;
  int epi;
  const float* bias;             // [N]
  uint16_t* Y;   int ldy;        // [M][N] bf16
  uint16_t* YT;  int ldyt;       // [N][M] bf16
  uint16_t* Z;   int ldz;        // [M][N] bf16 (pre-activation; read by EPI_DSILU)
  float* out;    int ldo;        // [M][N] fp32
  const float2* row_phase;       // EPI_LINEAR: row m's (re, im) column pairs times row_phase[m], or null
  int* status;
};

int gemm(const GemmArgs& g, cudaStream_t s);

// psf_mlp_forward with the output rows multiplied by the complex factors
// row_phase[B] (null: as psf_mlp_forward) inside the output layer's epilogue.
int forward_rows(const void* state, const float* query, int batch, float* out,
                 float* err_log10, void* ws, size_t ws_bytes, const float2* row_phase,
                 void* stream);

}  // namespace mlp
}  // namespace psf
