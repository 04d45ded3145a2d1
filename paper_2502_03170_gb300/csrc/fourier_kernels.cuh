// Kernel parameter blocks and launch wrappers of the Fourier (Cartesian)
// strategy, Eq. 8 with the correction factors of Eq. 12.
#pragma once

#include "psf_common.cuh"

namespace psf {

// Zernike phase grouped by azimuthal order (Eq. 15):
//   sum_j c_j Z_j(rho, phi) = sum_m [Pc_m(rho) cos(m phi) + Ps_m(rho) sin(m phi)]
// with Pc_m, Ps_m polynomials in rho (coefficient of rho^k at [m][k]).
constexpr int kZernMaxOrder = 10;   // Noll j <= 66
struct ZernPoly {
  int max_m;                                   // -1: no Zernike term
  int deg;                                     // highest power of rho present
  double c[kZernMaxOrder + 1][kZernMaxOrder + 1];
  double s[kZernMaxOrder + 1][kZernMaxOrder + 1];
};

// Gibson-Lanni optical path (Eq. 13) as a sum over layers:
//   W/(2 pi) = sum_l t_l sqrt(n_l^2 - n_i^2 sin^2 theta) / lambda   [cycles]
// with signed thicknesses t_l (design layers negative).
struct GLLayers {
  int n;
  double t[5];
  double n_idx[5];
};

struct NodeParams {
  int N;                 // pupil grid size
  double s_max;          // NA / n_i
  double inv_lambda;     // 1 / lambda (um^-1)
  double n_i;
  GLLayers gl;
  int apodize;
  double s_env;
  double pol[4];
  ZernPoly zp;
  const float* phase_map;  // [N][N] radians or null
  int model;               // 0 vectorial, 1 scalar (Eq. 3), 2 vectorial + Fresnel (Eq. 7)
  double n_s, n_g;         // sample and coverslip indices (Fresnel interfaces)
};

// Per-node table written once per call (structure of arrays, float):
//   amp[6][N*N]  A e^{-Im W} e_inf,c / cos(theta) (c = x, y, z; re, im)
//   wfr[N*N]     frac(Re W / 2 pi) in cycles
//   kh, kl[N*N]  n_i cos(theta) / lambda as a double-float (cycles per um)
//   rad          scratch of the build: the radial quantities (everything but
//                the Zernike / free phase and the azimuthal basis change) of
//                the node_rad_count(N) octant pairs, kNodeRad doubles each
struct NodeTable {
  float* amp;
  float* wfr;
  float* kh;
  float* kl;
  double* rad;
};
// radial record: [0] Re W / 2 pi mod 1, [1] amplitude (-1 outside the disk),
// [2] cos theta, [3] sin theta, [4, 5] q_s, [6, 7] q_p, [8, 9] min(|m_p|,
// |m_q|) / r and max / r (1, 0 at r = 0), [10 + 2m, 11 + 2m] the cos / sin
// Zernike radial sums of azimuthal order m (m <= kZernMaxOrder), radians
constexpr int kNodeRad = 10 + 2 * (kZernMaxOrder + 1);
// Octant pairs (k1 <= k2 < K, K = (N + 1) / 2) of |2p + 1 - N| values.
inline size_t node_rad_count(int N) {
  const size_t K = (size_t)(N + 1) / 2;
  return K * (K + 1) / 2;
}

void launch_node_table(const NodeParams& p, NodeTable t, cudaStream_t s);

// A[a][p] = exp(2 pi i (NA/lambda) u_p x_a), complex64 [n_out][N].
void launch_twiddle(int N, int n_out, double d, double na_over_lambda,
                    float2* A, cudaStream_t s);

// P[zc][c][p][q] (complex64) for the z-chunk [z0, z0 + nzc): z values as
// double-float pairs zz[nz] in device memory.
void launch_pupil_z_f32(NodeTable t, int N, const float2* zz, int z0, int nzc,
                        float2* P, cudaStream_t s);

// Stage 1 (FP32): U[zc][c][b][p] = sum_q Ay[b][q] P[zc][c][p][q].
void launch_stage1_f32(const float2* Ay, const float2* P, float2* U, int N,
                       int ny, int nzc, cudaStream_t s);

// Stage 2 (FP32) + intensity epilogue:
//   E[c][a][b] = C ds^2 sum_p Ax[a][p] U[zc][c][b][p],
//   I[z0+zc][a][b] = sum_c |E_c|^2; fields written if non-null.
void launch_stage2_f32(const float2* Ax, const float2* U, float* I,
                       float2* fields, int N, int nx, int ny, int nzc,
                       float ds2_over_2pi, cudaStream_t s);

}  // namespace psf

namespace psf {

// Generic batched FP32 complex GEMM C[b][m][n] = sum_k A[b][m][k] B[b][n][k].
void launch_cgemm_nt_f32(const float2* A, long long sA, const float2* B,
                         long long sB, float2* C, long long sC, int M, int N,
                         int K, int batch, cudaStream_t s);

// Conjugate-transposed zoom matrix AH[p][a] = conj(A[a][p]), [N][n_out].
void launch_twiddle_adj(int N, int n_out, double d, double na_over_lambda,
                        float2* AH, cudaStream_t s);

// Adjoint source (FP32): per (zc, a, b) recompute acc_c = sum_p Ax U_c for the
// three channels, I = scale^2 sum_c |acc_c|^2, g = 2 (I - T) (target) or
// grad_I, and store RT[zc][c][b][a] = 2 scale^2 g acc_c.  Loss partial sums
// sum (I - T)^2 per CTA go to loss_part[zc * tiles + tile] (target only).
void launch_stage2_adjsrc_f32(const float2* Ax, const float2* U,
                              const float* target, const float* grad_I,
                              float2* RT, float* loss_part, int N, int nx,
                              int ny, int nzc, float scale, cudaStream_t s);
int stage2_tiles(int nx, int ny);

// gW[p][q] += -sum_{zc,c} Im(conj(Gh[zc][c][p][q]) P[zc][c][p][q]).
void launch_grad_accum(const float2* Gh, const float2* P, float* gW, int NN,
                       int nzc, cudaStream_t s);

// Zernike basis of the pupil grid and the chain rule of Eq. 15:
// Zt[j][p][q] = Z_{j+1}(u_p, v_q) (FP64 evaluation, once per call), then
// grad_c[j] = sum_{p,q} Zt[j][p][q] gW[p][q] (fixed-order reduction).
struct ZernBasis {
  int n_zern;
  int m[66];                    // signed azimuthal order (Noll)
  int deg[66];                  // radial degree n: rc[j][k] = 0 for k > deg[j]
  double rc[66][11];            // radial coefficients (normalised)
};
void launch_zernike_table(const ZernBasis& zb, int N, float* Zt, cudaStream_t s);
// nb pupils: gW [nb][N][N] -> grad_c [nb][n_zern]; part: scratch of
// zernike_grad_part_bytes(n_zern, nb) bytes.
size_t zernike_grad_part_bytes(int n_zern, int nb);
void launch_zernike_grad(const ZernBasis& zb, int N, const float* Zt, const float* gW,
                         int nb, double* part, float* grad_c, cudaStream_t s);

// loss = sum of partials[0..n) in fixed order.
void launch_sum_partials(const float* part, int n, float* out, cudaStream_t s);

}  // namespace psf
