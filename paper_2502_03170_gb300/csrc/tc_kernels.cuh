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

#include "bessel_kernels.cuh"
#include "fourier_kernels.cuh"

namespace psf {

// Split-precision operands of the Bessel radial contraction
//   prof[s][(n, i)] = sum_j B[(n, i)][j] F[j][s]  (real B, complex F):
// B rows (n, i) x K columns (theta nodes, padded to Kp = 8k), F rows
// (s, re/im) interleaved, both split hi + lo.  With complex weights g_n
// (Fresnel coefficients) B = w_j J_n holds three planes of n_r_pad rows and
// F one plane per order, g_n F; the contraction runs per order.
struct TcBessel {
  uint16_t *B_hi, *B_lo;     // [3 N_r][Kp]  (complex weights: [3][n_r_pad][Kp])
  uint16_t *F_hi, *F_lo;     // [2 n_slices][Kp]  (complex weights: [3][2 n_slices][Kp])
  unsigned char* need;       // complex weights: per-order tile flags (all set)
  unsigned* amp_max;         // device max of |F0| (float bits), zeroed per call
  float* out_scale;          // device 1 / (S_B S_F)
};

int tc_bessel_kp(int n_theta);
void tc_bessel_carve(char* base, size_t* off, int n_theta, int n_r, int n_slices,
                     bool complex_g, TcBessel* out);
// J_n operand in split form (per call; layout from p.complex_g).
void tc_bessel_jmat(const BesselParams& p, ThetaTable t, double max_w,
                    int precision, const TcBessel& ops, cudaStream_t s);
// F operand from the per-emitter table and the contraction into prof;
// g_max bounds |g_n| over the nodes (used with complex weights).
int tc_bessel_contract(const BesselParams& p, ThetaTable t, EmitterTable et,
                       const int* slice_em, const float2* zz, double max_w, double g_max,
                       int precision, const TcBessel& ops, float2* prof,
                       int* status, cudaStream_t s);

// Split-precision operands of the Bessel adjoint contraction
//   g_F[s][j] = sum_row conj(Bt[j][row]) g_P[s][row]   (complex g_P):
// A rows j x K columns (3 N_r, pitch kp), g_P rows (s, re/im), BF16 hi + lo;
// a complex Bt (Fresnel weights) gives A rows (j, Re / Im).
// Harmonic radial contraction on the tensor cores (split hi + lo operands):
// per order l' = l + m_max + 2, prof[col][l'][i] = sum_j A[|l|][i][j] B[l'][col][j]
// over the columns col = 3 s + c of a slice chunk.
struct TcHarm {
  int kp, n_r_pad;
  size_t a_bytes;            // bytes of one of A_hi / A_lo
  uint16_t *A_hi, *A_lo;     // [(m_max + 3) n_r_pad][kp]: S_A w_j J_n(k r_i sin theta_j)
  uint16_t *B_hi, *B_lo;     // [n_ord][chunk columns][re/im][kp]: S_F D Bh
  unsigned char* need;       // [n_ord][tiles]: a column of the tile needs the order
  unsigned* bh_max;          // device max |Re Bh|, |Im Bh| (float bits), zeroed per call
  float* out_scale;          // device 1 / (S_A S_F)
};
int tc_harm_cols_per_tile();          // columns (s, c) per B tile
int tc_harm_n_r_pad(int n_r);         // N_r rounded up to the A tile height
void tc_harm_carve(char* base, size_t* off, int n_theta, int n_r, int m_max, int chunk,
                   TcHarm* out);
float tc_harm_scale_a(double max_w);  // S_A: power of two with max |A| < 2^14
// The contraction of n_cols columns (all orders; tiles flagged unneeded are
// skipped).  Returns PSF_OK or PSF_ERR_CUDA.
int tc_harm_contract(const TcHarm& ops, int n_theta, int n_r, int m_max, int n_cols,
                     int precision, float2* prof, int* status, cudaStream_t s);

struct TcBesselAdj {
  int kp;
  uint16_t *A_hi, *A_lo;     // [n_theta][kp] (complex weights: [2 n_theta][kp])
  uint16_t *G_hi, *G_lo;     // [2 n_slices][kp]
  float* scale;              // device 1.0 (BF16 needs no pre-scaling)
};
void tc_bessel_adj_carve(char* base, size_t* off, int n_theta, int n_r, int n_slices,
                         bool complex_g, TcBesselAdj* out);
// A operand from the FP32 J_n operand (Bt real, or BtC complex when
// non-null), then the contraction into gF.
int tc_bessel_adj_contract(const BesselParams& p, const float* Bt, const float2* BtC,
                           const TcBesselAdj& ops, float2* gF, int* status, cudaStream_t s);

struct TcOperands {
  uint16_t *Ax_hi, *Ax_lo;   // [2 nx][2 N] zoom-matrix blocks
  uint16_t *Ay_hi, *Ay_lo;   // [2 ny][2 N]
  uint16_t *P_hi, *P_lo;     // [zc][3][N][2 N] pupil fields of one z-chunk
  uint16_t *U_hi, *U_lo;     // [zc][3][ny][2 N] stage-1 output
};

// Operands of the symmetry-folded forward (fold_kernels.cu), 16-bit, split
// hi + lo, row pitch Kp = H rounded up to 16 (H = N/2; 16-bit elements, or
// 32-bit TF32 parts with the TF32 precisions):
//   Zx, Zy  zoom halves C = cos, S = sin over the first half p' < H of the
//           pupil and the first half of the outputs: [4][ceil(n/2)][Kp] with
//           the variants C hi, C lo, S hi, S lo;
//   P       pupil parity classes of a z-chunk: [zc][3][parity][re/im] slabs
//           of [4][H][Kp] with the variants X hi, X lo (q-even sum), Y hi,
//           Y lo (q-odd difference);
//   U       the p-folded stage-1 output: [zc][4][ny][3][re/im][Kp] with the
//           variants T+ hi, T+ lo, T- hi, T- lo.
struct TcFoldOperands {
  int H, Kp;
  uint16_t *Zx, *Zy, *P, *U;
};
int tc_fold_kp(int N);
const char* tc_fold_supported(int N, int nx, int ny);
// eb: operand element bytes, 2 (FP16 / BF16 parts) or 4 (TF32 parts)
int tc_fold_zchunk(int N, int nx, int ny, int nz, int eb = 2);
void tc_fold_carve(char* base, size_t* off, int N, int nx, int ny, int zc, TcFoldOperands* out,
                   int eb = 2);
// The folded forward over z-chunks of zc planes; arguments as
// tc_fourier_forward.  Returns PSF_ERR_CUDA when a launch is refused.
int tc_fold_forward(const TcFoldOperands& ops, NodeTable nodes, const float2* zz, int N,
                    int nx, int ny, double dx, double dy, int nz, int zc,
                    double na_over_lambda, float scale, double amp_bound, int precision,
                    float* intensity, float2* fields, float* host_out, int* status,
                    cudaStream_t s);

// nullptr if (N, nx, ny) can run on the split-precision path, else a reason.
const char* tc_fourier_supported(int N, int nx, int ny);

// Planes per z-chunk of the split path.
int tc_fourier_zchunk(int N, int nx, int ny, int nz);

// Carves the split-precision buffers from the workspace at *off.
void tc_fourier_carve(char* base, size_t* off, int N, int nx, int ny, int zc,
                      TcOperands* out);

// Upper bound of |P_c| over the pupil (for the power-of-two operand scales).
double tc_pupil_amplitude_bound(const NodeParams& np);

// The forward over the z-chunks of zc planes.  With host_out (pinned host
// memory of the whole stack) `intensity` is a device staging area of two
// chunks: each chunk is copied to host_out on a copy stream while the next
// one is computed, and the call completes on s once the stack is on the host.
int tc_fourier_forward(const TcOperands& ops, NodeTable nodes, const float2* zz,
                       int N, int nx, int ny, double dx, double dy, int nz,
                       int zc, double na_over_lambda, float scale,
                       double amp_bound, int precision, float* intensity,
                       float2* fields, float* host_out, int* status, cudaStream_t s);
bool tc_host_streaming_available();

// Split-precision Fourier adjoint (tensor cores).  Per z-chunk: pupil fields,
// stage 1, stage 2 recomputed with the adjoint source R = g E written as BF16
// operand rows, V = A_x^H R, Gh = V conj(A_y), then the phase gradient
// 2 s Re(conj(Gh) P) (s = ds^2 / 2 pi), summed over planes in order.
struct TcBwdOperands {
  TcOperands fwd;            // Ax, Ay, P, U (input precision)
  uint16_t *AxH_hi, *AxH_lo; // [2 N][2 nx] conj(Ax)^T blocks, BF16
  uint16_t *AyH_hi, *AyH_lo; // [2 N][2 ny]
  uint16_t *R_hi, *R_lo;     // [zc][3][ny][2 nx]
  uint16_t *V_hi, *V_lo;     // [zc][3][N][2 ny]
  float* gWz;                // [zc][3][re/im][N][N] Gh of a chunk (FP32)
  float* wfr;                // [group][N][N] phase tables of a group of pupils
  double* coef;              // [group][<= 66] Zernike coefficients of the group
  float* gW;                 // [group][N][N] dL/dW_0 of the group
  float* loss_part;          // [group * nz * tiles * 4]
  int group;                 // pupils per group (planes of a chunk span pupils)
};
const char* tc_fourier_bwd_supported(int N, int nx, int ny);
int tc_fourier_bwd_zchunk(int N, int nx, int ny, int nz, int max_planes);
int tc_fourier_bwd_group(int nz, int zc);
void tc_fourier_bwd_carve(char* base, size_t* off, int N, int nx, int ny, int nz, int zc,
                          TcBwdOperands* out);
// zoom matrices and their adjoints (once per call)
int tc_fourier_bwd_setup(const TcBwdOperands& ops, int N, int nx, int ny, double dx,
                         double dy, double na_over_lambda, int precision, cudaStream_t s);
// Phase tables of nb pupils into ops.wfr from the shared Gibson-Lanni phase
// wfr_gl, the Zernike basis Zt and the coefficients coef [nb][n_zern] (device)
// plus the free phase maps [nb][N][N] (device, or null).
void tc_group_phase(const TcBwdOperands& ops, const float* wfr_gl, const float* Zt,
                    const double* coef, int n_zern, const float* phase_map, int N, int nb,
                    cudaStream_t s);
// n_pupils (<= group) pupils whose phase tables are in ops.wfr: planes are
// flat over (pupil, z); gW[k][N][N] = dL/dW_0 of pupil k (overwritten);
// loss[k] (target only).  target / grad_intensity point at the group's first
// plane.  With grad_c non-null, grad_c[k][j] = sum Z_j gW[k] (chain rule of
// Eq. 15, Zt [n_zern][N][N]), formed as the fold finishes each pupil, through
// zpart (tc_zernike_parts_bytes(N, n_zern, n_pupils) bytes).
int tc_fourier_backward(const TcBwdOperands& ops, NodeTable nodes, const float2* zz,
                        int N, int nx, int ny, int nz, int n_pupils, int zc, float scale,
                        double amp_bound, int precision, const float* target,
                        const float* grad_intensity, float* gW, float* loss,
                        const float* Zt, int n_zern, double* zpart, float* grad_c,
                        int* status, cudaStream_t s);
size_t tc_zernike_parts_bytes(int N, int n_zern, int nb);

}  // namespace psf
