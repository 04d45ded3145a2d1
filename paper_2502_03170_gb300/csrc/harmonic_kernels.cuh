// Spherical (Bessel) strategy for pupils without axial symmetry, by
// azimuthal harmonics (Eq. 9 with the phi integral done by the
// Jacobi-Anger expansion, Eq. 6 split into its harmonics n = -2 .. 2).
//
//   A e^{i W(theta, phi)} = sum_{|m| <= M} P_m(theta) e^{i m phi},
//   E_c(rho, phi, z) = -i sum_{|l| <= M+2} i^l e^{i l phi} I_{c,l}(rho, z),
//   I_{c,l}(r, z) = sum_j w_j J_l(k r sin theta_j) e^{i k z cos theta_j}
//                   Bh_{c,l}(theta_j),
//   Bh_{c,l} = sum over the five kinds of coef[c][kind] g_kind P_{l+shift},
//   kinds (g_0, P_l), (g_2, P_{l-2}), (g_2, P_{l+2}), (g_1, P_{l-1}),
//   (g_1, P_{l+1}); J_{-l} = (-1)^l J_l is folded into Bh.
// P_m is a DFT (computed by FFT) over N_phi = 4 * pow2ceil(M + 1) azimuths
// of the non-axisymmetric part, times the axisymmetric integrand of the
// emitter table (A e^{i (W_GL + m = 0 Zernike)}); each emitter then keeps
// the harmonics up to its adaptive order M_e.
#pragma once

#include "bessel_kernels.cuh"
#include "psf_common.cuh"
#include "tc_kernels.cuh"

namespace psf {

constexpr int kHarmMaxM = 64;
constexpr int kHarmMaxNA = 60;   // m != 0 Noll indices j <= 66

struct HarmParams {
  int n_theta, n_r, nx, ny, n_em, n_zern;
  int m_max, n_phi, n_ord;       // n_ord = 2 m_max + 5 orders l = -(m_max+2) ..
  double k, dr, r_max, dx, dy;
  double tail_tol;               // adaptive order per emitter (0: M_e = m_max)
  int n_na;                      // m != 0 Noll terms j <= n_zern
  int na_j[kHarmMaxNA];          // their Noll indices
  int na_m[kHarmMaxNA];          // |m|
  int na_cos[kHarmMaxNA];        // 1: cos(m phi), 0: sin(m phi)
  double coef[3][5][2];          // channel x kind, complex (Jones vector of the model)
};

// Pupil harmonics Pm[e][m + M][theta] (complex) from the emitter table, the
// per-call radial table Zr [n_na][n_theta] (N_j R_n^{|m|}(sin theta / s_max))
// and the azimuth table cs [n_phi] = e^{2 pi i k / n_phi}; the emitter
// orders ord[e] = M_e (the largest |m| with max_theta |P_m| > tail_tol
// max_theta |P_0|, 0 if none; m_max with tail_tol = 0); and the
// channel/order mixtures Bh[e][c][l'][theta] from the harmonics |m| <= M_e.
void launch_harm_pupil(const HarmParams& p, ThetaTable t, EmitterTable e,
                       const double* zern, const float* Zr, const float2* cs,
                       float2* Pm, int* ord, float2* Bh, unsigned* bh_max, cudaStream_t s);

// Jt[n][i][j] = w_j J_n(k r_i sin theta_j), n = 0 .. m_max + 2 (FP64 by
// Miller's backward recurrence, all orders of one argument at once; stored
// FP32 when Jt is given, and as the split operand S_A w_j J_n of the
// tensor-core contraction when tc_ops is given).  bh_max of
// launch_harm_pupil (device max of |Re Bh|, |Im Bh|, or null) feeds the
// B operand's scale.
void launch_harm_jtab(const HarmParams& p, ThetaTable t, float* Jt, const TcHarm* tc_ops,
                      double sA, int bf16, cudaStream_t s);

// Split-precision path, per slice chunk: the defocus phasors D, the B
// operand of the orders each slice needs, and the tile flags of the
// contraction (tc_harm_contract runs it).
void launch_harm_operands(const HarmParams& p, ThetaTable t, const float2* Bh,
                          const int* slice_em, const int* valid, const int* ord,
                          const float2* zz, int s0, int ns, float2* D, const TcHarm& ops,
                          float sA, cudaStream_t s);

// Profiles of the slices [s0, s0 + ns) (D: scratch [ns][n_theta] for the
// defocus phasors e^{i k z_s cos theta_j}):
//   prof[s - s0][c][l'][i] = sum_j Jt[|l|][i][j] D[s][j] Bh[e(s)][c][l'][j]
// for |l| <= M_e(s) + 2 (other orders may be left unwritten).
void launch_harm_profiles(const HarmParams& p, ThetaTable t, const float* Jt,
                          const float2* Bh, const int* slice_em, const int* valid,
                          const int* ord, const float2* zz, int s0, int ns, float2* D,
                          float2* prof, cudaStream_t s);

// Octant pixel (a, b), b <= a, of a square grid with its radius sample i0,
// interpolation weight f and direction (cp, sp) = (x, y) / rho.
struct OctPix {
  int a, b, i0;
  float f, cp, sp;
  int pad[2];
};

// Square geometry (nx = ny, dx = dy): the epilogue works on octant pixels
// and their seven images.
bool harm_square(const HarmParams& p);
int harm_octant_pixels(const HarmParams& p);   // 0 unless square

// The octant pixels ordered by radius sample (a counting sort over i0: cnt
// [n_r] scratch, tab [harm_octant_pixels(p)]), so that the 32 pixels of a
// warp read nearly the same profile entries; the order within a sample is
// immaterial (every pixel is computed on its own).  No-op unless square.
void launch_harm_octant_table(const HarmParams& p, int* cnt, OctPix* tab, cudaStream_t s);

// I[s][a][b] = sum_c |sum_{|l| <= M_e + 2} i^l e^{i l phi}
//                     lerp(prof[s - s0][c][l'], rho)|^2
// for the slices [s0, s0 + ns) whose emitter is valid: by octant pixels
// (octab) on a square grid, else one thread per quarter pixel and its three
// mirrors, which share the radius.
void launch_harm_intensity(const HarmParams& p, const float2* prof,
                           const int* slice_em, const int* valid, const int* ord,
                           const OctPix* octab, int s0, int ns, float* I, cudaStream_t s);

}  // namespace psf
