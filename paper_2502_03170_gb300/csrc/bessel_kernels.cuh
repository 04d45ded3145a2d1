// Kernel parameter blocks and launch wrappers of the Bessel (spherical)
// strategy, Eq. 10-11 for batched emitters.
#pragma once

#include "psf_common.cuh"

namespace psf {

constexpr int kMaxM0 = 6;   // m = 0 Noll indices 1, 4, 11, 22, 37, 56 (j <= 66)

// Per-theta-node constants, FP64, filled on the host (structure of arrays,
// each [n_theta]).  W_GL(theta; t_s) of Eq. 13 with t_i from Eq. 14 is affine
// in the emitter depth t_s:  W/(2 pi) = t_s a(theta) + b(theta)  [cycles],
// with a, b complex where a layer is evanescent (im part = decay, cycles).
struct ThetaTable {
  const double* theta;   // GL nodes on [0, theta_max]
  const double* w;       // GL weights
  const double* sin_t;
  const double* cos_t;
  const double* a_re;
  const double* a_im;
  const double* b_re;
  const double* b_im;
  const double* amp0;    // A(theta): apodization x envelope (Eq. 16-17)
  const double* zm0;     // [kMaxM0][n_theta] Z_j(sin theta / s_max), m = 0 j
  const double* g;       // [3][re, im][n_theta] angular weights g_n of the model:
                         // sin(1+cos), sin^2, sin(cos-1) (Eq. 11); Fresnel:
                         // sin(q_s + q_p cos), q_p sin^2, sin(q_p cos - q_s);
                         // scalar (Eq. 5): 2 sin, 0, 0
  const float* kh;       // n_i cos(theta)/lambda as double-float
  const float* kl;
};

struct BesselParams {
  int n_theta, n_r, nx, ny, n_em, n_slices, n_zern;
  double k;              // 2 pi n_i / lambda
  double dr;             // r_max / (n_r - 1)
  double r_max;
  double dx, dy;
  int n_m0;              // number of m = 0 Noll indices <= n_zern
  int m0_j[kMaxM0];      // their Noll indices
  unsigned long long nonaxis_mask[2];  // bit j-1 set: Noll j has m != 0
  int project;
  double pol[4];
  int complex_g;         // the weights have imaginary parts (Fresnel)
};

// Per-emitter integrand table (float [n_em][n_theta]):
//   amp = A(theta) e^{-2 pi Im(W)/(2 pi)},  wfr = frac(Re W / 2 pi).
struct EmitterTable {
  float* amp;
  float* wfr;
  int* valid;            // [n_em] 0 if the emitter was rejected
};

void launch_bessel_jmat(const BesselParams& p, ThetaTable t, float* Bt,
                        cudaStream_t s);
// w0 (nullable): free radial phase [n_em][n_theta] in radians.
// amp_max (nullable): running maximum of the amplitudes (float bits).
void launch_bessel_emitters(const BesselParams& p, ThetaTable t,
                            const double* depth, const double* zern,
                            const float* w0, EmitterTable e, int* status,
                            unsigned* amp_max, cudaStream_t s);
void launch_slice_map(const BesselParams& p, const int* z_offsets,
                      const double* z, int* slice_em, float2* zz, int* status,
                      cudaStream_t s);
void launch_pixel_table(const BesselParams& p, int* pix_i0, float* pix_f,
                        float* pix_g, cudaStream_t s);
void launch_bessel_profiles_f32(const BesselParams& p, ThetaTable t,
                                const float* Bt, EmitterTable e,
                                const int* slice_em, const float2* zz,
                                float2* prof, cudaStream_t s);
// complex J_n operand (Fresnel weights): BtC [n_theta][3 N_r] complex
void launch_bessel_jmat_complex(const BesselParams& p, ThetaTable t, float2* BtC,
                                cudaStream_t s);
void launch_bessel_profiles_f32c(const BesselParams& p, ThetaTable t,
                                 const float2* BtC, EmitterTable e,
                                 const int* slice_em, const float2* zz,
                                 float2* prof, cudaStream_t s);
void launch_bessel_intensity(const BesselParams& p, const float2* prof,
                             const int* slice_em, const int* valid,
                             const int* pix_i0, const float* pix_f,
                             const float* pix_g, float* I, cudaStream_t s);

// Mirror epilogue.  The four pixels (a, b), (nx-1-a, b), (a, ny-1-b),
// (nx-1-a, ny-1-b) share their radius, hence the interpolated profiles and
// the terms alpha, beta of |E|^2; only the sign of sin 2phi differs.  Each
// thread interpolates one pixel of the quarter a < nx/2, b < ny/2 and writes
// its four mirrors.  qtab [nx/2][ny/2]: (i0 as int bits, f, S1 cos 2phi,
// S2 sin 2phi) of the quarter pixels (FP64 geometry, once per call).
bool bessel_mirror_fit(int nx, int ny, int n_r);
void launch_quarter_table(const BesselParams& p, float4* qtab, cudaStream_t s);
void launch_bessel_intensity_mirror(const BesselParams& p, const float2* prof,
                                    const int* slice_em, const int* valid,
                                    const float4* qtab, float* I,
                                    cudaStream_t s);

}  // namespace psf
