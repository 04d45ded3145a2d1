// Bessel (spherical) strategy kernels, Eq. 10-11: the J_n operand, the
// per-emitter integrand table, the radial contraction and the
// radial-to-Cartesian intensity epilogue.
#include "bessel_kernels.cuh"

namespace psf {

// ---------------------------------------------------------------------------
// J_n operand, emitter independent:
//   Bt[j][n N_r + i] = w_j g_n(theta_j) J_n(k r_i sin theta_j),
//   g_0 = sin(1+cos), g_1 = sin^2, g_2 = sin(cos-1)   (Eq. 11)
// FP64 via CUDA's double-precision Bessel functions, once per call.
// ---------------------------------------------------------------------------
__global__ void k_bessel_jmat(BesselParams p, ThetaTable t, float* Bt) {
  const int rows = 3 * p.n_r;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)rows * p.n_theta) return;
  const int j = (int)(idx / rows), row = (int)(idx - (long long)j * rows);
  const int n = row / p.n_r, i = row - n * p.n_r;
  const double st = t.sin_t[j];
  const double x = p.k * (i * p.dr) * st;
  double jn_v;
  if (n == 0) {
    jn_v = j0(x);
  } else if (n == 1) {
    jn_v = j1(x);
  } else {
    // J_2(0) = 0 exactly (the library routine is not used at x = 0)
    jn_v = x > 0.0 ? jn(2, x) : 0.0;
  }
  Bt[idx] = (float)(t.w[j] * t.g[(2 * n) * p.n_theta + j] * jn_v);
}

// Complex form for weights with imaginary parts (Fresnel coefficients past a
// critical angle).
__global__ void k_bessel_jmat_complex(BesselParams p, ThetaTable t, float2* BtC) {
  const int rows = 3 * p.n_r;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)rows * p.n_theta) return;
  const int j = (int)(idx / rows), row = (int)(idx - (long long)j * rows);
  const int n = row / p.n_r, i = row - n * p.n_r;
  const double x = p.k * (i * p.dr) * t.sin_t[j];
  const double jn_v = n == 0 ? j0(x) : (n == 1 ? j1(x) : (x > 0.0 ? jn(2, x) : 0.0));
  const double s = t.w[j] * jn_v;
  BtC[idx] = make_float2((float)(s * t.g[(2 * n) * p.n_theta + j]),
                         (float)(s * t.g[(2 * n + 1) * p.n_theta + j]));
}

void launch_bessel_jmat_complex(const BesselParams& p, ThetaTable t, float2* BtC,
                                cudaStream_t s) {
  const long long n = 3LL * p.n_r * p.n_theta;
  k_bessel_jmat_complex<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, t, BtC);
}

void launch_bessel_jmat(const BesselParams& p, ThetaTable t, float* Bt,
                        cudaStream_t s) {
  const long long n = 3LL * p.n_r * p.n_theta;
  k_bessel_jmat<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, t, Bt);
}

// ---------------------------------------------------------------------------
// Per-emitter integrand F0(theta) = A(theta) e^{i W_e(theta)} (Eq. 12):
// W_e = W_GL(t_s = depth[e]) + sum over m = 0 Noll terms c_{e,j} Z_j
//       (+ the free radial phase W_0[e][j] at the node, when given).
// FP64 phase, reduced mod one cycle.  Thread (e, j); j == 0 also checks that
// no m != 0 coefficient is set (the spherical form needs an axisymmetric
// pupil, Sec. 3.4) unless projection was requested.
// ---------------------------------------------------------------------------
__global__ void k_bessel_emitters(BesselParams p, ThetaTable t,
                                  const double* __restrict__ depth,
                                  const double* __restrict__ zern,
                                  const float* __restrict__ w0,
                                  EmitterTable et, int* status,
                                  unsigned* amp_max) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)p.n_em * p.n_theta) return;
  const int e = (int)(idx / p.n_theta), j = (int)(idx - (long long)e * p.n_theta);
  const double ts = depth[e];
  double w = ts * t.a_re[j] + t.b_re[j];
  const double dec = ts * t.a_im[j] + t.b_im[j];
  double wz = 0.0;
  for (int q = 0; q < p.n_m0; ++q)
    wz += zern[(size_t)e * p.n_zern + p.m0_j[q] - 1] * t.zm0[q * p.n_theta + j];
  if (w0) wz += (double)w0[idx];
  w += wz * (0.5 / kPi);
  w -= rint(w);
  double amp = t.amp0[j];
  if (dec != 0.0) amp *= exp(-2.0 * kPi * dec);
  et.amp[idx] = (float)amp;
  if (amp_max) atomicMax(amp_max, __float_as_uint((float)amp));   // amp >= 0
  et.wfr[idx] = (float)w;
  if (j == 0) {
    int ok = 1;
    if (!p.project) {
      for (int jj = 1; jj <= p.n_zern; ++jj) {
        const unsigned long long bit = 1ULL << ((jj - 1) & 63);
        if ((p.nonaxis_mask[(jj - 1) >> 6] & bit) &&
            zern[(size_t)e * p.n_zern + jj - 1] != 0.0)
          ok = 0;
      }
      if (!ok) set_status(status, PSF_ERR_NOT_AXISYMMETRIC);
    }
    et.valid[e] = ok;
  }
}

void launch_bessel_emitters(const BesselParams& p, ThetaTable t,
                            const double* depth, const double* zern,
                            const float* w0, EmitterTable e, int* status,
                            unsigned* amp_max, cudaStream_t s) {
  const long long n = (long long)p.n_em * p.n_theta;
  k_bessel_emitters<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, t, depth,
                                                                 zern, w0, e, status,
                                                                 amp_max);
}

// ---------------------------------------------------------------------------
// Slice -> emitter map and double-float z per slice.  Offsets outside
// [0, n_slices] or decreasing mark the status PSF_ERR_ARG and are skipped.
// ---------------------------------------------------------------------------
__global__ void k_slice_map(BesselParams p, const int* __restrict__ offs,
                            const double* __restrict__ z, int* slice_em,
                            float2* zz, int* status) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= p.n_em) return;
  const int a = offs[e], b = offs[e + 1];
  if (a < 0 || b < a || b > p.n_slices) {
    set_status(status, PSF_ERR_ARG);
    return;
  }
  for (int s = a; s < b; ++s) {
    slice_em[s] = e;
    const f2x v = split_double(z[s]);
    zz[s] = make_float2(v.hi, v.lo);
  }
}

void launch_slice_map(const BesselParams& p, const int* z_offsets,
                      const double* z, int* slice_em, float2* zz, int* status,
                      cudaStream_t s) {
  k_slice_map<<<ceil_div(p.n_em, 128), 128, 0, s>>>(p, z_offsets, z, slice_em,
                                                    zz, status);
}

// ---------------------------------------------------------------------------
// Pixel table: radius -> interpolation cell (i0, f) on r_i = i dr, and the
// polarisation-angle factor gamma = S1 cos 2phi + S2 sin 2phi with
// S1 = |p_x|^2 - |p_y|^2, S2 = 2 Re(conj(p_x) p_y).  FP64, once per call.
// ---------------------------------------------------------------------------
__global__ void k_pixel_table(BesselParams p, int* i0, float* f, float* g) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= p.nx * p.ny) return;
  const int a = idx / p.ny, b = idx - (idx / p.ny) * p.ny;
  const double x = (a - 0.5 * (p.nx - 1)) * p.dx;
  const double y = (b - 0.5 * (p.ny - 1)) * p.dy;
  const double rho = sqrt(x * x + y * y);
  const double tt = p.dr > 0 ? rho / p.dr : 0.0;   // r_max = 0: all r_i = 0
  int c = (int)floor(tt);
  c = c < 0 ? 0 : (c > p.n_r - 2 ? p.n_r - 2 : c);
  i0[idx] = c;
  f[idx] = (float)(tt - c);
  double c2 = 1.0, s2 = 0.0;
  if (rho > 0) {
    c2 = (x * x - y * y) / (rho * rho);
    s2 = 2.0 * x * y / (rho * rho);
  }
  const double S1 = p.pol[0] * p.pol[0] + p.pol[1] * p.pol[1] -
                    p.pol[2] * p.pol[2] - p.pol[3] * p.pol[3];
  const double S2 = 2.0 * (p.pol[0] * p.pol[2] + p.pol[1] * p.pol[3]);
  g[idx] = (float)(S1 * c2 + S2 * s2);
}

void launch_pixel_table(const BesselParams& p, int* pix_i0, float* pix_f,
                        float* pix_g, cudaStream_t s) {
  k_pixel_table<<<ceil_div(p.nx * p.ny, 256), 256, 0, s>>>(p, pix_i0, pix_f,
                                                           pix_g);
}

// ---------------------------------------------------------------------------
// Radial contraction (plain FP32): prof[s][row] = sum_j Bt[j][row] F[j][s],
// F[j][s] = amp[e(s)][j] exp(2 pi i (wfr[e(s)][j] + n_i z_s cos(theta_j)/lambda)).
// One CTA per 32 slices: F for the tile is generated once into shared memory
// (double-float defocus phase), then every 64-row band of the 3 N_r rows is
// contracted against it.  Thread = one row x 8 slices.
// ---------------------------------------------------------------------------
constexpr int BP_SL = 32;
template <bool CB>
__global__ void __launch_bounds__(256)
k_bessel_profiles_f32(BesselParams p, ThetaTable t, const float* __restrict__ Bt,
                      const float2* __restrict__ BtC,
                      EmitterTable et, const int* __restrict__ slice_em,
                      const float2* __restrict__ zz, float2* __restrict__ prof) {
  extern __shared__ float2 F[];   // [n_theta][BP_SL]
  const int s0 = blockIdx.x * BP_SL;
  const int tid = threadIdx.x;
  for (int q = tid; q < p.n_theta * BP_SL; q += blockDim.x) {
    const int j = q / BP_SL, sl = q - (q / BP_SL) * BP_SL;
    const int s = s0 + sl;
    float2 v = make_float2(0.f, 0.f);
    const int e = s < p.n_slices ? slice_em[s] : -1;
    if (e >= 0) {
      const size_t ej = (size_t)e * p.n_theta + j;
      const float2 z = zz[s];
      const float r = frac_mul_add(f2x{t.kh[j], t.kl[j]}, f2x{z.x, z.y}, et.wfr[ej]);
      const float2 c = cis_cycles(r);
      const float a = et.amp[ej];
      v = make_float2(a * c.x, a * c.y);
    }
    F[q] = v;
  }
  __syncthreads();
  const int rows = 3 * p.n_r;
  const int r_loc = tid & 63, sg = tid >> 6;   // 4 groups of 8 slices
  for (int r0 = 0; r0 < rows; r0 += 64) {
    const int row = r0 + r_loc;
    float2 acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = make_float2(0.f, 0.f);
    if (row < rows) {
      for (int j = 0; j < p.n_theta; ++j) {
        const float2* Fj = &F[j * BP_SL + sg * 8];
        if (CB) {
          const float2 b = __ldg(&BtC[(size_t)j * rows + row]);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            acc[k].x = fmaf(b.x, Fj[k].x, fmaf(-b.y, Fj[k].y, acc[k].x));
            acc[k].y = fmaf(b.x, Fj[k].y, fmaf(b.y, Fj[k].x, acc[k].y));
          }
        } else {
          const float b = __ldg(&Bt[(size_t)j * rows + row]);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            acc[k].x = fmaf(b, Fj[k].x, acc[k].x);
            acc[k].y = fmaf(b, Fj[k].y, acc[k].y);
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int s = s0 + sg * 8 + k;
        if (s < p.n_slices) prof[(size_t)s * rows + row] = acc[k];
      }
    }
  }
}

void launch_bessel_profiles_f32(const BesselParams& p, ThetaTable t,
                                const float* Bt, EmitterTable e,
                                const int* slice_em, const float2* zz,
                                float2* prof, cudaStream_t s) {
  const size_t smem = (size_t)p.n_theta * BP_SL * sizeof(float2);
  cudaFuncSetAttribute(k_bessel_profiles_f32<false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_bessel_profiles_f32<false><<<ceil_div(p.n_slices, BP_SL), 256, smem, s>>>(
      p, t, Bt, nullptr, e, slice_em, zz, prof);
}

void launch_bessel_profiles_f32c(const BesselParams& p, ThetaTable t,
                                 const float2* BtC, EmitterTable e,
                                 const int* slice_em, const float2* zz,
                                 float2* prof, cudaStream_t s) {
  const size_t smem = (size_t)p.n_theta * BP_SL * sizeof(float2);
  cudaFuncSetAttribute(k_bessel_profiles_f32<true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_bessel_profiles_f32<true><<<ceil_div(p.n_slices, BP_SL), 256, smem, s>>>(
      p, t, nullptr, BtC, e, slice_em, zz, prof);
}

// ---------------------------------------------------------------------------
// Radial -> Cartesian epilogue (Eq. 10).  With I_n^a = p_a I_n the intensity
// |E|^2 = |V|^2 / 4 (E = -(i/2) V) expands exactly into
//   |V|^2 = N (|I0|^2 + |I2|^2 + 2 |I1|^2) + gamma (2 |I1|^2 - 2 Re(conj(I0) I2)),
// N = |p_x|^2 + |p_y|^2, gamma from the pixel table; the I_n are the complex
// linear interpolants at the pixel radius.  One CTA per slice.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_bessel_intensity(BesselParams p, const float2* __restrict__ prof,
                   const int* __restrict__ slice_em, const int* __restrict__ valid,
                   const int* __restrict__ pix_i0, const float* __restrict__ pix_f,
                   const float* __restrict__ pix_g, float* __restrict__ I) {
  extern __shared__ float2 pr[];   // [3][n_r]
  const int s = blockIdx.x;
  const int e = slice_em[s];
  if (e < 0 || !valid[e]) return;
  const int rows = 3 * p.n_r;
  for (int q = threadIdx.x; q < rows; q += blockDim.x)
    pr[q] = prof[(size_t)s * rows + q];
  __syncthreads();
  const float Nn = (float)(p.pol[0] * p.pol[0] + p.pol[1] * p.pol[1] +
                           p.pol[2] * p.pol[2] + p.pol[3] * p.pol[3]);
  const int npix = p.nx * p.ny;
  float* out = I + (size_t)s * npix;
  for (int q = threadIdx.x; q < npix; q += blockDim.x) {
    const int c = pix_i0[q];
    const float f = pix_f[q], g = pix_g[q];
    float2 v[3];
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      const float2 lo = pr[n * p.n_r + c], hi = pr[n * p.n_r + c + 1];
      v[n] = make_float2(fmaf(f, hi.x - lo.x, lo.x), fmaf(f, hi.y - lo.y, lo.y));
    }
    const float m0 = v[0].x * v[0].x + v[0].y * v[0].y;
    const float m1 = v[1].x * v[1].x + v[1].y * v[1].y;
    const float m2 = v[2].x * v[2].x + v[2].y * v[2].y;
    const float re02 = v[0].x * v[2].x + v[0].y * v[2].y;
    const float alpha = Nn * (m0 + m2 + 2.f * m1);
    const float beta = 2.f * (m1 - re02);
    out[q] = 0.25f * fmaf(g, beta, alpha);
  }
}

void launch_bessel_intensity(const BesselParams& p, const float2* prof,
                             const int* slice_em, const int* valid,
                             const int* pix_i0, const float* pix_f,
                             const float* pix_g, float* I, cudaStream_t s) {
  const size_t smem = (size_t)3 * p.n_r * sizeof(float2);
  cudaFuncSetAttribute(k_bessel_intensity,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_bessel_intensity<<<p.n_slices, 256, smem, s>>>(p, prof, slice_em, valid,
                                                   pix_i0, pix_f, pix_g, I);
}

}  // namespace psf
