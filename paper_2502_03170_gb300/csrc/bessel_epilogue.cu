// Radial -> Cartesian epilogue of the Bessel strategy (Eq. 10) using the
// mirror symmetry of the centred output grid.
//
// With I_n^a = p_a I_n, |E|^2 = (alpha + gamma beta) / 4 where
//   alpha = N (|I0|^2 + |I2|^2 + 2 |I1|^2),  beta = 2 (|I1|^2 - Re(conj(I0) I2)),
//   gamma = S1 cos 2phi + S2 sin 2phi,  N = |p_x|^2 + |p_y|^2,
//   S1 = |p_x|^2 - |p_y|^2,  S2 = 2 Re(conj(p_x) p_y),
// and the I_n are the complex linear interpolants of the radial profiles at
// the pixel radius.  Mirroring x or y keeps the radius and cos 2phi and flips
// sin 2phi, so one evaluation serves four output pixels.
//
// Inside radial cell c the interpolant is I_n = P_n[c] + f D_n[c] with
// D_n[c] = P_n[c+1] - P_n[c], so alpha/4 and beta/4 are exact quadratics in f:
//   alpha/4 = A0 + A1 f + A2 f^2,  beta/4 = B0 + B1 f + B2 f^2,
// with per-cell coefficients built once per slice from |P|^2, 2 Re(conj(P) D),
// |D|^2 and the matching I0-I2 cross terms.  Each pixel then reads one cell
// record instead of six profile values.
#include "bessel_kernels.cuh"

namespace psf {

constexpr int MIR_THREADS = 256;
constexpr int MIR_SLICES = 32;       // slices per CTA
constexpr int MIR_REG_GROUPS = 4;    // quarter groups per thread kept in registers

bool bessel_mirror_fit(int nx, int ny, int n_r) {
  // shared memory: cell records (24 B) + two profile buffers (48 B) per radius
  return nx % 2 == 0 && ny % 8 == 0 && 72LL * n_r <= 100 * 1024;
}

__global__ void k_quarter_table(BesselParams p, float4* qtab) {
  const int QH = p.nx / 2, QW = p.ny / 2;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= QH * QW) return;
  const int a = idx / QW, b = idx - (idx / QW) * QW;
  const double x = (a - 0.5 * (p.nx - 1)) * p.dx;   // < 0 in the quarter
  const double y = (b - 0.5 * (p.ny - 1)) * p.dy;   // < 0 in the quarter
  const double rho = sqrt(x * x + y * y);
  const double tt = p.dr > 0 ? rho / p.dr : 0.0;
  int c = (int)floor(tt);
  c = c < 0 ? 0 : (c > p.n_r - 2 ? p.n_r - 2 : c);
  const double c2 = (x * x - y * y) / (rho * rho);
  const double s2 = 2.0 * x * y / (rho * rho);
  const double S1 = p.pol[0] * p.pol[0] + p.pol[1] * p.pol[1] -
                    p.pol[2] * p.pol[2] - p.pol[3] * p.pol[3];
  const double S2 = 2.0 * (p.pol[0] * p.pol[2] + p.pol[1] * p.pol[3]);
  qtab[idx] = make_float4(__int_as_float(c), (float)(tt - c), (float)(S1 * c2),
                          (float)(S2 * s2));
}

void launch_quarter_table(const BesselParams& p, float4* qtab, cudaStream_t s) {
  const int n = (p.nx / 2) * (p.ny / 2);
  k_quarter_table<<<ceil_div(n, 256), 256, 0, s>>>(p, qtab);
}

__device__ __forceinline__ float re_conj_mul(float2 a, float2 b) {
  return a.x * b.x + a.y * b.y;          // Re(conj(a) b)
}

template <bool REG>
__global__ void __launch_bounds__(MIR_THREADS)
k_bessel_intensity_mirror(BesselParams p, const float2* __restrict__ prof,
                          const int* __restrict__ slice_em,
                          const int* __restrict__ valid,
                          const float4* __restrict__ qtab, float* __restrict__ I) {
  extern __shared__ float4 smf[];
  const int rows = 3 * p.n_r;
  const int ncell = p.n_r - 1;
  float4* CA = smf;                                   // [ncell] (A0, A1, A2, B0)
  float2* CB = (float2*)(smf + ncell);                // [ncell] (B1, B2)
  float2* PB = (float2*)(CB + ((ncell + 1) & ~1));    // two profile buffers [2][rows]
  const int QW = p.ny / 2, QH = p.nx / 2;
  const int gw = QW / 4, G = QH * gw;                 // 4-pixel groups of the quarter
  const int npix = p.nx * p.ny;
  const float Nq = 0.25f * (float)(p.pol[0] * p.pol[0] + p.pol[1] * p.pol[1] +
                                   p.pol[2] * p.pol[2] + p.pol[3] * p.pol[3]);
  const int tid = threadIdx.x;
  const int s0 = blockIdx.x * MIR_SLICES;
  const int s1 = min(s0 + MIR_SLICES, p.n_slices);

  float4 qc[REG ? MIR_REG_GROUPS : 1][4];
  if (REG) {
#pragma unroll
    for (int k = 0; k < MIR_REG_GROUPS; ++k) {
      const int g = tid + k * MIR_THREADS;
#pragma unroll
      for (int j = 0; j < 4; ++j) qc[k][j] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (g < G) {
        const int a = g / gw, b4 = (g - (g / gw) * gw) * 4;
#pragma unroll
        for (int j = 0; j < 4; ++j) qc[k][j] = qtab[a * QW + b4 + j];
      }
    }
  }

  for (int q = tid; q < rows; q += MIR_THREADS) PB[q] = prof[(size_t)s0 * rows + q];
  int e_cur = slice_em[s0];
  bool ok_cur = e_cur >= 0 && valid[e_cur];
  int buf = 0;
  for (int s = s0; s < s1; ++s) {
    asm volatile("cp.async.wait_all;" ::: "memory");   // this thread's copies of P_s
    __syncthreads();                      // profile s ready; CA/CB free
    // asynchronous copy of the next slice's profile into the other buffer
    const bool has_next = s + 1 < s1;
    if (has_next) {
      float2* Q = PB + (buf ^ 1) * rows;
      for (int q = tid; q < rows; q += MIR_THREADS) {
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(Q + q);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst),
                     "l"(prof + (size_t)(s + 1) * rows + q)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    const int e_nxt = has_next ? slice_em[s + 1] : -1;
    const float2* P = PB + buf * rows;
    if (ok_cur) {
      // per-cell quadratic coefficients
      for (int c = tid; c < ncell; c += MIR_THREADS) {
        float2 v[3], d[3];
#pragma unroll
        for (int n = 0; n < 3; ++n) {
          v[n] = P[n * p.n_r + c];
          const float2 h = P[n * p.n_r + c + 1];
          d[n] = make_float2(h.x - v[n].x, h.y - v[n].y);
        }
        float q0[3], q1[3], q2[3];
#pragma unroll
        for (int n = 0; n < 3; ++n) {
          q0[n] = re_conj_mul(v[n], v[n]);
          q1[n] = 2.f * re_conj_mul(v[n], d[n]);
          q2[n] = re_conj_mul(d[n], d[n]);
        }
        const float x0 = re_conj_mul(v[0], v[2]);
        const float x1 = re_conj_mul(v[0], d[2]) + re_conj_mul(d[0], v[2]);
        const float x2 = re_conj_mul(d[0], d[2]);
        CA[c] = make_float4(Nq * (q0[0] + q0[2] + 2.f * q0[1]),
                            Nq * (q1[0] + q1[2] + 2.f * q1[1]),
                            Nq * (q2[0] + q2[2] + 2.f * q2[1]),
                            0.5f * (q0[1] - x0));
        CB[c] = make_float2(0.5f * (q1[1] - x1), 0.5f * (q2[1] - x2));
      }
    }
    __syncthreads();
    if (ok_cur) {
      float* out = I + (size_t)s * npix;
      const int kmax = REG ? MIR_REG_GROUPS : (G + MIR_THREADS - 1) / MIR_THREADS;
#pragma unroll
      for (int k = 0; k < (REG ? MIR_REG_GROUPS : 1); ++k) {
        for (int kk = (REG ? k : 0); kk < (REG ? k + 1 : kmax); ++kk) {
          const int g = tid + kk * MIR_THREADS;
          if (g >= G) break;
          const int a = g / gw, b4 = (g - (g / gw) * gw) * 4;
          float vp[4], vm[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float4 t = REG ? qc[k][j] : qtab[a * QW + b4 + j];
            const int c = __float_as_int(t.x);
            const float f = t.y;
            const float4 ca = CA[c];
            const float2 cb = CB[c];
            const float al = fmaf(fmaf(ca.z, f, ca.y), f, ca.x);
            const float be = fmaf(fmaf(cb.y, f, cb.x), f, ca.w);
            vp[j] = fmaf(t.z + t.w, be, al);   // (a, b) and (nx-1-a, ny-1-b)
            vm[j] = fmaf(t.z - t.w, be, al);   // one coordinate mirrored
          }
          const int am = p.nx - 1 - a, bm = p.ny - 4 - b4;
          *(float4*)(out + (size_t)a * p.ny + b4) = make_float4(vp[0], vp[1], vp[2], vp[3]);
          *(float4*)(out + (size_t)a * p.ny + bm) = make_float4(vm[3], vm[2], vm[1], vm[0]);
          *(float4*)(out + (size_t)am * p.ny + b4) = make_float4(vm[0], vm[1], vm[2], vm[3]);
          *(float4*)(out + (size_t)am * p.ny + bm) = make_float4(vp[3], vp[2], vp[1], vp[0]);
        }
      }
    }
    ok_cur = e_nxt >= 0 && valid[e_nxt];
    buf ^= 1;
  }
}

void launch_bessel_intensity_mirror(const BesselParams& p, const float2* prof,
                                    const int* slice_em, const int* valid,
                                    const float4* qtab, float* I,
                                    cudaStream_t s) {
  const int ncell = p.n_r - 1;
  const size_t smem = (size_t)ncell * sizeof(float4) +
                      (size_t)((ncell + 1) & ~1) * sizeof(float2) +
                      (size_t)2 * 3 * p.n_r * sizeof(float2);
  const int G = (p.nx / 2) * (p.ny / 8);
  const dim3 grid(ceil_div(p.n_slices, MIR_SLICES));
  if (G <= MIR_REG_GROUPS * MIR_THREADS) {
    cudaFuncSetAttribute(k_bessel_intensity_mirror<true>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_bessel_intensity_mirror<true><<<grid, MIR_THREADS, smem, s>>>(
        p, prof, slice_em, valid, qtab, I);
  } else {
    cudaFuncSetAttribute(k_bessel_intensity_mirror<false>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_bessel_intensity_mirror<false><<<grid, MIR_THREADS, smem, s>>>(
        p, prof, slice_em, valid, qtab, I);
  }
}

}  // namespace psf
