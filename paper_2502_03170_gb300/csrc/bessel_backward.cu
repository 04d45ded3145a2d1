// Adjoint of the Bessel (spherical) strategy, Eq. 10-11: gradients of a
// z-stack loss with respect to a free radial pupil phase W_0(theta_j), the
// m = 0 Zernike coefficients (Eq. 15) and the emitter depth (Eq. 13-14).
//
// The forward per slice is P = B F (radial contraction, B real), linear
// interpolation of P at each pixel radius and |E|^2 = (alpha + gamma beta)/4
// with alpha = N(|v0|^2 + |v2|^2 + 2|v1|^2), beta = 2(|v1|^2 - Re(conj(v0) v2)).
// With the complex gradient convention g = dL/dRe + i dL/dIm the pixel
// gradients are
//   g_v0 = G/2 (N v0 - gamma v2),  g_v1 = G (N + gamma) v1,
//   g_v2 = G/2 (N v2 - gamma v0),  G = dL/dI,
// and the interpolation transposes them onto the two radii of the pixel's
// cell.  Because v_n = u P_n[c] + f P_n[c+1] (u = 1 - f) is fixed by the cell,
// a cell needs only six moments of its pixels,
//   M_k = sum G u^(2-k) f^k,  K_k = sum G gamma u^(2-k) f^k   (k = 0, 1, 2),
// to produce its contribution to the radii c and c+1.  The pixels of a cell
// are visited in a fixed order (a per-call table sorted by cell), so every
// sum has a fixed order and the result is bitwise reproducible.
#include <cuda_bf16.h>

#include "bessel_backward.cuh"
#include "tc_ptx.cuh"

namespace psf {

// ---------------------------------------------------------------------------
// Kernel A: per slice, dL/dI -> cell moments -> g_P [3][n_r] (in place of P).
// One CTA per slice.  P is read into shared memory first and the CTA then
// overwrites the same profile row with its gradient, so no second
// [n_slices][3][n_r] buffer is needed.  With `target` the loss is
// sum (I - T)^2 and I is recomputed from P (G = 2 (I - T)); otherwise
// G = grad_intensity.  The slice's G (or T) is staged in shared memory when it
// fits (96 KB of shared memory in all), read from global memory otherwise.
// ---------------------------------------------------------------------------
template <bool TARGET, bool STAGE>
__global__ void __launch_bounds__(256)
k_bessel_adj_epilogue(BesselParams p, float2* __restrict__ prof,
                      const int* __restrict__ slice_em, const int* __restrict__ valid,
                      const PixGroup* __restrict__ groups,
                      const int* __restrict__ cell_start,
                      const float* __restrict__ T, const float* __restrict__ Gin,
                      float* __restrict__ loss_slice) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n_r = p.n_r, rows = 3 * n_r;
  float2* P = reinterpret_cast<float2*>(smem);          // [3][n_r]
  float2* lo = P + rows;                                  // [3][n_r] cell c -> radius c
  float2* hi = lo + rows;                                 // [3][n_r] cell c -> radius c+1
  float* red = reinterpret_cast<float*>(hi + rows);      // [8] warp partial losses
  float* Gs = red + 8;                                    // [npix] staged G or T
  const int s = blockIdx.x;
  const int tid = threadIdx.x;
  const int npix = p.nx * p.ny;
  float2* ps = prof + (size_t)s * rows;
  const int e = slice_em[s];
  if (e < 0 || !valid[e]) {
    for (int q = tid; q < rows; q += blockDim.x) ps[q] = make_float2(0.f, 0.f);
    if (TARGET && tid == 0) loss_slice[s] = 0.f;
    return;
  }
  const float* src = (TARGET ? T : Gin) + (size_t)s * npix;
  for (int q = tid; q < rows; q += blockDim.x) P[q] = ps[q];
  if (STAGE)
    for (int q = tid; q < npix; q += blockDim.x) Gs[q] = __ldg(&src[q]);
  __syncthreads();
  const float* gsrc = STAGE ? Gs : src;

  const float Nn = (float)(p.pol[0] * p.pol[0] + p.pol[1] * p.pol[1] +
                           p.pol[2] * p.pol[2] + p.pol[3] * p.pol[3]);
  float loss = 0.f;
  const int n_cells = n_r - 1;
  for (int c = tid; c < n_cells; c += blockDim.x) {
    float2 Pc[3], Pd[3];
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      Pc[n] = P[n * n_r + c];
      Pd[n] = P[n * n_r + c + 1];
    }
    float M0 = 0.f, M1 = 0.f, M2 = 0.f, K0 = 0.f, K1 = 0.f, K2 = 0.f;
    const int g0 = cell_start[c], g1 = cell_start[c + 1];
    for (int gi = g0; gi < g1; ++gi) {
      const PixGroup gr = groups[gi];
      const float f = gr.f, u = 1.f - f;
      float wsum = 0.f, wg = 0.f;
      if (TARGET) {
        float2 v[3];
#pragma unroll
        for (int n = 0; n < 3; ++n)
          v[n] = make_float2(fmaf(f, Pd[n].x - Pc[n].x, Pc[n].x),
                             fmaf(f, Pd[n].y - Pc[n].y, Pc[n].y));
        const float m0 = v[0].x * v[0].x + v[0].y * v[0].y;
        const float m1 = v[1].x * v[1].x + v[1].y * v[1].y;
        const float m2 = v[2].x * v[2].x + v[2].y * v[2].y;
        const float re02 = v[0].x * v[2].x + v[0].y * v[2].y;
        const float alpha = Nn * (m0 + m2 + 2.f * m1);
        const float beta = 2.f * (m1 - re02);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int px = gr.pix[k];
          if (px < 0) continue;
          const float gam = (k == 0 || k == 3) ? gr.gc + gr.gs : gr.gc - gr.gs;
          const float d = 0.25f * fmaf(gam, beta, alpha) - gsrc[px];
          loss = fmaf(d, d, loss);
          const float G = 2.f * d;
          wsum += G;
          wg = fmaf(G, gam, wg);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int px = gr.pix[k];
          if (px < 0) continue;
          const float gam = (k == 0 || k == 3) ? gr.gc + gr.gs : gr.gc - gr.gs;
          const float G = gsrc[px];
          wsum += G;
          wg = fmaf(G, gam, wg);
        }
      }
      const float uu = u * u, uf = u * f, ff = f * f;
      M0 = fmaf(wsum, uu, M0);
      M1 = fmaf(wsum, uf, M1);
      M2 = fmaf(wsum, ff, M2);
      K0 = fmaf(wg, uu, K0);
      K1 = fmaf(wg, uf, K1);
      K2 = fmaf(wg, ff, K2);
    }
    // sum over the cell's pixels of the weighted g_v_n, split onto c and c+1
    auto comb = [&](float a, float b, const float2& x, const float2& y) {
      return make_float2(fmaf(a, x.x, b * y.x), fmaf(a, x.y, b * y.y));
    };
    float2 dn[3], up[3];
    {
      const float2 A0 = comb(M0, M1, Pc[0], Pd[0]), A1 = comb(M0, M1, Pc[1], Pd[1]),
                   A2 = comb(M0, M1, Pc[2], Pd[2]);
      const float2 B0 = comb(K0, K1, Pc[0], Pd[0]), B1 = comb(K0, K1, Pc[1], Pd[1]),
                   B2 = comb(K0, K1, Pc[2], Pd[2]);
      dn[0] = make_float2(0.5f * (Nn * A0.x - B2.x), 0.5f * (Nn * A0.y - B2.y));
      dn[1] = make_float2(fmaf(Nn, A1.x, B1.x), fmaf(Nn, A1.y, B1.y));
      dn[2] = make_float2(0.5f * (Nn * A2.x - B0.x), 0.5f * (Nn * A2.y - B0.y));
    }
    {
      const float2 A0 = comb(M1, M2, Pc[0], Pd[0]), A1 = comb(M1, M2, Pc[1], Pd[1]),
                   A2 = comb(M1, M2, Pc[2], Pd[2]);
      const float2 B0 = comb(K1, K2, Pc[0], Pd[0]), B1 = comb(K1, K2, Pc[1], Pd[1]),
                   B2 = comb(K1, K2, Pc[2], Pd[2]);
      up[0] = make_float2(0.5f * (Nn * A0.x - B2.x), 0.5f * (Nn * A0.y - B2.y));
      up[1] = make_float2(fmaf(Nn, A1.x, B1.x), fmaf(Nn, A1.y, B1.y));
      up[2] = make_float2(0.5f * (Nn * A2.x - B0.x), 0.5f * (Nn * A2.y - B0.y));
    }
#pragma unroll
    for (int n = 0; n < 3; ++n) {
      lo[n * n_r + c] = dn[n];
      hi[n * n_r + c + 1] = up[n];
    }
  }
  if (tid == 0)
    for (int n = 0; n < 3; ++n) {
      hi[n * n_r] = make_float2(0.f, 0.f);               // radius 0: no cell below
      lo[n * n_r + n_r - 1] = make_float2(0.f, 0.f);     // last radius: no cell above
    }
  __syncthreads();
  // g_P[c] = lo(cell c) + hi(cell c - 1)
  for (int q = tid; q < rows; q += blockDim.x) {
    const float2 a = lo[q], b = hi[q];
    ps[q] = make_float2(a.x + b.x, a.y + b.y);
  }
  if (TARGET) {
    // fixed-order block reduction of the slice loss
    for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
    if ((tid & 31) == 0) red[tid >> 5] = loss;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      loss_slice[s] = t;
    }
  }
}

size_t bessel_adj_epilogue_smem(const BesselParams& p, bool stage) {
  size_t b = (size_t)9 * p.n_r * sizeof(float2) + 8 * sizeof(float);
  if (stage) b += (size_t)p.nx * p.ny * sizeof(float);
  return b;
}

bool bessel_adj_stage_fits(const BesselParams& p) {
  return bessel_adj_epilogue_smem(p, true) <= 96 * 1024;
}

void launch_bessel_adj_epilogue(const BesselParams& p, float2* prof, const int* slice_em,
                                const int* valid, const PixGroup* groups,
                                const int* cell_start, const float* target,
                                const float* grad_intensity, float* loss_slice,
                                cudaStream_t s) {
  const bool stage = bessel_adj_stage_fits(p);
  const size_t smem = bessel_adj_epilogue_smem(p, stage);
  const bool tgt = target != nullptr;
#define PSF_ADJ_LAUNCH(TG, ST)                                                        \
  do {                                                                                \
    cudaFuncSetAttribute(k_bessel_adj_epilogue<TG, ST>,                               \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     \
    k_bessel_adj_epilogue<TG, ST><<<p.n_slices, 256, smem, s>>>(                      \
        p, prof, slice_em, valid, groups, cell_start, target, grad_intensity,         \
        loss_slice);                                                                  \
  } while (0)
  if (tgt && stage) PSF_ADJ_LAUNCH(true, true);
  else if (tgt) PSF_ADJ_LAUNCH(true, false);
  else if (stage) PSF_ADJ_LAUNCH(false, true);
  else PSF_ADJ_LAUNCH(false, false);
#undef PSF_ADJ_LAUNCH
}

// ---------------------------------------------------------------------------
// Kernel A, sorted form (grids with at most a few thousand mirror groups):
// the same moments, computed in two passes per slice so that no pass waits on
// global memory inside a serial loop.
//   pass 1: thread per mirror group in natural order (coalesced reads of G
//           or T at the group's up to four pixels) -> (sum G, sum G gamma)
//           stored at the group's position in the cell-sorted order;
//   pass 2: thread per cell, a fixed-order sum over its contiguous run of the
//           sorted array (shared memory only) -> moments -> contributions.
// A CTA takes SE_SLICES slices; the sorted weights f and the cell starts are
// loaded into shared memory once per CTA.
// ---------------------------------------------------------------------------
constexpr int SE_THREADS = 256;
constexpr int SE_SLICES = 8;
constexpr int SE_GPT = 8;            // groups per thread per load batch

size_t bessel_adj_sorted_smem(const BesselParams& p) {
  const size_t ng = (size_t)((p.nx + 1) / 2) * ((p.ny + 1) / 2);
  return (size_t)9 * p.n_r * sizeof(float2) + ng * (sizeof(float2) + sizeof(float)) +
         (size_t)p.n_r * sizeof(int) + 8 * sizeof(float);
}

bool bessel_adj_sorted_fits(const BesselParams& p) {
  return bessel_adj_sorted_smem(p) <= 110 * 1024;
}

// SPLIT: g_P leaves as BF16 hi + lo planes (rows (s, re) and (s, im), row
// pitch kp) for the tensor-core contraction instead of in place of P.
__device__ __forceinline__ void split_bf16(float v, uint16_t& h, uint16_t& l) {
  const __nv_bfloat16 hb = __float2bfloat16_rn(v);
  h = __bfloat16_as_ushort(hb);
  l = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(hb)));
}

template <bool TARGET, bool SPLIT>
__global__ void __launch_bounds__(SE_THREADS)
k_bessel_adj_epilogue_sorted(BesselParams p, float2* __restrict__ prof,
                             const int* __restrict__ slice_em,
                             const int* __restrict__ valid,
                             const int2* __restrict__ gpc,      // natural g: (sorted pos, cell)
                             const float4* __restrict__ gfg,    // natural g: (f, gc, gs, 0)
                             const float* __restrict__ sorted_f,
                             const int* __restrict__ cell_start,
                             const float* __restrict__ T, const float* __restrict__ Gin,
                             float* __restrict__ loss_slice, uint16_t* __restrict__ g_hi,
                             uint16_t* __restrict__ g_lo, int kp) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n_r = p.n_r, rows = 3 * n_r, n_cells = n_r - 1;
  const int hb = (p.ny + 1) / 2, ng = ((p.nx + 1) / 2) * hb;
  const int npix = p.nx * p.ny;
  float2* P = reinterpret_cast<float2*>(smem);
  float2* lo = P + rows;
  float2* hi = lo + rows;
  float2* W = hi + rows;                                  // [ng] sorted order
  float* sf = reinterpret_cast<float*>(W + ng);          // [ng] sorted f
  int* cs = reinterpret_cast<int*>(sf + ng);             // [n_r]
  float* red = reinterpret_cast<float*>(cs + n_r);       // [8]
  const int tid = threadIdx.x;
  for (int q = tid; q < ng; q += SE_THREADS) sf[q] = sorted_f[q];
  for (int q = tid; q < n_r; q += SE_THREADS) cs[q] = cell_start[q];
  const float Nn = (float)(p.pol[0] * p.pol[0] + p.pol[1] * p.pol[1] +
                           p.pol[2] * p.pol[2] + p.pol[3] * p.pol[3]);
  for (int it = 0; it < SE_SLICES; ++it) {
    const int s = blockIdx.x * SE_SLICES + it;
    if (s >= p.n_slices) break;                           // uniform over the CTA
    float2* ps = prof + (size_t)s * rows;
    const int e = slice_em[s];
    __syncthreads();                                      // previous slice done
    if (e < 0 || !valid[e]) {
      for (int q = tid; q < rows; q += SE_THREADS) {
        if (SPLIT) {
          const size_t r0 = (size_t)(2 * s) * kp + q, r1 = r0 + kp;
          g_hi[r0] = g_lo[r0] = g_hi[r1] = g_lo[r1] = 0;
        } else {
          ps[q] = make_float2(0.f, 0.f);
        }
      }
      if (TARGET && tid == 0) loss_slice[s] = 0.f;
      continue;
    }
    for (int q = tid; q < rows; q += SE_THREADS) P[q] = ps[q];
    __syncthreads();
    const float* src = (TARGET ? T : Gin) + (size_t)s * npix;
    float loss = 0.f;
    // pass 1, in chunks of SE_GPT groups per thread: all loads of a chunk are
    // issued before any is used, so a thread keeps 4 SE_GPT reads in flight
    for (int g0 = 0; g0 < ng; g0 += SE_GPT * SE_THREADS) {
    float val[SE_GPT][4];
#pragma unroll
    for (int u = 0; u < SE_GPT; ++u) {
      const int g = g0 + u * SE_THREADS + tid;
      const int a = g / hb, b = g - (g / hb) * hb;
      const int a2 = p.nx - 1 - a, b2 = p.ny - 1 - b;
      const bool in = g < ng;
      val[u][0] = in ? __ldg(&src[a * p.ny + b]) : 0.f;
      val[u][1] = (in && a2 != a) ? __ldg(&src[a2 * p.ny + b]) : 0.f;
      val[u][2] = (in && b2 != b) ? __ldg(&src[a * p.ny + b2]) : 0.f;
      val[u][3] = (in && a2 != a && b2 != b) ? __ldg(&src[a2 * p.ny + b2]) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < SE_GPT; ++u) {
      const int g = g0 + u * SE_THREADS + tid;
      if (g >= ng) break;
      const int2 pc = gpc[g];
      const float4 fg = gfg[g];
      const int a = g / hb, b = g - (g / hb) * hb;
      const int a2 = p.nx - 1 - a, b2 = p.ny - 1 - b;
      int px[4];
      px[0] = a * p.ny + b;
      px[1] = a2 != a ? a2 * p.ny + b : -1;
      px[2] = b2 != b ? a * p.ny + b2 : -1;
      px[3] = (a2 != a && b2 != b) ? a2 * p.ny + b2 : -1;
      float alpha = 0.f, beta = 0.f;
      if (TARGET) {
        const int c = pc.y;
        const float f = fg.x;
        float2 v[3];
#pragma unroll
        for (int n = 0; n < 3; ++n) {
          const float2 x0 = P[n * n_r + c], x1 = P[n * n_r + c + 1];
          v[n] = make_float2(fmaf(f, x1.x - x0.x, x0.x), fmaf(f, x1.y - x0.y, x0.y));
        }
        const float m0 = v[0].x * v[0].x + v[0].y * v[0].y;
        const float m1 = v[1].x * v[1].x + v[1].y * v[1].y;
        const float m2 = v[2].x * v[2].x + v[2].y * v[2].y;
        const float re02 = v[0].x * v[2].x + v[0].y * v[2].y;
        alpha = Nn * (m0 + m2 + 2.f * m1);
        beta = 2.f * (m1 - re02);
      }
      float wsum = 0.f, wg = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (px[k] < 0) continue;
        const float gam = (k == 0 || k == 3) ? fg.y + fg.z : fg.y - fg.z;
        float G;
        if (TARGET) {
          const float d = 0.25f * fmaf(gam, beta, alpha) - val[u][k];
          loss = fmaf(d, d, loss);
          G = 2.f * d;
        } else {
          G = val[u][k];
        }
        wsum += G;
        wg = fmaf(G, gam, wg);
      }
      W[pc.x] = make_float2(wsum, wg);
    }
    }
    __syncthreads();
    // pass 2
    for (int c = tid; c < n_cells; c += SE_THREADS) {
      float M0 = 0.f, M1 = 0.f, M2 = 0.f, K0 = 0.f, K1 = 0.f, K2 = 0.f;
      const int k1 = cs[c + 1];
      for (int k = cs[c]; k < k1; ++k) {
        const float2 w = W[k];
        const float f = sf[k], u = 1.f - f;
        const float uu = u * u, uf = u * f, ff = f * f;
        M0 = fmaf(w.x, uu, M0);
        M1 = fmaf(w.x, uf, M1);
        M2 = fmaf(w.x, ff, M2);
        K0 = fmaf(w.y, uu, K0);
        K1 = fmaf(w.y, uf, K1);
        K2 = fmaf(w.y, ff, K2);
      }
      float2 Pc[3], Pd[3];
#pragma unroll
      for (int n = 0; n < 3; ++n) {
        Pc[n] = P[n * n_r + c];
        Pd[n] = P[n * n_r + c + 1];
      }
      auto comb = [&](float x, float y, const float2& u0, const float2& u1) {
        return make_float2(fmaf(x, u0.x, y * u1.x), fmaf(x, u0.y, y * u1.y));
      };
      {
        const float2 A0 = comb(M0, M1, Pc[0], Pd[0]), A1 = comb(M0, M1, Pc[1], Pd[1]),
                     A2 = comb(M0, M1, Pc[2], Pd[2]);
        const float2 B0 = comb(K0, K1, Pc[0], Pd[0]), B1 = comb(K0, K1, Pc[1], Pd[1]),
                     B2 = comb(K0, K1, Pc[2], Pd[2]);
        lo[c] = make_float2(0.5f * (Nn * A0.x - B2.x), 0.5f * (Nn * A0.y - B2.y));
        lo[n_r + c] = make_float2(fmaf(Nn, A1.x, B1.x), fmaf(Nn, A1.y, B1.y));
        lo[2 * n_r + c] = make_float2(0.5f * (Nn * A2.x - B0.x), 0.5f * (Nn * A2.y - B0.y));
      }
      {
        const float2 A0 = comb(M1, M2, Pc[0], Pd[0]), A1 = comb(M1, M2, Pc[1], Pd[1]),
                     A2 = comb(M1, M2, Pc[2], Pd[2]);
        const float2 B0 = comb(K1, K2, Pc[0], Pd[0]), B1 = comb(K1, K2, Pc[1], Pd[1]),
                     B2 = comb(K1, K2, Pc[2], Pd[2]);
        hi[c + 1] = make_float2(0.5f * (Nn * A0.x - B2.x), 0.5f * (Nn * A0.y - B2.y));
        hi[n_r + c + 1] = make_float2(fmaf(Nn, A1.x, B1.x), fmaf(Nn, A1.y, B1.y));
        hi[2 * n_r + c + 1] =
            make_float2(0.5f * (Nn * A2.x - B0.x), 0.5f * (Nn * A2.y - B0.y));
      }
    }
    if (tid == 0)
      for (int n = 0; n < 3; ++n) {
        hi[n * n_r] = make_float2(0.f, 0.f);
        lo[n * n_r + n_r - 1] = make_float2(0.f, 0.f);
      }
    if (TARGET) {
      for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
      if ((tid & 31) == 0) red[tid >> 5] = loss;
    }
    __syncthreads();
    for (int q = tid; q < rows; q += SE_THREADS) {
      const float2 x = lo[q], y = hi[q];
      const float2 v = make_float2(x.x + y.x, x.y + y.y);
      if (SPLIT) {
        const size_t r0 = (size_t)(2 * s) * kp + q, r1 = r0 + kp;
        uint16_t h, l;
        split_bf16(v.x, h, l);
        g_hi[r0] = h;
        g_lo[r0] = l;
        split_bf16(v.y, h, l);
        g_hi[r1] = h;
        g_lo[r1] = l;
      } else {
        ps[q] = v;
      }
    }
    if (TARGET && tid == 0) {
      float t = 0.f;
      for (int w = 0; w < SE_THREADS / 32; ++w) t += red[w];
      loss_slice[s] = t;
    }
  }
}

void launch_bessel_adj_epilogue_sorted(const BesselParams& p, float2* prof,
                                       const int* slice_em, const int* valid,
                                       const int2* gpc, const float4* gfg,
                                       const float* sorted_f, const int* cell_start,
                                       const float* target, const float* grad_intensity,
                                       float* loss_slice, uint16_t* g_hi, uint16_t* g_lo,
                                       int kp, cudaStream_t s) {
  const size_t smem = bessel_adj_sorted_smem(p);
  const unsigned grid = (unsigned)ceil_div(p.n_slices, SE_SLICES);
  const bool split = g_hi != nullptr;
#define PSF_ADJ_SORTED(TG, SP)                                                         \
  do {                                                                                 \
    cudaFuncSetAttribute(k_bessel_adj_epilogue_sorted<TG, SP>,                         \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);      \
    k_bessel_adj_epilogue_sorted<TG, SP><<<grid, SE_THREADS, smem, s>>>(               \
        p, prof, slice_em, valid, gpc, gfg, sorted_f, cell_start, target,              \
        grad_intensity, loss_slice, g_hi, g_lo, kp);                                   \
  } while (0)
  if (target && split) PSF_ADJ_SORTED(true, true);
  else if (target) PSF_ADJ_SORTED(true, false);
  else if (split) PSF_ADJ_SORTED(false, true);
  else PSF_ADJ_SORTED(false, false);
#undef PSF_ADJ_SORTED
}

// ---------------------------------------------------------------------------
// Kernel A, staged form (the benchmark-sized grids): the sorted two-pass
// reduction with each slice's dL/dI (or T) and profiles brought into shared
// memory by the TMA engine (cp.async.bulk, double-buffered on two mbarriers),
// so the next slice streams in while the current one is reduced.  One CTA
// per SM walks slices s = blockIdx.x, + gridDim.x, ...; each thread keeps its
// SB_GPT mirror groups' table entries in registers; the per-cell sums of pass
// 2 are split into two halves (threads t and t + 256) and added in a fixed
// order.  Every wait is bounded: on time-out the kernel records
// PSF_ERR_DEVICE_TIMEOUT, waits (bounded) for its own copy in flight and
// returns.
// ---------------------------------------------------------------------------
constexpr int SB_THREADS = 512;
constexpr int SB_GPT = 8;                    // groups per thread (<= 4096 groups)

struct SbLayout {
  size_t bars, flag, gbuf, pbuf, W, sf, cs, lo, hi, mp, red, bytes;
};

__host__ __device__ inline SbLayout sb_layout(int npix, int n_r, int ng) {
  SbLayout L;
  const size_t rows = 3 * (size_t)n_r, ncell = (size_t)n_r - 1;
  size_t o = 0;
  auto take = [&](size_t bytes, size_t align) {
    o = (o + align - 1) / align * align;
    const size_t r = o;
    o += bytes;
    return r;
  };
  L.bars = take(2 * sizeof(unsigned long long), 8);
  L.flag = take(sizeof(int), 4);
  L.gbuf = take(2 * (size_t)npix * sizeof(float), 128);
  L.pbuf = take(2 * rows * sizeof(float2), 128);
  // sorted per-group values, padded by one entry per cell (index k + cell):
  // the threads of pass 2a walk consecutive cells' runs in lockstep, and
  // without the padding runs of ~16 entries put their lanes on the same banks
  L.W = take(((size_t)ng + n_r) * sizeof(float2), 16);
  L.sf = take(((size_t)ng + n_r) * sizeof(float), 16);
  L.cs = take((size_t)n_r * sizeof(int), 16);
  L.lo = take(rows * sizeof(float2), 16);
  L.hi = take(rows * sizeof(float2), 16);
  L.mp = take(2 * ncell * 6 * sizeof(float), 16);
  L.red = take(SB_THREADS / 32 * sizeof(float), 16);
  L.bytes = (o + 127) / 128 * 128;
  return L;
}

bool bessel_adj_staged_fits(const BesselParams& p, const void* src) {
  const int ng = ((p.nx + 1) / 2) * ((p.ny + 1) / 2);
  const int npix = p.nx * p.ny;
  return ng <= SB_THREADS * SB_GPT && (npix % 4) == 0 && (p.n_r % 2) == 0 &&
         ((uintptr_t)src & 15) == 0 && sb_layout(npix, p.n_r, ng).bytes <= 227 * 1024;
}

template <bool TARGET, bool SPLIT, bool EVEN>
__global__ void __launch_bounds__(SB_THREADS, 1)
k_bessel_adj_epilogue_staged(BesselParams p, float2* __restrict__ prof,
                             const int* __restrict__ slice_em,
                             const int* __restrict__ valid,
                             const int2* __restrict__ gpc, const float4* __restrict__ gfg,
                             const float* __restrict__ sorted_f,
                             const int* __restrict__ cell_start,
                             const float* __restrict__ src_all,
                             float* __restrict__ loss_slice, uint16_t* __restrict__ g_hi,
                             uint16_t* __restrict__ g_lo, int kp, int* status) {
  using namespace tc;
  extern __shared__ __align__(128) unsigned char smem_sb[];
  const int n_r = p.n_r, rows = 3 * n_r, n_cells = n_r - 1;
  const int hb = (p.ny + 1) / 2, ng = ((p.nx + 1) / 2) * hb;
  const int npix = p.nx * p.ny;
  const SbLayout L = sb_layout(npix, n_r, ng);
  const uint32_t bar0 = smem_u32(smem_sb + L.bars);
  volatile int* flag = reinterpret_cast<volatile int*>(smem_sb + L.flag);
  float* Gb = reinterpret_cast<float*>(smem_sb + L.gbuf);
  float2* Pb = reinterpret_cast<float2*>(smem_sb + L.pbuf);
  float2* W = reinterpret_cast<float2*>(smem_sb + L.W);
  float* sf = reinterpret_cast<float*>(smem_sb + L.sf);
  int* cs = reinterpret_cast<int*>(smem_sb + L.cs);
  float2* lo = reinterpret_cast<float2*>(smem_sb + L.lo);
  float2* hi = reinterpret_cast<float2*>(smem_sb + L.hi);
  float* mp = reinterpret_cast<float*>(smem_sb + L.mp);
  float* red = reinterpret_cast<float*>(smem_sb + L.red);
  const int tid = threadIdx.x;
  const uint32_t g_bytes = (uint32_t)npix * 4u, p_bytes = (uint32_t)rows * 8u;

  auto issue = [&](int s, int b) {
    const uint32_t bar = bar0 + 8u * b;
    mbar_arrive_expect_tx(bar, g_bytes + p_bytes);
    bulk_load_1d(smem_u32(Gb + (size_t)b * npix), src_all + (size_t)s * npix, g_bytes, bar);
    bulk_load_1d(smem_u32(Pb + (size_t)b * rows), prof + (size_t)s * rows, p_bytes, bar);
  };
  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8, 1);
    *flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0 && (int)blockIdx.x < p.n_slices) issue(blockIdx.x, 0);

  // Slice-independent data of this thread's mirror groups, in registers:
  // pixel (a, b) and its mirrors, sorted position | cell << 16, f, and the
  // polarisation factors gamma of the unflipped (gp) and once-flipped (gm)
  // mirrors.
  int tpix[SB_GPT], tdx[SB_GPT], tdy[SB_GPT], tpc[SB_GPT];
  float tf[SB_GPT], tgp[SB_GPT], tgm[SB_GPT];
#pragma unroll
  for (int k = 0; k < SB_GPT; ++k) {
    const int g = tid + k * SB_THREADS;
    tpix[k] = -1;
    tdx[k] = tdy[k] = tpc[k] = 0;
    tf[k] = tgp[k] = tgm[k] = 0.f;
    if (g < ng) {
      const int a = g / hb, bb = g - (g / hb) * hb;
      const int2 pc = gpc[g];
      const float4 fg = gfg[g];
      tpix[k] = a * p.ny + bb;
      tdx[k] = (p.nx - 1 - 2 * a) * p.ny;        // (a, b) -> (nx-1-a, b); 0: same pixel
      tdy[k] = p.ny - 1 - 2 * bb;                // (a, b) -> (a, ny-1-b); 0: same pixel
      tpc[k] = pc.x | (pc.y << 16);
      tf[k] = fg.x;
      tgp[k] = fg.y + fg.z;
      tgm[k] = fg.y - fg.z;
    }
  }
  for (int c = tid; c < n_r - 1; c += SB_THREADS)
    for (int q = cell_start[c]; q < cell_start[c + 1]; ++q) sf[q + c] = sorted_f[q];
  for (int q = tid; q < n_r; q += SB_THREADS) cs[q] = cell_start[q];
  const float Nn = (float)(p.pol[0] * p.pol[0] + p.pol[1] * p.pol[1] +
                           p.pol[2] * p.pol[2] + p.pol[3] * p.pol[3]);
  uint32_t phase[2] = {0u, 0u};
  int it = 0;
  for (int s = blockIdx.x; s < p.n_slices; s += gridDim.x, ++it) {
    const int b = it & 1;
    const int s_next = s + gridDim.x;
    if (tid == 0) {
      if (s_next < p.n_slices) issue(s_next, b ^ 1);
      if (!mbar_wait(bar0 + 8u * b, phase[b], flag, status)) {
        // give up: let this CTA's copies in flight land (bounded) before leaving
        mbar_drain_wait(bar0 + 8u * b, phase[b]);
        if (s_next < p.n_slices) mbar_drain_wait(bar0 + 8u * (b ^ 1), phase[b ^ 1]);
        *flag = 1;
      }
    }
    __syncthreads();
    if (*flag) return;
    phase[b] ^= 1u;
    const float* Gs = Gb + (size_t)b * npix;
    const float2* P = Pb + (size_t)b * rows;
    const int e = slice_em[s];
    const bool ok = e >= 0 && valid[e];
    float loss = 0.f;
    if (ok) {
      // pass 1: mirror groups -> (sum G, sum G gamma) at their sorted positions
#pragma unroll
      for (int k = 0; k < SB_GPT; ++k) {
        if (tpix[k] < 0) continue;
        const int p0 = tpix[k], p1 = p0 + tdx[k], p2 = p0 + tdy[k], p3 = p1 + tdy[k];
        float alpha = 0.f, beta = 0.f;
        if (TARGET) {
          const int c = tpc[k] >> 16;
          const float f = tf[k];
          float2 v[3];
#pragma unroll
          for (int n = 0; n < 3; ++n) {
            const float2 x0 = P[n * n_r + c], x1 = P[n * n_r + c + 1];
            v[n] = make_float2(fmaf(f, x1.x - x0.x, x0.x), fmaf(f, x1.y - x0.y, x0.y));
          }
          const float m0 = v[0].x * v[0].x + v[0].y * v[0].y;
          const float m1 = v[1].x * v[1].x + v[1].y * v[1].y;
          const float m2 = v[2].x * v[2].x + v[2].y * v[2].y;
          const float re02 = v[0].x * v[2].x + v[0].y * v[2].y;
          alpha = Nn * (m0 + m2 + 2.f * m1);
          beta = 2.f * (m1 - re02);
        }
        // mirrors 0 and 3 take gamma = gp, mirrors 1 and 2 gamma = gm; a mirror
        // that coincides with an earlier pixel (odd grids) is skipped
        const bool h1 = EVEN || tdx[k] != 0, h2 = EVEN || tdy[k] != 0;
        const bool h3 = EVEN || (h1 && h2);
        float v0 = Gs[p0];
        float v1 = h1 ? Gs[p1] : 0.f, v2 = h2 ? Gs[p2] : 0.f, v3 = h3 ? Gs[p3] : 0.f;
        if (TARGET) {
          const float ip = 0.25f * fmaf(tgp[k], beta, alpha);
          const float im = 0.25f * fmaf(tgm[k], beta, alpha);
          const float d0 = ip - v0, d1 = im - v1, d2 = im - v2, d3 = ip - v3;
          loss = fmaf(d0, d0, loss);
          if (h1) loss = fmaf(d1, d1, loss);
          if (h2) loss = fmaf(d2, d2, loss);
          if (h3) loss = fmaf(d3, d3, loss);
          v0 = 2.f * d0;
          v1 = h1 ? 2.f * d1 : 0.f;
          v2 = h2 ? 2.f * d2 : 0.f;
          v3 = h3 ? 2.f * d3 : 0.f;
        }
        const float sp = v0 + v3, sm = v1 + v2;
        W[(tpc[k] & 0xFFFF) + (tpc[k] >> 16)] =
            make_float2(sp + sm, fmaf(tgp[k], sp, tgm[k] * sm));
      }
    }
    __syncthreads();
    if (ok) {
      // pass 2a: each cell's sorted run in two halves
      const int half = tid >> 8;
      for (int c = tid & 255; c < n_cells; c += 256) {
        const int k0 = cs[c], k1 = cs[c + 1], mid = (k0 + k1) >> 1;
        float M0 = 0.f, M1 = 0.f, M2 = 0.f, K0 = 0.f, K1 = 0.f, K2 = 0.f;
#pragma unroll 4
        for (int k = half ? mid : k0; k < (half ? k1 : mid); ++k) {
          const float2 w = W[k + c];
          const float f = sf[k + c], u = 1.f - f;
          const float uu = u * u, uf = u * f, ff = f * f;
          M0 = fmaf(w.x, uu, M0);
          M1 = fmaf(w.x, uf, M1);
          M2 = fmaf(w.x, ff, M2);
          K0 = fmaf(w.y, uu, K0);
          K1 = fmaf(w.y, uf, K1);
          K2 = fmaf(w.y, ff, K2);
        }
        float* m = mp + ((size_t)half * n_cells + c) * 6;
        m[0] = M0; m[1] = M1; m[2] = M2; m[3] = K0; m[4] = K1; m[5] = K2;
      }
    }
    if (TARGET) {
      for (int o = 16; o > 0; o >>= 1) loss += __shfl_down_sync(0xffffffffu, loss, o);
      if ((tid & 31) == 0) red[tid >> 5] = loss;
    }
    __syncthreads();
    if (ok) {
      // pass 2b: moments -> contributions to the radii c and c + 1
      for (int c = tid; c < n_cells; c += SB_THREADS) {
        const float* m0 = mp + (size_t)c * 6;
        const float* m1 = mp + ((size_t)n_cells + c) * 6;
        const float M0 = m0[0] + m1[0], M1 = m0[1] + m1[1], M2 = m0[2] + m1[2];
        const float K0 = m0[3] + m1[3], K1 = m0[4] + m1[4], K2 = m0[5] + m1[5];
        float2 Pc[3], Pd[3];
#pragma unroll
        for (int n = 0; n < 3; ++n) {
          Pc[n] = P[n * n_r + c];
          Pd[n] = P[n * n_r + c + 1];
        }
        auto comb = [&](float x, float y, const float2& u0, const float2& u1) {
          return make_float2(fmaf(x, u0.x, y * u1.x), fmaf(x, u0.y, y * u1.y));
        };
        {
          const float2 A0 = comb(M0, M1, Pc[0], Pd[0]), A1 = comb(M0, M1, Pc[1], Pd[1]),
                       A2 = comb(M0, M1, Pc[2], Pd[2]);
          const float2 B0 = comb(K0, K1, Pc[0], Pd[0]), B1 = comb(K0, K1, Pc[1], Pd[1]),
                       B2 = comb(K0, K1, Pc[2], Pd[2]);
          lo[c] = make_float2(0.5f * (Nn * A0.x - B2.x), 0.5f * (Nn * A0.y - B2.y));
          lo[n_r + c] = make_float2(fmaf(Nn, A1.x, B1.x), fmaf(Nn, A1.y, B1.y));
          lo[2 * n_r + c] =
              make_float2(0.5f * (Nn * A2.x - B0.x), 0.5f * (Nn * A2.y - B0.y));
        }
        {
          const float2 A0 = comb(M1, M2, Pc[0], Pd[0]), A1 = comb(M1, M2, Pc[1], Pd[1]),
                       A2 = comb(M1, M2, Pc[2], Pd[2]);
          const float2 B0 = comb(K1, K2, Pc[0], Pd[0]), B1 = comb(K1, K2, Pc[1], Pd[1]),
                       B2 = comb(K1, K2, Pc[2], Pd[2]);
          hi[c + 1] = make_float2(0.5f * (Nn * A0.x - B2.x), 0.5f * (Nn * A0.y - B2.y));
          hi[n_r + c + 1] = make_float2(fmaf(Nn, A1.x, B1.x), fmaf(Nn, A1.y, B1.y));
          hi[2 * n_r + c + 1] =
              make_float2(0.5f * (Nn * A2.x - B0.x), 0.5f * (Nn * A2.y - B0.y));
        }
      }
      if (tid == 0)
        for (int n = 0; n < 3; ++n) {
          hi[n * n_r] = make_float2(0.f, 0.f);
          lo[n * n_r + n_r - 1] = make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    for (int q = tid; q < rows; q += SB_THREADS) {
      float2 v = make_float2(0.f, 0.f);
      if (ok) {
        const float2 x = lo[q], y = hi[q];
        v = make_float2(x.x + y.x, x.y + y.y);
      }
      if (SPLIT) {
        const size_t r0 = (size_t)(2 * s) * kp + q, r1 = r0 + kp;
        uint16_t h, l;
        split_bf16(v.x, h, l);
        g_hi[r0] = h;
        g_lo[r0] = l;
        split_bf16(v.y, h, l);
        g_hi[r1] = h;
        g_lo[r1] = l;
      } else {
        prof[(size_t)s * rows + q] = v;
      }
    }
    if (TARGET && tid == 0) {
      float t = 0.f;
      if (ok)
        for (int w = 0; w < SB_THREADS / 32; ++w) t += red[w];
      loss_slice[s] = t;
    }
    __syncthreads();          // buffers b, W, lo/hi and red are free again
  }
}

void launch_bessel_adj_epilogue_staged(const BesselParams& p, float2* prof,
                                       const int* slice_em, const int* valid,
                                       const int2* gpc, const float4* gfg,
                                       const float* sorted_f, const int* cell_start,
                                       const float* target, const float* grad_intensity,
                                       float* loss_slice, uint16_t* g_hi, uint16_t* g_lo,
                                       int kp, int* status, cudaStream_t s) {
  const int ng = ((p.nx + 1) / 2) * ((p.ny + 1) / 2);
  const size_t smem = sb_layout(p.nx * p.ny, p.n_r, ng).bytes;
  int dev = 0, n_sm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = (unsigned)(p.n_slices < n_sm ? p.n_slices : n_sm);
  const float* src = target ? target : grad_intensity;
  const bool split = g_hi != nullptr;
  const bool even = (p.nx % 2) == 0 && (p.ny % 2) == 0;
#define PSF_ADJ_STAGED(TG, SP, EV)                                                     \
  do {                                                                                 \
    cudaFuncSetAttribute(k_bessel_adj_epilogue_staged<TG, SP, EV>,                     \
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);      \
    k_bessel_adj_epilogue_staged<TG, SP, EV><<<grid, SB_THREADS, smem, s>>>(           \
        p, prof, slice_em, valid, gpc, gfg, sorted_f, cell_start, src, loss_slice,     \
        g_hi, g_lo, kp, status);                                                       \
  } while (0)
#define PSF_ADJ_STAGED_EV(TG, SP)                                                      \
  do {                                                                                 \
    if (even) PSF_ADJ_STAGED(TG, SP, true);                                            \
    else PSF_ADJ_STAGED(TG, SP, false);                                                \
  } while (0)
  if (target && split) PSF_ADJ_STAGED_EV(true, true);
  else if (target) PSF_ADJ_STAGED_EV(true, false);
  else if (split) PSF_ADJ_STAGED_EV(false, true);
  else PSF_ADJ_STAGED_EV(false, false);
#undef PSF_ADJ_STAGED_EV
#undef PSF_ADJ_STAGED
}

// ---------------------------------------------------------------------------
// Kernel B: transposed radial contraction, g_F[s][j] = sum_row
// conj(Bt[j][row]) g_P[s][row] (rows = 3 N_r; Bt real, or complex with the
// Fresnel weights), FP32.  CTA tile 64 slices x 32 theta nodes, 128 threads
// with 4 x 4 complex accumulators, 32-row K chunks staged through shared
// memory.
// ---------------------------------------------------------------------------
constexpr int AT_S = 64, AT_J = 32, AT_K = 32;

PSF_D void adj_fma(float b, float2 p, float2& acc) {
  acc.x = fmaf(b, p.x, acc.x);
  acc.y = fmaf(b, p.y, acc.y);
}
PSF_D void adj_fma(float2 b, float2 p, float2& acc) {   // acc += conj(b) p
  acc.x = fmaf(b.x, p.x, fmaf(b.y, p.y, acc.x));
  acc.y = fmaf(b.x, p.y, fmaf(-b.y, p.x, acc.y));
}
PSF_D float adj_zero(float) { return 0.f; }
PSF_D float2 adj_zero(float2) { return make_float2(0.f, 0.f); }

template <typename TB>
__global__ void __launch_bounds__(128)
k_bessel_adj_contract(const TB* __restrict__ Bt, const float2* __restrict__ gP,
                      float2* __restrict__ gF, int n_slices, int n_theta, int rows) {
  // +1 padding: the transposing stores below hit distinct banks
  __shared__ float2 Ps[AT_K][AT_S + 1];
  __shared__ TB Bs[AT_K][AT_J + 1];
  const int tid = threadIdx.x;
  const int s0 = blockIdx.x * AT_S, j0 = blockIdx.y * AT_J;
  const int ts = tid & 15, tj = tid >> 4;       // 16 slice quads x 8 theta quads
  float2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
  for (int r0 = 0; r0 < rows; r0 += AT_K) {
    // g_P tile: 64 slices x 32 rows, rows fastest in global memory
    for (int q = tid; q < AT_S * AT_K; q += 128) {
      const int sl = q / AT_K, rr = q - sl * AT_K;
      const int sg = s0 + sl, rg = r0 + rr;
      Ps[rr][sl] = (sg < n_slices && rg < rows) ? gP[(size_t)sg * rows + rg]
                                                : make_float2(0.f, 0.f);
    }
    for (int q = tid; q < AT_J * AT_K; q += 128) {
      const int jj = q / AT_K, rr = q - jj * AT_K;
      const int jg = j0 + jj, rg = r0 + rr;
      Bs[rr][jj] = (jg < n_theta && rg < rows) ? __ldg(&Bt[(size_t)jg * rows + rg])
                                               : adj_zero(TB());
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < AT_K; ++k) {
      float2 pv[4];
      TB bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        pv[a] = Ps[k][ts * 4 + a];
        bv[a] = Bs[k][tj * 4 + a];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) adj_fma(bv[b], pv[a], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int sg = s0 + ts * 4 + a;
    if (sg >= n_slices) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int jg = j0 + tj * 4 + b;
      if (jg < n_theta) gF[(size_t)sg * n_theta + jg] = acc[a][b];
    }
  }
}

void launch_bessel_adj_contract(const BesselParams& p, const float* Bt, const float2* BtC,
                                const float2* gP, float2* gF, cudaStream_t s) {
  dim3 grid(ceil_div(p.n_slices, AT_S), ceil_div(p.n_theta, AT_J));
  if (BtC)
    k_bessel_adj_contract<float2><<<grid, 128, 0, s>>>(BtC, gP, gF, p.n_slices, p.n_theta,
                                                       3 * p.n_r);
  else
    k_bessel_adj_contract<float><<<grid, 128, 0, s>>>(Bt, gP, gF, p.n_slices, p.n_theta,
                                                      3 * p.n_r);
}

// ---------------------------------------------------------------------------
// Kernel C: per emitter, Q_j = sum over its slices of conj(g_F) F (F rebuilt
// exactly as the forward builds it), then
//   dL/dW_0(theta_j) = -Im Q_j,
//   dL/dt_s = sum_j Re(i D_j Q_j),  D_j = 2 pi (a_re + i a_im)_j,
//   dL/dc_q = sum_j Z_q(theta_j) dL/dW_0(theta_j)  (m = 0 Noll terms; others 0),
//   loss_e  = sum of the slice losses.
// One CTA per emitter; every sum runs in a fixed order.
// ---------------------------------------------------------------------------
constexpr int RED_THREADS = 256;

__device__ double block_sum(double v, double* buf) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) buf[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < RED_THREADS / 32; ++w) t += buf[w];
  return t;                                  // valid in thread 0
}

__global__ void __launch_bounds__(RED_THREADS)
k_bessel_adj_reduce(BesselParams p, ThetaTable t, EmitterTable et,
                    const int* __restrict__ z_offsets, const float2* __restrict__ zz,
                    const float2* __restrict__ gF, const float* __restrict__ loss_slice,
                    float* loss, float* grad_w, float* grad_zern, float* grad_depth) {
  __shared__ double buf[RED_THREADS / 32];
  const int e = blockIdx.x;
  const int tid = threadIdx.x;
  const int a = z_offsets[e], b = z_offsets[e + 1];
  const bool ok = et.valid[e] && a >= 0 && b >= a && b <= p.n_slices;
  double dep = 0.0;
  double zs[kMaxM0];
#pragma unroll
  for (int q = 0; q < kMaxM0; ++q) zs[q] = 0.0;
  for (int j = tid; j < p.n_theta; j += RED_THREADS) {
    double qr = 0.0, qi = 0.0;
    if (ok) {
      const size_t ej = (size_t)e * p.n_theta + j;
      const float amp = et.amp[ej], w = et.wfr[ej];
      const f2x kap{t.kh[j], t.kl[j]};
      for (int s = a; s < b; ++s) {
        const float2 z = zz[s];
        const float2 c = cis_cycles(frac_mul_add(kap, f2x{z.x, z.y}, w));
        const float fr = amp * c.x, fi = amp * c.y;
        const float2 g = gF[(size_t)s * p.n_theta + j];
        // conj(g) F
        qr += (double)(g.x * fr + g.y * fi);
        qi += (double)(g.x * fi - g.y * fr);
      }
    }
    const double gw = -qi;
    if (grad_w) grad_w[(size_t)e * p.n_theta + j] = (float)gw;
    const double dr = 2.0 * kPi * t.a_re[j], di = 2.0 * kPi * t.a_im[j];
    dep += -(dr * qi + di * qr);
    for (int q = 0; q < p.n_m0; ++q) zs[q] += t.zm0[(size_t)q * p.n_theta + j] * gw;
  }
  const double dsum = block_sum(dep, buf);
  if (tid == 0 && grad_depth) grad_depth[e] = (float)dsum;
  for (int q = 0; q < p.n_m0; ++q) {
    const double v = block_sum(zs[q], buf);
    if (tid == 0 && grad_zern) grad_zern[(size_t)e * p.n_zern + p.m0_j[q] - 1] = (float)v;
  }
  if (grad_zern)
    for (int k = tid; k < p.n_zern; k += RED_THREADS) {
      bool m0 = false;
      for (int q = 0; q < p.n_m0; ++q) m0 |= (p.m0_j[q] == k + 1);
      if (!m0) grad_zern[(size_t)e * p.n_zern + k] = 0.f;
    }
  if (tid == 0 && loss) {
    double l = 0.0;
    if (ok && loss_slice)
      for (int s = a; s < b; ++s) l += loss_slice[s];
    loss[e] = (float)l;
  }
}

void launch_bessel_adj_reduce(const BesselParams& p, ThetaTable t, EmitterTable et,
                              const int* z_offsets, const float2* zz, const float2* gF,
                              const float* loss_slice, float* loss, float* grad_w,
                              float* grad_zern, float* grad_depth, cudaStream_t s) {
  k_bessel_adj_reduce<<<p.n_em, RED_THREADS, 0, s>>>(p, t, et, z_offsets, zz, gF,
                                                     loss_slice, loss, grad_w, grad_zern,
                                                     grad_depth);
}

}  // namespace psf
