// Azimuthal-harmonic (non-axisymmetric) Bessel strategy: pupil harmonics by
// FFT, the per-emitter adaptive order, the channel/order mixtures, the J_n
// table, the FP32 per-order radial contraction (or the split operands of the
// tensor-core contraction, mode 5 of the persistent GEMM) and the Cartesian
// epilogues (FP32 arithmetic, FP64 tables).
#include "harmonic_kernels.cuh"
#include "tc_ptx.cuh"

namespace psf {

namespace {

// kinds: P index = l + shift, weight g_n
PSF_D int kind_shift(int kind) {
  return kind == 1 ? -2 : kind == 2 ? 2 : kind == 3 ? -1 : kind == 4 ? 1 : 0;
}
PSF_D int kind_g(int kind) { return kind == 0 ? 0 : (kind <= 2 ? 2 : 1); }

// ---------------------------------------------------------------------------
// One CTA (64 threads) per (emitter, group of HP_G theta nodes):
// e^{i W_na(theta_j, phi_k)} on the N_phi azimuths of each node, its DFT
// X_m = sum_k x_k e^{-2 pi i m k / N_phi} by a radix-2 decimation-in-time
// FFT in shared memory (inputs stored in bit-reversed order, log2 N_phi
// butterfly stages with twiddles conj(cs)), then P_m = A e^{i W_ax} X_m /
// N_phi for |m| <= M (X_{N_phi - m} for -m) -> Pm[e][m + M][j].  The
// products c_q N_q R_q(theta_j) of the m != 0 terms are formed once per CTA.
// ---------------------------------------------------------------------------
constexpr int HP_G = 4;
constexpr int HP_THREADS = 64;

__global__ void __launch_bounds__(HP_THREADS)
k_harm_pupil(HarmParams p, ThetaTable t, EmitterTable et, const double* __restrict__ zern,
             const float* __restrict__ Zr, const float2* __restrict__ cs,
             float2* __restrict__ Pm) {
  extern __shared__ float2 X[];                // [HP_G][n_phi]
  __shared__ float cz[kHarmMaxNA][HP_G];
  const int e = blockIdx.x, j0 = blockIdx.y * HP_G;
  const int N = p.n_phi, mask = N - 1, nP = 2 * p.m_max + 1;
  const int logN = 31 - __clz(N);
  for (int idx = threadIdx.x; idx < p.n_na * HP_G; idx += HP_THREADS) {
    const int q = idx / HP_G, g = idx - q * HP_G, j = j0 + g;
    cz[q][g] = j < p.n_theta
                   ? (float)zern[(size_t)e * p.n_zern + p.na_j[q] - 1] * Zr[q * p.n_theta + j]
                   : 0.f;
  }
  __syncthreads();
  // x_k = e^{i W_na(theta_j, phi_k)}, stored at the bit-reversed index of k
  for (int idx = threadIdx.x; idx < N * HP_G; idx += HP_THREADS) {
    const int g = idx / N, k = idx - g * N;
    float w = 0.f;
    for (int q = 0; q < p.n_na; ++q) {
      const float2 a = cs[(p.na_m[q] * k) & mask];   // e^{i m phi_k}
      w = fmaf(cz[q][g], p.na_cos[q] ? a.x : a.y, w);
    }
    float2 v;
    sincosf(w, &v.y, &v.x);
    X[g * N + (int)(__brev((unsigned)k) >> (32 - logN))] = v;
  }
  __syncthreads();
  // butterflies: stage h = 1, 2, 4, ..: (a, b) -> (a + w b, a - w b),
  // w = e^{-2 pi i r / (2 h)} = conj(cs[r N / (2 h)])
  for (int h = 1; h < N; h <<= 1) {
    const int step = N / (2 * h);
    for (int idx = threadIdx.x; idx < (N / 2) * HP_G; idx += HP_THREADS) {
      const int g = idx / (N / 2), bf = idx - g * (N / 2);
      const int r = bf & (h - 1), i0 = ((bf - r) << 1) + r;
      float2* base = X + g * N;
      const float2 c = cs[r * step];
      const float2 a = base[i0], b = base[i0 + h];
      const float2 wb = make_float2(fmaf(c.x, b.x, c.y * b.y), fmaf(c.x, b.y, -c.y * b.x));
      base[i0] = make_float2(a.x + wb.x, a.y + wb.y);
      base[i0 + h] = make_float2(a.x - wb.x, a.y - wb.y);
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < nP * HP_G; idx += HP_THREADS) {
    const int g = idx / nP, mi = idx - g * nP, j = j0 + g;
    if (j >= p.n_theta) continue;
    const int m = mi - p.m_max;
    const size_t ej = (size_t)e * p.n_theta + j;
    const float2 base = cis_cycles(et.wfr[ej]);
    const float scale = et.amp[ej] / (float)N;
    const float2 h = cmul(base, X[g * N + (m & mask)]);
    Pm[((size_t)e * nP + mi) * p.n_theta + j] = make_float2(scale * h.x, scale * h.y);
  }
}

// ---------------------------------------------------------------------------
// Adaptive order, one CTA per emitter: a_m = max_j |P_m(theta_j)| (one warp
// per harmonic), then M_e = the largest |m| <= M with a_m > tail_tol a_0 (0
// if none).  Each harmonic is tested on its own, not the summed tail: the
// rounding floor of the FP32 DFT (a few 1e-8 of a_0 on every harmonic)
// summed over tens of harmonics would exceed the tolerance.  tail_tol = 0
// keeps M_e = M.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_harm_order(HarmParams p, const float2* __restrict__ Pm, int* __restrict__ ord) {
  __shared__ float amax[2 * kHarmMaxM + 1];
  const int e = blockIdx.x, nP = 2 * p.m_max + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (!(p.tail_tol > 0.0)) {
    if (threadIdx.x == 0) ord[e] = p.m_max;
    return;
  }
  for (int mi = warp; mi < nP; mi += 8) {
    const float2* row = Pm + ((size_t)e * nP + mi) * p.n_theta;
    float v = 0.f;
    for (int j = lane; j < p.n_theta; j += 32) {
      const float2 x = row[j];
      v = fmaxf(v, sqrtf(x.x * x.x + x.y * x.y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) amax[mi] = v;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double lim = p.tail_tol * (double)amax[p.m_max];
  int M = 0;
  for (int m = p.m_max; m >= 1; --m)
    if ((double)amax[p.m_max + m] > lim || (double)amax[p.m_max - m] > lim) {
      M = m;
      break;
    }
  ord[e] = M;
}

// ---------------------------------------------------------------------------
// Channel/order mixtures from the harmonics |m| <= M_e: Bh[e][c][l'][j]
// (zero for |l| > M_e + 2).  One CTA (256 threads) per (emitter, 32 theta
// nodes): the lanes run over the nodes, so the harmonics are read and the
// mixtures written in coalesced rows; the eight warps share the outputs
// (c, l').  The coefficient x g products are formed once per node (the FP64
// tables are converted here only: on this GPU the conversions run on the
// narrow FP64 pipe).
// ---------------------------------------------------------------------------
constexpr int HM_NODES = 32;

__global__ void __launch_bounds__(256)
k_harm_mix(HarmParams p, ThetaTable t, EmitterTable et, const float2* __restrict__ Pm,
           const int* __restrict__ ord, float2* __restrict__ Bh, unsigned* bh_max) {
  __shared__ float2 pcol[2 * kHarmMaxM + 1][HM_NODES];   // P_m of the nodes
  __shared__ float2 cg[3][5][HM_NODES];                  // coef[c][kind] g_kind
  __shared__ bool cz[3][5];
  const int e = blockIdx.x, j0 = blockIdx.y * HM_NODES;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int j = j0 + tx;
  const bool jin = j < p.n_theta;
  const int nP = 2 * p.m_max + 1;
  for (int mi = ty; mi < nP; mi += 8)
    pcol[mi][tx] = jin ? Pm[((size_t)e * nP + mi) * p.n_theta + j] : make_float2(0.f, 0.f);
  for (int ck = ty; ck < 15; ck += 8) {
    const int c = ck / 5, kind = ck - 5 * c;
    const double cr = p.coef[c][kind][0], ci = p.coef[c][kind][1];
    const int gk = kind_g(kind);
    float2 g = make_float2(0.f, 0.f);
    if (jin)
      g = make_float2((float)t.g[(size_t)(2 * gk) * p.n_theta + j],
                      (float)t.g[(size_t)(2 * gk + 1) * p.n_theta + j]);
    cg[c][kind][tx] = cmul(make_float2((float)cr, (float)ci), g);
    if (tx == 0) cz[c][kind] = cr == 0.0 && ci == 0.0;
  }
  __syncthreads();
  const int Me = ord[e];
  const bool ok = et.valid[e] != 0;
  const int L = p.m_max + 2;
  float vmax = 0.f;
  if (jin)
    for (int o = ty; o < 3 * p.n_ord; o += 8) {
      const int c = o / p.n_ord, li = o - c * p.n_ord, l = li - L;
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int kind = 0; kind < 5; ++kind) {
        const int m = l + kind_shift(kind);
        if (m < -Me || m > Me) continue;
        if (cz[c][kind]) continue;
        const float2 v = cmul(cg[c][kind][tx], pcol[m + p.m_max][tx]);
        acc.x += v.x;
        acc.y += v.y;
      }
      if (l < 0 && ((-l) & 1)) acc = make_float2(-acc.x, -acc.y);   // J_{-n} = (-1)^n J_n
      if (!ok) acc = make_float2(0.f, 0.f);
      Bh[(((size_t)e * 3 + c) * p.n_ord + li) * p.n_theta + j] = acc;
      vmax = fmaxf(vmax, fmaxf(fabsf(acc.x), fabsf(acc.y)));
    }
  if (bh_max) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
      vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
    if (tx == 0) atomicMax(bh_max, __float_as_uint(vmax));   // vmax >= 0
  }
}

// J_0 .. J_nmax at one argument x >= 0 by Miller's backward recurrence
// J_{n-1} = (2n / x) J_n - J_{n+1}, started far above max(nmax, x) where the
// minimal solution dominates, normalised by J_0 + 2 sum_k J_{2k} = 1
// (FP64; values rescaled before they can overflow).
constexpr int kJMax = kHarmMaxM + 3;

PSF_D void bessel_j_all(double x, int nmax, double* out) {
  for (int n = 0; n <= nmax; ++n) out[n] = 0.0;
  if (x <= 0.0) {
    out[0] = 1.0;
    return;
  }
  const int start = 2 * ((max(nmax, (int)x) + 40 + (int)sqrt(40.0 * (max(nmax, (int)x) + 1))) / 2);
  const double two_x = 2.0 / x;
  double jp = 0.0, jc = 1.0, sum = 0.0;   // J_{n+1}, J_n (unnormalised)
  for (int n = start; n >= 1; --n) {
    const double jm = n * two_x * jc - jp;   // J_{n-1}
    jp = jc;
    jc = jm;
    const int m = n - 1;
    if (m <= nmax) out[m] = jc;
    if (m > 0 && (m & 1) == 0) sum += 2.0 * jc;
    if (fabs(jc) > 1e250) {
      jc *= 1e-250;
      jp *= 1e-250;
      sum *= 1e-250;
      for (int k = m; k <= nmax; ++k) out[k] *= 1e-250;
    }
  }
  const double norm = 1.0 / (sum + jc);
  for (int n = 0; n <= nmax; ++n) out[n] *= norm;
}

// one thread per (r_i, theta_j): every order at once; FP32 table Jt and/or
// the split operand S_A w_j J_n in hi / lo planes [n][n_r_pad][kp]
__global__ void k_harm_jtab(HarmParams p, ThetaTable t, float* __restrict__ Jt,
                            uint16_t* __restrict__ a_hi, uint16_t* __restrict__ a_lo, int kp,
                            int n_r_pad, double sA, int bf16) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)p.n_r * p.n_theta) return;
  const int i = (int)(idx / p.n_theta), j = (int)(idx - (long long)i * p.n_theta);
  const int nmax = p.m_max + 2;
  double J[kJMax];
  bessel_j_all(p.k * (i * p.dr) * t.sin_t[j], nmax, J);
  const double w = t.w[j];
  const size_t plane = (size_t)p.n_r * p.n_theta;
  if (Jt)
    for (int n = 0; n <= nmax; ++n) Jt[n * plane + idx] = (float)(w * J[n]);
  if (a_hi)
    for (int n = 0; n <= nmax; ++n) {
      uint16_t h, l;
      tc::split16d(sA * w * J[n], bf16, h, l);
      const size_t o = ((size_t)n * n_r_pad + i) * kp + j;
      a_hi[o] = h;
      a_lo[o] = l;
    }
}

// Split B operand of the tensor-core contraction for the slices [s0, s0+ns):
// rows (l', 3 sl + c, re/im), 2 * 3 ns rows per order, value
// S_F D[sl][j] Bh[e][c][l'][j] split into FP16 hi + lo; S_F is the power of two that
// keeps max |Bh| below 2^14.  Only (order, slice) pairs the epilogue reads
// (valid emitter, |l| <= M_e + 2) are written.  Block (64, 4): one
// (order, slice) pair per threadIdx.y, four theta nodes per thread.
constexpr int HB_TX = 64, HB_TY = 4;

// hi + lo FP16 parts of two values as packed pairs (low half = a): the same
// rounding as a scalar split, two conversions per instruction
PSF_D void split_pair16(float a, float b, uint32_t& h, uint32_t& l) {
  const __half2 hh = __floats2half2_rn(a, b);
  const float2 back = __half22float2(hh);
  const __half2 ll = __floats2half2_rn(a - back.x, b - back.y);
  h = *reinterpret_cast<const uint32_t*>(&hh);
  l = *reinterpret_cast<const uint32_t*>(&ll);
}

__global__ void __launch_bounds__(HB_TX * HB_TY)
k_harm_bgen(HarmParams p, const float2* __restrict__ Bh, const float2* __restrict__ D,
            const int* __restrict__ slice_em, const int* __restrict__ valid,
            const int* __restrict__ ord, int s0, int ns, int kp,
            const unsigned* __restrict__ bh_max, float sA, uint16_t* __restrict__ b_hi,
            uint16_t* __restrict__ b_lo, float* __restrict__ out_scale) {
  const float bm = __uint_as_float(*bh_max);
  const float sF = bm > 0.f ? exp2f(floorf(log2f(16384.f / bm))) : 1.f;
  if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) *out_scale = 1.f / (sA * sF);
  const long long pair = (long long)blockIdx.x * HB_TY + threadIdx.y;   // li * ns + sl
  if (pair >= (long long)p.n_ord * ns) return;
  const int li = (int)(pair / ns), sl = (int)(pair - (long long)li * ns);
  const int e = slice_em[s0 + sl];
  const int L = p.m_max + 2, n = li >= L ? li - L : L - li;
  if (e < 0 || !valid[e] || n > ord[e] + 2) return;
  const float2* d = D + (size_t)sl * p.n_theta;
  for (int q = threadIdx.x; q < (kp >> 2); q += HB_TX) {
    float2 v[3][4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = 4 * q + u;
      const bool in = j < p.n_theta;
      const float2 dj = in ? d[j] : make_float2(0.f, 0.f);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float2 x = make_float2(0.f, 0.f);
        if (in) x = cmul(dj, Bh[(((size_t)e * 3 + c) * p.n_ord + li) * p.n_theta + j]);
        v[c][u] = make_float2(sF * x.x, sF * x.y);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t row = (size_t)li * 6 * ns + (size_t)(3 * sl + c) * 2;
      uint2 hr, lr, hm, lm;
      split_pair16(v[c][0].x, v[c][1].x, hr.x, lr.x);
      split_pair16(v[c][2].x, v[c][3].x, hr.y, lr.y);
      split_pair16(v[c][0].y, v[c][1].y, hm.x, lm.x);
      split_pair16(v[c][2].y, v[c][3].y, hm.y, lm.y);
      *reinterpret_cast<uint2*>(b_hi + row * kp + 4 * q) = hr;
      *reinterpret_cast<uint2*>(b_lo + row * kp + 4 * q) = lr;
      *reinterpret_cast<uint2*>(b_hi + (row + 1) * kp + 4 * q) = hm;
      *reinterpret_cast<uint2*>(b_lo + (row + 1) * kp + 4 * q) = lm;
    }
  }
}

// need[li][nt] = some column of B tile nt (slices nt * spt .. + spt - 1 of
// the chunk) has a valid emitter with |l| <= M_e + 2
__global__ void k_harm_tile_need(HarmParams p, const int* __restrict__ slice_em,
                                 const int* __restrict__ valid, const int* __restrict__ ord,
                                 int s0, int ns, int cols_per_tile, int n_tiles,
                                 unsigned char* __restrict__ need) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)p.n_ord * n_tiles) return;
  const int li = (int)(idx / n_tiles), nt = (int)(idx - (long long)li * n_tiles);
  const int L = p.m_max + 2, n = li >= L ? li - L : L - li;
  const int c0 = nt * cols_per_tile, c1 = min(3 * ns, c0 + cols_per_tile);
  unsigned char f = 0;
  for (int sl = c0 / 3; sl * 3 < c1; ++sl) {
    const int e = slice_em[s0 + sl];
    if (e >= 0 && valid[e] && n <= ord[e] + 2) {
      f = 1;
      break;
    }
  }
  need[idx] = f;
}

// D[s][j] = e^{i k z_s cos theta_j} for the slices of a chunk
__global__ void k_harm_defocus(int n_theta, ThetaTable t, const float2* __restrict__ zz,
                               int s0, int ns, float2* __restrict__ D) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)ns * n_theta) return;
  const int sl = (int)(idx / n_theta), j = (int)(idx - (long long)sl * n_theta);
  const float2 z = zz[s0 + sl];
  D[idx] = cis_cycles(frac_mul_add(f2x{t.kh[j], t.kl[j]}, f2x{z.x, z.y}, 0.f));
}

// ---------------------------------------------------------------------------
// Radial contraction, one order per grid z: C[i][(s, c)] = sum_j Jt[|l|][i][j]
// D[s][j] Bh[e(s)][c][l'][j] (real x complex, FP32 FMA).  Tile 128 radii x 64
// columns, K step 16, double-buffered in shared memory; 256 threads on a
// 16 x 16 grid, each with 8 radii x 4 columns of complex accumulators (rows
// 4 tr + {0..3} and 64 + 4 tr + {0..3}, columns 2 tc + {0, 1} and
// 32 + 2 tc + {0, 1}; one float4 shared load feeds 16 FMAs).  A tile none of
// whose columns needs order l (|l| > M_e + 2, or no valid emitter) returns
// at once: the epilogue reads no profile beyond its emitter's orders.
// ---------------------------------------------------------------------------
constexpr int HP_BM = 128, HP_BN = 64, HP_BK = 16;
constexpr int HP_APAD = HP_BM + 4;   // floats per As row (16 B multiple; 2-way stores)
constexpr int HP_BPAD = HP_BN + 2;   // float2 per Bs row

__global__ void __launch_bounds__(256, 2)
k_harm_profiles(HarmParams p, const float* __restrict__ Jt, const float2* __restrict__ Bh,
                const int* __restrict__ slice_em, const int* __restrict__ valid,
                const int* __restrict__ ord, const float2* __restrict__ D, int s0, int ns,
                float2* __restrict__ prof) {
  __shared__ __align__(16) float As[2][HP_BK][HP_APAD];
  __shared__ __align__(16) float2 Bs[2][HP_BK][HP_BPAD];
  const int li = blockIdx.z, L = p.m_max + 2;
  const int n = li >= L ? li - L : L - li;
  const int i0 = blockIdx.y * HP_BM, c0 = blockIdx.x * HP_BN;
  const int ncol = 3 * ns;
  {
    bool need = false;
    if (threadIdx.x < HP_BN && c0 + (int)threadIdx.x < ncol) {
      const int e = slice_em[s0 + (c0 + (int)threadIdx.x) / 3];
      need = e >= 0 && valid[e] && n <= ord[e] + 2;
    }
    if (!__syncthreads_or(need)) return;
  }
  const float* A = Jt + (size_t)n * p.n_r * p.n_theta;
  const int tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
  // global -> register staging: A row tid / 2, k (tid & 1) * 8 + {0..7};
  // B column tid / 4, k (tid & 3) * 4 + {0..3}
  const int arow = tid >> 1, ak = (tid & 1) * 8;
  const int bcol = tid >> 2, bk = (tid & 3) * 4;
  const float* a_row = i0 + arow < p.n_r ? A + (size_t)(i0 + arow) * p.n_theta : nullptr;
  const float2* bh_col = nullptr;
  const float2* d_col = nullptr;
  if (c0 + bcol < ncol) {
    const int gc = c0 + bcol, sl = gc / 3, c = gc - 3 * sl;
    const int e = slice_em[s0 + sl];
    if (e >= 0 && valid[e]) {
      bh_col = Bh + (((size_t)e * 3 + c) * p.n_ord + li) * p.n_theta;
      d_col = D + (size_t)sl * p.n_theta;
    }
  }
  float ra[8];
  float2 rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int gk = k0 + ak + q;
      ra[q] = (a_row && gk < p.n_theta) ? a_row[gk] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int gk = k0 + bk + q;
      rb[q] = (bh_col && gk < p.n_theta) ? cmul(d_col[gk], bh_col[gk]) : make_float2(0.f, 0.f);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 8; ++q) As[buf][ak + q][arow] = ra[q];
#pragma unroll
    for (int q = 0; q < 4; ++q) Bs[buf][bk + q][bcol] = rb[q];
  };
  float2 acc[8][4];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[r][u] = make_float2(0.f, 0.f);
  const int nk = (p.n_theta + HP_BK - 1) / HP_BK;
  load(0);
  store(0);
  __syncthreads();
  for (int t = 0; t < nk; ++t) {
    const int buf = t & 1;
    if (t + 1 < nk) load((t + 1) * HP_BK);
#pragma unroll
    for (int kk = 0; kk < HP_BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * tr]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + 4 * tr]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][2 * tc]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][32 + 2 * tc]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float2 b[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w),
                           make_float2(b1.x, b1.y), make_float2(b1.z, b1.w)};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          acc[r][u].x = fmaf(a[r], b[u].x, acc[r][u].x);
          acc[r][u].y = fmaf(a[r], b[u].y, acc[r][u].y);
        }
    }
    if (t + 1 < nk) store(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int gc = c0 + (u < 2 ? 2 * tc + u : 32 + 2 * tc + (u - 2));
    if (gc >= ncol) continue;
    const int sl = gc / 3, c = gc - 3 * sl;
    float2* dst = prof + (((size_t)sl * 3 + c) * p.n_ord + li) * p.n_r;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int gi = i0 + (r < 4 ? 4 * tr + r : 64 + 4 * tr + (r - 4));
      if (gi < p.n_r) dst[gi] = acc[r][u];
    }
  }
}

// ---------------------------------------------------------------------------
// Epilogue: one thread per quarter pixel (a < ceil(nx/2), b < ceil(ny/2)) of
// one slice and its mirrors (+-x, +-y), which share the radius and so the
// interpolated I_{c,l}.  With T_l = (i e^{i phi})^l at (x, y):
//   (x, y): sum T_l v_l          (-x, -y): sum (-1)^l T_l v_l
//   (-x, y): sum conj(T_l) v_l   (x, -y): sum (-1)^l conj(T_l) v_l,
// kept as even and odd partial sums over |l| <= M_e + 2 (the slice's
// emitter order).  T_l by forward and backward
// recurrences from l = 0 (the large low orders carry the least rounding);
// |E_c|^2 = |sum|^2 (the -i prefactor has modulus 1).
// ---------------------------------------------------------------------------
struct MirrorAcc {
  float2 te, to, ce, co;   // sums of T v and conj(T) v over even / odd l
};

PSF_D void harm_add(MirrorAcc& m, float2 t, float2 v, bool odd) {
  const float2 a = cmul(t, v);
  const float2 b = cmul(make_float2(t.x, -t.y), v);
  if (odd) {
    m.to.x += a.x; m.to.y += a.y; m.co.x += b.x; m.co.y += b.y;
  } else {
    m.te.x += a.x; m.te.y += a.y; m.ce.x += b.x; m.ce.y += b.y;
  }
}

__global__ void __launch_bounds__(256)
k_harm_intensity(HarmParams p, const float2* __restrict__ prof,
                 const int* __restrict__ slice_em, const int* __restrict__ valid,
                 const int* __restrict__ ord, int s0, float* __restrict__ I) {
  const int sl = blockIdx.y, s = s0 + sl;
  const int e = slice_em[s];
  if (e < 0 || !valid[e]) return;
  const int ha = (p.nx + 1) / 2, hb = (p.ny + 1) / 2;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ha * hb) return;
  const int a = idx / hb, b = idx - a * hb;
  const double x = (a - 0.5 * (p.nx - 1)) * p.dx, y = (b - 0.5 * (p.ny - 1)) * p.dy;
  const double rho = sqrt(x * x + y * y);
  const double tt = p.dr > 0 ? rho / p.dr : 0.0;   // r_max = 0: all r_i = 0
  int i0 = (int)floor(tt);
  i0 = i0 < 0 ? 0 : (i0 > p.n_r - 2 ? p.n_r - 2 : i0);
  const float f = (float)(tt - i0);
  const float cp = rho > 0 ? (float)(x / rho) : 1.f, sp = rho > 0 ? (float)(y / rho) : 0.f;
  const float2 w = make_float2(-sp, cp);    // i e^{i phi}
  const float2 wc = make_float2(-sp, -cp);  // its inverse
  const int L = p.m_max + 2, Le = ord[e] + 2;
  const float2* base = prof + (size_t)sl * 3 * p.n_ord * p.n_r + i0;
  MirrorAcc acc[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) acc[c] = MirrorAcc{{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  float2 tf = make_float2(1.f, 0.f);
  for (int l = 0; l <= Le; ++l) {
    const bool odd = l & 1;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2* q = base + ((size_t)c * p.n_ord + (l + L)) * p.n_r;
      const float2 u = q[0], v = q[1];
      harm_add(acc[c], tf, make_float2(fmaf(f, v.x - u.x, u.x), fmaf(f, v.y - u.y, u.y)), odd);
    }
    tf = cmul(tf, w);
  }
  tf = wc;
  for (int l = -1; l >= -Le; --l) {
    const bool odd = (-l) & 1;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2* q = base + ((size_t)c * p.n_ord + (l + L)) * p.n_r;
      const float2 u = q[0], v = q[1];
      harm_add(acc[c], tf, make_float2(fmaf(f, v.x - u.x, u.x), fmaf(f, v.y - u.y, u.y)), odd);
    }
    tf = cmul(tf, wc);
  }
  float i_pp = 0.f, i_mm = 0.f, i_mp = 0.f, i_pm = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const MirrorAcc& m = acc[c];
    const float2 pp = make_float2(m.te.x + m.to.x, m.te.y + m.to.y);
    const float2 mm = make_float2(m.te.x - m.to.x, m.te.y - m.to.y);
    const float2 mp = make_float2(m.ce.x + m.co.x, m.ce.y + m.co.y);
    const float2 pm = make_float2(m.ce.x - m.co.x, m.ce.y - m.co.y);
    i_pp = fmaf(pp.x, pp.x, fmaf(pp.y, pp.y, i_pp));
    i_mm = fmaf(mm.x, mm.x, fmaf(mm.y, mm.y, i_mm));
    i_mp = fmaf(mp.x, mp.x, fmaf(mp.y, mp.y, i_mp));
    i_pm = fmaf(pm.x, pm.x, fmaf(pm.y, pm.y, i_pm));
  }
  float* out = I + (size_t)s * p.nx * p.ny;
  const int am = p.nx - 1 - a, bm = p.ny - 1 - b;
  out[(size_t)a * p.ny + b] = i_pp;
  out[(size_t)am * p.ny + bm] = i_mm;
  out[(size_t)am * p.ny + b] = i_mp;
  out[(size_t)a * p.ny + bm] = i_pm;
}

// ---------------------------------------------------------------------------
// Square geometry (nx = ny, dx = dy): each octant pixel (b <= a in the
// quarter) and its seven images share the radius, so one set of profile
// reads serves eight pixels.  With
// T_l = (i e^{i phi})^l at (x, y) the images take
//   (x, y): T_l            (-x, -y): (-1)^l T_l
//   (-y, x): i^l T_l       (y, -x): (-i)^l T_l
//   (-x, y): conj(T_l)     (x, -y): (-1)^l conj(T_l)
//   (y, x): (-i)^l conj(T_l)   (-y, -x): i^l conj(T_l),
// so the sums are kept by l mod 4 (S_r of T_l v_l, C_r of conj(T_l) v_l).
// On the diagonal (a = b) the swapped images are the pixels themselves and
// are not written again.
//
// A block holds 128 octant pixels x 3 channels (one thread per pixel and
// channel: 16 accumulators, two profile pointers), so that enough warps are
// resident to cover the profile-read latency; the channels' |E_c|^2 of the
// eight images meet in shared memory and are summed in channel order.
// The pixels are taken in the order of their radius sample (table built
// per call), so a block's 128 pixels span a short run [lo, hi] of radial
// samples: the block stages that window of its emitter's orders |l| <= Le
// for the three channels in shared memory (read once per slice in all)
// and reads the profiles from there; a window too long for the budget
// (large N_r on a small grid) is read from global memory, with an L2
// prefetch one order ahead.  Orders are taken in pairs +n, -n, read through
// pointers stepped by one row per order; T_{+n} = w^n and T_{-n} =
// conj(w)^n by recurrences outward from n = 0.
// ---------------------------------------------------------------------------
constexpr int HO_PIX = 128;
// staged profile window per block (dynamic; with the 12 KB of channel
// partials the block stays under the 48 KB default)
constexpr int HO_SMEM = 35 * 1024;
// prefetch distance in orders (256 workload emitters, split contraction:
// none 8.68 ms per call, 1 order 7.77, 2 orders 7.85, 3 orders 7.91; an L1
// prefetch measured the same as L2)
constexpr int kHarmPrefetch = 1;

struct OctAcc {
  float2 s[4], c[4];
};

// sum_r w^r X_r for w = 1, -1, i, -i
PSF_D float2 oct_sum(const float2* X, int w) {
  float2 r;
  if (w == 0) {          // 1
    r.x = X[0].x + X[1].x + X[2].x + X[3].x;
    r.y = X[0].y + X[1].y + X[2].y + X[3].y;
  } else if (w == 1) {   // -1
    r.x = X[0].x - X[1].x + X[2].x - X[3].x;
    r.y = X[0].y - X[1].y + X[2].y - X[3].y;
  } else if (w == 2) {   // i: X0 + i X1 - X2 - i X3
    r.x = X[0].x - X[1].y - X[2].x + X[3].y;
    r.y = X[0].y + X[1].x - X[2].y - X[3].x;
  } else {               // -i: X0 - i X1 - X2 + i X3
    r.x = X[0].x + X[1].y - X[2].x - X[3].y;
    r.y = X[0].y - X[1].x - X[2].y + X[3].x;
  }
  return r;
}

PSF_D float norm2(float2 v) { return fmaf(v.x, v.x, v.y * v.y); }

// one profile value pair at the thread's radius -> both sums of slot R
template <int R>
PSF_D void oct_add(OctAcc& acc, const float2* q, float f, float2 t) {
  const float2 u = q[0], v0 = q[1];
  const float2 v = make_float2(fmaf(f, v0.x - u.x, u.x), fmaf(f, v0.y - u.y, u.y));
  // S_R += t v, C_R += conj(t) v, each product folded into the sums
  acc.s[R].x = fmaf(-t.y, v.y, fmaf(t.x, v.x, acc.s[R].x));
  acc.s[R].y = fmaf(t.y, v.x, fmaf(t.x, v.y, acc.s[R].y));
  acc.c[R].x = fmaf(t.y, v.y, fmaf(t.x, v.x, acc.c[R].x));
  acc.c[R].y = fmaf(-t.y, v.x, fmaf(t.x, v.y, acc.c[R].y));
}

template <int J>
PSF_D void oct_pair(OctAcc& acc, const float2* pp, const float2* pm, int n, float f,
                    float2 tp, float2 tn) {
  oct_add<J>(acc, pp, f, tp);
  if (n > 0) oct_add<(4 - J) & 3>(acc, pm, f, tn);
}

// Octant pixel geometry of the square grid: radius sample i0, weight f and
// direction (cos, sin) of pixel (a, b), b <= a < ceil(n / 2).
PSF_D OctPix oct_pixel(const HarmParams& p, int a, int b) {
  const double x = (a - 0.5 * (p.nx - 1)) * p.dx, y = (b - 0.5 * (p.ny - 1)) * p.dy;
  const double rho = sqrt(x * x + y * y);
  const double tt = p.dr > 0 ? rho / p.dr : 0.0;   // r_max = 0: all r_i = 0
  int i0 = (int)floor(tt);
  i0 = i0 < 0 ? 0 : (i0 > p.n_r - 2 ? p.n_r - 2 : i0);
  OctPix q;
  q.a = a;
  q.b = b;
  q.i0 = i0;
  q.f = (float)(tt - i0);
  q.cp = rho > 0 ? (float)(x / rho) : 1.f;
  q.sp = rho > 0 ? (float)(y / rho) : 0.f;
  q.pad[0] = q.pad[1] = 0;
  return q;
}

PSF_D void oct_index(int idx, int& a, int& b) {
  // idx -> (a, b), b <= a: idx = a (a + 1) / 2 + b
  a = (int)((sqrtf(8.f * (float)idx + 1.f) - 1.f) * 0.5f);
  while (a * (a + 1) / 2 > idx) --a;
  while ((a + 1) * (a + 2) / 2 <= idx) ++a;
  b = idx - a * (a + 1) / 2;
}

__global__ void k_oct_count(HarmParams p, int npx, int* __restrict__ cnt) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= npx) return;
  int a, b;
  oct_index(idx, a, b);
  atomicAdd(&cnt[oct_pixel(p, a, b).i0], 1);
}

// exclusive prefix sum of cnt[0 .. n) in place (one block of 1024 threads,
// n <= 4096: four consecutive buckets per thread)
__global__ void __launch_bounds__(1024) k_oct_scan(int* __restrict__ cnt, int n) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  int v[4], sum = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = 4 * t + k;
    v[k] = i < n ? cnt[i] : 0;
    sum += v[k];
  }
  part[t] = sum;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int add = t >= o ? part[t - o] : 0;
    __syncthreads();
    part[t] += add;
    __syncthreads();
  }
  int run = part[t] - sum;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = 4 * t + k;
    if (i < n) cnt[i] = run;
    run += v[k];
  }
}

__global__ void k_oct_fill(HarmParams p, int npx, int* __restrict__ cursor,
                           OctPix* __restrict__ tab) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= npx) return;
  int a, b;
  oct_index(idx, a, b);
  const OctPix q = oct_pixel(p, a, b);
  tab[atomicAdd(&cursor[q.i0], 1)] = q;
}

// (four blocks of 384 threads per SM cap the registers at 40 with a small
// spill; 256 workload emitters, split contraction: 6.76 ms per call against
// 7.67 ms at three blocks)
__global__ void __launch_bounds__(3 * HO_PIX, 4)
k_harm_intensity_oct(HarmParams p, const float2* __restrict__ prof,
                     const int* __restrict__ slice_em, const int* __restrict__ valid,
                     const int* __restrict__ ord, const OctPix* __restrict__ tab, int s0,
                     float* __restrict__ I) {
  extern __shared__ float2 stg[];   // staged window [3][2 Le + 1][range]
  __shared__ float part[3][8][HO_PIX];
  const int sl = blockIdx.y, s = s0 + sl;
  const int e = slice_em[s];
  if (e < 0 || !valid[e]) return;   // uniform over the block
  const int ch = threadIdx.x / HO_PIX, t = threadIdx.x - ch * HO_PIX;
  const int h = (p.nx + 1) / 2, npx = h * (h + 1) / 2;
  const int first = blockIdx.x * HO_PIX, idx = first + t;
  const bool act = idx < npx;
  const int L = p.m_max + 2, Le = ord[e] + 2, n_r = p.n_r, nrow = 2 * Le + 1;
  // the block's pixels are sorted by radius sample: their radii lie in
  // [lo, hi] with lo, hi from the first and the last pixel
  const int lo = tab[first].i0;
  const int hi = tab[min(first + HO_PIX, npx) - 1].i0 + 1;
  const int range = hi - lo + 1;
  const bool staged = (size_t)3 * nrow * range * sizeof(float2) <= (size_t)HO_SMEM;
  const float2* slice_prof = prof + (size_t)sl * 3 * p.n_ord * n_r;
  if (staged) {
    for (int x = threadIdx.x; x < 3 * nrow * range; x += 3 * HO_PIX) {
      const int r = x / range, ii = x - r * range;
      const int c = r / nrow, li = r - c * nrow;   // order l = li - Le
      stg[x] = slice_prof[((size_t)c * p.n_ord + (li - Le + L)) * n_r + lo + ii];
    }
    __syncthreads();
  }
  int a = 0, b = 0;
  if (act) {
    const OctPix q = tab[idx];
    a = q.a;
    b = q.b;
    const float f = q.f;
    const float2 w = make_float2(-q.sp, q.cp);    // i e^{i phi}
    const float2 wc = make_float2(-q.sp, -q.cp);  // its inverse
    OctAcc acc;
#pragma unroll
    for (int r = 0; r < 4; ++r) acc.s[r] = acc.c[r] = make_float2(0.f, 0.f);
    // order +n / -n rows of this channel: in the staged window (row stride
    // range) or in the profiles (row stride n_r)
    const int stride = staged ? range : n_r;
    const float2* pp = staged ? stg + ((size_t)ch * nrow + Le) * range + (q.i0 - lo)
                              : slice_prof + ((size_t)ch * p.n_ord + L) * n_r + q.i0;
    const float2* pm = pp;
    float2 tp = make_float2(1.f, 0.f), tn = make_float2(1.f, 0.f);
    // after each order, unless staged, an L2 prefetch of the rows
    // kHarmPrefetch orders ahead (within |l| <= Le, so inside this
    // channel's rows)
    int nn = 0;
    auto step = [&]() {
      tp = cmul(tp, w);
      tn = cmul(tn, wc);
      pp += stride;
      pm -= stride;
      if (!staged) {
        ++nn;
        const int ahead = min(kHarmPrefetch, Le - nn);
        if (ahead > 0) {
          asm volatile("prefetch.global.L2 [%0];" ::"l"(pp + (size_t)ahead * n_r));
          asm volatile("prefetch.global.L2 [%0];" ::"l"(pm - (size_t)ahead * n_r));
        }
      }
    };
    for (int n0 = 0; n0 <= Le; n0 += 4) {
      oct_pair<0>(acc, pp, pm, n0, f, tp, tn);
      step();
      if (n0 + 1 > Le) break;
      oct_pair<1>(acc, pp, pm, n0 + 1, f, tp, tn);
      step();
      if (n0 + 2 > Le) break;
      oct_pair<2>(acc, pp, pm, n0 + 2, f, tp, tn);
      step();
      if (n0 + 3 > Le) break;
      oct_pair<3>(acc, pp, pm, n0 + 3, f, tp, tn);
      step();
    }
    // images: 0 (x,y) S.1, 1 (-x,-y) S.-1, 2 (-y,x) S.i, 3 (y,-x) S.-i,
    //         4 (-x,y) C.1, 5 (x,-y) C.-1, 6 (y,x) C.-i, 7 (-y,-x) C.i
    part[ch][0][t] = norm2(oct_sum(acc.s, 0));
    part[ch][1][t] = norm2(oct_sum(acc.s, 1));
    part[ch][2][t] = norm2(oct_sum(acc.s, 2));
    part[ch][3][t] = norm2(oct_sum(acc.s, 3));
    part[ch][4][t] = norm2(oct_sum(acc.c, 0));
    part[ch][5][t] = norm2(oct_sum(acc.c, 1));
    part[ch][6][t] = norm2(oct_sum(acc.c, 3));
    part[ch][7][t] = norm2(oct_sum(acc.c, 2));
  }
  __syncthreads();
  if (ch != 0 || !act) return;
  float iv[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) iv[k] = part[0][k][t] + part[1][k][t] + part[2][k][t];
  float* out = I + (size_t)s * p.nx * p.ny;
  const int n = p.nx, am = n - 1 - a, bm = n - 1 - b;
  out[(size_t)a * n + b] = iv[0];
  out[(size_t)am * n + bm] = iv[1];
  out[(size_t)am * n + b] = iv[4];
  out[(size_t)a * n + bm] = iv[5];
  if (a != b) {
    out[(size_t)bm * n + a] = iv[2];
    out[(size_t)b * n + am] = iv[3];
    out[(size_t)b * n + a] = iv[6];
    out[(size_t)bm * n + am] = iv[7];
  }
}

}  // namespace

void launch_harm_pupil(const HarmParams& p, ThetaTable t, EmitterTable e, const double* zern,
                       const float* Zr, const float2* cs, float2* Pm, int* ord, float2* Bh,
                       unsigned* bh_max, cudaStream_t s) {
  const size_t smem = sizeof(float2) * (size_t)p.n_phi * HP_G;
  k_harm_pupil<<<dim3(p.n_em, ceil_div(p.n_theta, HP_G)), HP_THREADS, smem, s>>>(
      p, t, e, zern, Zr, cs, Pm);
  k_harm_order<<<p.n_em, 256, 0, s>>>(p, Pm, ord);
  if (bh_max) cudaMemsetAsync(bh_max, 0, sizeof(unsigned), s);
  k_harm_mix<<<dim3(p.n_em, ceil_div(p.n_theta, HM_NODES)), 256, 0, s>>>(p, t, e, Pm, ord, Bh,
                                                                         bh_max);
}

void launch_harm_jtab(const HarmParams& p, ThetaTable t, float* Jt, const TcHarm* tc_ops,
                      double sA, int bf16, cudaStream_t s) {
  const long long total = (long long)p.n_r * p.n_theta;
  uint16_t* a_hi = tc_ops ? tc_ops->A_hi : nullptr;
  uint16_t* a_lo = tc_ops ? tc_ops->A_lo : nullptr;
  if (tc_ops) {
    cudaMemsetAsync(a_hi, 0, tc_ops->a_bytes, s);
    cudaMemsetAsync(a_lo, 0, tc_ops->a_bytes, s);
  }
  k_harm_jtab<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(
      p, t, Jt, a_hi, a_lo, tc_ops ? tc_ops->kp : 0, tc_ops ? tc_ops->n_r_pad : 0, sA, bf16);
}

void launch_harm_operands(const HarmParams& p, ThetaTable t, const float2* Bh,
                          const int* slice_em, const int* valid, const int* ord,
                          const float2* zz, int s0, int ns, float2* D, const TcHarm& ops,
                          float sA, cudaStream_t s) {
  const long long nd = (long long)ns * p.n_theta;
  k_harm_defocus<<<(unsigned)((nd + 255) / 256), 256, 0, s>>>(p.n_theta, t, zz, s0, ns, D);
  const long long pairs = (long long)p.n_ord * ns;
  k_harm_bgen<<<(unsigned)((pairs + HB_TY - 1) / HB_TY), dim3(HB_TX, HB_TY), 0, s>>>(
      p, Bh, D, slice_em, valid, ord, s0, ns, ops.kp, ops.bh_max, sA, ops.B_hi, ops.B_lo,
      ops.out_scale);
  const int cpt = tc_harm_cols_per_tile();
  const int n_tiles = ceil_div(3 * ns, cpt);
  const long long nf = (long long)p.n_ord * n_tiles;
  k_harm_tile_need<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(p, slice_em, valid, ord, s0, ns,
                                                                 cpt, n_tiles, ops.need);
}

void launch_harm_profiles(const HarmParams& p, ThetaTable t, const float* Jt,
                          const float2* Bh, const int* slice_em, const int* valid,
                          const int* ord, const float2* zz, int s0, int ns, float2* D,
                          float2* prof, cudaStream_t s) {
  const long long nd = (long long)ns * p.n_theta;
  k_harm_defocus<<<(unsigned)((nd + 255) / 256), 256, 0, s>>>(p.n_theta, t, zz, s0, ns, D);
  const dim3 grid(ceil_div(3 * ns, HP_BN), ceil_div(p.n_r, HP_BM), p.n_ord);
  k_harm_profiles<<<grid, 256, 0, s>>>(p, Jt, Bh, slice_em, valid, ord, D, s0, ns, prof);
}

bool harm_square(const HarmParams& p) { return p.nx == p.ny && p.dx == p.dy; }

int harm_octant_pixels(const HarmParams& p) {
  const int h = (p.nx + 1) / 2;
  return harm_square(p) ? h * (h + 1) / 2 : 0;
}

void launch_harm_octant_table(const HarmParams& p, int* cnt, OctPix* tab, cudaStream_t s) {
  const int npx = harm_octant_pixels(p);
  if (npx == 0) return;
  cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)p.n_r, s);
  k_oct_count<<<ceil_div(npx, 256), 256, 0, s>>>(p, npx, cnt);
  k_oct_scan<<<1, 1024, 0, s>>>(cnt, p.n_r);
  k_oct_fill<<<ceil_div(npx, 256), 256, 0, s>>>(p, npx, cnt, tab);
}

void launch_harm_intensity(const HarmParams& p, const float2* prof, const int* slice_em,
                           const int* valid, const int* ord, const OctPix* octab, int s0,
                           int ns, float* I, cudaStream_t s) {
  if (harm_square(p)) {
    const int h = (p.nx + 1) / 2;
    const dim3 grid(ceil_div(h * (h + 1) / 2, HO_PIX), ns);
    k_harm_intensity_oct<<<grid, 3 * HO_PIX, HO_SMEM, s>>>(p, prof, slice_em, valid, ord,
                                                           octab, s0, I);
    return;
  }
  const int quarter = ((p.nx + 1) / 2) * ((p.ny + 1) / 2);
  const dim3 grid(ceil_div(quarter, 256), ns);
  k_harm_intensity<<<grid, 256, 0, s>>>(p, prof, slice_em, valid, ord, s0, I);
}

}  // namespace psf
