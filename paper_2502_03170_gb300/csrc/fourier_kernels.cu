// Fourier (Cartesian) strategy kernels: pupil node table (FP64), zoom
// matrices (FP64 twiddles), per-z pupil fields (double-float defocus), and
// the plain-FP32 separable complex contractions with the |E|^2 epilogue.
#include "fourier_kernels.cuh"
#include "optics_models.cuh"

namespace psf {

// ---------------------------------------------------------------------------
// Node table: geometry of the cell-centred pupil grid (Sec. 3.4 footnote),
// Gibson-Lanni path (Eq. 13-14), Zernike + free phase (Eq. 15), apodization
// (Eq. 16), envelope (Eq. 17), far-field basis change (Eq. 6, q_s = q_p = 1
// unless Fresnel) and the 1/s_z of dOmega = ds_x ds_y / s_z (Eq. 8).  FP64
// throughout, once per call, in two passes:
//   radial pass: everything that depends on the node's radius only, once per
//     octant pair (|m_p|, |m_q|) with |m_p| <= |m_q| (m = 2p + 1 - N), an
//     eighth of the nodes: optical path in cycles (reduced mod 1), amplitude
//     (1/cos, apodization, envelope, evanescent decay), cos, sin, q_s, q_p,
//     |m| / r of both coordinates and the Zernike radial sums per azimuthal
//     order (FP64);
//   node pass: the azimuthal factors cos(m phi), sin(m phi) of the Zernike
//     sum and the free phase (FP64), the basis change of Eq. 6 (FP32: the
//     amplitudes are stored in FP32) and the double-float n_i cos / lambda.
// ---------------------------------------------------------------------------
__device__ __forceinline__ size_t node_tri(int k1, int k2) {
  return (size_t)k2 * (k2 + 1) / 2 + k1;
}

__global__ void k_node_radial(NodeParams p, double* __restrict__ rad) {
  const int N = p.N;
  const int K = (N + 1) / 2;
  // flat index over the triangle k1 <= k2 (FP64 issues at about 2 FMA per
  // clock per SM here: spread the pairs evenly over small blocks)
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)K * (K + 1) / 2) return;
  int k2 = (int)((sqrt(8.0 * (double)idx + 1.0) - 1.0) * 0.5);
  while ((long long)k2 * (k2 + 1) / 2 > idx) --k2;
  while ((long long)(k2 + 1) * (k2 + 2) / 2 <= idx) ++k2;
  const int k1 = (int)(idx - (long long)k2 * (k2 + 1) / 2);
  const int r0 = (N & 1) ? 0 : 1;          // |m| = 2k + r0
  const long long m1 = 2 * k1 + r0, m2 = 2 * k2 + r0;
  double* rec = rad + kNodeRad * node_tri(k1, k2);
  if (m1 * m1 + m2 * m2 > (long long)N * N) {
    for (int k = 0; k < kNodeRad; ++k) rec[k] = 0.0;
    rec[1] = -1.0;
    return;
  }
  const double rr = sqrt((double)(m1 * m1 + m2 * m2));
  const double rn = rr / N;
  const double sin_t = p.s_max * rn;
  const double cos_t = sqrt(fmax(0.0, 1.0 - sin_t * sin_t));
  // Eq. 13: optical path in cycles; evanescent layers add decay.
  double w_cyc = 0.0, decay_cyc = 0.0;
  const double nis = p.n_i * sin_t;
  for (int l = 0; l < p.gl.n; ++l) {
    const double arg = p.gl.n_idx[l] * p.gl.n_idx[l] - nis * nis;
    if (arg >= 0.0)
      w_cyc += p.gl.t[l] * sqrt(arg) * p.inv_lambda;
    else
      decay_cyc += p.gl.t[l] * sqrt(-arg) * p.inv_lambda;
  }
  w_cyc -= rint(w_cyc);
  double a = 1.0 / cos_t;
  if (p.apodize) a *= sqrt(cos_t);
  if (p.s_env > 0) a *= exp(-(sin_t * sin_t) / (p.s_env * p.s_env));
  if (decay_cyc != 0.0) a *= exp(-2.0 * kPi * decay_cyc);
  dcplx qs{1.0, 0.0}, qp{1.0, 0.0};
  if (p.model == 2) fresnel_q(p.n_s, p.n_g, p.n_i, sin_t, qs, qp);
  rec[0] = w_cyc;
  rec[1] = a;
  rec[2] = cos_t;
  rec[3] = sin_t;
  rec[4] = qs.re;
  rec[5] = qs.im;
  rec[6] = qp.re;
  rec[7] = qp.im;
  rec[8] = rr > 0 ? (double)m1 / rr : 1.0;
  rec[9] = rr > 0 ? (double)m2 / rr : 0.0;
  // Eq. 15: radial sums of the Zernike terms by azimuthal order (radians)
  for (int m = 0; m <= kZernMaxOrder; ++m) {
    double pc = 0.0, ps = 0.0;
    if (m <= p.zp.max_m) {
      for (int k = p.zp.deg; k >= 0; --k) {
        pc = pc * rn + p.zp.c[m][k];
        ps = ps * rn + p.zp.s[m][k];
      }
    }
    rec[10 + 2 * m] = pc;
    rec[11 + 2 * m] = ps;
  }
}

__global__ void k_node_table(NodeParams p, const double* __restrict__ rad, NodeTable t) {
  const int N = p.N;
  const int NN = N * N;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NN) return;
  const int ip = idx / N, iq = idx - (idx / N) * N;
  const int mp = 2 * ip + 1 - N, mq = 2 * iq + 1 - N;
  const int r0 = (N & 1) ? 0 : 1;
  const int ap = abs(mp), aq = abs(mq);
  const int ka = (ap - r0) >> 1, kb = (aq - r0) >> 1;
  const double* rec = rad + kNodeRad * node_tri(min(ka, kb), max(ka, kb));
  const double a = rec[1];
  if (a < 0.0) {
#pragma unroll
    for (int c = 0; c < 6; ++c) t.amp[c * NN + idx] = 0.f;
    t.wfr[idx] = 0.f;
    t.kh[idx] = 0.f;
    t.kl[idx] = 0.f;
    return;
  }
  const double cos_t = rec[2], sin_t = rec[3];
  // cos phi = m_p / r, sin phi = m_q / r from the octant's |m| / r
  double cp = ap <= aq ? rec[8] : rec[9];
  double sp = ap <= aq ? rec[9] : rec[8];
  if (mp < 0) cp = -cp;
  if (mq < 0) sp = -sp;
  // Eq. 15: sum over azimuthal orders of the radial sums times cos / sin(m phi)
  double wz = 0.0;
  if (p.zp.max_m >= 0) {
    double cm = 1.0, sm = 0.0;
    for (int m = 0; m <= p.zp.max_m; ++m) {
      wz += rec[10 + 2 * m] * cm + rec[11 + 2 * m] * sm;
      const double cn = cm * cp - sm * sp;
      sm = sm * cp + cm * sp;
      cm = cn;
    }
  }
  if (p.phase_map) wz += (double)p.phase_map[idx];
  double w_total = rec[0] + wz * (0.5 / kPi);
  w_total -= rint(w_total);

  float e[6];
  const float af = (float)a;
  if (p.model == 1) {
    // scalar model (Eq. 3): e_far = e_inc, carried in channel 0
    e[0] = af;
    e[1] = e[2] = e[3] = e[4] = e[5] = 0.f;
  } else {
    // Eq. 6, columns for e_inc^x and e_inc^y (each / 2); q_s = q_p = 1 unless
    // the Fresnel coefficients of Eq. 7 are requested (complex past the
    // critical angle of a layer)
    const float2 qs = make_float2((float)rec[4], (float)rec[5]);
    const float2 qp = make_float2((float)rec[6], (float)rec[7]);
    const float ct = (float)cos_t, st = (float)sin_t, cpf = (float)cp, spf = (float)sp;
    const float c2 = cpf * cpf - spf * spf, s2 = 2.f * spf * cpf;
    auto lin = [](float a1, float2 x, float a2, float2 y) {
      return make_float2(a1 * x.x + a2 * y.x, a1 * x.y + a2 * y.y);
    };
    // xx = [qs (1 - c2) + qp (1 + c2) cos] / 2, xy = (qp cos - qs) s2 / 2,
    // yy = [qs (1 + c2) + qp (1 - c2) cos] / 2, z = -qp (cos phi, sin phi) sin
    const float2 xx = lin(0.5f * (1.f - c2), qs, 0.5f * (1.f + c2) * ct, qp);
    const float2 xy = lin(-0.5f * s2, qs, 0.5f * s2 * ct, qp);
    const float2 yy = lin(0.5f * (1.f + c2), qs, 0.5f * (1.f - c2) * ct, qp);
    const float2 zx = make_float2(-cpf * st * qp.x, -cpf * st * qp.y);
    const float2 zy = make_float2(-spf * st * qp.x, -spf * st * qp.y);
    const float2 px = make_float2((float)p.pol[0], (float)p.pol[1]);
    const float2 py = make_float2((float)p.pol[2], (float)p.pol[3]);
    auto mac = [&](float2 m1, float2 v1, float2 m2, float2 v2) {
      const float2 u = cmul(m1, v1), w = cmul(m2, v2);
      return make_float2(af * (u.x + w.x), af * (u.y + w.y));
    };
    const float2 ex = mac(xx, px, xy, py), ey = mac(xy, px, yy, py), ez = mac(zx, px, zy, py);
    e[0] = ex.x; e[1] = ex.y; e[2] = ey.x; e[3] = ey.y; e[4] = ez.x; e[5] = ez.y;
  }
#pragma unroll
  for (int c = 0; c < 6; ++c) t.amp[c * NN + idx] = e[c];
  t.wfr[idx] = (float)w_total;
  const f2x kap = split_double(p.n_i * cos_t * p.inv_lambda);
  t.kh[idx] = kap.hi;
  t.kl[idx] = kap.lo;
}

void launch_node_table(const NodeParams& p, NodeTable t, cudaStream_t s) {
  const int pairs = (int)node_rad_count(p.N);
  k_node_radial<<<ceil_div(pairs, 32), 32, 0, s>>>(p, t.rad);
  const int NN = p.N * p.N;
  k_node_table<<<ceil_div(NN, 128), 128, 0, s>>>(p, t.rad, t);
}

// ---------------------------------------------------------------------------
// Zoom matrix A[a][p] = exp(2 pi i (NA/lambda) u_p x_a): the lateral phase
// k s_max u_p x_a of Eq. 8, in FP64 cycles reduced mod 1, FP64 sincospi.
// ---------------------------------------------------------------------------
__global__ void k_twiddle(int N, int n_out, double d, double f, float2* A) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_out * N) return;
  const int a = idx / N, pp = idx - (idx / N) * N;
  const double x = (a - 0.5 * (n_out - 1)) * d;
  const double u = (double)(2 * pp + 1 - N) / N;
  double cyc = f * u * x;
  cyc -= rint(cyc);
  double sn, cs;
  sincospi(2.0 * cyc, &sn, &cs);
  A[idx] = make_float2((float)cs, (float)sn);
}

void launch_twiddle(int N, int n_out, double d, double na_over_lambda,
                    float2* A, cudaStream_t s) {
  k_twiddle<<<ceil_div(n_out * N, 256), 256, 0, s>>>(N, n_out, d,
                                                      na_over_lambda, A);
}

// ---------------------------------------------------------------------------
// Per-z pupil fields: P_c = amp_c exp(2 pi i (W + n_i z cos(theta)/lambda)).
// The defocus k z cos(theta) of Eq. 8 is formed in double-float cycles.
// ---------------------------------------------------------------------------
__global__ void k_pupil_z_f32(NodeTable t, int NN, const float2* __restrict__ zz,
                              int z0, int nzc, float2* __restrict__ P) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NN) return;
  float2 amp[3];
#pragma unroll
  for (int c = 0; c < 3; ++c)
    amp[c] = make_float2(t.amp[(2 * c) * NN + idx], t.amp[(2 * c + 1) * NN + idx]);
  const float wfr = t.wfr[idx];
  const f2x kap = {t.kh[idx], t.kl[idx]};
  for (int zc = 0; zc < nzc; ++zc) {
    const float2 z = zz[z0 + zc];
    const float r = frac_mul_add(kap, f2x{z.x, z.y}, wfr);
    const float2 e = cis_cycles(r);
#pragma unroll
    for (int c = 0; c < 3; ++c)
      P[(size_t)(zc * 3 + c) * NN + idx] = cmul(amp[c], e);
  }
}

void launch_pupil_z_f32(NodeTable t, int N, const float2* zz, int z0, int nzc,
                        float2* P, cudaStream_t s) {
  const int NN = N * N;
  k_pupil_z_f32<<<ceil_div(NN, 256), 256, 0, s>>>(t, NN, zz, z0, nzc, P);
}

// ---------------------------------------------------------------------------
// Plain FP32 batched complex GEMM "NT": C[m][n] = sum_k A[m][k] B[n][k].
// 64 x 64 tile, K step 16, 256 threads, 4 x 4 complex outputs per thread.
// MODE 0 stores C; MODE 1 loops over the three field channels of B and
// accumulates |scale * C_c|^2 into an intensity tile (stage-2 epilogue).
// ---------------------------------------------------------------------------
constexpr int SB_M = 64, SB_N = 64, SB_K = 16;

template <int MODE>
__global__ void __launch_bounds__(256)
k_cgemm_nt_f32(const float2* __restrict__ A, long long sA,
               const float2* __restrict__ B, long long sB, long long sBc,
               float2* __restrict__ C, long long sC, int M, int N, int K,
               float* __restrict__ I, long long sI, float2* __restrict__ F,
               long long sF, float scale) {
  __shared__ float2 As[SB_K][SB_M + 1];
  __shared__ float2 Bs[SB_K][SB_N + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * SB_M, n0 = blockIdx.x * SB_N;
  const long long bz = blockIdx.z;
  const float2* Ab = A + bz * sA;

  float inten[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) inten[i][j] = 0.f;

  const int n_chan = MODE == 1 ? 3 : 1;
  for (int ch = 0; ch < n_chan; ++ch) {
    const float2* Bb = B + bz * sB + ch * sBc;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

    for (int k0 = 0; k0 < K; k0 += SB_K) {
      const int kk = tid & 15;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = (tid >> 4) + 16 * i;
        const int gm = m0 + r, gn = n0 + r, gk = k0 + kk;
        As[kk][r] = (gm < M && gk < K) ? Ab[(size_t)gm * K + gk] : make_float2(0.f, 0.f);
        Bs[kk][r] = (gn < N && gk < K) ? Bb[(size_t)gn * K + gk] : make_float2(0.f, 0.f);
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < SB_K; ++k) {
        float2 a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j].x = fmaf(a[i].x, b[j].x, fmaf(-a[i].y, b[j].y, acc[i][j].x));
            acc[i][j].y = fmaf(a[i].x, b[j].y, fmaf(a[i].y, b[j].x, acc[i][j].y));
          }
      }
      __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
        if (gm >= M || gn >= N) continue;
        if (MODE == 0) {
          C[bz * sC + (size_t)gm * N + gn] = acc[i][j];
        } else {
          inten[i][j] += acc[i][j].x * acc[i][j].x + acc[i][j].y * acc[i][j].y;
          if (F) {
            // E = (-i) * scale * acc  (C = -i/(2 pi), scale = ds^2/(2 pi))
            F[bz * sF + (size_t)ch * M * N + (size_t)gm * N + gn] =
                make_float2(scale * acc[i][j].y, -scale * acc[i][j].x);
          }
        }
      }
  }
  if (MODE == 1) {
    const float s2 = scale * scale;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
        if (gm < M && gn < N) I[bz * sI + (size_t)gm * N + gn] = s2 * inten[i][j];
      }
  }
}

void launch_stage1_f32(const float2* Ay, const float2* P, float2* U, int N,
                       int ny, int nzc, cudaStream_t s) {
  // M = ny (b), N = N_p (p), K = N_p (q); batch = nzc * 3
  dim3 grid(ceil_div(N, SB_N), ceil_div(ny, SB_M), nzc * 3);
  k_cgemm_nt_f32<0><<<grid, 256, 0, s>>>(Ay, 0, P, (long long)N * N, 0, U,
                                         (long long)ny * N, ny, N, N, nullptr,
                                         0, nullptr, 0, 1.f);
}

void launch_stage2_f32(const float2* Ax, const float2* U, float* I,
                       float2* fields, int N, int nx, int ny, int nzc,
                       float ds2_over_2pi, cudaStream_t s) {
  // M = nx (a), N = ny (b), K = N_p (p); batch = nzc, channels looped inside
  dim3 grid(ceil_div(ny, SB_N), ceil_div(nx, SB_M), nzc);
  k_cgemm_nt_f32<1><<<grid, 256, 0, s>>>(
      Ax, 0, U, 3LL * ny * N, (long long)ny * N, nullptr, 0, nx, ny, N, I,
      (long long)nx * ny, fields, 3LL * nx * ny, ds2_over_2pi);
}

}  // namespace psf

namespace psf {

void launch_cgemm_nt_f32(const float2* A, long long sA, const float2* B,
                         long long sB, float2* C, long long sC, int M, int N,
                         int K, int batch, cudaStream_t s) {
  dim3 grid(ceil_div(N, SB_N), ceil_div(M, SB_M), batch);
  k_cgemm_nt_f32<0><<<grid, 256, 0, s>>>(A, sA, B, sB, 0, C, sC, M, N, K,
                                         nullptr, 0, nullptr, 0, 1.f);
}

__global__ void k_twiddle_adj(int N, int n_out, double d, double f, float2* AH) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_out * N) return;
  const int pp = idx / n_out, a = idx - (idx / n_out) * n_out;
  const double x = (a - 0.5 * (n_out - 1)) * d;
  const double u = (double)(2 * pp + 1 - N) / N;
  double cyc = f * u * x;
  cyc -= rint(cyc);
  double sn, cs;
  sincospi(2.0 * cyc, &sn, &cs);
  AH[idx] = make_float2((float)cs, (float)-sn);
}

void launch_twiddle_adj(int N, int n_out, double d, double na_over_lambda,
                        float2* AH, cudaStream_t s) {
  k_twiddle_adj<<<ceil_div(n_out * N, 256), 256, 0, s>>>(N, n_out, d,
                                                          na_over_lambda, AH);
}

// Stage-2 recomputation for the adjoint: all three channels held at once.
__global__ void __launch_bounds__(256)
k_stage2_adjsrc_f32(const float2* __restrict__ A, const float2* __restrict__ B,
                    const float* __restrict__ T, const float* __restrict__ GI,
                    float2* __restrict__ RT, float* __restrict__ loss_part,
                    int M, int N, int K, float scale) {
  __shared__ float2 As[SB_K][SB_M + 1];
  __shared__ float2 Bs[SB_K][SB_N + 1];
  __shared__ float red[256];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * SB_M, n0 = blockIdx.x * SB_N;
  const long long zc = blockIdx.z;
  float2 acc[3][4][4];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[c][i][j] = make_float2(0.f, 0.f);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    const float2* Bb = B + (zc * 3 + ch) * (long long)N * K;
    for (int k0 = 0; k0 < K; k0 += SB_K) {
      const int kk = tid & 15;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = (tid >> 4) + 16 * i;
        const int gm = m0 + r, gn = n0 + r, gk = k0 + kk;
        As[kk][r] = (gm < M && gk < K) ? A[(size_t)gm * K + gk] : make_float2(0.f, 0.f);
        Bs[kk][r] = (gn < N && gk < K) ? Bb[(size_t)gn * K + gk] : make_float2(0.f, 0.f);
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < SB_K; ++k) {
        float2 a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[ch][i][j].x = fmaf(a[i].x, b[j].x, fmaf(-a[i].y, b[j].y, acc[ch][i][j].x));
            acc[ch][i][j].y = fmaf(a[i].x, b[j].y, fmaf(a[i].y, b[j].x, acc[ch][i][j].y));
          }
      }
      __syncthreads();
    }
  }
  const float s2 = scale * scale;
  float lsum = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + ty + 16 * i, gn = n0 + tx + 16 * j;
      if (gm >= M || gn >= N) continue;
      float I = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        I += acc[c][i][j].x * acc[c][i][j].x + acc[c][i][j].y * acc[c][i][j].y;
      I *= s2;
      const size_t o = (size_t)zc * M * N + (size_t)gm * N + gn;
      float g;
      if (T) {
        const float d = I - T[o];
        lsum += d * d;
        g = 2.f * d;
      } else {
        g = GI[o];
      }
      const float w = 2.f * s2 * g;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        RT[((size_t)zc * 3 + c) * M * N + (size_t)gn * M + gm] =
            make_float2(w * acc[c][i][j].x, w * acc[c][i][j].y);
    }
  if (loss_part) {
    red[tid] = lsum;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
      if (tid < st) red[tid] += red[tid + st];
      __syncthreads();
    }
    if (tid == 0)
      loss_part[zc * (gridDim.x * gridDim.y) + blockIdx.y * gridDim.x + blockIdx.x] = red[0];
  }
}

int stage2_tiles(int nx, int ny) { return ceil_div(ny, SB_N) * ceil_div(nx, SB_M); }

void launch_stage2_adjsrc_f32(const float2* Ax, const float2* U,
                              const float* target, const float* grad_I,
                              float2* RT, float* loss_part, int N, int nx,
                              int ny, int nzc, float scale, cudaStream_t s) {
  dim3 grid(ceil_div(ny, SB_N), ceil_div(nx, SB_M), nzc);
  k_stage2_adjsrc_f32<<<grid, 256, 0, s>>>(Ax, U, target, grad_I, RT,
                                           target ? loss_part : nullptr, nx, ny,
                                           N, scale);
}

__global__ void k_grad_accum(const float2* __restrict__ Gh,
                             const float2* __restrict__ P, float* gW, int NN,
                             int nzc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= NN) return;
  float acc = gW[idx];
  for (int b = 0; b < nzc * 3; ++b) {
    const float2 g = Gh[(size_t)b * NN + idx], p = P[(size_t)b * NN + idx];
    // Re(i conj(g) p) = -Im(conj(g) p) = -(g.x p.y - g.y p.x)
    acc -= g.x * p.y - g.y * p.x;
  }
  gW[idx] = acc;
}

void launch_grad_accum(const float2* Gh, const float2* P, float* gW, int NN,
                       int nzc, cudaStream_t s) {
  k_grad_accum<<<ceil_div(NN, 256), 256, 0, s>>>(Gh, P, gW, NN, nzc);
}

// Zernike basis on the pupil nodes, once per call: Zt[j][p][q] = Z_{j+1}(u_p, v_q)
// (Eq. 15).  FP64 radial polynomial; cos(m phi) and sin(m phi) are the real
// and imaginary parts of ((u + i v) / rho)^m, so no trigonometric call.
__global__ void k_zernike_table(ZernBasis zb, int N, float* __restrict__ Zt) {
  // one thread per node, every term: the azimuthal factors cos / sin(m phi)
  // once per node by the rotation recursion, the radial polynomial of each
  // term by Horner from its degree down (FP64; the coefficients above the
  // degree are zero, so starting higher would add exact zeros only)
  const int NN = N * N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NN) return;
  const int ip = i / N, iq = i - (i / N) * N;
  const double u = (double)(2 * ip + 1 - N) / N, v = (double)(2 * iq + 1 - N) / N;
  const double rn = sqrt(u * u + v * v);
  double cm[kZernMaxOrder + 1], sm[kZernMaxOrder + 1];
  cm[0] = 1.0;
  sm[0] = 0.0;
  const double c = rn > 0.0 ? u / rn : 1.0, sn = rn > 0.0 ? v / rn : 0.0;
#pragma unroll
  for (int k = 0; k < kZernMaxOrder; ++k) {
    cm[k + 1] = cm[k] * c - sm[k] * sn;
    sm[k + 1] = cm[k] * sn + sm[k] * c;
  }
  for (int j = 0; j < zb.n_zern; ++j) {
    const int m = zb.m[j], am = m < 0 ? -m : m;
    double r = 0.0;
    for (int k = zb.deg[j]; k >= 0; --k) r = r * rn + zb.rc[j][k];
    double ang = 1.0;
    if (am > 0 && rn == 0.0) {
      ang = 0.0;                                  // odd N: the centre node
    } else if (am > 0) {
#pragma unroll
      for (int q = 1; q <= kZernMaxOrder; ++q)
        if (q == am) ang = m > 0 ? cm[q] : sm[q];
    }
    Zt[(size_t)j * NN + i] = (float)(r * ang);
  }
}

void launch_zernike_table(const ZernBasis& zb, int N, float* Zt, cudaStream_t s) {
  const int NN = N * N;
  if (zb.n_zern > 0 && NN > 0) k_zernike_table<<<(unsigned)((NN + 255) / 256), 256, 0, s>>>(zb, N, Zt);
}

// dL/dc_j = sum_{p,q} Z_j[p][q] dL/dW_0[p][q] for `nb` pupils at once: CTA
// (j, part) takes its contiguous 1/kZgParts of the nodes, reads that slice of
// Z_j once and reduces it against every pupil's gradient (FP64, fixed order);
// one thread per (k, j) then adds the parts in order.
constexpr int kZgParts = 64;

// One CTA per (Zernike term j, node part): every pupil of the group at once.
// Each thread reads Z_j at its nodes once and keeps one FP32 partial per
// pupil (a few nodes each); the CTA reduces all of them in one pass (warp
// shuffles in FP64, then the warps in a fixed order).
constexpr int kZgMaxNb = 8;

__global__ void __launch_bounds__(256)
k_zernike_grad_part(const float* __restrict__ Zt, int NN, int nb,
                    const float* __restrict__ gW, double* part) {
  __shared__ double red[8][kZgMaxNb];
  const int j = blockIdx.x, sp = blockIdx.y;
  const int i0 = (int)((long long)NN * sp / kZgParts), i1 = (int)((long long)NN * (sp + 1) / kZgParts);
  const float* z = Zt + (size_t)j * NN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k0 = 0; k0 < nb; k0 += kZgMaxNb) {
    const int kn = min(kZgMaxNb, nb - k0);
    float acc[kZgMaxNb];
#pragma unroll
    for (int k = 0; k < kZgMaxNb; ++k) acc[k] = 0.f;
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const float zi = z[i];
#pragma unroll
      for (int k = 0; k < kZgMaxNb; ++k)
        if (k < kn) acc[k] = fmaf(zi, gW[(size_t)(k0 + k) * NN + i], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < kZgMaxNb; ++k) {
      double v = (double)acc[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kn) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
      part[((size_t)(k0 + threadIdx.x) * gridDim.x + j) * kZgParts + sp] = v;
    }
    __syncthreads();
  }
}

__global__ void k_zernike_grad_fin(const double* __restrict__ part, int n_zern, int nb,
                                   float* grad_c) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_zern * nb) return;
  double v = 0.0;
  for (int sp = 0; sp < kZgParts; ++sp) v += part[(size_t)t * kZgParts + sp];
  grad_c[t] = (float)v;          // t = k * n_zern + j
}

size_t zernike_grad_part_bytes(int n_zern, int nb) {
  return (size_t)n_zern * nb * kZgParts * sizeof(double);
}

void launch_zernike_grad(const ZernBasis& zb, int N, const float* Zt, const float* gW,
                         int nb, double* part, float* grad_c, cudaStream_t s) {
  if (zb.n_zern <= 0 || nb <= 0) return;
  k_zernike_grad_part<<<dim3(zb.n_zern, kZgParts), 256, 0, s>>>(Zt, N * N, nb, gW, part);
  k_zernike_grad_fin<<<ceil_div(zb.n_zern * nb, 128), 128, 0, s>>>(part, zb.n_zern, nb,
                                                                   grad_c);
}

__global__ void k_sum_partials(const float* __restrict__ part, int n, float* out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = (float)red[0];
}

void launch_sum_partials(const float* part, int n, float* out, cudaStream_t s) {
  k_sum_partials<<<1, 256, 0, s>>>(part, n, out);
}

}  // namespace psf
