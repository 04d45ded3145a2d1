// tcgen05 / TMEM / TMA kernels of the split-precision Fourier path.
//
// One persistent warp-specialised kernel serves both separable stages of
// Eq. 8 (stage 1: contraction over q, stage 2: contraction over p with the
// |E_x|^2 + |E_y|^2 + |E_z|^2 epilogue):
//   warp 0      TMA producer: zoom-matrix tile A (128 rows = 64 outputs x
//               re/im) and data tile B (192 rows = 3 channels x 64), hi and lo
//               planes, BK K-elements (2 BK-byte swizzled rows) per stage,
//               STAGES-deep ring;
//   warp 1      TMEM allocator + single-thread tcgen05.mma issuer: per
//               16-wide K step three MMAs (A_hi B_hi, A_lo B_hi, A_hi B_lo),
//               M = 128, N = 192, FP32 accumulation in TMEM (two 192-column
//               accumulators so the epilogue of one tile overlaps the next);
//   warps 2-5   epilogue: tcgen05.ld of the accumulator, then either the
//               stage-1 hi/lo split store or the stage-2 |E|^2 reduction.
// Every mbarrier wait is bounded; on time-out the kernel records
// PSF_ERR_DEVICE_TIMEOUT in the workspace status word, drains its own
// in-flight copies and MMAs (again with a bound), frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "split_pack.cuh"
#include "tc_kernels.cuh"
#include "tc_pair_ptx.cuh"
#include "tc_ptx.cuh"
#include "timing.cuh"

namespace psf {
namespace tc {

constexpr int BM = 128;             // A rows per tile (64 outputs x re/im)
constexpr int BN = 192;             // B rows per tile (3 channels x 64)
constexpr int BOUT = 64;            // outputs per tile along m and per channel along n
// Measured on GB300 (256^2 pupil, 512^2 px, 128 planes): BK 64 / 2 stages
// 1.009 ms per stack, BK 32 / 4 stages 1.022 ms, BK 32 / 5 stages 1.031 ms:
// the ring depth is not the limit (operand delivery into the SM is).
#ifndef PSF_TC_BK
#define PSF_TC_BK 64
#endif
#ifndef PSF_TC_STAGES
#define PSF_TC_STAGES 2
#endif
constexpr int BK = PSF_TC_BK;       // K elements per stage (32: 64-byte rows, 64: 128-byte rows)
constexpr int STAGES = PSF_TC_STAGES;
constexpr int SWZ = BK * 2;         // bytes per smem row = swizzle span
static_assert(BK == 32 || BK == 64, "BK must be 32 or 64");
constexpr int A_BYTES = BM * BK * 2;                 // 16 KB
constexpr int B_BYTES = BN * BK * 2;                 // 24 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int TMEM_COLS = 512;
constexpr int ACC_COL = 256;        // column offset of accumulator 1
constexpr int NUM_THREADS = 192;
constexpr int EPI_THREADS = 128;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*barriers*/ + 1024 /*align*/;

struct Params {
  int planes, m_tiles, n_tiles, k_chunks;
  int m_out;            // outputs along m (ny for stage 1, nx for stage 2)
  int n_rows;           // rows per channel along n (N for stage 1, ny for stage 2)
  int N;                // pupil size (K = 2 N)
  uint32_t idesc;
  int mode;             // 0: stage 1 -> U split store; 1: stage 2 -> intensity
  int bf16;             // operand type of the split (0 fp16, 1 bf16)
  float out_scale;      // stage 1: S_U / (S_A S_P); stage 2: field scale / (S_A S_U)
  uint16_t* U_hi;
  uint16_t* U_lo;
  float* I;             // [planes][nx][ny] (already offset to the chunk)
  float2* F;            // [planes][3][nx][ny] or null
  int nx, ny;
  int* status;
  // mode 2 (Bessel radial contraction): D rows = (n, i) rows of the J_n
  // operand, D columns = (slice, re/im) interleaved; prof[slice][row] complex
  float2* prof;
  int rows_total;       // 3 N_r
  int n_slices;
  // mode 2 with conj_pairs: A rows (r, Re / Im of a complex operand b_r),
  // prof[s][r] = conj(b_r) . x_s from the two rows' accumulators
  int conj_pairs;
  const float* scale_ptr;   // device scalar: 1 / (S_B S_F)
  int m_fastest;        // tile order: consecutive tiles share the B tile
  // mode 3 (adjoint source, stage-2 recomputation): g = 2 (I - T) or dL/dI,
  // R = g E written transposed as BF16 hi/lo rows (c, b), columns [Re a | Im a]
  const float* T;       // [planes][nx][ny] (offset to the chunk) or null
  const float* Gin;     // [planes][nx][ny] or null
  float* loss_part;     // [planes * m_tiles * n_tiles * 4] or null
  uint16_t* R_hi;
  uint16_t* R_lo;
  // mode 4 (adjoint stage 2): Gh stored as FP32 gWz[plane][c][re/im][p][q]
  float* gWz;
  // mode 5 (harmonic radial contraction, one plane per order l' = l + hL):
  // A rows (|l|, i) with n_r_pad rows per order, B rows (l', column, re/im)
  // with b_rows_per_plane rows per order; D columns = (column, re/im);
  // prof[column][l'][i] complex (rows_total = N_r, n_slices = columns);
  // tiles with need[plane * n_tiles + nt] == 0 are skipped by every role
  const unsigned char* need;
  int n_ord, hL, n_r_pad, b_rows_per_plane;
};

// Mode 5 tiles none of whose columns needs the tile's order.
PSF_D bool tile_skipped(const Params& p, int plane, int nt) {
  return p.mode == 5 && !p.need[(size_t)plane * p.n_tiles + nt];
}

// Tile index -> (plane, m-tile, n-tile).
PSF_D void decode_tile(const Params& p, int t, int& plane, int& mt, int& nt) {
  const int tpp = p.m_tiles * p.n_tiles;
  plane = t / tpp;
  const int rem = t - plane * tpp;
  if (p.m_fastest) {
    nt = rem / p.m_tiles;
    mt = rem - nt * p.m_tiles;
  } else {
    mt = rem / p.n_tiles;
    nt = rem - mt * p.n_tiles;
  }
}

PSF_D uint4 shfl_xor4(uint4 v, int m) {
  v.x = __shfl_xor_sync(0xffffffffu, v.x, m);
  v.y = __shfl_xor_sync(0xffffffffu, v.y, m);
  v.z = __shfl_xor_sync(0xffffffffu, v.z, m);
  v.w = __shfl_xor_sync(0xffffffffu, v.w, m);
  return v;
}

// Stores the 64-byte row pieces w[16] of the 32 lanes (row offset `off` in
// 16-bit elements, valid rows only) after a 4 x 4 transpose of 16-byte units
// within each group of four lanes (jj = lane & 3, k4 = lane & ~3).
PSF_D void store_rows_t4(uint16_t* base, const uint32_t (&w)[16], int jj, int k4, int lane,
                         bool row_ok, size_t off) {
  uint4 u0 = make_uint4(w[0], w[1], w[2], w[3]), u1 = make_uint4(w[4], w[5], w[6], w[7]);
  uint4 u2 = make_uint4(w[8], w[9], w[10], w[11]), u3 = make_uint4(w[12], w[13], w[14], w[15]);
  const bool b1 = (jj & 2) != 0, b0 = (jj & 1) != 0;
  // swap the off-diagonal 2 x 2 blocks (partner lane ^ 2)
  uint4 s0 = b1 ? u0 : u2, s1 = b1 ? u1 : u3;
  uint4 r0 = shfl_xor4(s0, 2), r1 = shfl_xor4(s1, 2);
  if (b1) { u0 = r0; u1 = r1; } else { u2 = r0; u3 = r1; }
  // then the off-diagonal units inside each 2 x 2 block (partner lane ^ 1)
  s0 = b0 ? u0 : u1;
  s1 = b0 ? u2 : u3;
  r0 = shfl_xor4(s0, 1);
  r1 = shfl_xor4(s1, 1);
  if (b0) { u0 = r0; u2 = r1; } else { u1 = r0; u3 = r1; }
  // u_i = unit jj of row k4 + i; row offsets and validity come from that lane
  const uint4 us[4] = {u0, u1, u2, u3};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const unsigned long long ro = __shfl_sync(0xffffffffu, (unsigned long long)off, k4 + i);
    const int ok = __shfl_sync(0xffffffffu, row_ok ? 1 : 0, k4 + i);
    if (ok) *(uint4*)(base + ro + (size_t)jj * 8) = us[i];
  }
  (void)lane;
}

// --------------------------------------------------------------------------
// Epilogue of one accumulator tile (tile plane / mt / nt; this warp's TMEM
// lane quarter `quad`), shared by the single-CTA and the CTA-pair kernels:
//   mode 0  stage 1 / V: split hi+lo store of out_scale * D (rows transposed
//           4 x 4 between lanes so each store writes 64-byte row pieces)
//   mode 1  stage 2: I = out_scale^2 sum_c |E_c|^2 (and the fields)
//   mode 2  Bessel radial profiles
//   mode 3  adjoint source R = g E with the loss partials
//   mode 4  Gh stored in FP32
//   mode 5  harmonic radial profiles of one order
// --------------------------------------------------------------------------
PSF_D void tile_epilogue(const Params& p, uint32_t tbase, int plane, int mt, int nt,
                         int quad, int lane) {
  const int row = quad * 32 + lane;          // accumulator row = A row
  const int oi = row >> 1, part = row & 1;   // output index within tile, re/im
  const int mo = mt * BOUT + oi;             // output index along m
      if (p.mode == 2) {
        // Bessel: prof[s][row] = scale * (D[row][2k], D[row][2k+1]), s = nt*96 + k
        const int grow = mt * BM + row;
        const float sc = *p.scale_ptr;
        if (p.conj_pairs) {
          // rows 2r (Re b) and 2r + 1 (Im b) sit in adjacent lanes:
          // conj(b) x = (Re b Re x + Im b Im x) + i (Re b Im x - Im b Re x)
          const int orow = grow >> 1;
          const bool odd = (lane & 1) != 0;
          for (int h = 0; h < BN / 32; ++h) {
            uint32_t r[32];
            tmem_ld32(tbase + (uint32_t)(h * 32), r);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const float xr = __uint_as_float(r[2 * k]), xi = __uint_as_float(r[2 * k + 1]);
              const float pr = __shfl_xor_sync(0xffffffffu, xr, 1);
              const float pi = __shfl_xor_sync(0xffffffffu, xi, 1);
              const int s = nt * (BN / 2) + h * 16 + k;
              if (!odd && orow < p.rows_total && s < p.n_slices)
                p.prof[(size_t)s * p.rows_total + orow] =
                    make_float2(sc * (xr + pi), sc * (xi - pr));
            }
          }
          return;
        }
        for (int h = 0; h < BN / 32; ++h) {
          uint32_t r[32];
          tmem_ld32(tbase + (uint32_t)(h * 32), r);
          if (grow < p.rows_total) {
            const int s0 = nt * (BN / 2) + h * 16;
            if (s0 + 16 <= p.n_slices) {
              // the whole chunk is in range: no per-slice test
              float2* d = p.prof + (size_t)s0 * p.rows_total + grow;
#pragma unroll
              for (int k = 0; k < 16; ++k)
                d[(size_t)k * p.rows_total] =
                    make_float2(sc * __uint_as_float(r[2 * k]), sc * __uint_as_float(r[2 * k + 1]));
              continue;
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const int s = s0 + k;
              if (s < p.n_slices)
                p.prof[(size_t)s * p.rows_total + grow] =
                    make_float2(sc * __uint_as_float(r[2 * k]), sc * __uint_as_float(r[2 * k + 1]));
            }
          }
        }
      } else if (p.mode == 5) {
        // harmonic: prof[col][plane][i] = scale * (D[i][2k], D[i][2k+1]),
        // col = nt * 96 + k, i = mt * 128 + row
        const int gi = mt * BM + row;
        const float sc = *p.scale_ptr;
        for (int h = 0; h < BN / 32; ++h) {
          uint32_t r[32];
          tmem_ld32(tbase + (uint32_t)(h * 32), r);
          if (gi < p.rows_total) {
            const int col0 = nt * (BN / 2) + h * 16;
            if (col0 + 16 <= p.n_slices) {
              // the whole chunk is in range: no per-column test
              const size_t cs = (size_t)p.n_ord * p.rows_total;
              float2* d = p.prof + ((size_t)col0 * p.n_ord + plane) * p.rows_total + gi;
#pragma unroll
              for (int k = 0; k < 16; ++k)
                d[(size_t)k * cs] =
                    make_float2(sc * __uint_as_float(r[2 * k]), sc * __uint_as_float(r[2 * k + 1]));
              continue;
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const int col = col0 + k;
              if (col < p.n_slices)
                p.prof[((size_t)col * p.n_ord + plane) * p.rows_total + gi] =
                    make_float2(sc * __uint_as_float(r[2 * k]), sc * __uint_as_float(r[2 * k + 1]));
            }
          }
        }
      } else if (p.mode == 3) {
        // adjoint source: I from the three channels, g = 2 (I - T) or dL/dI,
        // R_c = g E_c with E = out_scale (D_im - i D_re); the lane holding D_re
        // writes Im R, the lane holding D_im writes Re R (no exchange needed)
        float sq[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) sq[j] = 0.f;
        for (int c = 0; c < 3; ++c) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            uint32_t r[32];
            tmem_ld32(tbase + (uint32_t)(c * BOUT + h * 32), r);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float v = __uint_as_float(r[j]);
              sq[h * 32 + j] = fmaf(v, v, sq[h * 32 + j]);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 64; ++j) sq[j] += __shfl_xor_sync(0xffffffffu, sq[j], 1);
        const float sc2 = p.out_scale * p.out_scale;
        const int bb0 = nt * BOUT + part * 32;      // this lane's 32 outputs along b
        const bool row_ok = mo < p.nx;
        float g[32];
        float lsum = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int bb = bb0 + j;
          float gv = 0.f;
          if (row_ok && bb < p.ny) {
            const float I = sc2 * (part ? sq[32 + j] : sq[j]);
            const size_t pix = ((size_t)plane * p.nx + mo) * p.ny + bb;
            if (p.T) {
              const float d = I - p.T[pix];
              lsum = fmaf(d, d, lsum);
              gv = 2.f * d;
            } else {
              gv = p.Gin[pix];
            }
          }
          g[j] = gv;
        }
        float go[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) go[j] = __shfl_xor_sync(0xffffffffu, g[j], 1);
        const float sgn = part ? p.out_scale : -p.out_scale;
        const size_t col = (size_t)(part ? 0 : p.nx) + mo;
        for (int c = 0; c < 3; ++c) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            uint32_t r[32];
            tmem_ld32(tbase + (uint32_t)(c * BOUT + h * 32), r);
            if (!row_ok) continue;
            const int bb0 = nt * BOUT + h * 32;
            const size_t pitch = (size_t)(2 * p.nx);
            const size_t o0 = ((size_t)(plane * 3 + c) * p.ny + bb0) * pitch + col;
            if (bb0 + 32 <= p.ny) {
              // the whole chunk is in range: no per-row test
              uint16_t* rh = p.R_hi + o0;
              uint16_t* rl = p.R_lo + o0;
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                const float gj = (h == part) ? g[j] : go[j];
                uint16_t hh, ll;
                split16(sgn * gj * __uint_as_float(r[j]), 1, hh, ll);
                rh[(size_t)j * pitch] = hh;
                rl[(size_t)j * pitch] = ll;
              }
              continue;
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int bb = bb0 + j;
              if (bb >= p.ny) continue;
              // outputs h * 32 + j: the lane's own g for h == part, else the partner's
              const float gj = (h == part) ? g[j] : go[j];
              uint16_t hh, ll;
              split16(sgn * gj * __uint_as_float(r[j]), 1, hh, ll);
              const size_t o = o0 + (size_t)j * pitch;
              p.R_hi[o] = hh;
              p.R_lo[o] = ll;
            }
          }
        }
        if (p.loss_part) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
          if (lane == 0 && mt < p.m_tiles)
            p.loss_part[(((size_t)plane * p.m_tiles + mt) * p.n_tiles + nt) * 4 + quad] = lsum;
        }
      } else if (p.mode == 4) {
        // Gh: this lane holds Re (part 0) or Im (part 1) of Gh_c[p][q = mo] for
        // 64 p; stored as FP32 Ghf[plane][c][part][p][q] (stores only: the
        // pupil fields are folded in by a separate coalesced pass)
        const bool q_ok = mo < p.m_out;
        for (int c = 0; c < 3; ++c) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            uint32_t r[32];
            tmem_ld32(tbase + (uint32_t)(c * BOUT + h * 32), r);
            if (!q_ok) continue;
            float* dst = p.gWz + (((size_t)(plane * 3 + c) * 2 + part) * p.n_rows) * p.m_out + mo;
            const int pp0 = nt * BOUT + h * 32;
            if (pp0 + 32 <= p.n_rows) {
              // the whole chunk is in range: no per-row test
              float* d0 = dst + (size_t)pp0 * p.m_out;
#pragma unroll
              for (int j = 0; j < 32; ++j) d0[(size_t)j * p.m_out] = __uint_as_float(r[j]);
              continue;
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int pp = pp0 + j;
              if (pp < p.n_rows) dst[(size_t)pp * p.m_out] = __uint_as_float(r[j]);
            }
          }
        }
      } else if (p.mode == 0) {
        // stage 1: U[plane][c][b = mo][part * N + p] = split(out_scale * D)
        const bool row_ok = mo < p.m_out;
        for (int c = 0; c < 3; ++c) {
          for (int h = 0; h < 2; ++h) {
            uint32_t r[32];
            tmem_ld32(tbase + (uint32_t)(c * BOUT + h * 32), r);
            const int p0 = nt * BOUT + h * 32;
            if (p0 >= p.n_rows) continue;                 // uniform over the warp
            const size_t off = ((size_t)(plane * 3 + c) * p.m_out + mo) * (size_t)(2 * p.N) +
                               (size_t)part * p.N + p0;
            uint32_t hw[16], lw[16];
#pragma unroll
            for (int j = 0; j < 32; j += 2)
              split2(p.out_scale * __uint_as_float(r[j]), p.out_scale * __uint_as_float(r[j + 1]),
                     p.bf16, hw[j / 2], lw[j / 2]);
            if (p0 + 32 <= p.n_rows) {
              // Each lane holds 64 bytes (four 16-byte units) of its own row.
              // A 4 x 4 transpose of units inside every group of four lanes
              // gives lane 4k + j the unit j of rows 4k .. 4k + 3, so every
              // store instruction writes eight contiguous 64-byte row pieces.
              const int jj = lane & 3, k4 = lane & ~3;
              store_rows_t4(p.U_hi, hw, jj, k4, lane, row_ok, off);
              store_rows_t4(p.U_lo, lw, jj, k4, lane, row_ok, off);
            } else if (row_ok) {
#pragma unroll
              for (int j = 0; j < 32; ++j) {
                if (p0 + j < p.n_rows) {
                  p.U_hi[off + j] = (uint16_t)(hw[j / 2] >> (16 * (j & 1)));
                  p.U_lo[off + j] = (uint16_t)(lw[j / 2] >> (16 * (j & 1)));
                }
              }
            }
          }
        }
      } else {
        // stage 2: I[plane][a = mo][b] = (out_scale)^2 sum_c (Re^2 + Im^2)
        float s[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) s[j] = 0.f;
        const bool want_f = p.F != nullptr;
        for (int c = 0; c < 3; ++c) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            uint32_t r[32];
            tmem_ld32(tbase + (uint32_t)(c * BOUT + h * 32), r);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float v = __uint_as_float(r[j]);
              s[h * 32 + j] = fmaf(v, v, s[h * 32 + j]);
            }
            if (want_f) {
              // E = (-i) * out_scale * (Re + i Im): pair Re (even row) with Im
              const int b0 = nt * BOUT + h * 32;
              for (int j = 0; j < 32; ++j) {
                const float v = p.out_scale * __uint_as_float(r[j]);
                const float o = __shfl_xor_sync(0xffffffffu, v, 1);
                const float re = part ? o : v, im = part ? v : o;
                // even lane writes j < 16, odd lane j >= 16
                if ((j < 16) == (part == 0) && mo < p.nx && b0 + j < p.ny)
                  p.F[((size_t)(plane * 3 + c) * p.nx + mo) * p.ny + b0 + j] =
                      make_float2(im, -re);
              }
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 64; ++j) s[j] += __shfl_xor_sync(0xffffffffu, s[j], 1);
        const float sc = p.out_scale * p.out_scale;
        const int b0 = nt * BOUT + part * 32;
        // even lane (part 0) stores b0 + [0, 32), odd lane b0 + [32, 64):
        // select with compile-time indices so s[] stays in registers
        float o[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) o[j] = sc * (part ? s[32 + j] : s[j]);
        if (mo < p.nx && b0 < p.ny) {
          float* dst = p.I + ((size_t)plane * p.nx + mo) * p.ny + b0;
          if (b0 + 32 <= p.ny && (p.ny & 3) == 0) {
#pragma unroll
            for (int v = 0; v < 8; ++v)
              ((float4*)dst)[v] = make_float4(o[4 * v], o[4 * v + 1], o[4 * v + 2], o[4 * v + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (b0 + j < p.ny) dst[j] = o[j];
          }
        }
      }
}

// --------------------------------------------------------------------------
// The persistent GEMM kernel
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(NUM_THREADS, 1)
k_split_cgemm(const __grid_constant__ CUtensorMap mapA_hi,
              const __grid_constant__ CUtensorMap mapA_lo,
              const __grid_constant__ CUtensorMap mapB_hi,
              const __grid_constant__ CUtensorMap mapB_lo, const Params p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  // bars: full[STAGES], empty[STAGES], tfull[2], tempty[2], drain
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 5);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), EPI_THREADS);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int tiles_per_plane = p.m_tiles * p.n_tiles;
  const int total = p.planes * tiles_per_plane;

  if (warp == 0 && lane == 0) {
    // ------------------------------ TMA producer ------------------------------
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    int issued = 0;
    for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
      int plane, mt, nt;
      decode_tile(p, t, plane, mt, nt);
      if (tile_skipped(p, plane, nt)) continue;
      // mode 5: the order's A plane and B rows
      const int arow = p.mode == 5 ? abs(plane - p.hL) * p.n_r_pad + mt * BM : mt * BM;
      const int brow = p.mode == 5 ? plane * p.b_rows_per_plane + nt * BN : nt * BN;
      for (int kc = 0; kc < p.k_chunks; ++kc) {
        if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, p.status)) {
          ok = false;
          break;
        }
        const uint32_t base = smem_u32(smem + stage * STAGE_BYTES);
        mbar_arrive_expect_tx(full_bar(stage), STAGE_BYTES);
        tma_load_2d(base, &mapA_hi, kc * BK, arow, full_bar(stage));
        tma_load_2d(base + A_BYTES, &mapA_lo, kc * BK, arow, full_bar(stage));
        if (p.mode == 2 || p.mode == 5) {
          tma_load_2d(base + 2 * A_BYTES, &mapB_hi, kc * BK, brow, full_bar(stage));
          tma_load_2d(base + 2 * A_BYTES + B_BYTES, &mapB_lo, kc * BK, brow,
                      full_bar(stage));
        } else {
          tma_load_3d(base + 2 * A_BYTES, &mapB_hi, kc * BK, nt * BOUT, plane * 3,
                      full_bar(stage));
          tma_load_3d(base + 2 * A_BYTES + B_BYTES, &mapB_lo, kc * BK, nt * BOUT,
                      plane * 3, full_bar(stage));
        }
        ++issued;
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    if (!ok) {
      // drain: wait (bounded) for the copies still in flight before exiting
      for (int k = 0; k < STAGES && k < issued; ++k) {
        if (--stage < 0) {
          stage = STAGES - 1;
          phase ^= 1u;
        }
        mbar_drain_wait(full_bar(stage), phase);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ------------------------------ MMA issuer --------------------------------
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    bool any = false;   // an MMA was issued (mode 5 may skip every tile of a CTA)
    for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
      if (p.mode == 5) {
        int plane, mt, nt;
        decode_tile(p, t, plane, mt, nt);
        if (tile_skipped(p, plane, nt)) continue;
      }
      any = true;
      if (!mbar_wait(tempty_bar(acc), acc_phase ^ 1u, abort_flag, p.status)) {
        ok = false;
        break;
      }
      tmem_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(acc * ACC_COL);
      for (int kc = 0; kc < p.k_chunks; ++kc) {
        if (!mbar_wait(full_bar(stage), phase, abort_flag, p.status)) {
          ok = false;
          break;
        }
        tmem_fence_after();
        const uint32_t base = smem_u32(smem + stage * STAGE_BYTES);
        const uint64_t dAh = smem_desc<SWZ>(base), dAl = smem_desc<SWZ>(base + A_BYTES);
        const uint64_t dBh = smem_desc<SWZ>(base + 2 * A_BYTES);
        const uint64_t dBl = smem_desc<SWZ>(base + 2 * A_BYTES + B_BYTES);
#pragma unroll
        for (int k = 0; k < BK / 16; ++k) {
          const uint64_t adv = (uint64_t)((k * 32) >> 4);   // 16 elements = 32 bytes
          const uint32_t first = (kc == 0 && k == 0) ? 0u : 1u;
          mma_f16(d_tmem, dAh + adv, dBh + adv, p.idesc, first);
          mma_f16(d_tmem, dAl + adv, dBh + adv, p.idesc, 1u);
          mma_f16(d_tmem, dAh + adv, dBl + adv, p.idesc, 1u);
        }
        mma_commit(empty_bar(stage));      // frees the smem slot when done
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (!ok) break;
      mma_commit(tfull_bar(acc));          // accumulator ready
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1u;
      }
    }
    // make sure every issued MMA has finished before TMEM is released
    if (any) {
      mma_commit(drain_bar);
      mbar_drain_wait(drain_bar, 0);
    }
  } else if (warp >= 2) {
    // ------------------------------ epilogue ----------------------------------
    const int quad = warp & 3;                 // TMEM lanes 32*quad .. +31
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
      int plane, mt, nt;
      decode_tile(p, t, plane, mt, nt);
      if (tile_skipped(p, plane, nt)) continue;
      int okw = 1;
      if (lane == 0) okw = mbar_wait(tfull_bar(acc), acc_phase, abort_flag, p.status) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) break;
      tmem_fence_after();
      const uint32_t tbase = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * ACC_COL);
      tile_epilogue(p, tbase, plane, mt, nt, quad, lane);
      tmem_fence_before();
      mbar_arrive(tempty_bar(acc));
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1u;
      }
    }
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// --------------------------------------------------------------------------
// Operand producers
// --------------------------------------------------------------------------
// Zoom-matrix blocks: rows (i, re) = [Re A | -Im A], (i, im) = [Im A | Re A],
// A[i][p] = exp(2 pi i f u_p x_i), scaled by S_A.  With m = 2p+1-N and
// n = 2i+1-n_out (exact integers) the angle is f d m n / (2N) cycles: one FP64
// product, reduced mod 1 in FP64, then sin/cos of the reduced angle.
// One thread per (i, p) writes the four block entries.
__global__ void k_twiddle_split(int N, int n_out, double alpha, float sA, int bf16,
                                uint16_t* hi, uint16_t* lo) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_out * N) return;
  const int i = idx / N, pp = idx - (idx / N) * N;
  const long long mn = (long long)(2 * pp + 1 - N) * (long long)(2 * i + 1 - n_out);
  double cyc = alpha * (double)mn;
  cyc -= rint(cyc);
  float sn, cs;
  sincospif(2.0f * (float)cyc, &sn, &cs);
  const size_t K = 2 * (size_t)N;
  const size_t re = (size_t)(2 * i) * K, im = re + K;
  uint16_t h, l;
  split16(sA * cs, bf16, h, l);
  hi[re + pp] = h;  lo[re + pp] = l;           // (i, re): Re A
  hi[im + N + pp] = h;  lo[im + N + pp] = l;   // (i, im): Re A
  split16(-sA * sn, bf16, h, l);
  hi[re + N + pp] = h;  lo[re + N + pp] = l;   // (i, re): -Im A
  split16(sA * sn, bf16, h, l);
  hi[im + pp] = h;  lo[im + pp] = l;           // (i, im): Im A
}

// Adjoint zoom-matrix blocks (BF16 hi + lo, unscaled): rows (q, re/im) over
// the pupil index, columns [Re | Im] over the output index b,
//   A'[q][b] = conj(A[b][q]) = exp(-2 pi i f u_q x_b),
// the same exact integer angle as k_twiddle_split with the roles swapped.
__global__ void k_twiddle_adj_split(int N, int n_out, double alpha, uint16_t* hi,
                                    uint16_t* lo) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_out * N) return;
  const int q = idx / n_out, bo = idx - (idx / n_out) * n_out;
  const long long mn = (long long)(2 * q + 1 - N) * (long long)(2 * bo + 1 - n_out);
  double cyc = -alpha * (double)mn;
  cyc -= rint(cyc);
  float sn, cs;
  sincospif(2.0f * (float)cyc, &sn, &cs);
  const size_t K = 2 * (size_t)n_out;
  const size_t re = (size_t)(2 * q) * K, im = re + K;
  uint16_t h, l;
  split16(cs, 1, h, l);
  hi[re + bo] = h;  lo[re + bo] = l;               // (q, re): Re A'
  hi[im + n_out + bo] = h;  lo[im + n_out + bo] = l;   // (q, im): Re A'
  split16(-sn, 1, h, l);
  hi[re + n_out + bo] = h;  lo[re + n_out + bo] = l;   // (q, re): -Im A'
  split16(sn, 1, h, l);
  hi[im + bo] = h;  lo[im + bo] = l;               // (q, im): Im A'
}

// Phase gradient of a chunk: for node (p, q) and each flat plane of the chunk
// (planes p0 .. p0 + planes over (pupil, z), nz_per per pupil)
//   2 s Re(conj(Gh_c) P_c) summed over c = scale * sum_c (Gh_re P_re + Gh_im P_im),
// with the pupil field P_c = amp_c e^{2 pi i (wfr_k + n_i z cos / lambda)}
// rebuilt from the node table exactly as the pupil planes were built, summed
// into gW[pupil] in plane order (a pupil's first plane starts its sum).  One
// thread per (pupil of the chunk, node).
// When the chunk holds a pupil's last plane its gW is final here, and the
// chain rule of Eq. 15 follows at once (Zt non-null): each warp reduces
// Z_j gW over its 32 nodes for every j and writes one FP64 partial to
// zpart[pupil][j][warp]; k_zernike_parts_fin sums them in a fixed order.
constexpr int kGwPlanes = 4;   // planes whose Gh loads are in flight together
__global__ void __launch_bounds__(256)
k_gw_fold(const float* __restrict__ Ghf, NodeTable t, const float2* __restrict__ zz, int N,
          int p0, int planes, int nz_per, float scale, float* gW,
          const float* __restrict__ Zt, int n_zern, double* __restrict__ zpart) {
  const int NN = N * N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int pk = p0 / nz_per + (int)blockIdx.y;           // pupil of this CTA
  const int a = max(pk * nz_per - p0, 0), b = min((pk + 1) * nz_per - p0, planes);
  const bool act = i < NN && a < b;
  float v = 0.f;
  if (act) {
    float amp[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) amp[c] = t.amp[(size_t)c * NN + i];
    const float w = t.wfr[(size_t)pk * NN + i];
    const f2x kap{t.kh[i], t.kl[i]};
    float* dst = gW + (size_t)pk * NN + i;
    v = (p0 + a - pk * nz_per == 0) ? 0.f : *dst;
    // one plane's contribution, its six Gh values already loaded
    auto plane_term = [&](int pl, const float (&gh)[6]) {
      const float2 z = zz[p0 + pl - pk * nz_per];
      const float2 e = cis_cycles(frac_mul_add(kap, f2x{z.x, z.y}, w));
      float acc = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float pr = amp[2 * c] * e.x - amp[2 * c + 1] * e.y;
        const float pi = amp[2 * c] * e.y + amp[2 * c + 1] * e.x;
        acc = fmaf(gh[2 * c], pr, acc);
        acc = fmaf(gh[2 * c + 1], pi, acc);
      }
      v = fmaf(scale, acc, v);
    };
    // the Gh values of kGwPlanes planes are loaded before any is used: the
    // kernel streams Gh once, and these loads in flight are what keeps HBM
    // busy (the sum still runs plane by plane, in order)
    int pl = a;
    for (; pl + kGwPlanes <= b; pl += kGwPlanes) {
      float gh[kGwPlanes][6];
#pragma unroll
      for (int u = 0; u < kGwPlanes; ++u)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const size_t gb = ((size_t)((pl + u) * 3 + c) * 2) * NN + i;
          gh[u][2 * c] = Ghf[gb];
          gh[u][2 * c + 1] = Ghf[gb + NN];
        }
#pragma unroll
      for (int u = 0; u < kGwPlanes; ++u) plane_term(pl + u, gh[u]);
    }
    for (; pl < b; ++pl) {
      float gh[6];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const size_t gb = ((size_t)(pl * 3 + c) * 2) * NN + i;
        gh[2 * c] = Ghf[gb];
        gh[2 * c + 1] = Ghf[gb + NN];
      }
      plane_term(pl, gh);
    }
    *dst = v;
  }
  // uniform over the CTA: does this chunk finish pupil pk?
  const bool last = a < b && (pk + 1) * nz_per - p0 <= planes;
  if (Zt == nullptr || !last) return;
  const int n_warps = (NN + 31) / 32, wg = i >> 5, lane = threadIdx.x & 31;
  for (int j = 0; j < n_zern; ++j) {
    float c = act ? Zt[(size_t)j * NN + i] * v : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0 && wg < n_warps) zpart[((size_t)pk * n_zern + j) * n_warps + wg] = (double)c;
  }
}

// grad_c[k][j] = sum of zpart[k][j][0 .. n_parts) in order (FP64)
__global__ void k_zernike_parts_fin(const double* __restrict__ zpart, int n_zern, int nb,
                                    int n_parts, float* grad_c) {
  __shared__ double red[8];
  const int kj = blockIdx.x;
  if (kj >= n_zern * nb) return;
  const double* pp = zpart + (size_t)kj * n_parts;
  double acc = 0.0;
  for (int q = threadIdx.x; q < n_parts; q += blockDim.x) acc += pp[q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    grad_c[kj] = (float)v;
  }
}

// Phases of a group of pupils from the shared Gibson-Lanni phase:
//   wfr[k][i] = frac(wfr_gl[i] + (sum_j c[k][j] Z_j[i] + W_0[k][i]) / 2 pi)
// (Zernike basis table Zt [n_zern][N N]; the Zernike and free phases are
// O(1) rad, so FP32 terms keep ~1e-7 rad).
// Eight pupils per thread (grid y): each basis value is read once for all of
// them; every pupil's sum runs over j in order, as for one pupil alone.  The
// block's coefficients are rounded to FP32 once, into shared memory (a
// double-to-float conversion issues at the FP64 rate).
constexpr int kGpPupils = 8;
constexpr int kGpMaxZern = 66;
__global__ void k_group_phase(const float* __restrict__ wfr_gl, const float* __restrict__ Zt,
                              const double* __restrict__ coef, int n_zern,
                              const float* __restrict__ phase_map, int NN, int nb,
                              float* wfr) {
  __shared__ float cf[kGpPupils][kGpMaxZern];
  const int k0 = blockIdx.y * kGpPupils;
  for (int e = threadIdx.x; e < kGpPupils * n_zern; e += blockDim.x) {
    const int u = e / n_zern, j = e - u * n_zern;
    cf[u][j] = k0 + u < nb ? (float)coef[(size_t)(k0 + u) * n_zern + j] : 0.f;
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NN) return;
  float w[kGpPupils];
#pragma unroll
  for (int u = 0; u < kGpPupils; ++u) w[u] = 0.f;
  for (int j = 0; j < n_zern; ++j) {
    const float z = Zt[(size_t)j * NN + i];
#pragma unroll
    for (int u = 0; u < kGpPupils; ++u) w[u] = fmaf(cf[u][j], z, w[u]);
  }
  const float g = wfr_gl[i];
#pragma unroll
  for (int u = 0; u < kGpPupils; ++u) {
    const int k = k0 + u;
    if (k >= nb) break;
    float wk = w[u];
    if (phase_map) wk += phase_map[(size_t)k * NN + i];
    float cyc = g + wk * (float)(0.5 / kPi);
    cyc -= rintf(cyc);
    wfr[(size_t)k * NN + i] = cyc;
  }
}

// loss[k] = sum of the partials of pupil k (n_per each), FP64, fixed order.
__global__ void k_loss_group(const float* __restrict__ part, int n_per, float* loss) {
  __shared__ double red[256];
  const float* pp = part + (size_t)blockIdx.x * n_per;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n_per; i += blockDim.x) acc += pp[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss[blockIdx.x] = (float)red[0];
}

// Pupil fields of a z-chunk as split operand rows: P[zc][c][p][q] -> row
// (zc, c, p), columns [Re q | Im q], scaled by S_P.  Four consecutive nodes
// (same p, N % 4 == 0) per thread and one plane per grid row, 8-byte stores.
// Planes are numbered flat over (pupil, z) with nz_per planes per pupil; the
// phase table of pupil k is t.wfr + k * wfr_stride (the amplitude and defocus
// tables are shared).  A single pupil passes wfr_stride = 0.
__global__ void k_pupil_z_split(NodeTable t, int N, const float2* __restrict__ zz,
                                int z0, int nzc, int nz_per, long long wfr_stride,
                                float sP, int bf16,
                                uint16_t* __restrict__ hi, uint16_t* __restrict__ lo) {
  const int NN = N * N;
  const int idx4 = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx4 * 4 >= NN) return;
  const int idx = idx4 * 4;
  const int ip = idx / N, iq = idx - (idx / N) * N;
  const int flat = z0 + (int)blockIdx.y;
  const int pk = flat / nz_per, zi = flat - pk * nz_per;
  float4 a4[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) a4[c] = *(const float4*)(t.amp + (size_t)c * NN + idx);
  const float4 w4 = *(const float4*)(t.wfr + (size_t)pk * wfr_stride + idx);
  const float4 kh4 = *(const float4*)(t.kh + idx);
  const float4 kl4 = *(const float4*)(t.kl + idx);
  const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
  const float khv[4] = {kh4.x, kh4.y, kh4.z, kh4.w};
  const float klv[4] = {kl4.x, kl4.y, kl4.z, kl4.w};
  float2 amp[3][4];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float re[4] = {a4[2 * c].x, a4[2 * c].y, a4[2 * c].z, a4[2 * c].w};
    const float imv[4] = {a4[2 * c + 1].x, a4[2 * c + 1].y, a4[2 * c + 1].z, a4[2 * c + 1].w};
#pragma unroll
    for (int k = 0; k < 4; ++k) amp[c][k] = make_float2(sP * re[k], sP * imv[k]);
  }
  {
    const int zc = blockIdx.y;                 // one plane per grid row
    const float2 z = zz[zi];
    float2 e[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      e[k] = cis_cycles(frac_mul_add(f2x{khv[k], klv[k]}, f2x{z.x, z.y}, wv[k]));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) v[k] = cmul(amp[c][k], e[k]);
      // packed pairs of consecutive nodes: node k in the low half
      uint32_t hr0, lr0, hr1, lr1, hm0, lm0, hm1, lm1;
      split2(v[0].x, v[1].x, bf16, hr0, lr0);
      split2(v[2].x, v[3].x, bf16, hr1, lr1);
      split2(v[0].y, v[1].y, bf16, hm0, lm0);
      split2(v[2].y, v[3].y, bf16, hm1, lm1);
      const size_t row = ((size_t)(zc * 3 + c) * N + ip) * (size_t)(2 * N);
      *(uint2*)(hi + row + iq) = make_uint2(hr0, hr1);
      *(uint2*)(lo + row + iq) = make_uint2(lr0, lr1);
      *(uint2*)(hi + row + N + iq) = make_uint2(hm0, hm1);
      *(uint2*)(lo + row + N + iq) = make_uint2(lm0, lm1);
    }
  }
}

// --------------------------------------------------------------------------
// Host side
// --------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t,
                                  void*, const cuuint64_t*, const cuuint64_t*,
                                  const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// rows x (2N) 16-bit matrix, box BK x box_rows, SWZ-byte swizzle
static bool make_map_2d(CUtensorMap* m, const uint16_t* base, int K, int rows,
                        int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, (void*)base, dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            SWZ == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// planes x rows x (2N), box BK x 64 x 3 (three channels stacked = 192 rows)
static bool make_map_3d(CUtensorMap* m, const uint16_t* base, int K, int rows,
                        int planes) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)K * 2, (cuuint64_t)K * 2 * rows};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)BOUT, 3};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, (void*)base, dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            SWZ == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static uint32_t make_idesc(int bf16) {
  const uint32_t fmt = bf16 ? 1u : 0u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(BM >> 4) << 24);
}

static int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

static int launch_gemm(const CUtensorMap& Ah, const CUtensorMap& Al,
                       const CUtensorMap& Bh, const CUtensorMap& Bl,
                       const Params& p, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_split_cgemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             SMEM_BYTES) != cudaSuccess)
      return PSF_ERR_CUDA;
    attr = true;
  }
  const int total = p.planes * p.m_tiles * p.n_tiles;
  const int grid = total < num_sms() ? total : num_sms();
  k_split_cgemm<<<grid, NUM_THREADS, SMEM_BYTES, s>>>(Ah, Al, Bh, Bl, p);
  return cudaPeekAtLastError() == cudaSuccess ? PSF_OK : PSF_ERR_CUDA;
}


// --------------------------------------------------------------------------
// CTA-pair form (cta_group::2) of the forward stages (modes 0 and 1).
// A cluster of two CTAs owns a 256-row tile (two m-tiles): each CTA loads its
// own 128 rows of the zoom-matrix operand and half (96 of 192 rows) of the
// data operand, so a CTA receives 56 KB per K chunk instead of 80 KB; the
// leader (rank 0) issues M = 256 MMAs that read both CTAs' shared memory and
// write both CTAs' TMEM, and multicasts its commits to both CTAs' barriers.
// Each CTA's epilogue reads its own 128 TMEM lanes exactly as in the single
// CTA kernel and returns the accumulator to the leader (remote arrival).
// Every wait is bounded as in k_split_cgemm.
// --------------------------------------------------------------------------
constexpr int PS_STAGES = 3;
constexpr int PS_ACCS = 2;                            // accumulators in TMEM
constexpr int PS_TMEM_COLS = 512;                     // two 192-column accumulators
constexpr int PB_ROWS = BN / 2;                       // 96 data rows per CTA
constexpr int PB_BYTES = PB_ROWS * BK * 2;            // 12 KB
constexpr int PSTAGE_BYTES = 2 * A_BYTES + 2 * PB_BYTES;
constexpr int PSMEM_BYTES = PS_STAGES * PSTAGE_BYTES + 1024 + 1024;


// Returns the accumulator to the leader: an arrival on its mbarrier (a
// shared::cluster address) with the default release.cta semantics.  A
// cluster-scope release would first wait until every global store of the
// tile just written is visible cluster-wide, holding the accumulator for the
// stores' latency; the hand-off orders only TMEM reads, which
// tcgen05.wait::ld has completed and tcgen05.fence::before_thread_sync
// orders before this arrival.
PSF_D void release_acc_remote(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}

PSF_D void decode_pair(const Params& p, int t, int& plane, int& mp, int& nt) {
  const int m_pairs = (p.m_tiles + 1) / 2;
  const int tpp = m_pairs * p.n_tiles;
  plane = t / tpp;
  const int rem = t - plane * tpp;
  nt = rem / m_pairs;
  mp = rem - nt * m_pairs;
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
k_split_cgemm_pair(const __grid_constant__ CUtensorMap mapA_hi,
                   const __grid_constant__ CUtensorMap mapA_lo,
                   const __grid_constant__ CUtensorMap mapB_hi,
                   const __grid_constant__ CUtensorMap mapB_lo, const Params p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + PS_STAGES * PSTAGE_BYTES);
  // bars: full[S], empty[S], tfull[2], tempty[2], drain
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * PS_STAGES + 5);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();
  const bool leader = rank == 0;
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (PS_STAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * PS_STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * PS_STAGES + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * PS_STAGES + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < PS_STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), 2 * EPI_THREADS);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc_pair(smem_u32(tmem_slot), PS_TMEM_COLS);
  tmem_fence_before();
  __syncthreads();
  cluster_sync_all();          // both CTAs' barriers exist before any remote use
  tmem_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int m_pairs = (p.m_tiles + 1) / 2;
  const int total = p.planes * m_pairs * p.n_tiles;
  const int cluster = blockIdx.x >> 1, n_clusters = gridDim.x >> 1;

  if (warp == 0 && lane == 0) {
    // ------------------------------ TMA producer ------------------------------
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    int issued = 0;
    for (int t = cluster; t < total && ok; t += n_clusters) {
      int plane, mp, nt;
      decode_pair(p, t, plane, mp, nt);
      const int mt = 2 * mp + (int)rank;
      for (int kc = 0; kc < p.k_chunks; ++kc) {
        if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, p.status)) {
          ok = false;
          break;
        }
        const uint32_t base = smem_u32(smem + stage * PSTAGE_BYTES);
        const uint32_t fb = mapa_shared(full_bar(stage), 0);   // the leader's barrier
        if (leader) mbar_arrive_expect_tx(full_bar(stage), 2 * PSTAGE_BYTES);
        tma_load_2d_pair(base, &mapA_hi, kc * BK, mt * BM, fb);
        tma_load_2d_pair(base + A_BYTES, &mapA_lo, kc * BK, mt * BM, fb);
        // this CTA's 96 rows of the 192 (3 channels x 64) data rows, 32 at a time
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const int r = (int)rank * PB_ROWS + i * 32;
          const int ch = r >> 6, ro = r & 63;
          tma_load_3d_pair(base + 2 * A_BYTES + i * 4096, &mapB_hi, kc * BK, nt * BOUT + ro,
                           plane * 3 + ch, fb);
          tma_load_3d_pair(base + 2 * A_BYTES + PB_BYTES + i * 4096, &mapB_lo, kc * BK,
                           nt * BOUT + ro, plane * 3 + ch, fb);
        }
        ++issued;
        if (++stage == PS_STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    if (!ok && leader) {
      // drain: wait (bounded) for the copies still in flight before exiting
      for (int k = 0; k < PS_STAGES && k < issued; ++k) {
        if (--stage < 0) {
          stage = PS_STAGES - 1;
          phase ^= 1u;
        }
        mbar_drain_wait(full_bar(stage), phase);
      }
    }
  } else if (warp == 1 && lane == 0 && leader) {
    // ------------------------------ MMA issuer (leader) -----------------------
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int t = cluster; t < total && ok; t += n_clusters) {
      if (!mbar_wait(tempty_bar(acc), acc_phase ^ 1u, abort_flag, p.status)) {
        ok = false;
        break;
      }
      tmem_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(acc * ACC_COL);
      for (int kc = 0; kc < p.k_chunks; ++kc) {
        if (!mbar_wait(full_bar(stage), phase, abort_flag, p.status)) {
          ok = false;
          break;
        }
        tmem_fence_after();
        const uint32_t base = smem_u32(smem + stage * PSTAGE_BYTES);
        const uint64_t dAh = smem_desc<SWZ>(base), dAl = smem_desc<SWZ>(base + A_BYTES);
        const uint64_t dBh = smem_desc<SWZ>(base + 2 * A_BYTES);
        const uint64_t dBl = smem_desc<SWZ>(base + 2 * A_BYTES + PB_BYTES);
#pragma unroll
        for (int k = 0; k < BK / 16; ++k) {
          const uint64_t adv = (uint64_t)((k * 32) >> 4);   // 16 elements = 32 bytes
          const uint32_t first = (kc == 0 && k == 0) ? 0u : 1u;
          mma_f16_pair(d_tmem, dAh + adv, dBh + adv, p.idesc, first);
          mma_f16_pair(d_tmem, dAl + adv, dBh + adv, p.idesc, 1u);
          mma_f16_pair(d_tmem, dAh + adv, dBl + adv, p.idesc, 1u);
        }
        mma_commit_pair(empty_bar(stage), 3);   // frees the stage in both CTAs
        if (++stage == PS_STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (!ok) break;
      mma_commit_pair(tfull_bar(acc), 3);       // accumulator ready in both CTAs
      if (++acc == PS_ACCS) {
        acc = 0;
        acc_phase ^= 1u;
      }
    }
    mma_commit_pair(drain_bar, 1);
    mbar_drain_wait(drain_bar, 0);
  } else if (warp >= 2) {
    // ------------------------------ epilogue ----------------------------------
    const int quad = warp & 3;                 // TMEM lanes 32*quad .. +31
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int t = cluster; t < total; t += n_clusters) {
      int okw = 1;
      if (lane == 0) okw = mbar_wait(tfull_bar(acc), acc_phase, abort_flag, p.status) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) break;
      tmem_fence_after();
      int plane, mp, nt;
      decode_pair(p, t, plane, mp, nt);
      const int mt = 2 * mp + (int)rank;
      const uint32_t tbase = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * ACC_COL);
      tile_epilogue(p, tbase, plane, mt, nt, quad, lane);
      tmem_fence_before();
      release_acc_remote(mapa_shared(tempty_bar(acc), 0));   // the leader's barrier
      if (++acc == PS_ACCS) {
        acc = 0;
        acc_phase ^= 1u;
      }
    }
  }
  tmem_fence_before();
  __syncthreads();
  cluster_sync_all();          // every MMA done and every TMEM read done in both CTAs
  tmem_fence_after();
  if (warp == 1) tmem_dealloc_pair(tmem_base, PS_TMEM_COLS);
}

// 3D map with 32-row boxes (one channel) for the pair kernel's data operand
static bool make_map_3d_rows32(CUtensorMap* m, const uint16_t* base, int K, int rows,
                               int planes) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)K * 2, (cuuint64_t)K * 2 * rows};
  cuuint32_t box[3] = {(cuuint32_t)BK, 32, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, (void*)base, dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            SWZ == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static uint32_t make_idesc_pair(int bf16) {
  const uint32_t fmt = bf16 ? 1u : 0u;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)((2 * BM) >> 4) << 24);
}

// Pair launch of a contraction (modes 0, 1, 3, 4): Bh, Bl must be 32-row maps.
static int launch_gemm_pair(const CUtensorMap& Ah, const CUtensorMap& Al,
                            const CUtensorMap& Bh, const CUtensorMap& Bl, Params p,
                            cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_split_cgemm_pair, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             PSMEM_BYTES) != cudaSuccess)
      return PSF_ERR_CUDA;
    attr = true;
  }
  p.idesc = make_idesc_pair(p.bf16);
  const int total = p.planes * ((p.m_tiles + 1) / 2) * p.n_tiles;
  int clusters = num_sms() / 2;
  if (total < clusters) clusters = total;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(2 * clusters);
  cfg.blockDim = dim3(NUM_THREADS);
  cfg.dynamicSmemBytes = PSMEM_BYTES;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_split_cgemm_pair, Ah, Al, Bh, Bl, p) != cudaSuccess)
    return PSF_ERR_CUDA;
  return cudaPeekAtLastError() == cudaSuccess ? PSF_OK : PSF_ERR_CUDA;
}
}  // namespace tc

// ==========================================================================
// Interface used by psf_api.cu
// ==========================================================================
const char* tc_fourier_supported(int N, int nx, int ny) {
  if (N % 8 != 0 || N < 16) return "n_pupil must be a multiple of 8 and >= 16";
  if (nx < 1 || ny < 1) return "empty output grid";
  return nullptr;
}

int tc_fourier_zchunk(int N, int nx, int ny, int nz) {
  // P (hi+lo) + U (hi+lo) per plane; a chunk holds up to 256 planes and 4 GB.
  // Longer launches beat keeping U in L2 (stage 2 leaves HBM mostly idle):
  // 256^2 / 512^2 / 128 planes takes 0.665 ms as one chunk against 0.774 ms
  // in 19-plane chunks that fit 96 MB.  Among the sizes from half the cap up
  // to it, take the one whose chunks fill the persistent CTA-pair rounds best
  // (stage-1 and stage-2 tile pairs over SMs / 2 clusters, summed over the
  // stack); ties keep the larger.
  const double per_z = 3.0 * 2.0 * 2.0 * 2.0 * N * ((double)N + ny);
  int cap = (int)(4096.0 * 1048576.0 / per_z);
  if (cap < 1) cap = 1;
  if (cap > 256) cap = 256;
  if (cap > nz) cap = nz;
  int sms = tc::num_sms();
  if (sms < 2) sms = 152;   // no device here: size for the target part
  const long long clusters = sms / 2;
  const long long per1 = (long long)((ceil_div(ny, tc::BOUT) + 1) / 2) * ceil_div(N, tc::BOUT);
  const long long per2 = (long long)((ceil_div(nx, tc::BOUT) + 1) / 2) * ceil_div(ny, tc::BOUT);
  int best = cap;
  long long best_rounds = -1;
  const int lo = cap / 2 > 1 ? cap / 2 : 1;
  for (int zc = cap; zc >= lo; --zc) {
    long long rounds = 0;
    for (int z0 = 0; z0 < nz; z0 += zc) {
      const long long n = nz - z0 < zc ? nz - z0 : zc;
      rounds += (n * per1 + clusters - 1) / clusters + (n * per2 + clusters - 1) / clusters;
    }
    if (best_rounds < 0 || rounds < best_rounds) {
      best_rounds = rounds;
      best = zc;
    }
  }
  return best;
}

void tc_fourier_carve(char* base, size_t* off, int N, int nx, int ny, int zc,
                      TcOperands* out) {
  auto take = [&](size_t elems) -> uint16_t* {
    *off = align_up(*off, 1024);
    uint16_t* p = base ? (uint16_t*)(base + *off) : nullptr;
    *off += elems * sizeof(uint16_t);
    return p;
  };
  const size_t K = 2 * (size_t)N;
  out->Ax_hi = take(2 * (size_t)nx * K);
  out->Ax_lo = take(2 * (size_t)nx * K);
  out->Ay_hi = take(2 * (size_t)ny * K);
  out->Ay_lo = take(2 * (size_t)ny * K);
  out->P_hi = take((size_t)zc * 3 * N * K);
  out->P_lo = take((size_t)zc * 3 * N * K);
  out->U_hi = take((size_t)zc * 3 * ny * K);
  out->U_lo = take((size_t)zc * 3 * ny * K);
}

double tc_pupil_amplitude_bound(const NodeParams& np) {
  // |P_c| <= A(theta)/cos(theta) * decay(theta) * |pol| (Eq. 6 is unitary)
  const double pol = sqrt(np.pol[0] * np.pol[0] + np.pol[1] * np.pol[1] +
                          np.pol[2] * np.pol[2] + np.pol[3] * np.pol[3]);
  double best = 0.0;
  const int S = 4096;
  for (int i = 0; i <= S; ++i) {
    const double st = np.s_max * i / S;
    const double ct = sqrt(fmax(0.0, 1.0 - st * st));
    double a = 1.0 / ct;
    if (np.apodize) a *= sqrt(ct);
    double dec = 0.0;
    for (int l = 0; l < np.gl.n; ++l) {
      const double arg = np.gl.n_idx[l] * np.gl.n_idx[l] - (np.n_i * st) * (np.n_i * st);
      if (arg < 0) dec += np.gl.t[l] * sqrt(-arg) * np.inv_lambda;
    }
    a *= exp(-2.0 * kPi * dec);
    if (a > best) best = a;
  }
  // Fresnel coefficients scale the unitary Eq. 6 by at most max|q| <= 2
  return 1.05 * best * (pol > 0 ? pol : 1.0) * (np.model == 2 ? 2.0 : 1.0);
}

static float pow2_scale(double bound, double target) {
  // largest power of two S with bound * S <= target
  if (!(bound > 0)) return 1.0f;
  return (float)exp2(floor(log2(target / bound)));
}

// Per-thread, per-device side stream and fork/join events (created once).
struct SideStream {
  int dev = -1;
  cudaStream_t s = nullptr;
  cudaEvent_t consumed = nullptr, ready = nullptr;
};

static SideStream* side_stream() {
  static thread_local SideStream ss[16];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return nullptr;
  SideStream& x = ss[dev];
  if (x.dev != dev) {
    if (cudaStreamCreateWithFlags(&x.s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&x.consumed, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&x.ready, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    x.dev = dev;
  }
  return &x;
}

// Copies of finished z-chunks to a pinned host output run on a per-device
// stream of their own: stage 2 of chunk i writes staging buffer i mod 2, an
// event hands it to the copy stream, and stage 2 of chunk i + 2 waits for
// that copy before it reuses the buffer.
struct CopyStream {
  int dev = -1;
  cudaStream_t s = nullptr;
  cudaEvent_t done[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
};

static CopyStream* copy_stream() {
  static thread_local CopyStream cs[16];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return nullptr;
  CopyStream& x = cs[dev];
  if (x.dev != dev) {
    bool ok = cudaStreamCreateWithFlags(&x.s, cudaStreamNonBlocking) == cudaSuccess;
    for (int b = 0; b < 2 && ok; ++b)
      ok = cudaEventCreateWithFlags(&x.done[b], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&x.copied[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      return nullptr;
    }
    x.dev = dev;
  }
  return &x;
}

bool tc_host_streaming_available() { return copy_stream() != nullptr; }

int tc_fourier_forward(const TcOperands& ops, NodeTable nodes, const float2* zz,
                       int N, int nx, int ny, double dx, double dy, int nz,
                       int zc, double na_over_lambda, float scale,
                       double amp_bound, int precision, float* intensity,
                       float2* fields, float* host_out, int* status, cudaStream_t s) {
  using namespace tc;
  CopyStream* cps = host_out ? copy_stream() : nullptr;
  if (host_out && !cps) return PSF_ERR_CUDA;
  const int bf16 = precision == PSF_PREC_SPLIT_BF16 ? 1 : 0;
  const int K = 2 * N;
  const double target = 16384.0;             // keep |scaled value| <= 2^14
  const float sA = pow2_scale(1.0, target);
  const float sP = pow2_scale(amp_bound, target);
  const float sU = pow2_scale(amp_bound * N, target);
  {
    TimingScope ts(kTimeSetup, s);
    k_twiddle_split<<<ceil_div(nx * N, 256), 256, 0, s>>>(
        N, nx, na_over_lambda * dx / (2.0 * N), sA, bf16, ops.Ax_hi, ops.Ax_lo);
  }
  {
    TimingScope ts(kTimeSetup, s);
    k_twiddle_split<<<ceil_div(ny * N, 256), 256, 0, s>>>(
        N, ny, na_over_lambda * dy / (2.0 * N), sA, bf16, ops.Ay_hi, ops.Ay_lo);
  }
  CUtensorMap mAx_h, mAx_l, mAy_h, mAy_l, mP_h, mP_l, mU_h, mU_l;
  bool ok = make_map_2d(&mAx_h, ops.Ax_hi, K, 2 * nx, BM) &&
            make_map_2d(&mAx_l, ops.Ax_lo, K, 2 * nx, BM) &&
            make_map_2d(&mAy_h, ops.Ay_hi, K, 2 * ny, BM) &&
            make_map_2d(&mAy_l, ops.Ay_lo, K, 2 * ny, BM) &&
            make_map_3d(&mP_h, ops.P_hi, K, N, 3 * zc) &&
            make_map_3d(&mP_l, ops.P_lo, K, N, 3 * zc) &&
            make_map_3d(&mU_h, ops.U_hi, K, ny, 3 * zc) &&
            make_map_3d(&mU_l, ops.U_lo, K, ny, 3 * zc);
  if (!ok) return PSF_ERR_CUDA;
  // CTA-pair contraction by default; PSF_TC_PAIR=0 in the environment selects
  // the single-CTA kernel (same arithmetic, bitwise identical results)
  const char* pe = getenv("PSF_TC_PAIR");
  bool pair = !(pe && pe[0] == '0');
  CUtensorMap mP2_h, mP2_l, mU2_h, mU2_l;
  if (pair)
    pair = make_map_3d_rows32(&mP2_h, ops.P_hi, K, N, 3 * zc) &&
           make_map_3d_rows32(&mP2_l, ops.P_lo, K, N, 3 * zc) &&
           make_map_3d_rows32(&mU2_h, ops.U_hi, K, ny, 3 * zc) &&
           make_map_3d_rows32(&mU2_l, ops.U_lo, K, ny, 3 * zc);
  const uint32_t idesc = make_idesc(bf16);
  // The pupil planes of chunk i + 1 are built on a side stream while stage 2
  // of chunk i runs (stage 2 does not read them); the side stream forks after
  // stage 1 of chunk i has consumed the buffer and joins before stage 1 of
  // chunk i + 1, so the caller's stream order is kept.
  SideStream* side = side_stream();
  auto pupil = [&](int zc0, cudaStream_t st) {
    const int n = nz - zc0 < zc ? nz - zc0 : zc;
    TimingScope ts(kTimePupil, st);
    const dim3 pg(ceil_div(N * N / 4, 128), n);
    k_pupil_z_split<<<pg, 128, 0, st>>>(nodes, N, zz, zc0, n, nz, 0, sP, bf16, ops.P_hi,
                                        ops.P_lo);
  };
  pupil(0, s);
  for (int z0 = 0; z0 < nz; z0 += zc) {
    const int nzc = nz - z0 < zc ? nz - z0 : zc;
    const bool more = z0 + zc < nz;
    Params p1;
    memset(&p1, 0, sizeof(p1));
    p1.planes = nzc;
    p1.m_tiles = ceil_div(ny, BOUT);
    p1.n_tiles = ceil_div(N, BOUT);
    p1.k_chunks = ceil_div(K, BK);
    p1.m_out = ny;
    p1.n_rows = N;
    p1.N = N;
    p1.idesc = idesc;
    p1.mode = 0;
    p1.bf16 = bf16;
    p1.out_scale = sU / (sA * sP);
    p1.U_hi = ops.U_hi;
    p1.U_lo = ops.U_lo;
    p1.nx = nx;
    p1.ny = ny;
    p1.status = status;
    int r;
    {
      TimingScope ts(kTimeStage1, s);
      r = pair ? launch_gemm_pair(mAy_h, mAy_l, mP2_h, mP2_l, p1, s) : PSF_ERR_CUDA;
      if (r) {                   // no cluster launch: the single-CTA kernel
        cudaGetLastError();
        pair = false;
        r = launch_gemm(mAy_h, mAy_l, mP_h, mP_l, p1, s);
      }
    }
    if (r) return r;
    if (more) {
      if (side) {
        cudaEventRecord(side->consumed, s);
        cudaStreamWaitEvent(side->s, side->consumed, 0);
        pupil(z0 + zc, side->s);
        cudaEventRecord(side->ready, side->s);
      }
    }
    Params p2 = p1;
    p2.m_tiles = ceil_div(nx, BOUT);
    p2.n_tiles = ceil_div(ny, BOUT);
    p2.m_out = nx;
    p2.n_rows = ny;
    p2.mode = 1;
    p2.out_scale = scale / (sA * sU);
    const int ci = z0 / zc, buf = ci & 1;
    const size_t plane = (size_t)nx * ny;
    if (cps) {
      // `intensity` is the two-chunk staging area; wait until the copy of
      // chunk i - 2 of this call has left this buffer (only events recorded
      // in this call are waited on, so the call holds no dependency on an
      // earlier one)
      p2.I = intensity + (size_t)buf * zc * plane;
      if (ci >= 2) cudaStreamWaitEvent(s, cps->copied[buf], 0);
    } else {
      p2.I = intensity + (size_t)z0 * plane;
    }
    p2.F = fields ? fields + (size_t)z0 * 3 * nx * ny : nullptr;
    {
      TimingScope ts(kTimeStage2, s);
      r = pair ? launch_gemm_pair(mAx_h, mAx_l, mU2_h, mU2_l, p2, s)
               : launch_gemm(mAx_h, mAx_l, mU_h, mU_l, p2, s);
    }
    if (r) return r;
    if (cps) {
      cudaEventRecord(cps->done[buf], s);
      cudaStreamWaitEvent(cps->s, cps->done[buf], 0);
      cudaMemcpyAsync(host_out + (size_t)z0 * plane, p2.I, (size_t)nzc * plane * sizeof(float),
                      cudaMemcpyDeviceToHost, cps->s);
      cudaEventRecord(cps->copied[buf], cps->s);
    }
    if (more) {
      if (side)
        cudaStreamWaitEvent(s, side->ready, 0);
      else
        pupil(z0 + zc, s);
    }
  }
  if (cps) {
    // the call completes on the caller's stream once the stack is on the host
    const int n_chunks = (nz + zc - 1) / zc;
    if (n_chunks >= 1) cudaStreamWaitEvent(s, cps->copied[0], 0);
    if (n_chunks >= 2) cudaStreamWaitEvent(s, cps->copied[1], 0);
  }
  return PSF_OK;
}

// ==========================================================================
// Fourier adjoint on the split-precision path
// ==========================================================================
const char* tc_fourier_bwd_supported(int N, int nx, int ny) {
  if (const char* why = tc_fourier_supported(N, nx, ny)) return why;
  if (nx % 8 != 0 || ny % 8 != 0)
    return "the split-precision adjoint needs nx and ny multiples of 8";
  return nullptr;
}

static double tc_bwd_plane_bytes(int N, int nx, int ny) {
  // P, U (input precision) + R, V (BF16), hi + lo, and gWz, per plane
  return 3.0 * 2.0 * 2.0 * 2.0 *
             ((double)N * N + (double)ny * N + (double)ny * nx + (double)N * ny) +
         24.0 * N * N;
}

int tc_fourier_bwd_zchunk(int N, int nx, int ny, int nz, int max_planes) {
  // As many planes as asked for (up to whole batches of pupils), at most
  // 2048 and 16 GB: longer launches fill the persistent contractions and
  // amortise the per-group work (batch 64 x 32 planes: 7.4 ms with 128-plane
  // groups, 5.1 ms as one group).
  (void)nz;
  int zc = (int)(16384.0 * 1048576.0 / tc_bwd_plane_bytes(N, nx, ny));
  const int cap = max_planes < 2048 ? max_planes : 2048;
  if (zc > cap) zc = cap;
  if (zc < 1) zc = 1;
  return zc;
}

int tc_fourier_bwd_group(int nz, int zc) { return nz <= zc ? zc / nz : 1; }

void tc_fourier_bwd_carve(char* base, size_t* off, int N, int nx, int ny, int nz, int zc,
                          TcBwdOperands* out) {
  auto take = [&](size_t bytes) -> char* {
    *off = align_up(*off, 1024);
    char* p = base ? base + *off : nullptr;
    *off += bytes;
    return p;
  };
  const int gp = tc_fourier_bwd_group(nz, zc);
  tc_fourier_carve(base, off, N, nx, ny, zc, &out->fwd);
  const size_t K2 = 2 * (size_t)N, NN = (size_t)N * N;
  out->AxH_hi = (uint16_t*)take(K2 * 2 * nx * 2);
  out->AxH_lo = (uint16_t*)take(K2 * 2 * nx * 2);
  out->AyH_hi = (uint16_t*)take(K2 * 2 * ny * 2);
  out->AyH_lo = (uint16_t*)take(K2 * 2 * ny * 2);
  out->R_hi = (uint16_t*)take((size_t)zc * 3 * ny * 2 * nx * 2);
  out->R_lo = (uint16_t*)take((size_t)zc * 3 * ny * 2 * nx * 2);
  out->V_hi = (uint16_t*)take((size_t)zc * 3 * N * 2 * ny * 2);
  out->V_lo = (uint16_t*)take((size_t)zc * 3 * N * 2 * ny * 2);
  out->gWz = (float*)take((size_t)zc * 6 * NN * 4);
  out->wfr = (float*)take((size_t)gp * NN * 4);
  out->coef = (double*)take((size_t)gp * 66 * 8);
  out->gW = (float*)take((size_t)gp * NN * 4);
  const size_t parts = (size_t)gp * nz * ceil_div(nx, tc::BOUT) * ceil_div(ny, tc::BOUT) * 4;
  out->loss_part = (float*)take(parts * 4);
  out->group = gp;
}

int tc_fourier_bwd_setup(const TcBwdOperands& ops, int N, int nx, int ny, double dx,
                         double dy, double na_over_lambda, int precision, cudaStream_t s) {
  using namespace tc;
  const int bf16 = precision == PSF_PREC_SPLIT_BF16 ? 1 : 0;
  const float sA = pow2_scale(1.0, 16384.0);
  k_twiddle_split<<<ceil_div(nx * N, 256), 256, 0, s>>>(
      N, nx, na_over_lambda * dx / (2.0 * N), sA, bf16, ops.fwd.Ax_hi, ops.fwd.Ax_lo);
  k_twiddle_split<<<ceil_div(ny * N, 256), 256, 0, s>>>(
      N, ny, na_over_lambda * dy / (2.0 * N), sA, bf16, ops.fwd.Ay_hi, ops.fwd.Ay_lo);
  k_twiddle_adj_split<<<ceil_div(nx * N, 256), 256, 0, s>>>(
      N, nx, na_over_lambda * dx / (2.0 * N), ops.AxH_hi, ops.AxH_lo);
  k_twiddle_adj_split<<<ceil_div(ny * N, 256), 256, 0, s>>>(
      N, ny, na_over_lambda * dy / (2.0 * N), ops.AyH_hi, ops.AyH_lo);
  return cudaPeekAtLastError() == cudaSuccess ? PSF_OK : PSF_ERR_CUDA;
}

struct TcBwdMaps {
  CUtensorMap Ax_h, Ax_l, Ay_h, Ay_l, P_h, P_l, U_h, U_l;
  CUtensorMap AxH_h, AxH_l, AyH_h, AyH_l, R_h, R_l, V_h, V_l;
  CUtensorMap P2_h, P2_l, R2_h, R2_l, U2_h, U2_l, V2_h, V2_l;   // 32-row (pair) maps
};

void tc_group_phase(const TcBwdOperands& ops, const float* wfr_gl, const float* Zt,
                    const double* coef, int n_zern, const float* phase_map, int N, int nb,
                    cudaStream_t s) {
  tc::k_group_phase<<<dim3(ceil_div(N * N, 256), ceil_div(nb, tc::kGpPupils)), 256, 0, s>>>(
      wfr_gl, Zt, coef, n_zern, phase_map, N * N, nb, ops.wfr);
}

size_t tc_zernike_parts_bytes(int N, int n_zern, int nb) {
  return (size_t)nb * (n_zern > 0 ? n_zern : 1) * (((size_t)N * N + 31) / 32) * sizeof(double) +
         sizeof(double);
}

int tc_fourier_backward(const TcBwdOperands& ops, NodeTable nodes, const float2* zz,
                        int N, int nx, int ny, int nz, int n_pupils, int zc, float scale,
                        double amp_bound, int precision, const float* target,
                        const float* grad_intensity, float* gW, float* loss,
                        const float* Zt, int n_zern, double* zpart, float* grad_c,
                        int* status, cudaStream_t s) {
  using namespace tc;
  const int bf16 = precision == PSF_PREC_SPLIT_BF16 ? 1 : 0;
  const int K = 2 * N;
  const double tgt = 16384.0;
  const float sA = pow2_scale(1.0, tgt);
  const float sP = pow2_scale(amp_bound, tgt);
  const float sU = pow2_scale(amp_bound * N, tgt);
  const TcOperands& f = ops.fwd;
  static thread_local TcBwdMaps m;      // encoded per call (host work only)
  bool ok = make_map_2d(&m.Ax_h, f.Ax_hi, K, 2 * nx, BM) &&
            make_map_2d(&m.Ax_l, f.Ax_lo, K, 2 * nx, BM) &&
            make_map_2d(&m.Ay_h, f.Ay_hi, K, 2 * ny, BM) &&
            make_map_2d(&m.Ay_l, f.Ay_lo, K, 2 * ny, BM) &&
            make_map_3d(&m.P_h, f.P_hi, K, N, 3 * zc) &&
            make_map_3d(&m.P_l, f.P_lo, K, N, 3 * zc) &&
            make_map_3d(&m.U_h, f.U_hi, K, ny, 3 * zc) &&
            make_map_3d(&m.U_l, f.U_lo, K, ny, 3 * zc) &&
            make_map_2d(&m.AxH_h, ops.AxH_hi, 2 * nx, 2 * N, BM) &&
            make_map_2d(&m.AxH_l, ops.AxH_lo, 2 * nx, 2 * N, BM) &&
            make_map_2d(&m.AyH_h, ops.AyH_hi, 2 * ny, 2 * N, BM) &&
            make_map_2d(&m.AyH_l, ops.AyH_lo, 2 * ny, 2 * N, BM) &&
            make_map_3d(&m.R_h, ops.R_hi, 2 * nx, ny, 3 * zc) &&
            make_map_3d(&m.R_l, ops.R_lo, 2 * nx, ny, 3 * zc) &&
            make_map_3d(&m.V_h, ops.V_hi, 2 * ny, N, 3 * zc) &&
            make_map_3d(&m.V_l, ops.V_lo, 2 * ny, N, 3 * zc);
  if (!ok) return PSF_ERR_CUDA;
  // the four contractions run on the CTA-pair kernel unless PSF_TC_PAIR=0 or
  // the cluster launch is refused (then the single-CTA kernel, same results)
  const char* pe = getenv("PSF_TC_PAIR");
  bool pair = !(pe && pe[0] == '0');
  if (pair)
    pair = make_map_3d_rows32(&m.P2_h, f.P_hi, K, N, 3 * zc) &&
           make_map_3d_rows32(&m.P2_l, f.P_lo, K, N, 3 * zc) &&
           make_map_3d_rows32(&m.R2_h, ops.R_hi, 2 * nx, ny, 3 * zc) &&
           make_map_3d_rows32(&m.R2_l, ops.R_lo, 2 * nx, ny, 3 * zc) &&
           make_map_3d_rows32(&m.U2_h, f.U_hi, K, ny, 3 * zc) &&
           make_map_3d_rows32(&m.U2_l, f.U_lo, K, ny, 3 * zc) &&
           make_map_3d_rows32(&m.V2_h, ops.V_hi, 2 * ny, N, 3 * zc) &&
           make_map_3d_rows32(&m.V2_l, ops.V_lo, 2 * ny, N, 3 * zc);
  auto gemm_any = [&](const CUtensorMap& Ah, const CUtensorMap& Al, const CUtensorMap& Bh,
                   const CUtensorMap& Bl, const CUtensorMap& Bh2, const CUtensorMap& Bl2,
                   const Params& p) {
    if (pair) {
      if (launch_gemm_pair(Ah, Al, Bh2, Bl2, p, s) == PSF_OK) return PSF_OK;
      cudaGetLastError();
      pair = false;
    }
    return launch_gemm(Ah, Al, Bh, Bl, p, s);
  };
  const uint32_t idesc = make_idesc(bf16), idesc_b = make_idesc(1);
  const int tiles2 = ceil_div(nx, BOUT) * ceil_div(ny, BOUT);
  const int total = n_pupils * nz;                 // flat planes of this group
  NodeTable tn = nodes;
  tn.wfr = ops.wfr;
  int r;
  for (int z0 = 0; z0 < total; z0 += zc) {
    const int nzc = total - z0 < zc ? total - z0 : zc;
    {
      TimingScope ts(kTimePupil, s);
      const dim3 pg(ceil_div(N * N / 4, 128), nzc);
      k_pupil_z_split<<<pg, 128, 0, s>>>(tn, N, zz, z0, nzc, nz, (long long)N * N, sP,
                                         bf16, f.P_hi, f.P_lo);
    }
    Params p1;
    memset(&p1, 0, sizeof(p1));
    p1.planes = nzc;
    p1.m_tiles = ceil_div(ny, BOUT);
    p1.n_tiles = ceil_div(N, BOUT);
    p1.k_chunks = ceil_div(K, BK);
    p1.m_out = ny;
    p1.n_rows = N;
    p1.N = N;
    p1.idesc = idesc;
    p1.mode = 0;
    p1.bf16 = bf16;
    p1.out_scale = sU / (sA * sP);
    p1.U_hi = f.U_hi;
    p1.U_lo = f.U_lo;
    p1.nx = nx;
    p1.ny = ny;
    p1.status = status;
    {
      TimingScope ts(kTimeStage1, s);
      if ((r = gemm_any(m.Ay_h, m.Ay_l, m.P_h, m.P_l, m.P2_h, m.P2_l, p1))) return r;
    }
    // stage 2 recomputed: I, loss partials and R^T (BF16)
    Params p3 = p1;
    p3.m_tiles = ceil_div(nx, BOUT);
    p3.n_tiles = ceil_div(ny, BOUT);
    p3.m_out = nx;
    p3.n_rows = ny;
    p3.mode = 3;
    p3.out_scale = scale / (sA * sU);
    const size_t zoff = (size_t)z0 * nx * ny;
    p3.T = target ? target + zoff : nullptr;
    p3.Gin = target ? nullptr : grad_intensity + zoff;
    p3.loss_part = target ? ops.loss_part + (size_t)z0 * tiles2 * 4 : nullptr;
    p3.R_hi = ops.R_hi;
    p3.R_lo = ops.R_lo;
    {
      TimingScope ts(kTimeAdjoint, s);
      if ((r = gemm_any(m.Ax_h, m.Ax_l, m.U_h, m.U_l, m.U2_h, m.U2_l, p3))) return r;
    }
    // V[c][p][b] = sum_a conj(Ax[a][p]) R_c[a][b]   (split BF16, stored like U)
    Params pv = p1;
    pv.m_tiles = ceil_div(N, BOUT);
    pv.n_tiles = ceil_div(ny, BOUT);
    pv.k_chunks = ceil_div(2 * nx, BK);
    pv.m_out = N;
    pv.n_rows = ny;
    pv.N = ny;
    pv.idesc = idesc_b;
    pv.bf16 = 1;
    pv.out_scale = 1.f;
    pv.U_hi = ops.V_hi;
    pv.U_lo = ops.V_lo;
    {
      TimingScope ts(kTimeAdjoint, s);
      if ((r = gemm_any(m.AxH_h, m.AxH_l, m.R_h, m.R_l, m.R2_h, m.R2_l, pv))) return r;
    }
    // Gh^T[q][p] = sum_b conj(Ay[b][q]) V[p][b] -> Ghf; then 2 s Re(conj(Gh) P)
    Params p4 = p1;
    p4.m_tiles = ceil_div(N, BOUT);
    p4.n_tiles = ceil_div(N, BOUT);
    p4.k_chunks = ceil_div(2 * ny, BK);
    p4.m_out = N;
    p4.n_rows = N;
    p4.N = N;
    p4.idesc = idesc_b;
    p4.bf16 = 1;
    p4.mode = 4;
    p4.gWz = ops.gWz;
    {
      TimingScope ts(kTimeAdjoint, s);
      if ((r = gemm_any(m.AyH_h, m.AyH_l, m.V_h, m.V_l, m.V2_h, m.V2_l, p4))) return r;
      const int pk0 = z0 / nz, pk1 = (z0 + nzc - 1) / nz;
      k_gw_fold<<<dim3(ceil_div(N * N, 256), pk1 - pk0 + 1), 256, 0, s>>>(
          ops.gWz, tn, zz, N, z0, nzc, nz, 2.f * scale, gW, grad_c ? Zt : nullptr, n_zern,
          zpart);
    }
  }
  if (target && loss)
    k_loss_group<<<n_pupils, 256, 0, s>>>(ops.loss_part, nz * tiles2 * 4, loss);
  if (grad_c && n_zern > 0)
    k_zernike_parts_fin<<<n_zern * n_pupils, 256, 0, s>>>(zpart, n_zern, n_pupils,
                                                          (N * N + 31) / 32, grad_c);
  return cudaPeekAtLastError() == cudaSuccess ? PSF_OK : PSF_ERR_CUDA;
}

// ==========================================================================
// Bessel radial contraction on the split-precision path
// ==========================================================================
namespace tc {

// B[(n, i)][j] = S_B w_j g_n(theta_j) J_n(k r_i sin theta_j) (Eq. 11), FP64,
// columns j >= n_theta zero.  row_pitch rows per order (rows i >= N_r zero);
// with complex weights (Fresnel) g_n stays out of this operand (with_g 0)
// and rides on the per-order F operand instead.
__global__ void k_bessel_jmat_split(BesselParams p, ThetaTable t, double sB,
                                    int bf16, int Kp, int row_pitch, int with_g,
                                    uint16_t* hi, uint16_t* lo) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int rows = 3 * row_pitch;
  if (idx >= (long long)rows * Kp) return;
  const int row = (int)(idx / Kp), j = (int)(idx - (long long)row * Kp);
  double v = 0.0;
  const int n = row / row_pitch, i = row - n * row_pitch;
  if (j < p.n_theta && i < p.n_r) {
    const double st = t.sin_t[j];
    const double x = p.k * (i * p.dr) * st;
    double jn_v;
    if (n == 0) {
      jn_v = j0(x);
    } else if (n == 1) {
      jn_v = j1(x);
    } else {
      jn_v = x > 0.0 ? jn(2, x) : 0.0;   // J_2(0) = 0
    }
    v = sB * t.w[j] * (with_g ? t.g[(2 * n) * p.n_theta + j] : 1.0) * jn_v;
  }
  uint16_t h, l;
  split16d(v, bf16, h, l);
  hi[idx] = h;
  lo[idx] = l;
}

// F rows (s, re) and (s, im): S_F amp e^{2 pi i (wfr + n_i z_s cos / lambda)};
// S_F is the power of two that keeps the largest |F0| (times g_max) below
// 2^14.  With complex weights (n_ord 3) the operand holds one plane of rows
// per order, g_n(theta_j) F: rows (n, s, re/im).  Block (64, 4): one slice
// per threadIdx.y, each thread four consecutive theta nodes (Kp is a
// multiple of 8), stored as 8-byte packs of four 16-bit values per row.
constexpr int FG_TX = 64, FG_TY = 4;

__global__ void __launch_bounds__(FG_TX * FG_TY)
k_bessel_fgen_split(BesselParams p, ThetaTable t, EmitterTable et,
                    const int* __restrict__ slice_em, const float2* __restrict__ zz,
                    const unsigned* __restrict__ amp_max, int Kp, int bf16, float sB,
                    int n_ord, float g_max, uint16_t* hi, uint16_t* lo, float* out_scale) {
  const float am = __uint_as_float(*amp_max) * g_max;
  const float sF = am > 0.f ? exp2f(floorf(log2f(16384.f / am))) : 1.f;
  if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) *out_scale = 1.f / (sB * sF);
  const int s = blockIdx.x * FG_TY + threadIdx.y;
  if (s >= p.n_slices) return;
  const int e = slice_em[s];
  const float2 z = zz[s];
  const size_t plane_rows = 2 * (size_t)p.n_slices;
  for (int q = threadIdx.x; q < (Kp >> 2); q += FG_TX) {
    float2 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = 4 * q + u;
      v[u] = make_float2(0.f, 0.f);
      if (j < p.n_theta && e >= 0) {
        const size_t ej = (size_t)e * p.n_theta + j;
        const float2 c =
            cis_cycles(frac_mul_add(f2x{t.kh[j], t.kl[j]}, f2x{z.x, z.y}, et.wfr[ej]));
        const float a = sF * et.amp[ej];
        v[u] = make_float2(a * c.x, a * c.y);
      }
    }
    for (int n = 0; n < n_ord; ++n) {
      float2 w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = 4 * q + u;
        w[u] = v[u];
        if (n_ord > 1 && j < p.n_theta) {
          const float2 g = make_float2((float)t.g[(2 * n) * p.n_theta + j],
                                       (float)t.g[(2 * n + 1) * p.n_theta + j]);
          w[u] = cmul(g, w[u]);
        }
      }
      // packed pairs of consecutive nodes: node 4q + u in the low half
      uint32_t hr0, lr0, hr1, lr1, hm0, lm0, hm1, lm1;
      split2(w[0].x, w[1].x, bf16, hr0, lr0);
      split2(w[2].x, w[3].x, bf16, hr1, lr1);
      split2(w[0].y, w[1].y, bf16, hm0, lm0);
      split2(w[2].y, w[3].y, bf16, hm1, lm1);
      const size_t r0 = ((size_t)n * plane_rows + 2 * (size_t)s) * Kp + 4 * q, r1 = r0 + Kp;
      *reinterpret_cast<uint2*>(hi + r0) = make_uint2(hr0, hr1);
      *reinterpret_cast<uint2*>(lo + r0) = make_uint2(lr0, lr1);
      *reinterpret_cast<uint2*>(hi + r1) = make_uint2(hm0, hm1);
      *reinterpret_cast<uint2*>(lo + r1) = make_uint2(lm0, lm1);
    }
  }
}

// Adjoint operand: A[j][row] = Bt[j][row] (FP32 J_n operand, theta-major)
// split into BF16 hi + lo with row pitch kp (columns >= rows zero); thread 0
// also stores the unit output scale of the contraction.  With the complex
// operand BtC (Fresnel weights) the rows interleave A[2j] = Re BtC[j] and
// A[2j + 1] = Im BtC[j].
__global__ void k_bessel_adj_bt_split(const float* __restrict__ Bt,
                                      const float2* __restrict__ BtC, int n_theta, int rows,
                                      int kp, uint16_t* hi, uint16_t* lo, float* scale) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx == 0) *scale = 1.f;
  const int a_rows = BtC ? 2 * n_theta : n_theta;
  if (idx >= (long long)a_rows * kp) return;
  const int ar = (int)(idx / kp), q = (int)(idx - (long long)ar * kp);
  float v = 0.f;
  if (q < rows) {
    if (BtC) {
      const float2 b = BtC[(size_t)(ar >> 1) * rows + q];
      v = (ar & 1) ? b.y : b.x;
    } else {
      v = Bt[(size_t)ar * rows + q];
    }
  }
  uint16_t h, l;
  split16(v, 1, h, l);
  hi[idx] = h;
  lo[idx] = l;
}

}  // namespace tc

int tc_bessel_kp(int n_theta) { return (n_theta + 7) / 8 * 8; }

void tc_bessel_adj_carve(char* base, size_t* off, int n_theta, int n_r, int n_slices,
                         bool complex_g, TcBesselAdj* out) {
  auto take = [&](size_t bytes) -> char* {
    *off = align_up(*off, 1024);
    char* p = base ? base + *off : nullptr;
    *off += bytes;
    return p;
  };
  out->kp = tc_bessel_kp(3 * n_r);
  const size_t kp = out->kp;
  const size_t a_rows = (complex_g ? 2 : 1) * (size_t)n_theta;
  out->A_hi = (uint16_t*)take(a_rows * kp * 2);
  out->A_lo = (uint16_t*)take(a_rows * kp * 2);
  out->G_hi = (uint16_t*)take(2 * (size_t)n_slices * kp * 2 + 2);
  out->G_lo = (uint16_t*)take(2 * (size_t)n_slices * kp * 2 + 2);
  out->scale = (float*)take(sizeof(float));
}

int tc_bessel_adj_contract(const BesselParams& p, const float* Bt, const float2* BtC,
                           const TcBesselAdj& ops, float2* gF, int* status, cudaStream_t s) {
  using namespace tc;
  const int rows = 3 * p.n_r, kp = ops.kp;
  const int a_rows = BtC ? 2 * p.n_theta : p.n_theta;
  {
    const long long n = (long long)a_rows * kp;
    k_bessel_adj_bt_split<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        Bt, BtC, p.n_theta, rows, kp, ops.A_hi, ops.A_lo, ops.scale);
  }
  // K extent = 3 N_r (columns past it read as zero), row pitch kp
  auto map2 = [&](CUtensorMap* m, const uint16_t* base, int nrows, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)nrows};
    cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, (void*)base, dims, strides, box,
              es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              SWZ == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  CUtensorMap mAh, mAl, mGh, mGl;
  if (!(map2(&mAh, ops.A_hi, a_rows, BM) && map2(&mAl, ops.A_lo, a_rows, BM) &&
        map2(&mGh, ops.G_hi, 2 * p.n_slices, BN) && map2(&mGl, ops.G_lo, 2 * p.n_slices, BN)))
    return PSF_ERR_CUDA;
  Params q;
  memset(&q, 0, sizeof(q));
  q.planes = 1;
  q.m_tiles = ceil_div(a_rows, BM);
  q.n_tiles = ceil_div(2 * p.n_slices, BN);
  q.k_chunks = ceil_div(rows, BK);
  q.idesc = make_idesc(1);
  q.mode = 2;
  q.bf16 = 1;
  q.prof = gF;                 // gF[s][j]: "rows" of this contraction are theta nodes
  q.rows_total = p.n_theta;
  q.conj_pairs = BtC ? 1 : 0;  // rows (j, Re / Im of the complex operand)
  q.n_slices = p.n_slices;
  q.scale_ptr = ops.scale;
  q.m_fastest = 1;
  q.status = status;
  return launch_gemm(mAh, mAl, mGh, mGl, q, s);
}

void tc_bessel_carve(char* base, size_t* off, int n_theta, int n_r, int n_slices,
                     bool complex_g, TcBessel* out) {
  auto take = [&](size_t bytes) -> char* {
    *off = align_up(*off, 1024);
    char* p = base ? base + *off : nullptr;
    *off += bytes;
    return p;
  };
  const size_t Kp = tc_bessel_kp(n_theta);
  // complex weights: J_n planes of n_r_pad rows, F planes per order
  const size_t b_rows = 3 * (size_t)(complex_g ? tc_harm_n_r_pad(n_r) : n_r);
  const size_t f_rows = (complex_g ? 3 : 1) * 2 * (size_t)n_slices;
  out->B_hi = (uint16_t*)take(b_rows * Kp * 2);
  out->B_lo = (uint16_t*)take(b_rows * Kp * 2);
  out->F_hi = (uint16_t*)take(f_rows * Kp * 2 + 2);
  out->F_lo = (uint16_t*)take(f_rows * Kp * 2 + 2);
  out->need = complex_g ? (unsigned char*)take(3 * (size_t)ceil_div(2 * n_slices, tc::BN) + 1)
                        : nullptr;
  out->amp_max = (unsigned*)take(sizeof(unsigned));
  out->out_scale = (float*)take(sizeof(float));
}

static float bessel_sB(const BesselParams& p, double max_w) {
  // |B| <= max_j w_j * |g_n| (<= 2 for the real weights) * |J_n| (<= 1);
  // complex weights leave B = w_j J_n
  return pow2_scale((p.complex_g ? 1.0 : 2.0) * max_w, 16384.0);
}

void tc_bessel_jmat(const BesselParams& p, ThetaTable t, double max_w,
                    int precision, const TcBessel& ops, cudaStream_t s) {
  const int Kp = tc_bessel_kp(p.n_theta);
  const int pitch = p.complex_g ? tc_harm_n_r_pad(p.n_r) : p.n_r;
  const long long n = 3LL * pitch * Kp;
  tc::k_bessel_jmat_split<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
      p, t, (double)bessel_sB(p, max_w), precision == PSF_PREC_SPLIT_BF16 ? 1 : 0, Kp,
      pitch, p.complex_g ? 0 : 1, ops.B_hi, ops.B_lo);
}

int tc_bessel_contract(const BesselParams& p, ThetaTable t, EmitterTable et,
                       const int* slice_em, const float2* zz, double max_w, double g_max,
                       int precision, const TcBessel& ops, float2* prof,
                       int* status, cudaStream_t s) {
  using namespace tc;
  const int bf16 = precision == PSF_PREC_SPLIT_BF16 ? 1 : 0;
  const int Kp = tc_bessel_kp(p.n_theta);
  const float sB = bessel_sB(p, max_w);
  const int n_ord = p.complex_g ? 3 : 1;
  {
    TimingScope ts(kTimeSetup, s);
    const unsigned nb = (unsigned)(p.n_slices > 0 ? ceil_div(p.n_slices, FG_TY) : 1);
    k_bessel_fgen_split<<<nb, dim3(FG_TX, FG_TY), 0, s>>>(
        p, t, et, slice_em, zz, ops.amp_max, Kp, bf16, sB, n_ord,
        p.complex_g ? (float)g_max : 1.f, ops.F_hi, ops.F_lo, ops.out_scale);
  }
  // K extent = n_theta (columns past it read as zero), row pitch Kp
  auto map2 = [&](CUtensorMap* m, const uint16_t* base, int rows, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)p.n_theta, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, (void*)base, dims, strides, box,
              es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              SWZ == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  CUtensorMap mBh, mBl, mFh, mFl;
  const int rows = 3 * p.n_r;
  if (p.complex_g) {
    // complex weights: per order n a tile grid over (radius, slice column)
    // with A = S_B w_j J_n (plane n of n_r_pad rows) and B = S_F g_n F
    // (plane n of 2 n_slices rows) -- the per-order contraction of the
    // harmonic path with orders 0..2
    const int n_r_pad = tc_harm_n_r_pad(p.n_r);
    const int n_tiles = ceil_div(2 * p.n_slices, BN);
    if (!(map2(&mBh, ops.B_hi, 3 * n_r_pad, BM) && map2(&mBl, ops.B_lo, 3 * n_r_pad, BM) &&
          map2(&mFh, ops.F_hi, 6 * p.n_slices, BN) && map2(&mFl, ops.F_lo, 6 * p.n_slices, BN)))
      return PSF_ERR_CUDA;
    cudaMemsetAsync(ops.need, 1, 3 * (size_t)n_tiles, s);
    Params q;
    memset(&q, 0, sizeof(q));
    q.planes = 3;
    q.m_tiles = n_r_pad / BM;
    q.n_tiles = n_tiles;
    q.k_chunks = ceil_div(p.n_theta, BK);
    q.idesc = make_idesc(bf16);
    q.mode = 5;
    q.bf16 = bf16;
    q.prof = prof;
    q.rows_total = p.n_r;
    q.n_slices = p.n_slices;
    q.scale_ptr = ops.out_scale;
    q.m_fastest = 1;
    q.status = status;
    q.need = ops.need;
    q.n_ord = 3;
    q.hL = 0;
    q.n_r_pad = n_r_pad;
    q.b_rows_per_plane = 2 * p.n_slices;
    TimingScope ts(kTimeBesselRadial, s);
    return launch_gemm(mBh, mBl, mFh, mFl, q, s);
  }
  if (!(map2(&mBh, ops.B_hi, rows, BM) && map2(&mBl, ops.B_lo, rows, BM) &&
        map2(&mFh, ops.F_hi, 2 * p.n_slices, BN) && map2(&mFl, ops.F_lo, 2 * p.n_slices, BN)))
    return PSF_ERR_CUDA;
  Params q;
  memset(&q, 0, sizeof(q));
  q.planes = 1;
  q.m_tiles = ceil_div(rows, BM);
  q.n_tiles = ceil_div(2 * p.n_slices, BN);
  q.k_chunks = ceil_div(p.n_theta, BK);
  q.idesc = make_idesc(bf16);
  q.mode = 2;
  q.bf16 = bf16;
  q.prof = prof;
  q.rows_total = rows;
  q.n_slices = p.n_slices;
  q.scale_ptr = ops.out_scale;
  q.m_fastest = 1;
  q.status = status;
  TimingScope ts(kTimeBesselRadial, s);
  return launch_gemm(mBh, mBl, mFh, mFl, q, s);
}

// ---------------------------------------------------------------------------
// Harmonic radial contraction (mode 5): per order l' a tile grid over
// (radius, column) with A = S_A w_j J_|l|(k r_i sin theta_j) and
// B = S_F D[s][j] Bh[e][c][l'][j], split hi + lo; K = theta.
// ---------------------------------------------------------------------------
int tc_harm_cols_per_tile() { return tc::BN / 2; }

int tc_harm_n_r_pad(int n_r) { return ceil_div(n_r, tc::BM) * tc::BM; }

void tc_harm_carve(char* base, size_t* off, int n_theta, int n_r, int m_max, int chunk,
                   TcHarm* out) {
  using namespace tc;
  auto take = [&](size_t bytes) -> char* {
    *off = align_up(*off, 1024);
    char* p = base ? base + *off : nullptr;
    *off += bytes;
    return p;
  };
  out->kp = tc_bessel_kp(n_theta);
  out->n_r_pad = tc_harm_n_r_pad(n_r);
  const size_t kp = out->kp, n_ord = 2 * (size_t)m_max + 5;
  const size_t a_rows = (size_t)(m_max + 3) * out->n_r_pad;
  const size_t b_rows = n_ord * 6 * (size_t)chunk;
  out->a_bytes = a_rows * kp * 2;
  out->A_hi = (uint16_t*)take(out->a_bytes);
  out->A_lo = (uint16_t*)take(out->a_bytes);
  out->B_hi = (uint16_t*)take(b_rows * kp * 2);
  out->B_lo = (uint16_t*)take(b_rows * kp * 2);
  const size_t tiles = (size_t)ceil_div(6 * chunk, BN);
  out->need = (unsigned char*)take(n_ord * tiles);
  out->bh_max = (unsigned*)take(sizeof(unsigned));
  out->out_scale = (float*)take(sizeof(float));
}

float tc_harm_scale_a(double max_w) { return pow2_scale(max_w, 16384.0); }

int tc_harm_contract(const TcHarm& ops, int n_theta, int n_r, int m_max, int n_cols,
                     int precision, float2* prof, int* status, cudaStream_t s) {
  using namespace tc;
  const int bf16 = precision == PSF_PREC_SPLIT_BF16 ? 1 : 0;
  const int n_ord = 2 * m_max + 5;
  auto map2 = [&](CUtensorMap* m, const uint16_t* base, long long rows, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)n_theta, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ops.kp * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, (void*)base, dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE,
              SWZ == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  CUtensorMap mAh, mAl, mBh, mBl;
  const long long a_rows = (long long)(m_max + 3) * ops.n_r_pad;
  const long long b_rows = (long long)n_ord * 2 * n_cols;
  if (!(map2(&mAh, ops.A_hi, a_rows, BM) && map2(&mAl, ops.A_lo, a_rows, BM) &&
        map2(&mBh, ops.B_hi, b_rows, BN) && map2(&mBl, ops.B_lo, b_rows, BN)))
    return PSF_ERR_CUDA;
  Params q;
  memset(&q, 0, sizeof(q));
  q.planes = n_ord;
  q.m_tiles = ops.n_r_pad / BM;
  q.n_tiles = ceil_div(2 * n_cols, BN);
  q.k_chunks = ceil_div(n_theta, BK);
  q.idesc = make_idesc(bf16);
  q.mode = 5;
  q.bf16 = bf16;
  q.prof = prof;
  q.rows_total = n_r;
  q.n_slices = n_cols;
  q.scale_ptr = ops.out_scale;
  q.m_fastest = 1;
  q.status = status;
  q.need = ops.need;
  q.n_ord = n_ord;
  q.hL = m_max + 2;
  q.n_r_pad = ops.n_r_pad;
  q.b_rows_per_plane = 2 * n_cols;
  return launch_gemm(mAh, mAl, mBh, mBl, q, s);
}

}  // namespace psf
