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
#include <string.h>

#include "tc_kernels.cuh"
#include "tc_ptx.cuh"
#include "timing.cuh"

namespace psf {
namespace tc {

constexpr int BM = 128;             // A rows per tile (64 outputs x re/im)
constexpr int BN = 192;             // B rows per tile (3 channels x 64)
constexpr int BOUT = 64;            // outputs per tile along m and per channel along n
// Measured on GB300 (256^2 pupil, 512^2 px, 128 planes): BK 64 / 2 stages
// 1.009 ms per stack, BK 32 / 4 stages 1.022 ms, BK 32 / 5 stages 1.031 ms:
// the ring depth is not the limit (operand delivery is, see the design notes).
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
  const float* scale_ptr;   // device scalar: 1 / (S_B S_F)
  int m_fastest;        // tile order: consecutive tiles share the B tile
};

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
      for (int kc = 0; kc < p.k_chunks; ++kc) {
        if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, p.status)) {
          ok = false;
          break;
        }
        const uint32_t base = smem_u32(smem + stage * STAGE_BYTES);
        mbar_arrive_expect_tx(full_bar(stage), STAGE_BYTES);
        tma_load_2d(base, &mapA_hi, kc * BK, mt * BM, full_bar(stage));
        tma_load_2d(base + A_BYTES, &mapA_lo, kc * BK, mt * BM, full_bar(stage));
        if (p.mode == 2) {
          tma_load_2d(base + 2 * A_BYTES, &mapB_hi, kc * BK, nt * BN, full_bar(stage));
          tma_load_2d(base + 2 * A_BYTES + B_BYTES, &mapB_lo, kc * BK, nt * BN,
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
    for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
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
    mma_commit(drain_bar);
    mbar_drain_wait(drain_bar, 0);
  } else if (warp >= 2) {
    // ------------------------------ epilogue ----------------------------------
    const int quad = warp & 3;                 // TMEM lanes 32*quad .. +31
    const int row = quad * 32 + lane;          // accumulator row = A row
    const int oi = row >> 1, part = row & 1;   // output index within tile, re/im
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
      int okw = 1;
      if (lane == 0) okw = mbar_wait(tfull_bar(acc), acc_phase, abort_flag, p.status) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) break;
      tmem_fence_after();
      int plane, mt, nt;
      decode_tile(p, t, plane, mt, nt);
      const uint32_t tbase = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * ACC_COL);
      const int mo = mt * BOUT + oi;           // output index along m
      if (p.mode == 2) {
        // Bessel: prof[s][row] = scale * (D[row][2k], D[row][2k+1]), s = nt*96 + k
        const int grow = mt * BM + row;
        const float sc = *p.scale_ptr;
        for (int h = 0; h < BN / 32; ++h) {
          uint32_t r[32];
          tmem_ld32(tbase + (uint32_t)(h * 32), r);
          if (grow < p.rows_total) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const int s = nt * (BN / 2) + h * 16 + k;
              if (s < p.n_slices)
                p.prof[(size_t)s * p.rows_total + grow] =
                    make_float2(sc * __uint_as_float(r[2 * k]), sc * __uint_as_float(r[2 * k + 1]));
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
            if (!row_ok || p0 >= p.n_rows) continue;
            const size_t off = ((size_t)(plane * 3 + c) * p.m_out + mo) * (size_t)(2 * p.N) +
                               (size_t)part * p.N + p0;
            uint32_t hw[16], lw[16];
#pragma unroll
            for (int j = 0; j < 32; j += 2) {
              uint16_t h0, l0, h1, l1;
              split16(p.out_scale * __uint_as_float(r[j]), p.bf16, h0, l0);
              split16(p.out_scale * __uint_as_float(r[j + 1]), p.bf16, h1, l1);
              hw[j / 2] = (uint32_t)h0 | ((uint32_t)h1 << 16);
              lw[j / 2] = (uint32_t)l0 | ((uint32_t)l1 << 16);
            }
            if (p0 + 32 <= p.n_rows) {
              uint4* dh = (uint4*)(p.U_hi + off);
              uint4* dl = (uint4*)(p.U_lo + off);
#pragma unroll
              for (int v = 0; v < 4; ++v) {
                dh[v] = make_uint4(hw[4 * v], hw[4 * v + 1], hw[4 * v + 2], hw[4 * v + 3]);
                dl[v] = make_uint4(lw[4 * v], lw[4 * v + 1], lw[4 * v + 2], lw[4 * v + 3]);
              }
            } else {
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

// Pupil fields of a z-chunk as split operand rows: P[zc][c][p][q] -> row
// (zc, c, p), columns [Re q | Im q], scaled by S_P.  Four consecutive nodes
// (same p, N % 4 == 0) per thread and one plane per grid row, 8-byte stores.
__global__ void k_pupil_z_split(NodeTable t, int N, const float2* __restrict__ zz,
                                int z0, int nzc, float sP, int bf16,
                                uint16_t* __restrict__ hi, uint16_t* __restrict__ lo) {
  const int NN = N * N;
  const int idx4 = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx4 * 4 >= NN) return;
  const int idx = idx4 * 4;
  const int ip = idx / N, iq = idx - (idx / N) * N;
  float4 a4[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) a4[c] = *(const float4*)(t.amp + (size_t)c * NN + idx);
  const float4 w4 = *(const float4*)(t.wfr + idx);
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
    const float2 z = zz[z0 + zc];
    float2 e[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
      e[k] = cis_cycles(frac_mul_add(f2x{khv[k], klv[k]}, f2x{z.x, z.y}, wv[k]));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      uint16_t hr[4], lr[4], hm[4], lm[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 v = cmul(amp[c][k], e[k]);
        split16(v.x, bf16, hr[k], lr[k]);
        split16(v.y, bf16, hm[k], lm[k]);
      }
      const size_t row = ((size_t)(zc * 3 + c) * N + ip) * (size_t)(2 * N);
      auto pack = [](const uint16_t* s) {
        return make_uint2((uint32_t)s[0] | ((uint32_t)s[1] << 16),
                          (uint32_t)s[2] | ((uint32_t)s[3] << 16));
      };
      *(uint2*)(hi + row + iq) = pack(hr);
      *(uint2*)(lo + row + iq) = pack(lr);
      *(uint2*)(hi + row + N + iq) = pack(hm);
      *(uint2*)(lo + row + N + iq) = pack(lm);
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
  (void)nx;
  // P (hi+lo) + U (hi+lo) per plane, keep the chunk near 64 MB
  const double per_z = 3.0 * 2.0 * 2.0 * 2.0 * N * ((double)N + ny);
  int zc = (int)(64.0 * 1048576.0 / per_z);
  if (zc < 1) zc = 1;
  if (zc > 64) zc = 64;
  if (zc > nz) zc = nz;
  return zc;
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
  return 1.05 * best * (pol > 0 ? pol : 1.0);
}

static float pow2_scale(double bound, double target) {
  // largest power of two S with bound * S <= target
  if (!(bound > 0)) return 1.0f;
  return (float)exp2(floor(log2(target / bound)));
}

int tc_fourier_forward(const TcOperands& ops, NodeTable nodes, const float2* zz,
                       int N, int nx, int ny, double dx, double dy, int nz,
                       int zc, double na_over_lambda, float scale,
                       double amp_bound, int precision, float* intensity,
                       float2* fields, int* status, cudaStream_t s) {
  using namespace tc;
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
  const uint32_t idesc = make_idesc(bf16);
  for (int z0 = 0; z0 < nz; z0 += zc) {
    const int nzc = nz - z0 < zc ? nz - z0 : zc;
    {
      TimingScope ts(kTimePupil, s);
      const dim3 pg(ceil_div(N * N / 4, 128), nzc);
      k_pupil_z_split<<<pg, 128, 0, s>>>(nodes, N, zz, z0, nzc, sP, bf16, ops.P_hi,
                                         ops.P_lo);
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
    p1.U_hi = ops.U_hi;
    p1.U_lo = ops.U_lo;
    p1.nx = nx;
    p1.ny = ny;
    p1.status = status;
    int r;
    {
      TimingScope ts(kTimeStage1, s);
      r = launch_gemm(mAy_h, mAy_l, mP_h, mP_l, p1, s);
    }
    if (r) return r;
    Params p2 = p1;
    p2.m_tiles = ceil_div(nx, BOUT);
    p2.n_tiles = ceil_div(ny, BOUT);
    p2.m_out = nx;
    p2.n_rows = ny;
    p2.mode = 1;
    p2.out_scale = scale / (sA * sU);
    p2.I = intensity + (size_t)z0 * nx * ny;
    p2.F = fields ? fields + (size_t)z0 * 3 * nx * ny : nullptr;
    {
      TimingScope ts(kTimeStage2, s);
      r = launch_gemm(mAx_h, mAx_l, mU_h, mU_l, p2, s);
    }
    if (r) return r;
  }
  return PSF_OK;
}

// ==========================================================================
// Bessel radial contraction on the split-precision path
// ==========================================================================
namespace tc {

PSF_D void split16d(double v, int bf16, uint16_t& hi, uint16_t& lo) {
  if (bf16) {
    const __nv_bfloat16 h = __double2bfloat16(v);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(__double2bfloat16(v - (double)__bfloat162float(h)));
  } else {
    const __half h = __double2half(v);
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(__double2half(v - (double)__half2float(h)));
  }
}

// B[(n, i)][j] = S_B w_j g_n(theta_j) J_n(k r_i sin theta_j) (Eq. 11), FP64,
// columns j >= n_theta zero.
__global__ void k_bessel_jmat_split(BesselParams p, ThetaTable t, double sB,
                                    int bf16, int Kp, uint16_t* hi, uint16_t* lo) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int rows = 3 * p.n_r;
  if (idx >= (long long)rows * Kp) return;
  const int row = (int)(idx / Kp), j = (int)(idx - (long long)row * Kp);
  double v = 0.0;
  if (j < p.n_theta) {
    const int n = row / p.n_r, i = row - n * p.n_r;
    const double st = t.sin_t[j], ct = t.cos_t[j];
    const double x = p.k * (i * p.dr) * st;
    double jn_v, g;
    if (n == 0) {
      jn_v = j0(x);
      g = st * (1.0 + ct);
    } else if (n == 1) {
      jn_v = j1(x);
      g = st * st;
    } else {
      jn_v = x > 0.0 ? jn(2, x) : 0.0;   // J_2(0) = 0
      g = st * (ct - 1.0);
    }
    v = sB * t.w[j] * g * jn_v;
  }
  uint16_t h, l;
  split16d(v, bf16, h, l);
  hi[idx] = h;
  lo[idx] = l;
}

// F rows (s, re) and (s, im): S_F amp e^{2 pi i (wfr + n_i z_s cos / lambda)};
// S_F is the power of two that keeps the largest |F0| below 2^14.
__global__ void k_bessel_fgen_split(BesselParams p, ThetaTable t, EmitterTable et,
                                    const int* __restrict__ slice_em,
                                    const float2* __restrict__ zz,
                                    const unsigned* __restrict__ amp_max, int Kp,
                                    int bf16, float sB, uint16_t* hi, uint16_t* lo,
                                    float* out_scale) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= (long long)p.n_slices * Kp) return;
  const float am = __uint_as_float(*amp_max);
  const float sF = am > 0.f ? exp2f(floorf(log2f(16384.f / am))) : 1.f;
  if (idx == 0) *out_scale = 1.f / (sB * sF);
  const int s = (int)(idx / Kp), j = (int)(idx - (long long)s * Kp);
  const int e = slice_em[s];
  float2 v = make_float2(0.f, 0.f);
  if (j < p.n_theta && e >= 0) {
    const size_t ej = (size_t)e * p.n_theta + j;
    const float2 z = zz[s];
    const float2 c = cis_cycles(frac_mul_add(f2x{t.kh[j], t.kl[j]}, f2x{z.x, z.y}, et.wfr[ej]));
    const float a = sF * et.amp[ej];
    v = make_float2(a * c.x, a * c.y);
  }
  const size_t r0 = (size_t)(2 * s) * Kp + j, r1 = r0 + Kp;
  uint16_t h, l;
  split16(v.x, bf16, h, l);
  hi[r0] = h;
  lo[r0] = l;
  split16(v.y, bf16, h, l);
  hi[r1] = h;
  lo[r1] = l;
}

// Adjoint operand: A[j][row] = Bt[j][row] (FP32 J_n operand, theta-major)
// split into BF16 hi + lo with row pitch kp (columns >= rows zero); thread 0
// also stores the unit output scale of the contraction.
__global__ void k_bessel_adj_bt_split(const float* __restrict__ Bt, int n_theta, int rows,
                                      int kp, uint16_t* hi, uint16_t* lo, float* scale) {
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx == 0) *scale = 1.f;
  if (idx >= (long long)n_theta * kp) return;
  const int j = (int)(idx / kp), q = (int)(idx - (long long)j * kp);
  const float v = q < rows ? Bt[(size_t)j * rows + q] : 0.f;
  uint16_t h, l;
  split16(v, 1, h, l);
  hi[idx] = h;
  lo[idx] = l;
}

}  // namespace tc

int tc_bessel_kp(int n_theta) { return (n_theta + 7) / 8 * 8; }

void tc_bessel_adj_carve(char* base, size_t* off, int n_theta, int n_r, int n_slices,
                         TcBesselAdj* out) {
  auto take = [&](size_t bytes) -> char* {
    *off = align_up(*off, 1024);
    char* p = base ? base + *off : nullptr;
    *off += bytes;
    return p;
  };
  out->kp = tc_bessel_kp(3 * n_r);
  const size_t kp = out->kp;
  out->A_hi = (uint16_t*)take((size_t)n_theta * kp * 2);
  out->A_lo = (uint16_t*)take((size_t)n_theta * kp * 2);
  out->G_hi = (uint16_t*)take(2 * (size_t)n_slices * kp * 2 + 2);
  out->G_lo = (uint16_t*)take(2 * (size_t)n_slices * kp * 2 + 2);
  out->scale = (float*)take(sizeof(float));
}

int tc_bessel_adj_contract(const BesselParams& p, const float* Bt, const TcBesselAdj& ops,
                           float2* gF, int* status, cudaStream_t s) {
  using namespace tc;
  const int rows = 3 * p.n_r, kp = ops.kp;
  {
    const long long n = (long long)p.n_theta * kp;
    k_bessel_adj_bt_split<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        Bt, p.n_theta, rows, kp, ops.A_hi, ops.A_lo, ops.scale);
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
  if (!(map2(&mAh, ops.A_hi, p.n_theta, BM) && map2(&mAl, ops.A_lo, p.n_theta, BM) &&
        map2(&mGh, ops.G_hi, 2 * p.n_slices, BN) && map2(&mGl, ops.G_lo, 2 * p.n_slices, BN)))
    return PSF_ERR_CUDA;
  Params q;
  memset(&q, 0, sizeof(q));
  q.planes = 1;
  q.m_tiles = ceil_div(p.n_theta, BM);
  q.n_tiles = ceil_div(2 * p.n_slices, BN);
  q.k_chunks = ceil_div(rows, BK);
  q.idesc = make_idesc(1);
  q.mode = 2;
  q.bf16 = 1;
  q.prof = gF;                 // gF[s][j]: "rows" of this contraction are theta nodes
  q.rows_total = p.n_theta;
  q.n_slices = p.n_slices;
  q.scale_ptr = ops.scale;
  q.m_fastest = 1;
  q.status = status;
  return launch_gemm(mAh, mAl, mGh, mGl, q, s);
}

void tc_bessel_carve(char* base, size_t* off, int n_theta, int n_r, int n_slices,
                     TcBessel* out) {
  auto take = [&](size_t bytes) -> char* {
    *off = align_up(*off, 1024);
    char* p = base ? base + *off : nullptr;
    *off += bytes;
    return p;
  };
  const size_t Kp = tc_bessel_kp(n_theta);
  out->B_hi = (uint16_t*)take(3 * (size_t)n_r * Kp * 2);
  out->B_lo = (uint16_t*)take(3 * (size_t)n_r * Kp * 2);
  out->F_hi = (uint16_t*)take(2 * (size_t)n_slices * Kp * 2 + 2);
  out->F_lo = (uint16_t*)take(2 * (size_t)n_slices * Kp * 2 + 2);
  out->amp_max = (unsigned*)take(sizeof(unsigned));
  out->out_scale = (float*)take(sizeof(float));
}

static float bessel_sB(double max_w) {
  // |B| <= max_j w_j * |g_n| (<= 2) * |J_n| (<= 1)
  return pow2_scale(2.0 * max_w, 16384.0);
}

void tc_bessel_jmat(const BesselParams& p, ThetaTable t, double max_w,
                    int precision, const TcBessel& ops, cudaStream_t s) {
  const int Kp = tc_bessel_kp(p.n_theta);
  const long long n = 3LL * p.n_r * Kp;
  tc::k_bessel_jmat_split<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
      p, t, (double)bessel_sB(max_w), precision == PSF_PREC_SPLIT_BF16 ? 1 : 0, Kp,
      ops.B_hi, ops.B_lo);
}

int tc_bessel_contract(const BesselParams& p, ThetaTable t, EmitterTable et,
                       const int* slice_em, const float2* zz, double max_w,
                       int precision, const TcBessel& ops, float2* prof,
                       int* status, cudaStream_t s) {
  using namespace tc;
  const int bf16 = precision == PSF_PREC_SPLIT_BF16 ? 1 : 0;
  const int Kp = tc_bessel_kp(p.n_theta);
  const float sB = bessel_sB(max_w);
  {
    TimingScope ts(kTimeSetup, s);
    const long long n = (long long)p.n_slices * Kp;
    k_bessel_fgen_split<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        p, t, et, slice_em, zz, ops.amp_max, Kp, bf16, sB, ops.F_hi, ops.F_lo,
        ops.out_scale);
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

}  // namespace psf
