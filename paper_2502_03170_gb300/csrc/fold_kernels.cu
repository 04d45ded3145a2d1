// Symmetry-folded tcgen05 contractions of the Fourier forward (Eq. 8).
//
// The pupil nodes u_p = (2p+1-N)/N and the output pixels x_a = (a-(n-1)/2) dx
// are both symmetric about zero, so with the mirror indices p~ = N-1-p and
// a~ = n-1-a the zoom matrix obeys
//   A[a][p~] = conj(A[a][p]),   A[a~][p] = conj(A[a][p]).
// Writing A[a][p'] = C + iS for the first half p' < N/2 of the pupil, any
// contraction over p splits into two real contractions over half of K:
//   sum_p A[a][p] X[p] = sum_p' C X+[p'] + i S X-[p'],  X+- = X[p'] +- X[p~'],
// and the mirrored output a~ reuses both sums with the sign of the S term
// flipped.  Each separable stage of Eq. 8 therefore needs a quarter of the
// real multiply-adds of the complex 2x2-block form:
//   stage 1 (over q):  X1 = C_y . P[s+], Y1 = S_y . P[s-]  ->  T[b'], T[b~']
//   stage 2 (over p):  X2 = C_x . T+,    Y2 = S_x . T-     ->  E[a'], E[a~']
// with the pupil combined over both mirrors before stage 1 (four parity
// classes P[s r] = (P[p'][q'] + s P[p'][q~']) + r (P[p~'][q'] + s P[p~'][q~'])),
// so stage 1 directly writes the p-folded T+ (r = +) and T- (r = -) that
// stage 2 contracts.
//
// Kernel: a CTA pair (cta_group::2, M = 256 zoom rows) per tile, as in the
// unfolded contraction, with two operand streams per side: the zoom halves
// C and S (each CTA its 128 rows) and the data halves for X and Y (each CTA
// half the tile's columns), all split hi + lo.  Per 16-wide K step the
// leader issues six MMAs (three split products into each of the X and Y
// accumulators, FP32 in TMEM).  Warp roles, bounded waits and the drain on
// time-out are those of the unfolded pair kernel.
//
// TF32 (template flag): the operand parts are 32-bit TF32 values (x = hi + lo
// rounded with cvt.rna.tf32, or hi alone for single-pass TF32), a 128-byte
// stage row holds 32 K elements, and the leader issues kind::tf32 MMAs of
// K = 8 (three split products, or one product per accumulator in the single
// pass).  Everything else -- layout of the variants, the tiles, the
// epilogues -- is shared with the 16-bit form.
#include <cuda.h>
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
namespace fold {

constexpr int BM = 128;                 // zoom rows per CTA
constexpr int BK = 64;                  // 16-bit K elements per stage (128-byte swizzled rows)
constexpr int SWZ = 128;
constexpr int EPI_WARPS = 8;            // two per TMEM lane quarter
constexpr int NUM_THREADS = 64 + 32 * EPI_WARPS;
constexpr int TMEM_COLS = 512;
constexpr int S1_PB = 64;               // stage 1: p' per tile
constexpr int S2_BOUT = 16;             // stage 2: outputs b per tile
constexpr int S2_HB = S2_BOUT / 2;      // stage 2: outputs b per CTA of the pair
constexpr int A_BYTES = BM * BK * 2;    // one variant of a zoom-half chunk: 16 KB
constexpr int A_CHUNK = 4 * A_BYTES;    // C hi, C lo, S hi, S lo of one K chunk
constexpr int RES_CHUNKS = 2;           // resident zoom halves: K <= 128 (N <= 256)
constexpr int SMEM_LIMIT = 227 * 1024;

// Tile shape of each stage: BN accumulator columns (= data rows of the pair),
// NACC accumulator sets (X and Y) in TMEM.  With RES the CTA's zoom-half rows
// for the whole K range stay in shared memory for the kernel's lifetime and
// the ring carries only the data operand; otherwise every ring stage holds
// one K chunk of both operands.  Each operand's four variants (hi/lo of the
// X and Y sides, or of C and S) are one TMA box.
template <int MODE, bool RES>
struct Shape {
  static constexpr int BN = MODE == 0 ? 2 * S1_PB : 6 * S2_BOUT;   // 128 / 96
  static constexpr int PB_ROWS = BN / 2;                            // data rows per CTA
  static constexpr int PB_BYTES = PB_ROWS * BK * 2;                 // one variant
  static constexpr int A_RES = RES ? RES_CHUNKS * A_CHUNK : 0;
  static constexpr int STAGE_BYTES = (RES ? 0 : A_CHUNK) + 4 * PB_BYTES;
  static constexpr int NACC = (4 * BN <= TMEM_COLS) ? 2 : 1;
  static constexpr int STAGES_FIT = (SMEM_LIMIT - 2048 - A_RES) / STAGE_BYTES;
  static constexpr int STAGES = STAGES_FIT > 6 ? 6 : STAGES_FIT;
  static constexpr int SMEM_BYTES = A_RES + STAGES * STAGE_BYTES + 2048;
  static_assert(STAGES >= 2, "operand ring needs two stages");
};

struct FoldParams {
  int planes, m_pairs, n_tiles, k_chunks;
  int H;                // folded K extent (N / 2)
  int Kp;               // row pitch of every operand (elements, multiple of 16)
  int m_rows;           // folded zoom rows: ceil(n_out / 2)
  int n_out;            // ny (stage 1) or nx (stage 2): mirror index n_out - 1 - i
  int nx, ny;
  int pblk;             // stage 1: p'-blocks of S1_PB per (channel, parity)
  uint32_t idesc;
  int bf16;
  int passes;           // TF32 operands: 3 (hi.hi + lo.hi + hi.lo) or 1 (hi.hi)
  float out_scale;
  uint16_t* U;          // stage 1 output [planes][4][6 ny][Kp]: T+ hi, T+ lo, T- hi, T- lo
                        // (32-bit elements with TF32 operands)
  float* I;             // stage 2: [planes][nx][ny]
  float2* F;            // stage 2: [planes][3][nx][ny] or null
  int* status;
};

// 32 / 16 consecutive TMEM columns of this warp's lanes; the wait is in the
// same asm block, so no use of r[] can be scheduled before the data arrive.
PSF_D void tmem_ld32w(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32"
      " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15,"
      " %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31},"
      " [%32];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
        "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
        "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]),
        "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

PSF_D void tmem_ld16w(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32"
      " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15},"
      " [%16];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
        "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
        "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

// Four 16-column loads (addresses a0..a3) and one wait, in one asm block.
PSF_D void tmem_ld16x4w(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                        uint32_t (&r0)[16], uint32_t (&r1)[16], uint32_t (&r2)[16],
                        uint32_t (&r3)[16]) {
#define PSF_R16(r) "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), \
    "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),  \
    "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32"
      " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%64];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32"
      " {%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31},"
      " [%65];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32"
      " {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47},"
      " [%66];\n"
      "tcgen05.ld.sync.aligned.32x32b.x16.b32"
      " {%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63},"
      " [%67];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : PSF_R16(r0), PSF_R16(r1), PSF_R16(r2), PSF_R16(r3)
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3)
      : "memory");
#undef PSF_R16
}

// One 32-byte sector per lane (8 words, 32-byte aligned address).
PSF_D void st_global_v8(void* ptr, const uint32_t (&w)[8]) {
  asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(ptr),
               "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]),
               "r"(w[7])
               : "memory");
}

PSF_D void decode(const FoldParams& p, int t, int& plane, int& mp, int& nt) {
  const int tpp = p.m_pairs * p.n_tiles;
  plane = t / tpp;
  const int rem = t - plane * tpp;
  nt = rem / p.m_pairs;
  mp = rem - nt * p.m_pairs;
}

// 16 split values of one output row piece: one 32-byte store each for hi
// (at off) and lo (at off + lo_delta); the row pitch is a multiple of 16
// elements and the piece starts at a multiple of 16.  Element-wise where
// the piece runs past the valid K extent.
PSF_D void store_piece16(uint16_t* base, size_t off, size_t lo_delta, const float (&v)[16],
                         int bf16, int n_valid) {
  uint32_t hw[8], lw[8];
#pragma unroll
  for (int j = 0; j < 16; j += 2) split2(v[j], v[j + 1], bf16, hw[j / 2], lw[j / 2]);
  if (n_valid >= 16) {
    st_global_v8(base + off, hw);
    st_global_v8(base + off + lo_delta, lw);
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j < n_valid) {
        base[off + j] = (uint16_t)(hw[j / 2] >> (16 * (j & 1)));
        base[off + lo_delta + j] = (uint16_t)(lw[j / 2] >> (16 * (j & 1)));
      }
    }
  }
}

// The TF32 form of store_piece16: 16 values split into TF32 hi + lo (lo 0
// with one pass), 32-bit elements, two 32-byte stores each for hi and lo.
PSF_D void store_piece32(uint32_t* base, size_t off, size_t lo_delta, const float (&v)[16],
                         int passes, int n_valid) {
  uint32_t h[16], l[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) split_tf32(v[j], passes, h[j], l[j]);
  if (n_valid >= 16) {
    const uint32_t h0[8] = {h[0], h[1], h[2], h[3], h[4], h[5], h[6], h[7]};
    const uint32_t h1[8] = {h[8], h[9], h[10], h[11], h[12], h[13], h[14], h[15]};
    const uint32_t l0[8] = {l[0], l[1], l[2], l[3], l[4], l[5], l[6], l[7]};
    const uint32_t l1[8] = {l[8], l[9], l[10], l[11], l[12], l[13], l[14], l[15]};
    st_global_v8(base + off, h0);
    st_global_v8(base + off + 8, h1);
    st_global_v8(base + off + lo_delta, l0);
    st_global_v8(base + off + lo_delta + 8, l1);
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j < n_valid) {
        base[off + j] = h[j];
        base[off + lo_delta + j] = l[j];
      }
    }
  }
}

template <bool TF32>
PSF_D void store_piece(const FoldParams& p, size_t off, size_t lo_delta, const float (&v)[16],
                       int n_valid) {
  if (TF32)
    store_piece32((uint32_t*)p.U, off, lo_delta, v, p.passes, n_valid);
  else
    store_piece16(p.U, off, lo_delta, v, p.bf16, n_valid);
}

// Releases the accumulator on the leader's barrier once this warp has read
// its columns (before the arithmetic and the stores of the tile).  The
// arrival keeps the default release.cta semantics: a cluster-scope release
// would first wait until the warp's earlier global stores (the previous
// tile's output, often still in flight) are visible cluster-wide, while the
// hand-off orders only the TMEM reads, which tcgen05.wait::ld has completed
// and tcgen05.fence::before_thread_sync orders before the arrival.
PSF_D void release_acc(int lane, uint32_t bar_cluster) {
  tmem_fence_before();
  __syncwarp();
  if (lane == 0)
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}

// ---------------------------------------------------------------------------
// Epilogue of stage 1: tile (plane, channel c, parity r, p'-block); this
// thread's accumulator row is b' (TMEM lane), columns (re/im, 64 p'), of
// which the warp's half of the chunks is read:
//   T^r[p'][b'] = X + i Y,  T^r[p'][b~'] = X - i Y   (X, Y complex)
// written split hi + lo as rows (b, c, re/im) of U^r for b = b' and b~'.
// ---------------------------------------------------------------------------
template <bool TF32>
PSF_D void epilogue_stage1(const FoldParams& p, uint32_t tx, uint32_t ty, int plane, int mt,
                           int nt, int row, int half, int lane, uint32_t release_bar) {
  const int c = nt / (2 * p.pblk);
  const int rem = nt - c * 2 * p.pblk;
  const int par = rem / p.pblk, blk = rem - par * p.pblk;
  const int b = mt * BM + row;
  const bool ok_b = b < p.m_rows;
  const int bm = p.n_out - 1 - b;
  const bool ok_m = ok_b && bm != b;
  constexpr int CH = S1_PB / 32;          // 16-wide p' chunks per warp
  uint32_t v[CH][4][16];                  // X re, X im, Y re, Y im
#pragma unroll
  for (int u = 0; u < CH; ++u) {
    const int h = half * CH + u;
    tmem_ld16x4w(tx + (uint32_t)(h * 16), tx + (uint32_t)(S1_PB + h * 16),
                 ty + (uint32_t)(h * 16), ty + (uint32_t)(S1_PB + h * 16), v[u][0], v[u][1],
                 v[u][2], v[u][3]);
  }
  release_acc(lane, release_bar);
  if (!ok_b) return;
  const float sc = p.out_scale;
  const size_t kp = (size_t)p.Kp;
  const size_t var = (size_t)6 * p.ny * kp;             // elements per variant
  // row (b, c, re) of variant hi of parity par; im is the next row
  const size_t base_v = ((size_t)plane * 4 + 2 * par) * var;
  const size_t rb = base_v + ((size_t)b * 6 + 2 * c) * kp;
  const size_t rm = base_v + ((size_t)bm * 6 + 2 * c) * kp;
#pragma unroll
  for (int u = 0; u < CH; ++u) {
    const int p0 = blk * S1_PB + (half * CH + u) * 16;
    const int n_valid = p.H - p0;
    if (n_valid <= 0) continue;
    float t[16];
#pragma unroll
    for (int j = 0; j < 16; ++j)
      t[j] = sc * (__uint_as_float(v[u][0][j]) - __uint_as_float(v[u][3][j]));
    store_piece<TF32>(p, rb + p0, var, t, n_valid);
#pragma unroll
    for (int j = 0; j < 16; ++j)
      t[j] = sc * (__uint_as_float(v[u][1][j]) + __uint_as_float(v[u][2][j]));
    store_piece<TF32>(p, rb + kp + p0, var, t, n_valid);
    if (ok_m) {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        t[j] = sc * (__uint_as_float(v[u][0][j]) + __uint_as_float(v[u][3][j]));
      store_piece<TF32>(p, rm + p0, var, t, n_valid);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        t[j] = sc * (__uint_as_float(v[u][1][j]) - __uint_as_float(v[u][2][j]));
      store_piece<TF32>(p, rm + kp + p0, var, t, n_valid);
    }
  }
}

// ---------------------------------------------------------------------------
// Epilogue of stage 2: tile (plane, b-block of S2_BOUT); this thread's
// accumulator row is a' (TMEM lane).  CTA h of the pair supplied the data
// rows (b, c, re/im) of the outputs b0 + h S2_HB .. + S2_HB, so the tile's
// columns are (h, b, c, re/im); the epilogue warps of half h read those 48.
// Per channel
//   E[a'] = X + i Y,  E[a~'] = X - i Y,
// I = out_scale^2 sum_c |E_c|^2 at a' and a~'; the optional fields carry the
// -i of the Eq. 8 prefactor.
// ---------------------------------------------------------------------------
PSF_D void epilogue_stage2(const FoldParams& p, uint32_t tx, uint32_t ty, int plane, int mt,
                           int nt, int row, int half, int lane, uint32_t release_bar) {
  const int a = mt * BM + row;
  const bool ok_a = a < p.m_rows;
  const int am = p.n_out - 1 - a;
  const bool ok_m = ok_a && am != a;
  const int b0 = nt * S2_BOUT + half * S2_HB;
  uint32_t xa[32], xb[16], ya[32], yb[16];
  const uint32_t col = (uint32_t)(half * 6 * S2_HB);
  tmem_ld32w(tx + col, xa);
  tmem_ld16w(tx + col + 32, xb);
  tmem_ld32w(ty + col, ya);
  tmem_ld16w(ty + col + 32, yb);
  release_acc(lane, release_bar);
  auto xv = [&](int k) { return __uint_as_float(k < 32 ? xa[k] : xb[k - 32]); };
  auto yv = [&](int k) { return __uint_as_float(k < 32 ? ya[k] : yb[k - 32]); };
  const float sc = p.out_scale;
  float s[S2_HB], sm[S2_HB];
#pragma unroll
  for (int j = 0; j < S2_HB; ++j) s[j] = sm[j] = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float er[S2_HB], ei[S2_HB], mr[S2_HB], mi[S2_HB];
#pragma unroll
    for (int j = 0; j < S2_HB; ++j) {
      const int kr = j * 6 + 2 * c, ki = kr + 1;
      const float xr_ = xv(kr), xi_ = xv(ki), yr_ = yv(kr), yi_ = yv(ki);
      er[j] = xr_ - yi_;
      ei[j] = xi_ + yr_;
      mr[j] = xr_ + yi_;
      mi[j] = xi_ - yr_;
      s[j] = fmaf(er[j], er[j], fmaf(ei[j], ei[j], s[j]));
      sm[j] = fmaf(mr[j], mr[j], fmaf(mi[j], mi[j], sm[j]));
    }
    if (p.F && ok_a) {
      // E = -i * out_scale * (re + i im) = out_scale * (im, -re)
      float2* fa = p.F + (((size_t)plane * 3 + c) * p.nx + a) * p.ny + b0;
      float2* fm = p.F + (((size_t)plane * 3 + c) * p.nx + am) * p.ny + b0;
#pragma unroll
      for (int j = 0; j < S2_HB; ++j) {
        if (b0 + j < p.ny) {
          fa[j] = make_float2(sc * ei[j], -sc * er[j]);
          if (ok_m) fm[j] = make_float2(sc * mi[j], -sc * mr[j]);
        }
      }
    }
  }
  if (!ok_a || b0 >= p.ny) return;
  const float sc2 = sc * sc;
  float* da = p.I + ((size_t)plane * p.nx + a) * p.ny + b0;
  float* dm = p.I + ((size_t)plane * p.nx + am) * p.ny + b0;
  if (b0 + S2_HB <= p.ny && (p.ny & 3) == 0) {
#pragma unroll
    for (int v = 0; v < S2_HB / 4; ++v) {
      ((float4*)da)[v] = make_float4(sc2 * s[4 * v], sc2 * s[4 * v + 1], sc2 * s[4 * v + 2],
                                     sc2 * s[4 * v + 3]);
      if (ok_m)
        ((float4*)dm)[v] = make_float4(sc2 * sm[4 * v], sc2 * sm[4 * v + 1],
                                       sc2 * sm[4 * v + 2], sc2 * sm[4 * v + 3]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < S2_HB; ++j) {
      if (b0 + j < p.ny) {
        da[j] = sc2 * s[j];
        if (ok_m) dm[j] = sc2 * sm[j];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The persistent CTA-pair kernel of both folded stages.
//   mA: zoom halves [4][m_rows][H] (C hi, C lo, S hi, S lo), box BK x 128 x 4
//   mB: data, four variants (X hi, X lo, Y hi, Y lo) per box
// TF32: 32-bit operands, kind::tf32 MMAs with K = 8; a stage holds the same
// 128-byte rows (32 elements), so the shared-memory layout, the four 32-byte
// K steps per stage and the descriptors are those of the 16-bit form.
// ---------------------------------------------------------------------------
template <int MODE, bool RES, bool TF32>
__global__ void __launch_bounds__(NUM_THREADS, 1)
k_fold_pair(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
            const FoldParams p) {
  using Sh = Shape<MODE, RES>;
  constexpr int BKE = TF32 ? BK / 2 : BK;      // K elements per stage
  constexpr int STAGES = Sh::STAGES, BN = Sh::BN, NACC = Sh::NACC;
  constexpr int PB_BYTES = Sh::PB_BYTES, STAGE_BYTES = Sh::STAGE_BYTES;
  constexpr int B_OFF = RES ? 0 : A_CHUNK;      // data operand within a stage
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* ring = smem + Sh::A_RES;
  uint64_t* bars = (uint64_t*)(ring + STAGES * STAGE_BYTES);
  // bars: full[S], empty[S], tfull[NACC], tempty[NACC], drain, a_full
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * STAGES + 2 * NACC + 2);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();
  const bool leader = rank == 0;
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (STAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * STAGES + NACC + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * STAGES + 2 * NACC);
  const uint32_t afull_bar = drain_bar + 8u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < NACC; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), 2 * EPI_WARPS);    // one arrival per epilogue warp
    }
    mbar_init(drain_bar, 1);
    mbar_init(afull_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc_pair(smem_u32(tmem_slot), TMEM_COLS);
  tmem_fence_before();
  __syncthreads();
  cluster_sync_all();          // both CTAs' barriers exist before any remote use
  tmem_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  const int total = p.planes * p.m_pairs * p.n_tiles;
  const int cluster = blockIdx.x >> 1, n_clusters = gridDim.x >> 1;

  if (warp == 0 && lane == 0) {
    // ------------------------------ TMA producer ------------------------------
    bool ok = true;
    if (RES) {
      // this CTA's 128 zoom rows over the whole K range, once per kernel
      // (m_pairs == 1: every tile uses them)
      const uint32_t fa = mapa_shared(afull_bar, 0);
      if (leader) mbar_arrive_expect_tx(afull_bar, 2u * p.k_chunks * A_CHUNK);
      for (int kc = 0; kc < p.k_chunks; ++kc)
        tma_load_3d_pair(smem_u32(smem) + kc * A_CHUNK, &mA, kc * BKE, (int)rank * BM, 0, fa);
    }
    int stage = 0;
    uint32_t phase = 0;
    int issued = 0;
    for (int t = cluster; t < total && ok; t += n_clusters) {
      int plane, mp, nt;
      decode(p, t, plane, mp, nt);
      const int mt = 2 * mp + (int)rank;
      for (int kc = 0; kc < p.k_chunks; ++kc) {
        if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, p.status)) {
          ok = false;
          break;
        }
        const uint32_t base = smem_u32(ring + stage * STAGE_BYTES);
        const uint32_t fb = mapa_shared(full_bar(stage), 0);   // the leader's barrier
        if (leader) mbar_arrive_expect_tx(full_bar(stage), 2 * STAGE_BYTES);
        const int k0 = kc * BKE;
        if (!RES) tma_load_3d_pair(base, &mA, k0, mt * BM, 0, fb);
        if (MODE == 0) {
          // rows (plane, c, parity, re/im = rank) x 64 p' of the p'-block
          const int c = nt / (2 * p.pblk);
          const int rem = nt - c * 2 * p.pblk;
          const int par = rem / p.pblk, blk = rem - par * p.pblk;
          const int slab = ((plane * 3 + c) * 2 + par) * 2 + (int)rank;
          tma_load_3d_pair(base + B_OFF, &mB, k0, blk * S1_PB, 4 * slab, fb);
        } else {
          // rows (b, c, re/im) of this CTA's S2_HB outputs b
          tma_load_3d_pair(base + B_OFF, &mB, k0, (nt * S2_BOUT + (int)rank * S2_HB) * 6,
                           4 * plane, fb);
        }
        ++issued;
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    if (!ok && leader) {
      // drain: wait (bounded) for the copies still in flight before exiting
      if (RES) mbar_drain_wait(afull_bar, 0);
      for (int k = 0; k < STAGES && k < issued; ++k) {
        if (--stage < 0) {
          stage = STAGES - 1;
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
    if (RES) {
      ok = mbar_wait(afull_bar, 0, abort_flag, p.status);
      tmem_fence_after();
    }
    for (int t = cluster; t < total && ok; t += n_clusters) {
      if (!mbar_wait(tempty_bar(acc), acc_phase ^ 1u, abort_flag, p.status)) {
        ok = false;
        break;
      }
      tmem_fence_after();
      const uint32_t d_x = tmem_base + (uint32_t)(acc * 2 * BN);
      const uint32_t d_y = d_x + (uint32_t)BN;
      for (int kc = 0; kc < p.k_chunks; ++kc) {
        if (!mbar_wait(full_bar(stage), phase, abort_flag, p.status)) {
          ok = false;
          break;
        }
        tmem_fence_after();
        const uint32_t base = smem_u32(ring + stage * STAGE_BYTES);
        const uint32_t ab = RES ? smem_u32(smem) + kc * A_CHUNK : base;
        const uint64_t dCh = smem_desc<SWZ>(ab), dCl = smem_desc<SWZ>(ab + A_BYTES);
        const uint64_t dSh = smem_desc<SWZ>(ab + 2 * A_BYTES);
        const uint64_t dSl = smem_desc<SWZ>(ab + 3 * A_BYTES);
        const uint32_t bx = base + B_OFF;
        const uint64_t dXh = smem_desc<SWZ>(bx), dXl = smem_desc<SWZ>(bx + PB_BYTES);
        const uint64_t dYh = smem_desc<SWZ>(bx + 2 * PB_BYTES);
        const uint64_t dYl = smem_desc<SWZ>(bx + 3 * PB_BYTES);
#pragma unroll
        for (int k = 0; k < BK / 16; ++k) {
          const uint64_t adv = (uint64_t)((k * 32) >> 4);   // 16 elements = 32 bytes
          const uint32_t first = (kc == 0 && k == 0) ? 0u : 1u;
          if (TF32) {
            mma_tf32_pair(d_x, dCh + adv, dXh + adv, p.idesc, first);
            if (p.passes == 3) {
              mma_tf32_pair(d_x, dCl + adv, dXh + adv, p.idesc, 1u);
              mma_tf32_pair(d_x, dCh + adv, dXl + adv, p.idesc, 1u);
            }
            mma_tf32_pair(d_y, dSh + adv, dYh + adv, p.idesc, first);
            if (p.passes == 3) {
              mma_tf32_pair(d_y, dSl + adv, dYh + adv, p.idesc, 1u);
              mma_tf32_pair(d_y, dSh + adv, dYl + adv, p.idesc, 1u);
            }
          } else {
            mma_f16_pair(d_x, dCh + adv, dXh + adv, p.idesc, first);
            mma_f16_pair(d_x, dCl + adv, dXh + adv, p.idesc, 1u);
            mma_f16_pair(d_x, dCh + adv, dXl + adv, p.idesc, 1u);
            mma_f16_pair(d_y, dSh + adv, dYh + adv, p.idesc, first);
            mma_f16_pair(d_y, dSl + adv, dYh + adv, p.idesc, 1u);
            mma_f16_pair(d_y, dSh + adv, dYl + adv, p.idesc, 1u);
          }
        }
        mma_commit_pair(empty_bar(stage), 3);   // frees the stage in both CTAs
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (!ok) break;
      mma_commit_pair(tfull_bar(acc), 3);       // accumulators ready in both CTAs
      if (++acc == NACC) {
        acc = 0;
        acc_phase ^= 1u;
      }
    }
    mma_commit_pair(drain_bar, 1);
    mbar_drain_wait(drain_bar, 0);
  } else if (warp >= 2) {
    // ------------------------------ epilogue ----------------------------------
    const int quad = warp & 3;                 // TMEM lanes 32*quad .. +31
    const int half = (warp - 2) >> 2;          // which half of the tile's columns
    const int row = quad * 32 + lane;
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int t = cluster; t < total; t += n_clusters) {
      int okw = 1;
      if (lane == 0) okw = mbar_wait(tfull_bar(acc), acc_phase, abort_flag, p.status) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) break;
      tmem_fence_after();
      int plane, mp, nt;
      decode(p, t, plane, mp, nt);
      const int mt = 2 * mp + (int)rank;
      const uint32_t tx = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * 2 * BN);
      const uint32_t ty = tx + (uint32_t)BN;
      // each epilogue warp releases the accumulator (on the leader's barrier)
      // as soon as it has read its columns, before its arithmetic and stores
      const uint32_t rel = mapa_shared(tempty_bar(acc), 0);
      if (MODE == 0)
        epilogue_stage1<TF32>(p, tx, ty, plane, mt, nt, row, half, lane, rel);
      else
        epilogue_stage2(p, tx, ty, plane, mt, nt, row, half, lane, rel);
      if (++acc == NACC) {
        acc = 0;
        acc_phase ^= 1u;
      }
    }
  }
  tmem_fence_before();
  __syncthreads();
  cluster_sync_all();          // every MMA done and every TMEM read done in both CTAs
  tmem_fence_after();
  if (warp == 1) tmem_dealloc_pair(tmem_base, TMEM_COLS);
}

// ---------------------------------------------------------------------------
// Operand producers
// ---------------------------------------------------------------------------
// Folded zoom halves Z[4][m_rows][Kp] (C hi, C lo, S hi, S lo): for
// i' < m_rows (= ceil(n_out/2)) and p' < H,
//   C[i'][p'] = S_A cos(2 pi f u_p' x_i'),  S[i'][p'] = S_A sin(...),
// the angle f d m n / (2N) cycles from the exact integers m = 2p'+1-N and
// n = 2i'+1-n_out (one FP64 product, reduced mod 1).
// (TF32 operands: 32-bit elements, split into TF32 hi + lo, lo 0 with one pass.)
template <bool TF32>
__global__ void k_fold_twiddle(int N, int n_out, int m_rows, int H, int Kp, double alpha,
                               float sA, int bf16, int passes, void* __restrict__ Zv) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m_rows * H) return;
  const int i = idx / H, pp = idx - (idx / H) * H;
  const long long mn = (long long)(2 * pp + 1 - N) * (long long)(2 * i + 1 - n_out);
  double cyc = alpha * (double)mn;
  cyc -= rint(cyc);
  float sn, cs;
  sincospif(2.0f * (float)cyc, &sn, &cs);
  const size_t var = (size_t)m_rows * Kp;
  const size_t o = (size_t)i * Kp + pp;
  if (TF32) {
    uint32_t* Z = (uint32_t*)Zv;
    uint32_t h, l;
    split_tf32(sA * cs, passes, h, l);
    Z[o] = h;
    Z[var + o] = l;
    split_tf32(sA * sn, passes, h, l);
    Z[2 * var + o] = h;
    Z[3 * var + o] = l;
  } else {
    uint16_t* Z = (uint16_t*)Zv;
    uint16_t h, l;
    split16(sA * cs, bf16, h, l);
    Z[o] = h;
    Z[var + o] = l;
    split16(sA * sn, bf16, h, l);
    Z[2 * var + o] = h;
    Z[3 * var + o] = l;
  }
}

// Pupil fields of a z-chunk folded over both mirrors.  For node (p', q') of
// the first quadrant (p', q' < H) and the mirrors p~' = N-1-p',
// q~' = N-1-q', with P_c = amp_c e^{2 pi i (W + n_i z cos / lambda)} rebuilt
// from the node table:
//   P[s r] = (P[p'][q'] + s P[p'][q~']) + r (P[p~'][q'] + s P[p~'][q~'])
// stored split (scale S_P): slab ((plane, c, r, re/im)), variants X hi, X lo
// (s = +), Y hi, Y lo (s = -), row p', column q' (pitch Kp).  Four
// consecutive q' per thread, one plane per grid row; planes are numbered
// flat over (pupil, z) with nz_per planes per pupil (a single pupil:
// wfr_stride 0).
template <bool TF32>
__global__ void __launch_bounds__(128)
k_fold_pupil(NodeTable t, int N, int H, int Kp, const float2* __restrict__ zz, int z0,
             int nz_per, long long wfr_stride, float sP, int bf16, int passes,
             void* __restrict__ Pout) {
  const int NN = N * N;
  const int H4 = H / 4;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= H * H4) return;
  const int pp = idx / H4, q0 = (idx - (idx / H4) * H4) * 4;
  const int flat = z0 + (int)blockIdx.y;
  const int pk = flat / nz_per, zi = flat - pk * nz_per;
  const float2 z = zz[zi];
  const f2x zf{z.x, z.y};
  // node index of the four mirror images: [0] (p', q'), [1] (p', q~'),
  // [2] (p~', q'), [3] (p~', q~'); the q~' runs are stored reversed
  const int pm = N - 1 - pp;
  const int base[4] = {pp * N + q0, pp * N + (N - 4 - q0), pm * N + q0, pm * N + (N - 4 - q0)};
  const float* wfr = t.wfr + (size_t)pk * wfr_stride;
  float2 e[4][4];                       // [image][k], k = q' - q0
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const float4 w4 = *(const float4*)(wfr + base[g]);
    const float4 kh4 = *(const float4*)(t.kh + base[g]);
    const float4 kl4 = *(const float4*)(t.kl + base[g]);
    const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
    const float khv[4] = {kh4.x, kh4.y, kh4.z, kh4.w};
    const float klv[4] = {kl4.x, kl4.y, kl4.z, kl4.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = (g & 1) ? 3 - j : j;     // reversed runs for the q~' images
      e[g][k] = cis_cycles(frac_mul_add(f2x{khv[j], klv[j]}, zf, wv[j]));
    }
  }
  const size_t var = (size_t)H * Kp;          // elements per (slab, variant)
#pragma unroll 1
  for (int c = 0; c < 3; ++c) {
    float2 Pv[4][4];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const float4 ar = *(const float4*)(t.amp + (size_t)(2 * c) * NN + base[g]);
      const float4 ai = *(const float4*)(t.amp + (size_t)(2 * c + 1) * NN + base[g]);
      const float arv[4] = {ar.x, ar.y, ar.z, ar.w};
      const float aiv[4] = {ai.x, ai.y, ai.z, ai.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = (g & 1) ? 3 - j : j;
        Pv[g][k] = cmul(make_float2(sP * arv[j], sP * aiv[j]), e[g][k]);
      }
    }
    // parity combinations, k = 0..3
    float v[2][2][2][4];                  // [s: 0 '+', 1 '-'][r][re/im][k]
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 sp = make_float2(Pv[0][k].x + Pv[1][k].x, Pv[0][k].y + Pv[1][k].y);
      const float2 dp = make_float2(Pv[0][k].x - Pv[1][k].x, Pv[0][k].y - Pv[1][k].y);
      const float2 sm = make_float2(Pv[2][k].x + Pv[3][k].x, Pv[2][k].y + Pv[3][k].y);
      const float2 dm = make_float2(Pv[2][k].x - Pv[3][k].x, Pv[2][k].y - Pv[3][k].y);
      v[0][0][0][k] = sp.x + sm.x;  v[0][0][1][k] = sp.y + sm.y;
      v[0][1][0][k] = sp.x - sm.x;  v[0][1][1][k] = sp.y - sm.y;
      v[1][0][0][k] = dp.x + dm.x;  v[1][0][1][k] = dp.y + dm.y;
      v[1][1][0][k] = dp.x - dm.x;  v[1][1][1][k] = dp.y - dm.y;
    }
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int ri = 0; ri < 2; ++ri) {
          const size_t slab = (((size_t)blockIdx.y * 3 + c) * 2 + r) * 2 + ri;
          const size_t o = (slab * 4 + 2 * s) * var + (size_t)pp * Kp + q0;
          if (TF32) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) split_tf32(v[s][r][ri][k], passes, h[k], l[k]);
            uint32_t* P = (uint32_t*)Pout;
            *(uint4*)(P + o) = make_uint4(h[0], h[1], h[2], h[3]);
            *(uint4*)(P + o + var) = make_uint4(l[0], l[1], l[2], l[3]);
          } else {
            // packed pairs: element k in the low half, k + 1 in the high half
            uint32_t h01, l01, h23, l23;
            split2(v[s][r][ri][0], v[s][r][ri][1], bf16, h01, l01);
            split2(v[s][r][ri][2], v[s][r][ri][3], bf16, h23, l23);
            uint16_t* P = (uint16_t*)Pout;
            *(uint2*)(P + o) = make_uint2(h01, h23);
            *(uint2*)(P + o + var) = make_uint2(l01, l23);
          }
        }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* q = nullptr;
    cudaDriverEntryPointQueryResult r;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &q, 12000, cudaEnableDefault,
                                         &r) == cudaSuccess &&
        r == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)q;
  }
  return fn;
}

// [slabs][rows][K] 16-bit tensor with row pitch Kp (elements), K extent H;
// boxes BK x box_rows x 4 (four consecutive slabs: the four variants).
// Columns H .. Kp-1 and rows past `rows` read as zeros.
// eb: element bytes (2: 16-bit operands, 4: TF32), a box row is 128 bytes.
static bool make_map(CUtensorMap* m, const void* base, int H, int Kp, int rows, int slabs,
                     int box_rows, int eb) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)H, (cuuint64_t)rows, (cuuint64_t)slabs};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * eb, (cuuint64_t)Kp * eb * rows};
  cuuint32_t box[3] = {(cuuint32_t)(128 / eb), (cuuint32_t)box_rows, 4};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, eb == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 3,
            (void*)base, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// operand format: 0 fp16, 1 bf16, 2 tf32
static uint32_t make_idesc(int fmt_code, int bn) {
  const uint32_t fmt = (uint32_t)fmt_code;
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(bn >> 3) << 17) |
         ((uint32_t)((2 * BM) >> 4) << 24);
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

template <int MODE, bool RES, bool TF32>
static int launch(const CUtensorMap& mA, const CUtensorMap& mB, FoldParams p,
                  cudaStream_t s) {
  using Sh = Shape<MODE, RES>;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_fold_pair<MODE, RES, TF32>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             Sh::SMEM_BYTES) != cudaSuccess)
      return PSF_ERR_CUDA;
    attr = true;
  }
  p.idesc = make_idesc(TF32 ? 2 : p.bf16, Sh::BN);
  const int total = p.planes * p.m_pairs * p.n_tiles;
  int clusters = num_sms() / 2;
  if (total < clusters) clusters = total;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(2 * clusters);
  cfg.blockDim = dim3(NUM_THREADS);
  cfg.dynamicSmemBytes = Sh::SMEM_BYTES;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_fold_pair<MODE, RES, TF32>, mA, mB, p) != cudaSuccess)
    return PSF_ERR_CUDA;
  return cudaPeekAtLastError() == cudaSuccess ? PSF_OK : PSF_ERR_CUDA;
}

// Resident zoom halves when one pair tile covers every zoom row and the
// whole K range fits the resident area.
template <int MODE>
static int launch_any(const CUtensorMap& mA, const CUtensorMap& mB, const FoldParams& p,
                      bool tf32, cudaStream_t s) {
  const bool res = p.m_pairs == 1 && p.k_chunks <= RES_CHUNKS;
  if (tf32)
    return res ? launch<MODE, true, true>(mA, mB, p, s) : launch<MODE, false, true>(mA, mB, p, s);
  return res ? launch<MODE, true, false>(mA, mB, p, s) : launch<MODE, false, false>(mA, mB, p, s);
}

static float pow2_scale(double bound, double target) {
  // largest power of two S with bound * S <= target
  if (!(bound > 0)) return 1.0f;
  return (float)exp2(floor(log2(target / bound)));
}

}  // namespace fold
}  // namespace tc

// ==========================================================================
// Interface used by psf_api.cu
// ==========================================================================
int tc_fold_kp(int N) { return ((N / 2) + 15) / 16 * 16; }

const char* tc_fold_supported(int N, int nx, int ny) {
  if (N % 8 != 0 || N < 16) return "n_pupil must be a multiple of 8 and >= 16";
  if (nx < 1 || ny < 1) return "empty output grid";
  return nullptr;
}

static double fold_plane_bytes(int N, int ny, int eb) {
  const double H = N / 2, Kp = tc_fold_kp(N);
  // P: 4 variants x 12 H rows; U: 4 variants x 6 ny rows (eb-byte elements, pitch Kp)
  return eb * Kp * (4.0 * 12.0 * H + 4.0 * 6.0 * ny);
}

int tc_fold_zchunk(int N, int nx, int ny, int nz, int eb) {
  // P and U of a chunk up to 4 GB and 256 planes (long launches fill the
  // persistent contractions); the planes are then spread evenly over the
  // chunks so the last one is not short
  (void)nx;
  int cap = (int)(4096.0 * 1048576.0 / fold_plane_bytes(N, ny, eb));
  if (cap < 1) cap = 1;
  if (cap > 256) cap = 256;
  if (cap > nz) cap = nz;
  const int n_chunks = (nz + cap - 1) / cap;
  return (nz + n_chunks - 1) / n_chunks;
}

void tc_fold_carve(char* base, size_t* off, int N, int nx, int ny, int zc, TcFoldOperands* out,
                   int eb) {
  auto take = [&](size_t elems) -> uint16_t* {
    *off = align_up(*off, 1024);
    uint16_t* p = base ? (uint16_t*)(base + *off) : nullptr;
    *off += elems * (size_t)eb;
    return p;
  };
  const int H = N / 2, Kp = tc_fold_kp(N);
  const size_t mx = (size_t)(nx + 1) / 2, my = (size_t)(ny + 1) / 2;
  out->H = H;
  out->Kp = Kp;
  out->Zx = take(4 * mx * Kp);
  out->Zy = take(4 * my * Kp);
  out->P = take((size_t)zc * 48 * H * Kp);
  out->U = take((size_t)zc * 24 * ny * Kp);
}

// Per-thread, per-device side stream (pupil planes of the next chunk) and
// the copy stream of a pinned host output; see tc_fourier_forward.
struct FoldStreams {
  int dev = -1;
  cudaStream_t side = nullptr, copy = nullptr;
  cudaEvent_t consumed = nullptr, ready = nullptr;
  cudaEvent_t done[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
};

static FoldStreams* fold_streams() {
  static thread_local FoldStreams fs[16];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return nullptr;
  FoldStreams& x = fs[dev];
  if (x.dev != dev) {
    bool ok = cudaStreamCreateWithFlags(&x.side, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&x.copy, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&x.consumed, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&x.ready, cudaEventDisableTiming) == cudaSuccess;
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

int tc_fold_forward(const TcFoldOperands& ops, NodeTable nodes, const float2* zz, int N,
                    int nx, int ny, double dx, double dy, int nz, int zc,
                    double na_over_lambda, float scale, double amp_bound, int precision,
                    float* intensity, float2* fields, float* host_out, int* status,
                    cudaStream_t s) {
  using namespace tc;
  using namespace tc::fold;
  FoldStreams* fs = fold_streams();
  if (host_out && !fs) return PSF_ERR_CUDA;
  const int bf16 = precision == PSF_PREC_SPLIT_BF16 ? 1 : 0;
  const bool tf32 = precision == PSF_PREC_SPLIT_TF32 || precision == PSF_PREC_TF32;
  const int passes = precision == PSF_PREC_TF32 ? 1 : 3;
  const int eb = tf32 ? 4 : 2;
  const int bke = tf32 ? BK / 2 : BK;        // K elements per stage
  const int H = ops.H, Kp = ops.Kp;
  const int mx = (nx + 1) / 2, my = (ny + 1) / 2;
  const double target = 16384.0;             // keep |scaled value| <= 2^14
  const float sA = fold::pow2_scale(1.0, target);
  const float sP = fold::pow2_scale(4.0 * amp_bound, target);
  const float sU = fold::pow2_scale(2.0 * amp_bound * N, target);
  {
    TimingScope ts(kTimeSetup, s);
    auto twiddle = [&](int n_out, int m, double d, void* Z) {
      if (tf32)
        k_fold_twiddle<true><<<ceil_div(m * H, 256), 256, 0, s>>>(
            N, n_out, m, H, Kp, na_over_lambda * d / (2.0 * N), sA, bf16, passes, Z);
      else
        k_fold_twiddle<false><<<ceil_div(m * H, 256), 256, 0, s>>>(
            N, n_out, m, H, Kp, na_over_lambda * d / (2.0 * N), sA, bf16, passes, Z);
    };
    twiddle(nx, mx, dx, ops.Zx);
    twiddle(ny, my, dy, ops.Zy);
  }
  CUtensorMap mZy, mP, mZx, mU;
  bool ok = make_map(&mZy, ops.Zy, H, Kp, my, 4, BM, eb) &&
            make_map(&mP, ops.P, H, Kp, H, 48 * zc, S1_PB, eb) &&
            make_map(&mZx, ops.Zx, H, Kp, mx, 4, BM, eb) &&
            make_map(&mU, ops.U, H, Kp, 6 * ny, 4 * zc, 6 * S2_HB, eb);
  if (!ok) return PSF_ERR_CUDA;
  auto pupil = [&](int zc0, cudaStream_t st) {
    const int n = nz - zc0 < zc ? nz - zc0 : zc;
    TimingScope ts(kTimePupil, st);
    const dim3 pg(ceil_div(H * (H / 4), 128), n);
    if (tf32)
      k_fold_pupil<true><<<pg, 128, 0, st>>>(nodes, N, H, Kp, zz, zc0, nz, 0, sP, bf16, passes,
                                             ops.P);
    else
      k_fold_pupil<false><<<pg, 128, 0, st>>>(nodes, N, H, Kp, zz, zc0, nz, 0, sP, bf16,
                                              passes, ops.P);
  };
  pupil(0, s);
  for (int z0 = 0; z0 < nz; z0 += zc) {
    const int nzc = nz - z0 < zc ? nz - z0 : zc;
    const bool more = z0 + zc < nz;
    FoldParams p1;
    memset(&p1, 0, sizeof(p1));
    p1.planes = nzc;
    p1.m_pairs = ceil_div(my, 2 * BM);
    p1.pblk = ceil_div(H, S1_PB);
    p1.n_tiles = 3 * 2 * p1.pblk;
    p1.k_chunks = ceil_div(H, bke);
    p1.H = H;
    p1.Kp = Kp;
    p1.m_rows = my;
    p1.n_out = ny;
    p1.nx = nx;
    p1.ny = ny;
    p1.bf16 = bf16;
    p1.passes = passes;
    p1.out_scale = sU / (sA * sP);
    p1.U = ops.U;
    p1.status = status;
    int r;
    {
      TimingScope ts(kTimeStage1, s);
      r = launch_any<0>(mZy, mP, p1, tf32, s);
    }
    if (r) return r;
    if (more && fs) {
      // the pupil planes of the next chunk on the side stream, overlapping
      // stage 2 of this one (which does not read them)
      cudaEventRecord(fs->consumed, s);
      cudaStreamWaitEvent(fs->side, fs->consumed, 0);
      pupil(z0 + zc, fs->side);
      cudaEventRecord(fs->ready, fs->side);
    }
    FoldParams p2 = p1;
    p2.m_pairs = ceil_div(mx, 2 * BM);
    p2.n_tiles = ceil_div(ny, S2_BOUT);
    p2.m_rows = mx;
    p2.n_out = nx;
    p2.out_scale = scale / (sA * sU);
    const int ci = z0 / zc, buf = ci & 1;
    const size_t plane = (size_t)nx * ny;
    if (host_out) {
      // `intensity` is the two-chunk staging area (see tc_fourier_forward)
      p2.I = intensity + (size_t)buf * zc * plane;
      if (ci >= 2) cudaStreamWaitEvent(s, fs->copied[buf], 0);
    } else {
      p2.I = intensity + (size_t)z0 * plane;
    }
    p2.F = fields ? fields + (size_t)z0 * 3 * plane : nullptr;
    {
      TimingScope ts(kTimeStage2, s);
      r = launch_any<1>(mZx, mU, p2, tf32, s);
    }
    if (r) return r;
    if (host_out) {
      cudaEventRecord(fs->done[buf], s);
      cudaStreamWaitEvent(fs->copy, fs->done[buf], 0);
      cudaMemcpyAsync(host_out + (size_t)z0 * plane, p2.I, (size_t)nzc * plane * sizeof(float),
                      cudaMemcpyDeviceToHost, fs->copy);
      cudaEventRecord(fs->copied[buf], fs->copy);
    }
    if (more) {
      if (fs)
        cudaStreamWaitEvent(s, fs->ready, 0);
      else
        pupil(z0 + zc, s);
    }
  }
  if (host_out) {
    const int n_chunks = (nz + zc - 1) / zc;
    if (n_chunks >= 1) cudaStreamWaitEvent(s, fs->copied[0], 0);
    if (n_chunks >= 2) cudaStreamWaitEvent(s, fs->copied[1], 0);
  }
  return PSF_OK;
}

}  // namespace psf
