// tcgen05 BF16 GEMM with the MLP epilogues (bias + SiLU, linear, SiLU'
// backward, plain store).  Warp roles as in the Fourier kernels: warp 0 TMA
// producer (A tile 128 x 64, B tile n_tile x 64, 128-byte swizzle, 4-deep
// ring), warp 1 TMEM allocator + single-thread MMA issuer (M = 128,
// N = n_tile <= 256, K = 16 per instruction, FP32 accumulation in one of two
// TMEM accumulators), warps 2-5 epilogue.  Waits are bounded (status word).
#include <math.h>
#include <string.h>

#include "mlp_kernels.cuh"
#include "tc_ptx.cuh"

namespace psf {
namespace mlp {

ParamLayout param_layout() {
  ParamLayout L;
  size_t o = 0;
  for (int l = 0; l < NLAYER; ++l) {
    L.W[l] = o;
    o += (size_t)layer_out(l) * layer_in(l);
    L.b[l] = o;
    o += layer_out(l);
  }
  L.We = o;
  o += HID;
  L.be = o;
  o += 1;
  L.total = o;
  return L;
}

namespace {

using namespace tc;

constexpr int GM = 128;                 // A rows per tile
constexpr int GNMAX = 256;              // max B rows per tile
constexpr int GK = 64;                  // K per stage (128-byte rows)
constexpr int GSTAGES = 3;
constexpr int GA_BYTES = GM * GK * 2;
constexpr int GB_BYTES = GNMAX * GK * 2;
constexpr int GSTAGE = GA_BYTES + GB_BYTES;   // 48 KB
constexpr int GEPI_WARPS = 16;          // four per TMEM lane quarter
constexpr int GTHREADS = 64 + 32 * GEPI_WARPS;
constexpr int GCH = 16;                 // epilogue columns per TMEM load
// FP32 outputs of a chunk staged per epilogue warp (32 rows, stride 20 floats:
// 16-byte aligned rows, conflict-free 16-byte writes) and stored 8 rows of
// 64 bytes per instruction
constexpr int GSTG_LD = GCH + 4;
constexpr int GSTG_BYTES = GEPI_WARPS * 32 * GSTG_LD * 4;
constexpr int GSMEM = GSTAGES * GSTAGE + GSTG_BYTES + 1024 + 1024;

struct KArgs {
  GemmArgs g;
  int n_tile, m_tiles, n_tiles, k_chunks;
  uint32_t idesc;
};

PSF_D float bf2f(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }

// (re, im) pairs of a float4 times the complex e
PSF_D float4 cmul2(float4 w, float2 e) {
  return make_float4(w.x * e.x - w.y * e.y, w.x * e.y + w.y * e.x,
                     w.z * e.x - w.w * e.y, w.z * e.y + w.w * e.x);
}

// bias[n0 .. n0 + GCH) (0 past N), as four 16-byte loads when the chunk is full
PSF_D void load_bias(const GemmArgs& g, int n0, bool full, float (&b)[GCH]) {
  if (full && (((uintptr_t)(g.bias + n0) & 15) == 0)) {
#pragma unroll
    for (int q = 0; q < GCH / 4; ++q) {
      const float4 w = __ldg((const float4*)(g.bias + n0) + q);
      b[4 * q] = w.x;
      b[4 * q + 1] = w.y;
      b[4 * q + 2] = w.z;
      b[4 * q + 3] = w.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < GCH; ++j) b[j] = n0 + j < g.N ? g.bias[n0 + j] : 0.f;
  }
}

// 16 consecutive TMEM columns of this warp's lanes, waited in the same asm.
PSF_D void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32"
      " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
        "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
        "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
PSF_D uint16_t f2bf(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

__global__ void __launch_bounds__(GTHREADS, 1)
k_gemm_bf16(const __grid_constant__ CUtensorMap mapA,
            const __grid_constant__ CUtensorMap mapB, const KArgs ka) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* gstg = (float*)(smem + GSTAGES * GSTAGE);
  uint64_t* bars = (uint64_t*)(smem + GSTAGES * GSTAGE + GSTG_BYTES);
  uint32_t* tmem_slot = (uint32_t*)(bars + 2 * GSTAGES + 5);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const GemmArgs& g = ka.g;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar0 = smem_u32(bars);
  auto full_bar = [&](int s) { return bar0 + 8u * s; };
  auto empty_bar = [&](int s) { return bar0 + 8u * (GSTAGES + s); };
  auto tfull_bar = [&](int b) { return bar0 + 8u * (2 * GSTAGES + b); };
  auto tempty_bar = [&](int b) { return bar0 + 8u * (2 * GSTAGES + 2 + b); };
  const uint32_t drain_bar = bar0 + 8u * (2 * GSTAGES + 4);

  if (threadIdx.x == 0) {
    for (int s = 0; s < GSTAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull_bar(b), 1);
      mbar_init(tempty_bar(b), 32 * GEPI_WARPS);
    }
    mbar_init(drain_bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const int total = ka.m_tiles * ka.n_tiles;
  const uint32_t stage_tx = (uint32_t)(GA_BYTES + ka.n_tile * GK * 2);

  if (warp == 0 && lane == 0) {
    int stage = 0, issued = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
      const int nt = t / ka.m_tiles, mt = t - (t / ka.m_tiles) * ka.m_tiles;
      for (int kc = 0; kc < ka.k_chunks; ++kc) {
        if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, g.status)) {
          ok = false;
          break;
        }
        const uint32_t base = smem_u32(smem + stage * GSTAGE);
        mbar_arrive_expect_tx(full_bar(stage), stage_tx);
        tma_load_2d(base, &mapA, kc * GK, mt * GM, full_bar(stage));
        tma_load_2d(base + GA_BYTES, &mapB, kc * GK, nt * ka.n_tile, full_bar(stage));
        ++issued;
        if (++stage == GSTAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
    if (!ok) {
      for (int k = 0; k < GSTAGES && k < issued; ++k) {
        if (--stage < 0) {
          stage = GSTAGES - 1;
          phase ^= 1u;
        }
        mbar_drain_wait(full_bar(stage), phase);
      }
    }
  } else if (warp == 1 && lane == 0) {
    int stage = 0, acc = 0;
    uint32_t phase = 0, acc_phase = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
      if (!mbar_wait(tempty_bar(acc), acc_phase ^ 1u, abort_flag, g.status)) break;
      tmem_fence_after();
      const uint32_t d_tmem = tmem_base + (uint32_t)(acc * 256);
      for (int kc = 0; kc < ka.k_chunks; ++kc) {
        if (!mbar_wait(full_bar(stage), phase, abort_flag, g.status)) {
          ok = false;
          break;
        }
        tmem_fence_after();
        const uint32_t base = smem_u32(smem + stage * GSTAGE);
        const uint64_t da = smem_desc<128>(base), db = smem_desc<128>(base + GA_BYTES);
#pragma unroll
        for (int k = 0; k < GK / 16; ++k) {
          const uint64_t adv = (uint64_t)((k * 32) >> 4);
          mma_f16(d_tmem, da + adv, db + adv, ka.idesc, (kc == 0 && k == 0) ? 0u : 1u);
        }
        mma_commit(empty_bar(stage));
        if (++stage == GSTAGES) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (!ok) break;
      mma_commit(tfull_bar(acc));
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1u;
      }
    }
    mma_commit(drain_bar);
    mbar_drain_wait(drain_bar, 0);
  } else if (warp >= 2) {
    // epilogue: warp (quad, part) reads the 16-column chunks part, part + 4, ..
    // of its lane quarter (four warps per quarter hide the latency of the
    // activation arithmetic and the row-wise stores)
    const int quad = warp & 3, part = (warp - 2) >> 2;
    const int row = quad * 32 + lane;
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
      int okw = 1;
      if (lane == 0) okw = mbar_wait(tfull_bar(acc), acc_phase, abort_flag, g.status) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) break;
      tmem_fence_after();
      const int nt = t / ka.m_tiles, mt = t - (t / ka.m_tiles) * ka.m_tiles;
      const int m = mt * GM + row;
      const bool mok = m < g.M;
      const uint32_t tbase = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * 256);
      for (int c0 = part * GCH; c0 < ka.n_tile; c0 += 4 * GCH) {
        uint32_t r[GCH];
        tmem_ld16(tbase + (uint32_t)c0, r);
        const int n0 = nt * ka.n_tile + c0;
        if (n0 >= g.N) continue;                    // the same for the whole warp
        const bool full = n0 + GCH <= g.N;
        float* ow = g.out ? g.out + n0 : nullptr;
        if ((g.epi == EPI_LINEAR || g.epi == EPI_STORE) && full && (g.ldo & 3) == 0 &&
            ((uintptr_t)ow & 15) == 0) {
          // FP32 output through the warp's staging rows
          float* st = gstg + (warp - 2) * 32 * GSTG_LD;
          // the row's complex factor applies to (re, im) column pairs (n0 even)
          const bool rp_ok = g.row_phase != nullptr && mok;
          const float2 e_row = rp_ok ? g.row_phase[m] : make_float2(1.f, 0.f);
          float bias[GCH];
          if (g.epi == EPI_LINEAR) load_bias(g, n0, true, bias);
#pragma unroll
          for (int q = 0; q < GCH / 4; ++q) {
            float4 w = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                   __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
            if (g.epi == EPI_LINEAR) {
              w.x += bias[4 * q];
              w.y += bias[4 * q + 1];
              w.z += bias[4 * q + 2];
              w.w += bias[4 * q + 3];
              if (rp_ok) w = cmul2(w, e_row);
            }
            ((float4*)(st + lane * GSTG_LD))[q] = w;
          }
          __syncwarp();
          const int m0 = mt * GM + quad * 32;
#pragma unroll
          for (int it = 0; it < 4; ++it) {
            const int rr = it * 8 + (lane >> 2), q = lane & 3;
            if (m0 + rr < g.M)
              ((float4*)(ow + (size_t)(m0 + rr) * g.ldo))[q] =
                  ((const float4*)(st + rr * GSTG_LD))[q];
          }
          __syncwarp();
          continue;
        }
        if (!mok) continue;
        if (g.epi == EPI_HIDDEN || g.epi == EPI_DSILU) {
          uint16_t v16[GCH], z16[GCH];
          if (g.epi == EPI_DSILU) {
            const uint16_t* zp = g.Z + (size_t)m * g.ldz + n0;
            if (full) {
#pragma unroll
              for (int q = 0; q < GCH / 8; ++q) {
                const uint4 w = ((const uint4*)zp)[q];
                const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                  z16[8 * q + 2 * h] = (uint16_t)(ww[h] & 0xFFFFu);
                  z16[8 * q + 2 * h + 1] = (uint16_t)(ww[h] >> 16);
                }
              }
            } else {
#pragma unroll
              for (int j = 0; j < GCH; ++j) z16[j] = n0 + j < g.N ? zp[j] : (uint16_t)0;
            }
          }
          float bias[GCH];
          if (g.epi == EPI_HIDDEN) load_bias(g, n0, full, bias);
          // the logistic through the fast exp and reciprocal: its FP32 error
          // (a few ulp) is far below the BF16 rounding that follows
#pragma unroll
          for (int j = 0; j < GCH; ++j) {
            const float a = __uint_as_float(r[j]);
            if (g.epi == EPI_HIDDEN) {
              const uint16_t zb = f2bf(a + bias[j]);
              const float zr = bf2f(zb);
              z16[j] = zb;
              v16[j] = f2bf(zr * __frcp_rn(1.f + __expf(-zr)));   // SiLU of the stored z
            } else {
              const float z = bf2f(z16[j]);
              const float sg = __frcp_rn(1.f + __expf(-z));
              v16[j] = f2bf(a * sg * (1.f + z * (1.f - sg)));
            }
          }
          uint16_t* yp = g.Y + (size_t)m * g.ldy + n0;
          if (full) {
#pragma unroll
            for (int q = 0; q < GCH / 8; ++q)
              ((uint4*)yp)[q] = make_uint4(
                  (uint32_t)v16[8 * q] | ((uint32_t)v16[8 * q + 1] << 16),
                  (uint32_t)v16[8 * q + 2] | ((uint32_t)v16[8 * q + 3] << 16),
                  (uint32_t)v16[8 * q + 4] | ((uint32_t)v16[8 * q + 5] << 16),
                  (uint32_t)v16[8 * q + 6] | ((uint32_t)v16[8 * q + 7] << 16));
            if (g.epi == EPI_HIDDEN && g.Z) {
              uint16_t* zp = g.Z + (size_t)m * g.ldz + n0;
#pragma unroll
              for (int q = 0; q < GCH / 8; ++q)
                ((uint4*)zp)[q] = make_uint4(
                    (uint32_t)z16[8 * q] | ((uint32_t)z16[8 * q + 1] << 16),
                    (uint32_t)z16[8 * q + 2] | ((uint32_t)z16[8 * q + 3] << 16),
                    (uint32_t)z16[8 * q + 4] | ((uint32_t)z16[8 * q + 5] << 16),
                    (uint32_t)z16[8 * q + 6] | ((uint32_t)z16[8 * q + 7] << 16));
            }
          } else {
#pragma unroll
            for (int j = 0; j < GCH; ++j)
              if (n0 + j < g.N) {
                yp[j] = v16[j];
                if (g.epi == EPI_HIDDEN && g.Z) g.Z[(size_t)m * g.ldz + n0 + j] = z16[j];
              }
          }
          if (g.YT) {
#pragma unroll
            for (int j = 0; j < GCH; ++j)
              if (n0 + j < g.N) g.YT[(size_t)(n0 + j) * g.ldyt + m] = v16[j];
          }
        } else {
          float* op = g.out + (size_t)m * g.ldo + n0;
          float v[GCH], bias[GCH];
          if (g.epi == EPI_LINEAR) load_bias(g, n0, full, bias);
#pragma unroll
          for (int j = 0; j < GCH; ++j) {
            v[j] = __uint_as_float(r[j]);
            if (g.epi == EPI_LINEAR) v[j] += bias[j];
          }
          if (g.epi == EPI_LINEAR && g.row_phase) {
            const float2 e = g.row_phase[m];
#pragma unroll
            for (int j = 0; j < GCH; j += 2) {
              const float re = v[j] * e.x - v[j + 1] * e.y;
              v[j + 1] = v[j] * e.y + v[j + 1] * e.x;
              v[j] = re;
            }
          }
          if (full && (g.ldo & 3) == 0) {
#pragma unroll
            for (int q = 0; q < GCH / 4; ++q)
              ((float4*)op)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < GCH; ++j)
              if (n0 + j < g.N) op[j] = v[j];
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
                 "r"(512)
                 : "memory");
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t,
                                  void*, const cuuint64_t*, const cuuint64_t*,
                                  const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
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

bool make_map(CUtensorMap* m, const uint16_t* base, int K, int rows, int ld,
              int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)GK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, (void*)base, dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace

int gemm(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.K <= 0) return PSF_ERR_ARG;
  if ((g.lda & 7) || (g.ldb & 7) || (g.N % 16 && g.N > 256)) return PSF_ERR_ARG;
  KArgs ka;
  memset(&ka, 0, sizeof(ka));
  ka.g = g;
  ka.n_tile = g.N >= GNMAX ? GNMAX : (g.N + 15) / 16 * 16;
  ka.m_tiles = ceil_div(g.M, GM);
  ka.n_tiles = ceil_div(g.N, ka.n_tile);
  ka.k_chunks = ceil_div(g.K, GK);
  // kind::f16, BF16 A and B (format 1), FP32 D, K-major, N >> 3, M >> 4
  ka.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(ka.n_tile >> 3) << 17) |
             ((uint32_t)(GM >> 4) << 24);
  CUtensorMap mA, mB;
  if (!make_map(&mA, g.A, g.K, g.M, g.lda, GM) ||
      !make_map(&mB, g.B, g.K, g.N, g.ldb, ka.n_tile))
    return PSF_ERR_CUDA;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             GSMEM) != cudaSuccess)
      return PSF_ERR_CUDA;
    attr = true;
  }
  const int total = ka.m_tiles * ka.n_tiles;
  const int grid = total < num_sms() ? total : num_sms();
  k_gemm_bf16<<<grid, GTHREADS, GSMEM, s>>>(mA, mB, ka);
  return cudaPeekAtLastError() == cudaSuccess ? PSF_OK : PSF_ERR_CUDA;
}

}  // namespace mlp
}  // namespace psf
