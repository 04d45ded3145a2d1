// Chirp-Z stage 2: the zoom along x for every output column, three field
// channels, intensity sum_c |E_c|^2 (and the fields on request).  Each
// thread carries two adjacent output columns (b, b + 1) through the paired
// FFT; CS channel slots of a column pair run side by side (CS = 3) or in
// turn (CS = 1, the longest FFT).  A CTA walks a group of z-planes and, where
// shared memory allows, prefetches the next item's input rows with cp.async
// while the current one is transformed.  The FFT passes synchronise one
// barrier group (the warps of one slot); only the channel sum of CS = 3,
// which reads the three channel slots, synchronises the CTA.
#include "czt_fft.cuh"

namespace psf {
namespace {

using namespace czt;

PSF_D void cp_async8(void* dst, const void* src, int bytes) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(bytes)
               : "memory");
}
PSF_D void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
PSF_D void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// CS channel slots, CP column pairs per CTA (about 192 threads below L = 2048)
template <int L, int NIN>
struct Stage2Shape {
  static constexpr int T = L / 16;
  static constexpr int CS = L <= 2048 ? 3 : 1;
  static constexpr int CP = T * 3 * 4 <= 192 ? 4 : (T * 3 * 2 <= 192 ? 2 : 1);
  using S = Shape<L, CS * CP, 1>;
  // shared after the FFT buffers: acc [SLOTS][L] float2 (CS = 1 only),
  // staging [SLOTS][NIN][T] 16-byte elements (prefetch only), post^x [nx]
  static constexpr size_t ACC = CS == 1 ? (size_t)S::SLOTS * L * 8 : 0;
  static constexpr size_t STG = (size_t)S::SLOTS * NIN * T * 16;
  static constexpr bool PREFETCH = S::SMEM + ACC + STG + (size_t)L * 8 <= 227 * 1024;
  static constexpr size_t FIXED = S::SMEM + ACC + (PREFETCH ? STG : 0);
};

// grid (ceil(ny / (2 CP)) column blocks, z-groups of zg planes); slot = cs CP + cp
template <int L, int NIN>
__global__ void __launch_bounds__(Stage2Shape<L, NIN>::S::THREADS,
                                  Stage2Shape<L, NIN>::S::THREADS <= 192 ? 2 : 1)
k_czt_stage2(const float2* __restrict__ Tin, int N, int nx, int ny, int nzc, int zg,
             CztDir cx, float* __restrict__ I, float2* __restrict__ F) {
  using G = Stage2Shape<L, NIN>;
  using S = typename G::S;
  constexpr int CS = G::CS, CP = G::CP, T = S::T;
  extern __shared__ float4 sm4[];
  float2* tab = reinterpret_cast<float2*>(sm4);
  char* tail = reinterpret_cast<char*>(sm4 + S::TAB4 + S::SLOTS * S::STRIDE);
  float2* acc_all = reinterpret_cast<float2*>(tail);
  float4* stg_all = reinterpret_cast<float4*>(tail + G::ACC);
  float2* post = reinterpret_cast<float2*>(tail + G::ACC + (G::PREFETCH ? G::STG : 0));
  int slot, t;
  lane_split<S>(threadIdx.x, &slot, &t);
  const int cs = slot / CP, cp = slot % CP;
  float4* buf = sm4 + S::TAB4 + slot * S::STRIDE;
  float4* stg = stg_all + (size_t)slot * NIN * T;
  float2* acc = acc_all + (size_t)slot * L;
  const int b = (blockIdx.x * CP + cp) * 2;   // columns b (A) and b + 1 (B)
  const bool okA = b < ny, okB = b + 1 < ny;
  load_tables<S>(cx, tab);
  for (int i = threadIdx.x; i < nx; i += S::THREADS) post[i] = cx.post[i];
  __syncthreads();
  const int zb = blockIdx.z * zg, ze = min(zb + zg, nzc);
  // items: (plane, channel) with channel = cs (CS = 3) or 0, 1, 2 (CS = 1)
  const int per = 3 / CS, n_items = (ze - zb) * per;
  auto row_of = [&](int it) {
    const int zc = zb + it / per, c = CS == 3 ? cs : it % per;
    return Tin + ((size_t)(zc * 3 + c) * ny + b) * N;
  };
  auto prefetch = [&](int it) {
    const float2* src = row_of(it);
#pragma unroll
    for (int r = 0; r < NIN; ++r) {
      const int p = t + T * r;
      const bool in = p < N;
      float4* d = stg + r * T + t;
      cp_async8(d, in && okA ? src + p : Tin, in && okA ? 8 : 0);
      cp_async8(reinterpret_cast<char*>(d) + 8, in && okB ? src + N + p : Tin,
                in && okB ? 8 : 0);
    }
    cp_async_commit();
  };
  if constexpr (G::PREFETCH) {
    if (n_items > 0) prefetch(0);
  }
  for (int it = 0; it < n_items; ++it) {
    const int zc = zb + it / per, c = CS == 3 ? cs : it % per;
    c2 v[16];
    if constexpr (G::PREFETCH) {
      cp_async_wait_all();   // this thread's own copies; it alone reads them
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        if (r < NIN) {
          const float4 f = stg[r * T + t];
          v[r] = c2{make_float2(f.x, f.z), make_float2(f.y, f.w)};
        } else {
          v[r] = c2{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        }
      }
    } else {
      const float2* src = row_of(it);
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int p = t + T * r;
        float2 xa = make_float2(0.f, 0.f), xb = xa;
        if (r < NIN && p < N) {
          if (okA) xa = src[p];
          if (okB) xb = src[N + p];
        }
        v[r] = c2{make_float2(xa.x, xb.x), make_float2(xa.y, xb.y)};
      }
    }
    fft_block<S, NIN>(v, buf, tab, t);
    // the staged values went through a barrier above: refill the stage
    if constexpr (G::PREFETCH) {
      if (it + 1 < n_items) prefetch(it + 1);
    }
    {
      const float2* Hc = tab + kCztTw2 + kCztTwL;
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = conj_mulw(v[r], Hc[t + T * r]);
    }
    fft_block<S, 16>(v, buf, tab, t);
    float2* fo = F ? F + (size_t)(zc * 3 + c) * nx * ny + b : nullptr;
    float2* red = reinterpret_cast<float2*>(buf);
    if constexpr (CS == 3) group_sync<S>();   // the last pass has read buf
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int a = t + T * r;
      if (a < nx) {
        const float2 pa = post[a];
        const float2 ea = cmul(make_float2(v[r].re.x, -v[r].im.x), pa);
        const float2 eb = cmul(make_float2(v[r].re.y, -v[r].im.y), pa);
        const float2 pw = make_float2(fmaf(ea.x, ea.x, ea.y * ea.y),
                                      fmaf(eb.x, eb.x, eb.y * eb.y));
        if constexpr (CS == 3) {
          red[a] = pw;
        } else {
          const float2 prev = c == 0 ? make_float2(0.f, 0.f) : acc[a];
          acc[a] = make_float2(prev.x + pw.x, prev.y + pw.y);
        }
        if (fo && okA) {
          fo[(size_t)a * ny] = ea;
          if (okB) fo[(size_t)a * ny + 1] = eb;
        }
      }
    }
    if (it % per != per - 1) continue;   // CS = 1: more channels of this plane
    if constexpr (CS == 3) __syncthreads();   // the three channel slots are written
    if (cs == 0 && okA) {
      float* io = I + (size_t)zc * nx * ny + b;
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int a = t + T * r;
        if (a < nx) {
          float2 s;
          if constexpr (CS == 3) {
            const float2* r0 = reinterpret_cast<const float2*>(sm4 + S::TAB4 + cp * S::STRIDE);
            const float2* r1 = reinterpret_cast<const float2*>(sm4 + S::TAB4 +
                                                               (CP + cp) * S::STRIDE);
            const float2* r2 = reinterpret_cast<const float2*>(sm4 + S::TAB4 +
                                                               (2 * CP + cp) * S::STRIDE);
            s = make_float2(r0[a].x + r1[a].x + r2[a].x, r0[a].y + r1[a].y + r2[a].y);
          } else {
            s = acc[a];
          }
          io[(size_t)a * ny] = s.x;
          if (okB) io[(size_t)a * ny + 1] = s.y;
        }
      }
    }
    // the channel slots read above are rewritten by the next item's FFT,
    // whose barriers span one group only
    if constexpr (CS == 3) __syncthreads();
  }
  if constexpr (G::PREFETCH) cp_async_wait_all();
}

// planes per CTA: enough CTAs for about four waves of two per SM
inline int z_group(int base_ctas, int nzc) {
  const int want = 152 * 2 * 4;
  int groups = (want + base_ctas - 1) / base_ctas;
  if (groups > nzc) groups = nzc;
  if (groups < 1) groups = 1;
  return (nzc + groups - 1) / groups;
}

template <int L, int NIN>
void launch(const float2* T, int N, int nx, int ny, int nzc, const CztDir& cx, float* I,
            float2* F, cudaStream_t s) {
  using G = Stage2Shape<L, NIN>;
  const size_t smem = G::FIXED + (size_t)nx * sizeof(float2);
  cudaFuncSetAttribute(k_czt_stage2<L, NIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  const int cols = ceil_div(ny, 2 * G::CP);
  const int zg = z_group(cols, nzc);
  const dim3 grid(cols, 1, ceil_div(nzc, zg));
  k_czt_stage2<L, NIN><<<grid, G::S::THREADS, smem, s>>>(T, N, nx, ny, nzc, zg, cx, I, F);
}

template <int L>
void launch_nin(const float2* T, int N, int nx, int ny, int nzc, const CztDir& cx,
                float* I, float2* F, cudaStream_t s) {
  switch (czt_nin<typename Stage2Shape<L, 16>::S>(N)) {
    case 4: launch<L, 4>(T, N, nx, ny, nzc, cx, I, F, s); break;
    case 8: launch<L, 8>(T, N, nx, ny, nzc, cx, I, F, s); break;
    default: launch<L, 16>(T, N, nx, ny, nzc, cx, I, F, s); break;
  }
}

}  // namespace

void launch_czt_stage2(const float2* T, int N, int nx, int ny, int nzc, const CztDir& cx,
                       float* I, float2* fields, cudaStream_t s) {
  switch (cx.L) {
    case 256: launch_nin<256>(T, N, nx, ny, nzc, cx, I, fields, s); break;
    case 512: launch_nin<512>(T, N, nx, ny, nzc, cx, I, fields, s); break;
    case 1024: launch_nin<1024>(T, N, nx, ny, nzc, cx, I, fields, s); break;
    case 2048: launch_nin<2048>(T, N, nx, ny, nzc, cx, I, fields, s); break;
    default: launch_nin<4096>(T, N, nx, ny, nzc, cx, I, fields, s); break;
  }
}

}  // namespace psf
