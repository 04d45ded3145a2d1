// Chirp-Z stage 1: the zoom along y for every pupil row, with the pupil
// field of Eq. 8 / Eq. 12 formed from the node table on the fly.  Each
// thread carries two adjacent pupil rows (p, p + 1) through the paired FFT;
// a CTA walks a group of z-planes, so after the first plane its node reads
// hit L1.
#include "czt_fft.cuh"

namespace psf {
namespace {

using namespace czt;

// pupil value of node idx at defocus z, with the y pre-chirp (cycles)
PSF_D float2 pupil_node(const NodeTable& nt, const float* amp_re, const float* amp_im,
                        size_t idx, float pre_cyc, f2x z) {
  const f2x kap = {__ldg(nt.kh + idx), __ldg(nt.kl + idx)};
  const float ph = frac_mul_add(kap, z, __ldg(nt.wfr + idx) + pre_cyc);
  return cmul(make_float2(__ldg(amp_re + idx), __ldg(amp_im + idx)), cis_cycles(ph));
}

// grid (ceil(N / (2 SLOTS)) row blocks, 3 channels, z-groups of zg planes);
// QL = 2 pairs interleaved per warp, so the stores (rows p .. p + 3) fill
// 32-byte sectors; the node reads run along q.  Shared: tables, buffers,
// then post^y [ny] and pre_cyc^y [N].
template <class S, int NIN>
__global__ void __launch_bounds__(S::THREADS, 512 / S::THREADS)
k_czt_stage1(NodeTable nt, int N, const float2* __restrict__ zz, int z0, int nzc, int zg,
             CztDir cx, CztDir cy, int ny, float2* __restrict__ Tout) {
  extern __shared__ float4 sm4[];
  float2* tab = reinterpret_cast<float2*>(sm4);
  float2* post = reinterpret_cast<float2*>(sm4 + S::TAB4 + S::SLOTS * S::STRIDE);
  float* pre_cyc = reinterpret_cast<float*>(post + ny);
  int slot, t;
  lane_split<S>(threadIdx.x, &slot, &t);
  float4* buf = sm4 + S::TAB4 + slot * S::STRIDE;
  const int p = (blockIdx.x * S::SLOTS + slot) * 2;   // rows p (A) and p + 1 (B)
  const bool okA = p < N, okB = p + 1 < N;
  const int c = blockIdx.y;
  load_tables<S>(cy, tab);
  for (int i = threadIdx.x; i < ny; i += S::THREADS) post[i] = cy.post[i];
  for (int i = threadIdx.x; i < N; i += S::THREADS) pre_cyc[i] = cy.pre_cyc[i];
  __syncthreads();
  const size_t NN = (size_t)N * N;
  const float* amp_re = nt.amp + (2 * c) * NN;
  const float* amp_im = nt.amp + (2 * c + 1) * NN;
  const size_t rowA = (size_t)p * N, rowB = rowA + N;
  const float2 wa = okA ? cx.pre[p] : make_float2(0.f, 0.f);
  const float2 wb = okB ? cx.pre[p + 1] : make_float2(0.f, 0.f);
  const int zb = blockIdx.z * zg, ze = min(zb + zg, nzc);
  for (int zc = zb; zc < ze; ++zc) {
    const float2 zv = zz[z0 + zc];
    const f2x z = {zv.x, zv.y};
    c2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int q = t + S::T * r;
      float2 xa = make_float2(0.f, 0.f), xb = xa;
      if (r < NIN && q < N) {
        const float pc = pre_cyc[q];
        if (okA) xa = pupil_node(nt, amp_re, amp_im, rowA + q, pc, z);
        if (okB) xb = pupil_node(nt, amp_re, amp_im, rowB + q, pc, z);
      }
      v[r] = c2{make_float2(xa.x, xb.x), make_float2(xa.y, xb.y)};
    }
    convolve<S, NIN>(v, buf, tab, t);
    if (okA) {
      float2* out = Tout + (size_t)(zc * 3 + c) * ny * N + p;
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int b = t + S::T * r;
        if (b < ny) {
          const float2 pb = post[b];
          float2* o = out + (size_t)b * N;
          o[0] = cmul(cmul(make_float2(v[r].re.x, -v[r].im.x), pb), wa);
          if (okB) o[1] = cmul(cmul(make_float2(v[r].re.y, -v[r].im.y), pb), wb);
        }
      }
    }
  }
}

template <int L>
using Shape1 = Shape<L, (256 / (L / 16) < 8 ? (256 / (L / 16) > 1 ? 256 / (L / 16) : 1) : 8),
                     (256 / (L / 16) >= 2 ? 2 : 1)>;

// planes per CTA: enough CTAs for about four waves of two per SM
inline int z_group(int base_ctas, int nzc) {
  const int want = 152 * 2 * 4;
  int groups = (want + base_ctas - 1) / base_ctas;
  if (groups > nzc) groups = nzc;
  if (groups < 1) groups = 1;
  return (nzc + groups - 1) / groups;
}

template <class S, int NIN>
void launch(NodeTable nt, int N, const float2* zz, int z0, int nzc, const CztDir& cx,
            const CztDir& cy, int ny, float2* T, cudaStream_t s) {
  const size_t smem = S::SMEM + (size_t)ny * sizeof(float2) + (size_t)N * sizeof(float);
  cudaFuncSetAttribute(k_czt_stage1<S, NIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  const int rows = ceil_div(N, 2 * S::SLOTS);
  const int zg = z_group(rows * 3, nzc);
  const dim3 grid(rows, 3, ceil_div(nzc, zg));
  k_czt_stage1<S, NIN><<<grid, S::THREADS, smem, s>>>(nt, N, zz, z0, nzc, zg, cx, cy, ny, T);
}

template <int L>
void launch_nin(NodeTable nt, int N, const float2* zz, int z0, int nzc, const CztDir& cx,
                const CztDir& cy, int ny, float2* T, cudaStream_t s) {
  using S = Shape1<L>;
  switch (czt_nin<S>(N)) {
    case 4: launch<S, 4>(nt, N, zz, z0, nzc, cx, cy, ny, T, s); break;
    case 8: launch<S, 8>(nt, N, zz, z0, nzc, cx, cy, ny, T, s); break;
    default: launch<S, 16>(nt, N, zz, z0, nzc, cx, cy, ny, T, s); break;
  }
}

}  // namespace

void launch_czt_stage1(NodeTable t, int N, const float2* zz, int z0, int nzc,
                       const CztDir& cx, const CztDir& cy, int ny, float2* T,
                       cudaStream_t s) {
  switch (cy.L) {
    case 256: launch_nin<256>(t, N, zz, z0, nzc, cx, cy, ny, T, s); break;
    case 512: launch_nin<512>(t, N, zz, z0, nzc, cx, cy, ny, T, s); break;
    case 1024: launch_nin<1024>(t, N, zz, z0, nzc, cx, cy, ny, T, s); break;
    case 2048: launch_nin<2048>(t, N, zz, z0, nzc, cx, cy, ny, T, s); break;
    default: launch_nin<4096>(t, N, zz, z0, nzc, cx, cy, ny, T, s); break;
  }
}

}  // namespace psf
