// Surrogate profiles with the Bessel path as fallback: the MLP answers every
// query, its error head flags the queries whose predicted relative error is
// above the caller's bound, and those are recomputed by psf_bessel_vectorial
// (profiles only) and scattered back into the output.
#include <math.h>
#include <string.h>

#include "mlp_kernels.cuh"
#include "timing.cuh"

namespace psf {
void set_last_error(const char* msg);
void psf_axis_path_cycles(const psf_optics* o, double* a0, double* a1);
void psf_axis_zernike(int n_zern, double* z0);
}

namespace {

using namespace psf;

constexpr int kNR = 256;     // radii of the surrogate's profiles (1536 = 3 x 256 x 2)

__global__ void k_flag(const float* __restrict__ errp, int B, float thr_log10, int* idx,
                       int* count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  if (!(errp[b] <= thr_log10)) idx[atomicAdd(count, 1)] = b;   // NaN -> fallback
}

__global__ void k_gather(const float* __restrict__ q, const int* __restrict__ idx, int n,
                         double* depth, double* zern, int* offs, double* z) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > n) return;
  offs[k] = k;
  if (k == n) return;
  const float* qb = q + (size_t)idx[k] * mlp::IN;
  for (int j = 0; j < 21; ++j) zern[(size_t)k * 21 + j] = qb[j];
  depth[k] = qb[21];
  z[k] = qb[22];
}

__global__ void k_scatter(const float* __restrict__ prof, const int* __restrict__ idx, int n,
                          float* out) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)n * mlp::OUT) return;
  const int k = (int)(i / mlp::OUT), e = (int)(i - (long long)k * mlp::OUT);
  out[(size_t)idx[k] * mlp::OUT + e] = prof[i];
}

// The profiles' on-axis phase (theta = 0 in Eq. 10-11): Gibson-Lanni path
// (Eq. 13) a0 + a1 t_s and the m = 0 Zernike terms at rho = 0 (Eq. 15) of the
// pupil, plus the defocus n_i z / lambda, in cycles.  The network learns the
// profiles with this phase divided out (a smoother function of z and t_s);
// k_axis_phase multiplies [B][3 x 256] complex values by e^{dir 2 pi i phi}.
struct AxisPhase {
  double a0, a1, n_over_lambda;
  double z0[21];
};

PSF_D float2 axis_phasor(const float* __restrict__ qb, const AxisPhase& ap, int dir) {
  double cyc = ap.a0 + ap.a1 * (double)qb[21] + ap.n_over_lambda * (double)qb[22];
  double zs = 0.0;
  for (int j = 0; j < 21; ++j) zs += ap.z0[j] * (double)qb[j];
  cyc += zs * (0.5 / 3.14159265358979323846);
  cyc -= rint(cyc);
  double sn, cs;
  sincospi(2.0 * cyc, &sn, &cs);
  return make_float2((float)cs, (float)(dir > 0 ? sn : -sn));
}

// e^{dir 2 pi i phi} of each query, one thread per query (FP64 phase
// reduced mod 1 cycle, then the FP64 sincospi)
__global__ void k_axis_phasor(const float* __restrict__ q, int B, AxisPhase ap, int dir,
                              float2* ph) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  ph[b] = axis_phasor(q + (size_t)b * mlp::IN, ap, dir);
}

// data [B][768] complex times the phasor of its query: 16 queries per block,
// their phasors computed in parallel into shared memory first
constexpr int kRowsPerBlock = 16;
__global__ void __launch_bounds__(256)
k_rows_phase(const float* __restrict__ q, int B, AxisPhase ap, int dir, float4* data) {
  __shared__ float2 ph[kRowsPerBlock];
  const int b0 = blockIdx.x * kRowsPerBlock;
  if (threadIdx.x < kRowsPerBlock && b0 + threadIdx.x < B)
    ph[threadIdx.x] = axis_phasor(q + (size_t)(b0 + threadIdx.x) * mlp::IN, ap, dir);
  __syncthreads();
  const int nb = min(kRowsPerBlock, B - b0);
  constexpr int PER = mlp::OUT / 4;                       // float4 per query
  float4* d = data + (size_t)b0 * PER;
  for (int i = threadIdx.x; i < nb * PER; i += blockDim.x) {
    const float2 e = ph[i / PER];
    const float4 w = d[i];
    d[i] = make_float4(w.x * e.x - w.y * e.y, w.x * e.y + w.y * e.x,
                       w.z * e.x - w.w * e.y, w.z * e.y + w.w * e.x);
  }
}

AxisPhase axis_phase(const psf_optics* o) {
  AxisPhase ap;
  psf_axis_path_cycles(o, &ap.a0, &ap.a1);
  ap.n_over_lambda = o->n_i / o->lambda;
  psf_axis_zernike(21, ap.z0);
  return ap;
}

struct SurLayout {
  size_t mlp_ws, bessel_ws;
  int* idx;
  int* count;
  float* errp;
  double *depth, *zern, *z;
  int* offs;
  float* prof;
  float2* phase;
  char* mlp;
  char* bessel;
  size_t bytes;
};

SurLayout sur_layout(void* base, const psf_optics* opt, int B, int n_theta, int nx, int ny,
                     int precision) {
  SurLayout L;
  memset(&L, 0, sizeof(L));
  char* b = (char*)base;
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    off = align_up(off, 1024);
    char* p = b ? b + off : nullptr;
    off += bytes;
    return p;
  };
  L.mlp_ws = psf_mlp_workspace_size(B);
  L.bessel_ws = psf_bessel_workspace_size(opt, B, B, n_theta, kNR, nx, ny, precision);
  L.mlp = take(L.mlp_ws);
  L.idx = (int*)take((size_t)B * 4);
  L.count = (int*)take(4);
  L.errp = (float*)take((size_t)B * 4);
  L.depth = (double*)take((size_t)B * 8);
  L.zern = (double*)take((size_t)B * 21 * 8);
  L.z = (double*)take((size_t)B * 8);
  L.offs = (int*)take((size_t)(B + 1) * 4);
  L.prof = (float*)take((size_t)B * mlp::OUT * 4);
  L.phase = (float2*)take((size_t)B * 8);
  L.bessel = take(L.bessel_ws);
  L.bytes = align_up(off, 256);
  return L;
}

}  // namespace

extern "C" size_t psf_surrogate_workspace_size(const psf_optics* base, int batch,
                                               int n_theta, int nx, int ny, int precision) {
  if (batch < 1 || batch > (1 << 20)) return 0;
  const SurLayout L = sur_layout(nullptr, base, batch, n_theta, nx, ny, precision);
  if (!L.mlp_ws || !L.bessel_ws) return 0;
  return L.bytes;
}

extern "C" int psf_surrogate_profiles(const void* state, const psf_optics* base,
                                      const float* query, int batch, double max_rel_err,
                                      int n_theta, int nx, int ny, double dx, double dy,
                                      int precision, float* out, int* n_fallback, void* ws,
                                      size_t ws_bytes, void* stream) {
  if (!state || !base || !query || !out || !ws) {
    set_last_error("surrogate: NULL pointer");
    return PSF_ERR_ARG;
  }
  if (!(max_rel_err > 0)) {
    set_last_error("surrogate: max_rel_err must be > 0");
    return PSF_ERR_ARG;
  }
  const size_t need = psf_surrogate_workspace_size(base, batch, n_theta, nx, ny, precision);
  if (!need) return PSF_ERR_ARG;
  if (ws_bytes < need) {
    set_last_error("surrogate: workspace too small");
    return PSF_ERR_WORKSPACE;
  }
  const SurLayout L = sur_layout(ws, base, batch, n_theta, nx, ny, precision);
  cudaStream_t s = (cudaStream_t)stream;
  // the MLP answers all queries; its error head gives log10(rel. error)
  float* errp = L.errp;
  // the network's profiles carry the on-axis phase divided out: the output
  // layer's epilogue restores it row by row
  k_axis_phasor<<<ceil_div(batch, 256), 256, 0, s>>>(query, batch, axis_phase(base), 1,
                                                     L.phase);
  int r = mlp::forward_rows(state, query, batch, out, errp, L.mlp, L.mlp_ws, L.phase, stream);
  if (r) return r;
  cudaMemsetAsync(L.count, 0, 4, s);
  // accept a prediction only if twice its predicted error is within the bound
  k_flag<<<ceil_div(batch, 256), 256, 0, s>>>(errp, batch,
                                              (float)(log10(max_rel_err) - log10(2.0)),
                                              L.idx, L.count);
  int h = 0;
  if (cudaMemcpyAsync(&h, L.count, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    set_last_error("surrogate: reading the fallback count failed");
    return PSF_ERR_CUDA;
  }
  if (n_fallback) *n_fallback = h;
  if (h > 0) {
    k_gather<<<ceil_div(h + 1, 256), 256, 0, s>>>(query, L.idx, h, L.depth, L.zern, L.offs,
                                                  L.z);
    psf_optics o = *base;
    o.flags |= PSF_PROJECT_AXISYMMETRIC;
    r = psf_bessel_vectorial(&o, h, L.depth, L.zern, 21, nullptr, L.offs, L.z, h, n_theta, kNR, nx,
                             ny, dx, dy, precision, nullptr, L.prof, L.bessel, L.bessel_ws,
                             stream);
    if (r) return r;
    const long long n = (long long)h * mlp::OUT;
    k_scatter<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(L.prof, L.idx, h, out);
  }
  if (cudaPeekAtLastError() != cudaSuccess) {
    set_last_error("surrogate: launch failed");
    return PSF_ERR_CUDA;
  }
  return PSF_OK;
}

extern "C" int psf_surrogate_phase(const psf_optics* base, const float* query, int batch,
                                   float* data, int direction, void* stream) {
  if (!base || !query || !data) {
    set_last_error("surrogate phase: NULL pointer");
    return PSF_ERR_ARG;
  }
  if (batch < 0 || batch > (1 << 20) || (direction != 1 && direction != -1)) {
    set_last_error("surrogate phase: batch outside [0, 1048576] or direction not +-1");
    return PSF_ERR_ARG;
  }
  if (batch == 0) return PSF_OK;
  k_rows_phase<<<ceil_div(batch, kRowsPerBlock), 256, 0, (cudaStream_t)stream>>>(
      query, batch, axis_phase(base), direction, (float4*)data);
  if (cudaPeekAtLastError() != cudaSuccess) {
    set_last_error("surrogate phase: launch failed");
    return PSF_ERR_CUDA;
  }
  return PSF_OK;
}
