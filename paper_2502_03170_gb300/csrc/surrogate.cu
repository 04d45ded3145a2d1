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

struct SurLayout {
  size_t mlp_ws, bessel_ws;
  int* idx;
  int* count;
  float* errp;
  double *depth, *zern, *z;
  int* offs;
  float* prof;
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
  int r = psf_mlp_forward(state, query, batch, out, errp, L.mlp, L.mlp_ws, stream);
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
