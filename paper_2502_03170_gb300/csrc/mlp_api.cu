// Host side and elementwise kernels of the learned surrogate (see the MLP
// section of include/psf.h): input normalisation, loss and error-head
// kernels, fixed-order reductions, Adam, deterministic initialisation, the
// forward / backward GEMM sequence and the surrogate-with-fallback driver.
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "mlp_kernels.cuh"
#include "timing.cuh"

namespace psf {
void set_last_error(const char* msg);
}

namespace psf {
namespace mlp {
namespace {

constexpr int MAX_BATCH = 1 << 20;

PSF_D float bf(uint16_t h) { return __uint_as_float((uint32_t)h << 16); }
PSF_D uint16_t tobf(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

int err(int code, const char* msg) {
  set_last_error(msg);
  return code;
}

int pad8(int b) { return (b + 7) / 8 * 8; }

struct State {
  float *params, *m, *v;
  uint16_t* Wb[NLAYER];
  uint16_t* WbT[NLAYER];
  size_t bytes;
};

State state_layout(void* base) {
  State S;
  memset(&S, 0, sizeof(S));
  const ParamLayout P = param_layout();
  char* b = (char*)base;
  size_t off = 0;
  auto take = [&](size_t bytes) -> void* {
    off = align_up(off, 256);
    void* p = b ? b + off : nullptr;
    off += bytes;
    return p;
  };
  S.params = (float*)take(P.total * 4);
  S.m = (float*)take(P.total * 4);
  S.v = (float*)take(P.total * 4);
  for (int l = 0; l < NLAYER; ++l) {
    S.Wb[l] = (uint16_t*)take((size_t)layer_out(l) * layer_in(l) * 2);
    S.WbT[l] = (uint16_t*)take((size_t)layer_out(l) * layer_in(l) * 2);
  }
  S.bytes = align_up(off, 256);
  return S;
}

struct Work {
  uint16_t *X0, *X0T;
  uint16_t *Y[NHID], *YT[NHID], *Z[NHID];
  float* out;
  uint16_t *G4, *G4T;
  uint16_t *dZ[2], *dZT[2];
  float *grads, *relerr, *lossp, *errp, *resid, *lossp2;
  size_t bytes;
};

Work work_layout(void* base, int B, bool train) {
  Work W;
  memset(&W, 0, sizeof(W));
  const int Bp = pad8(B);
  char* b = (char*)base;
  size_t off = kStatusBytes;
  auto take = [&](size_t bytes) -> void* {
    off = align_up(off, 1024);
    void* p = b ? b + off : nullptr;
    off += bytes;
    return p;
  };
  W.X0 = (uint16_t*)take((size_t)B * IN_PAD * 2);
  W.X0T = (uint16_t*)take((size_t)IN_PAD * Bp * 2);
  for (int l = 0; l < NHID; ++l) {
    W.Y[l] = (uint16_t*)take((size_t)B * HID * 2);
    if (train) {
      W.YT[l] = (uint16_t*)take((size_t)HID * Bp * 2);
      W.Z[l] = (uint16_t*)take((size_t)B * HID * 2);
    }
  }
  W.errp = (float*)take((size_t)B * 4);
  if (train) {
    W.out = (float*)take((size_t)B * OUT * 4);
    W.G4 = (uint16_t*)take((size_t)B * OUT * 2);
    W.G4T = (uint16_t*)take((size_t)OUT * Bp * 2);
    for (int k = 0; k < 2; ++k) {
      W.dZ[k] = (uint16_t*)take((size_t)B * HID * 2);
      W.dZT[k] = (uint16_t*)take((size_t)HID * Bp * 2);
    }
    W.grads = (float*)take(param_layout().total * 4);
    W.relerr = (float*)take((size_t)B * 4);
    W.lossp = (float*)take((size_t)B * 4);
    W.resid = (float*)take((size_t)B * 4);
    W.lossp2 = (float*)take((size_t)B * 4);
  }
  W.bytes = align_up(off, 256);
  return W;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// Network input (BF16, + transpose): c_1..c_21 / 0.05, d = depth / 5 - 1,
// u = z / 2, then for k = 0..NFREQ-1 sin/cos(2 pi f_k u) with
// f_k = 0.5 * 16^(k/(NFREQ-1)) and sin/cos(2 pi g_k d) with
// g_k = 0.5 * 40^(k/(NFREQ-1)) (geometric frequency ladders), zero padding.
__global__ void k_prep(const float* __restrict__ q, int B, int Bp, uint16_t* X0,
                       uint16_t* X0T) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= B * IN_PAD) return;
  const int b = idx / IN_PAD, k = idx - (idx / IN_PAD) * IN_PAD;
  const float d = q[(size_t)b * IN + 21] * 0.2f - 1.f;
  const float u = q[(size_t)b * IN + 22] * 0.5f;
  float v = 0.f;
  if (k < 21) {
    v = q[(size_t)b * IN + k] * 20.f;
  } else if (k == 21) {
    v = d;
  } else if (k == 22) {
    v = u;
  } else if (k < IN_FEAT) {
    const int f = (k - IN) >> 2, kind = (k - IN) & 3;   // (sin u, cos u, sin d, cos d)
    const float frac = (float)f / (NFREQ - 1);
    const float fr = kind < 2 ? 0.5f * exp2f(4.f * frac) : 0.5f * exp2f(log2f(40.f) * frac);
    float cyc = fr * (kind < 2 ? u : d);
    cyc -= rintf(cyc);
    float sn, cs;
    sincospif(2.0f * cyc, &sn, &cs);
    v = (kind & 1) ? cs : sn;
  }
  const uint16_t h = tobf(v);
  X0[idx] = h;
  if (X0T) X0T[(size_t)k * Bp + b] = h;
}

// Per sample: relative error and dL/dout = (2/B)(out - t)/|t|^2 (BF16, + T).
__global__ void k_loss(const float* __restrict__ out, const float* __restrict__ t,
                       int B, int Bp, uint16_t* G, uint16_t* GT, float* relerr,
                       float* lossp) {
  __shared__ float red[2][256];
  const int b = blockIdx.x;
  const float* o = out + (size_t)b * OUT;
  const float* tt = t + (size_t)b * OUT;
  float n2 = 0.f, e2 = 0.f;
  for (int k = threadIdx.x; k < OUT; k += 256) {
    const float d = o[k] - tt[k];
    n2 += tt[k] * tt[k];
    e2 += d * d;
  }
  red[0][threadIdx.x] = n2;
  red[1][threadIdx.x] = e2;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      red[0][threadIdx.x] += red[0][threadIdx.x + st];
      red[1][threadIdx.x] += red[1][threadIdx.x + st];
    }
    __syncthreads();
  }
  const float N2 = fmaxf(red[0][0], 1e-30f), E2 = red[1][0];
  const float sc = 2.f / ((float)B * N2);
  for (int k = threadIdx.x; k < OUT; k += 256) {
    const uint16_t h = tobf(sc * (o[k] - tt[k]));
    G[(size_t)b * OUT + k] = h;
    GT[(size_t)k * Bp + b] = h;
  }
  if (threadIdx.x == 0) {
    relerr[b] = sqrtf(E2 / N2);
    lossp[b] = E2 / N2 / (float)B;
  }
}

// Row sums of a transposed BF16 matrix XT [N][ld] over b < B (fixed order).
__global__ void k_rowsum(const uint16_t* __restrict__ XT, int B, int ld, float* out) {
  __shared__ float red[256];
  const uint16_t* r = XT + (size_t)blockIdx.x * ld;
  float s = 0.f;
  for (int b = threadIdx.x; b < B; b += 256) s += bf(r[b]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

// Error head e_b = w_e . Y3[b] + b_e; with relerr: residual to log10(relerr).
__global__ void k_err_fwd(const uint16_t* __restrict__ Y3, const float* __restrict__ we,
                          const float* __restrict__ be, int B,
                          const float* __restrict__ relerr, float* errp, float* resid,
                          float* lossp2) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= B) return;
  const uint16_t* y = Y3 + (size_t)warp * HID;
  float s = 0.f;
  for (int k = lane; k < HID; k += 32) s += we[k] * bf(y[k]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    const float e = s + be[0];
    errp[warp] = e;
    if (relerr) {
      const float r = e - log10f(fmaxf(relerr[warp], 1e-7f));
      resid[warp] = r;
      lossp2[warp] = r * r / (float)B;
    }
  }
}

// dL_e/dw_e[k] = (2/B) sum_b resid_b Y3T[k][b]; block HID: dL_e/db_e.
__global__ void k_err_grad(const uint16_t* __restrict__ Y3T, int B, int ld,
                           const float* __restrict__ resid, float* gwe, float* gbe) {
  __shared__ float red[256];
  const int k = blockIdx.x;
  float s = 0.f;
  for (int b = threadIdx.x; b < B; b += 256)
    s += resid[b] * (k < HID ? bf(Y3T[(size_t)k * ld + b]) : 1.f);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float g = 2.f * red[0] / (float)B;
    if (k < HID)
      gwe[k] = g;
    else
      gbe[0] = g;
  }
}

// Fixed-order sum of n floats (one block).
__global__ void k_sum(const float* __restrict__ v, int n, float* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) s += v[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = (float)red[0];
}

struct LayerPtrs {
  size_t W[NLAYER];
  uint16_t* Wb[NLAYER];
  uint16_t* WbT[NLAYER];
};

// Writes the BF16 copies W_l and W_l^T of the FP32 weight at packed index i.
PSF_D void write_copies(const LayerPtrs& L, size_t i, float p) {
#pragma unroll
  for (int l = 0; l < NLAYER; ++l) {
    const size_t n = (size_t)layer_out(l) * layer_in(l);
    if (i >= L.W[l] && i < L.W[l] + n) {
      const size_t e = i - L.W[l];
      const int in = layer_in(l), outn = layer_out(l);
      const int o = (int)(e / in), k = (int)(e - (e / in) * in);
      const uint16_t h = tobf(p);
      L.Wb[l][e] = h;
      L.WbT[l][(size_t)k * outn + o] = h;
    }
  }
}

// Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= lr mhat / (sqrt(vhat) + eps), mhat = m / (1 - b1^t), vhat = v / (1 - b2^t).
__global__ void k_adam(float* p, float* m, float* v, const float* __restrict__ g,
                       size_t n, float lr, float c1, float c2, LayerPtrs L) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
  p[i] = pi;
  write_copies(L, i, pi);
}

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based uniform generator.
PSF_D double uniform01(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void k_init(float* p, float* m, float* v, size_t n, unsigned long long seed,
                       LayerPtrs L) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float val = 0.f;
  for (int l = 0; l < NLAYER; ++l) {
    const size_t nw = (size_t)layer_out(l) * layer_in(l);
    if (i >= L.W[l] && i < L.W[l] + nw) {
      const int in = layer_in(l);
      const int k = (int)((i - L.W[l]) % in);
      const int fan_in = l == 0 ? IN_FEAT : HID;
      if (k < fan_in) {
        const double a = (l == NLAYER - 1 ? 0.5 : 1.0) * sqrt(6.0 / fan_in);
        val = (float)((2.0 * uniform01(seed, i) - 1.0) * a);
      }
    }
  }
  p[i] = val;
  m[i] = 0.f;
  v[i] = 0.f;
  write_copies(L, i, val);
}

__global__ void k_copies(const float* p, size_t n, LayerPtrs L) {
  const size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) write_copies(L, i, p[i]);
}

LayerPtrs layer_ptrs(const State& S) {
  LayerPtrs L;
  const ParamLayout P = param_layout();
  for (int l = 0; l < NLAYER; ++l) {
    L.W[l] = P.W[l];
    L.Wb[l] = S.Wb[l];
    L.WbT[l] = S.WbT[l];
  }
  return L;
}

// ---------------------------------------------------------------------------
// forward / backward sequences
// ---------------------------------------------------------------------------
int forward(const State& S, const Work& W, const float* q, int B, float* out,
            bool train, int* status, cudaStream_t s, const float2* row_phase = nullptr) {
  const ParamLayout P = param_layout();
  const int Bp = pad8(B);
  k_prep<<<ceil_div(B * IN_PAD, 256), 256, 0, s>>>(q, B, Bp, W.X0, train ? W.X0T : nullptr);
  for (int l = 0; l < NLAYER; ++l) {
    GemmArgs g;
    memset(&g, 0, sizeof(g));
    g.A = l == 0 ? W.X0 : W.Y[l - 1];
    g.lda = l == 0 ? IN_PAD : HID;
    g.B = S.Wb[l];
    g.ldb = layer_in(l);
    g.M = B;
    g.N = layer_out(l);
    g.K = layer_in(l);
    g.bias = S.params + P.b[l];
    g.status = status;
    if (l < NLAYER - 1) {
      g.epi = EPI_HIDDEN;
      g.Y = W.Y[l];
      g.ldy = HID;
      g.YT = train ? W.YT[l] : nullptr;
      g.ldyt = Bp;
      g.Z = train ? W.Z[l] : nullptr;
      g.ldz = HID;
    } else {
      g.epi = EPI_LINEAR;
      g.out = out;
      g.ldo = OUT;
      g.row_phase = row_phase;
    }
    const int r = gemm(g, s);
    if (r) return r;
  }
  return PSF_OK;
}

int backward(const State& S, const Work& W, const float* target, int B, float* loss,
             int* status, cudaStream_t s) {
  const ParamLayout P = param_layout();
  const int Bp = pad8(B);
  k_loss<<<B, 256, 0, s>>>(W.out, target, B, Bp, W.G4, W.G4T, W.relerr, W.lossp);
  // output layer: dW4 = G4^T Y3, db4 = rows of G4T, dZ3 = (G4 W4) SiLU'(Z3)
  const uint16_t* gT = W.G4T;
  const uint16_t* gN = W.G4;
  int ldg = OUT;
  int cur = 0;
  for (int l = NLAYER - 1; l >= 0; --l) {
    const int outn = layer_out(l), in = layer_in(l);
    GemmArgs dw;
    memset(&dw, 0, sizeof(dw));
    dw.A = gT;
    dw.lda = Bp;
    dw.B = l == 0 ? W.X0T : W.YT[l - 1];
    dw.ldb = Bp;
    dw.M = outn;
    dw.N = in;
    dw.K = B;
    dw.epi = EPI_STORE;
    dw.out = W.grads + P.W[l];
    dw.ldo = in;
    dw.status = status;
    int r = gemm(dw, s);
    if (r) return r;
    k_rowsum<<<outn, 256, 0, s>>>(gT, B, Bp, W.grads + P.b[l]);
    if (l == 0) break;
    GemmArgs dx;
    memset(&dx, 0, sizeof(dx));
    dx.A = gN;
    dx.lda = ldg;
    dx.B = S.WbT[l];
    dx.ldb = outn;
    dx.M = B;
    dx.N = in;
    dx.K = outn;
    dx.epi = EPI_DSILU;
    dx.Z = W.Z[l - 1];
    dx.ldz = HID;
    dx.Y = W.dZ[cur];
    dx.ldy = HID;
    dx.YT = W.dZT[cur];
    dx.ldyt = Bp;
    dx.status = status;
    r = gemm(dx, s);
    if (r) return r;
    gN = W.dZ[cur];
    gT = W.dZT[cur];
    ldg = HID;
    cur ^= 1;
  }
  // error head (no gradient into the trunk)
  k_err_fwd<<<ceil_div(B * 32, 256), 256, 0, s>>>(W.Y[NHID - 1], S.params + P.We,
                                                  S.params + P.be, B, W.relerr, W.errp,
                                                  W.resid, W.lossp2);
  k_err_grad<<<HID + 1, 256, 0, s>>>(W.YT[NHID - 1], B, Bp, W.resid, W.grads + P.We,
                                     W.grads + P.be);
  if (loss) {
    k_sum<<<1, 256, 0, s>>>(W.lossp, B, loss);
    k_sum<<<1, 256, 0, s>>>(W.lossp2, B, loss + 1);
  }
  return PSF_OK;
}

int check_batch(int B) {
  if (B < 1 || B > MAX_BATCH) return err(PSF_ERR_ARG, "mlp: batch outside [1, 1048576]");
  return PSF_OK;
}

}  // namespace
}  // namespace mlp
}  // namespace psf

using namespace psf;
using namespace psf::mlp;

extern "C" size_t psf_mlp_param_count(void) { return param_layout().total; }

extern "C" size_t psf_mlp_state_bytes(void) { return state_layout(nullptr).bytes; }

extern "C" int psf_mlp_init(void* state, unsigned long long seed, void* stream) {
  if (!state) return err(PSF_ERR_ARG, "mlp: state is NULL");
  const State S = state_layout(state);
  const size_t n = param_layout().total;
  k_init<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      S.params, S.m, S.v, n, seed, layer_ptrs(S));
  return cudaPeekAtLastError() == cudaSuccess ? PSF_OK : err(PSF_ERR_CUDA, "mlp: init launch");
}

extern "C" size_t psf_mlp_workspace_size(int batch) {
  if (batch < 1 || batch > MAX_BATCH) return 0;
  return work_layout(nullptr, batch, true).bytes;
}

static int mlp_train_or_grad(void* state, const float* query, const float* target,
                             int batch, float lr, int step, float* loss, float* grads_out,
                             void* ws, size_t ws_bytes, void* stream, bool update) {
  int r = check_batch(batch);
  if (r) return r;
  if (!state || !query || !target || !ws) return err(PSF_ERR_ARG, "mlp: NULL pointer");
  if (update && (step < 1 || !(lr > 0.f))) return err(PSF_ERR_ARG, "mlp: step >= 1 and lr > 0");
  const Work W = work_layout(ws, batch, true);
  if (ws_bytes < W.bytes) return err(PSF_ERR_WORKSPACE, "mlp: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const State S = state_layout(state);
  cudaMemsetAsync(ws, 0, sizeof(int), s);
  {
    TimingScope ts(kTimeSetup, s);
    r = forward(S, W, query, batch, W.out, true, (int*)ws, s);
    if (!r) r = backward(S, W, target, batch, loss, (int*)ws, s);
  }
  if (r) return err(r, "mlp: GEMM launch failed");
  const size_t n = param_layout().total;
  if (update) {
    const float c1 = 1.f - powf(0.9f, (float)step), c2 = 1.f - powf(0.999f, (float)step);
    k_adam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(S.params, S.m, S.v, W.grads, n, lr, c1,
                                                       c2, layer_ptrs(S));
  } else if (grads_out) {
    cudaMemcpyAsync(grads_out, W.grads, n * 4, cudaMemcpyDeviceToDevice, s);
  }
  return cudaPeekAtLastError() == cudaSuccess ? PSF_OK : err(PSF_ERR_CUDA, "mlp: launch");
}

extern "C" int psf_mlp_train_step(void* state, const float* query, const float* target,
                                  int batch, float lr, int step, float* loss, void* ws,
                                  size_t ws_bytes, void* stream) {
  return mlp_train_or_grad(state, query, target, batch, lr, step, loss, nullptr, ws,
                           ws_bytes, stream, true);
}

extern "C" int psf_mlp_gradients(void* state, const float* query, const float* target,
                                 int batch, float* grads, float* loss, void* ws,
                                 size_t ws_bytes, void* stream) {
  if (!grads) return err(PSF_ERR_ARG, "mlp: grads is NULL");
  return mlp_train_or_grad(state, query, target, batch, 0.f, 0, loss, grads, ws, ws_bytes,
                           stream, false);
}

extern "C" int psf_mlp_forward(const void* state, const float* query, int batch, float* out,
                               float* err_log10, void* ws, size_t ws_bytes, void* stream) {
  return psf::mlp::forward_rows(state, query, batch, out, err_log10, ws, ws_bytes, nullptr,
                                stream);
}

int psf::mlp::forward_rows(const void* state, const float* query, int batch, float* out,
                           float* err_log10, void* ws, size_t ws_bytes,
                           const float2* row_phase, void* stream) {
  int r = check_batch(batch);
  if (r) return r;
  if (!state || !query || !out || !ws) return err(PSF_ERR_ARG, "mlp: NULL pointer");
  const Work W = work_layout(ws, batch, false);
  if (ws_bytes < W.bytes) return err(PSF_ERR_WORKSPACE, "mlp: workspace too small");
  cudaStream_t s = (cudaStream_t)stream;
  const State S = state_layout((void*)state);
  cudaMemsetAsync(ws, 0, sizeof(int), s);
  r = forward(S, W, query, batch, out, false, (int*)ws, s, row_phase);
  if (r) return err(r, "mlp: GEMM launch failed");
  if (err_log10) {
    const ParamLayout P = param_layout();
    k_err_fwd<<<ceil_div(batch * 32, 256), 256, 0, s>>>(W.Y[NHID - 1], S.params + P.We,
                                                        S.params + P.be, batch, nullptr,
                                                        err_log10, nullptr, nullptr);
  }
  return cudaPeekAtLastError() == cudaSuccess ? PSF_OK : err(PSF_ERR_CUDA, "mlp: launch");
}

extern "C" int psf_mlp_get_params(const void* state, float* params, void* stream) {
  if (!state || !params) return err(PSF_ERR_ARG, "mlp: NULL pointer");
  const State S = state_layout((void*)state);
  cudaMemcpyAsync(params, S.params, param_layout().total * 4, cudaMemcpyDeviceToDevice,
                  (cudaStream_t)stream);
  return cudaPeekAtLastError() == cudaSuccess ? PSF_OK : err(PSF_ERR_CUDA, "mlp: copy");
}

extern "C" int psf_mlp_set_params(void* state, const float* params, void* stream) {
  if (!state || !params) return err(PSF_ERR_ARG, "mlp: NULL pointer");
  const State S = state_layout(state);
  const size_t n = param_layout().total;
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemcpyAsync(S.params, params, n * 4, cudaMemcpyDeviceToDevice, s);
  k_copies<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(S.params, n, layer_ptrs(S));
  return cudaPeekAtLastError() == cudaSuccess ? PSF_OK : err(PSF_ERR_CUDA, "mlp: set");
}
