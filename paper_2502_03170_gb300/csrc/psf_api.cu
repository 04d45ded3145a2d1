// Host side of libpsf: argument validation, FP64 parameter preparation
// (Eq. 13-15, Gauss-Legendre nodes), workspace layout and kernel launches.
// Every exported symbol is declared in include/psf.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "bessel_backward.cuh"
#include "bessel_kernels.cuh"
#include "czt_kernels.cuh"
#include "harmonic_kernels.cuh"
#include "fourier_kernels.cuh"
#include "optics_models.cuh"
#include "tc_kernels.cuh"
#include "timing.cuh"
#include "upload.cuh"

namespace psf {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

static int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

// Sets the thread's last-error message (for entry points in other files).
void set_last_error(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

static int cuda_check(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(PSF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return PSF_OK;
}

static bool finite_pos(double v) { return isfinite(v) && v > 0; }

// ---------------------------------------------------------------------------
// Accuracy envelope of the split precisions.  A forward call in a split mode
// is accepted only at sizes where its measured intensity error against the
// FP64 oracle stays within half the 1e-5 bound on the benchmark workloads
// (Gibson-Lanni + Noll 4..21, 512^2 px):
//   Fourier, folded contractions: split FP16 4.3e-6 at n_pupil 512 (8.7e-6 at
//     1024, 1.7e-5 at 2048); split BF16 4.2e-6 at 1024 (7.6e-6 at 2048);
//   split TF32 (three TF32 products) 3.0e-6 at 256 (6.1e-6 at 512, 1.2e-5
//     at 1024); single-pass TF32 1.3e-4 to 3.4e-4 at every pupil;
//   spherical (Bessel and harmonic) split FP16: 5.2e-6 at 448 Gauss-Legendre
//     nodes (9.9e-6 at 880); split BF16 5.2e-5 on the Bessel workload.
// The error grows with the contraction length (the K extent that each FP32
// tensor-core accumulator sums).  PSF_PREC_AUTO picks the fastest mode that
// stays inside.
// ---------------------------------------------------------------------------
constexpr int kSplitFp16MaxPupil = 512;
constexpr int kSplitBf16MaxPupil = 1024;
constexpr int kSplitTf32MaxPupil = 256;
constexpr int kSplitMaxTheta = 448;

static bool outside_allowed(const psf_optics* opt) {
  return opt && (opt->flags & PSF_OUTSIDE_ENVELOPE);
}

static int fourier_envelope(const psf_optics* opt, int N, int precision) {
  if (outside_allowed(opt)) return PSF_OK;
  if (precision == PSF_PREC_TF32)
    return fail(PSF_ERR_PRECISION,
                "TF32 with one product per multiply-add keeps 11 significant bits per "
                "operand (measured 1.3e-4 to 3.4e-4 from the FP64 oracle): outside the "
                "1e-5 envelope; use PSF_PREC_SPLIT_TF32 or set PSF_OUTSIDE_ENVELOPE");
  if (precision == PSF_PREC_SPLIT_TF32 && N > kSplitTf32MaxPupil)
    return fail(PSF_ERR_PRECISION,
                "split TF32 is accepted up to n_pupil %d (measured 3.0e-6 at 256, 6.1e-6 "
                "at 512); n_pupil %d: use PSF_PREC_SPLIT_FP16, PSF_PREC_FP32_CHIRPZ or "
                "PSF_PREC_AUTO", kSplitTf32MaxPupil, N);
  if (precision == PSF_PREC_SPLIT_FP16 && N > kSplitFp16MaxPupil)
    return fail(PSF_ERR_PRECISION,
                "split FP16 holds the 1e-5 bound up to n_pupil %d (measured 4.3e-6 at 512, "
                "8.7e-6 at 1024); n_pupil %d: use PSF_PREC_SPLIT_BF16 (up to %d), "
                "PSF_PREC_FP32_CHIRPZ, PSF_PREC_FP32 or PSF_PREC_AUTO",
                kSplitFp16MaxPupil, N, kSplitBf16MaxPupil);
  if (precision == PSF_PREC_SPLIT_BF16 && N > kSplitBf16MaxPupil)
    return fail(PSF_ERR_PRECISION,
                "split BF16 holds the 1e-5 bound up to n_pupil %d (measured 4.2e-6 at 1024, "
                "7.6e-6 at 2048); n_pupil %d: use PSF_PREC_FP32_CHIRPZ, PSF_PREC_FP32 or "
                "PSF_PREC_AUTO",
                kSplitBf16MaxPupil, N);
  return PSF_OK;
}

static int spherical_envelope(const psf_optics* opt, int n_theta, int precision) {
  if (outside_allowed(opt)) return PSF_OK;
  if (precision == PSF_PREC_SPLIT_BF16)
    return fail(PSF_ERR_PRECISION,
                "split BF16 keeps 16 significant bits per operand: 5.2e-5 from the FP64 "
                "oracle on the Bessel workload, over the 1e-5 bound; use PSF_PREC_SPLIT_FP16, "
                "PSF_PREC_FP32 or PSF_PREC_AUTO");
  if (precision == PSF_PREC_SPLIT_FP16 && n_theta > kSplitMaxTheta)
    return fail(PSF_ERR_PRECISION,
                "split FP16 holds the 1e-5 bound up to %d theta nodes (measured 5.2e-6 at "
                "448, 9.9e-6 at 880); n_theta %d: use PSF_PREC_FP32 or PSF_PREC_AUTO",
                kSplitMaxTheta, n_theta);
  return PSF_OK;
}

static int czt_fits(int N, int nx, int ny);   // defined with the Fourier strategy

// PSF_PREC_AUTO of the Fourier forward: the dense split contraction inside
// its envelope (FP16 up to n_pupil 512, BF16 up to 1024), else the chirp-Z
// zoom when its FFT length fits, else FP32.
static int resolve_fourier_precision(int N, int nx, int ny, int precision) {
  if (precision != PSF_PREC_AUTO) return precision;
  const bool tc = N % 8 == 0 && N >= 16;
  if (tc && N <= kSplitFp16MaxPupil) return PSF_PREC_SPLIT_FP16;
  if (tc && N <= kSplitBf16MaxPupil) return PSF_PREC_SPLIT_BF16;
  if (czt_fits(N, nx, ny)) return PSF_PREC_FP32_CHIRPZ;
  return PSF_PREC_FP32;
}

// PSF_PREC_AUTO of the spherical forwards: split FP16 inside its envelope.
static int resolve_spherical_precision(int n_theta, int precision) {
  if (precision != PSF_PREC_AUTO) return precision;
  return n_theta <= kSplitMaxTheta ? PSF_PREC_SPLIT_FP16 : PSF_PREC_FP32;
}

// PSF_PREC_AUTO of the adjoints (gradient bound 1e-4): the tensor-core split
// FP16 form wherever it runs.
static int resolve_fourier_backward_precision(int N, int nx, int ny, int precision) {
  if (precision != PSF_PREC_AUTO) return precision;
  return tc_fourier_bwd_supported(N, nx, ny) ? PSF_PREC_FP32 : PSF_PREC_SPLIT_FP16;
}
static int resolve_bessel_backward_precision(int precision) {
  return precision == PSF_PREC_AUTO ? PSF_PREC_SPLIT_FP16 : precision;
}

static int check_optics(const psf_optics* o) {
  if (!o) return fail(PSF_ERR_ARG, "optics is NULL");
  if (!finite_pos(o->NA) || !finite_pos(o->lambda) || !finite_pos(o->n_i))
    return fail(PSF_ERR_ARG, "NA, lambda and n_i must be finite and > 0");
  if (!(o->NA < o->n_i))
    return fail(PSF_ERR_ARG, "NA (%g) must be below n_i (%g)", o->NA, o->n_i);
  if (!finite_pos(o->n_s) || !finite_pos(o->n_g) || !finite_pos(o->n_i_design) ||
      !finite_pos(o->n_g_design))
    return fail(PSF_ERR_ARG, "refractive indices must be finite and > 0");
  if (!isfinite(o->t_g) || !isfinite(o->t_g_design) || !isfinite(o->t_i_design) ||
      !isfinite(o->depth) || !isfinite(o->s_env))
    return fail(PSF_ERR_ARG, "thicknesses / depth / s_env must be finite");
  for (int i = 0; i < 4; ++i)
    if (!isfinite(o->pol[i])) return fail(PSF_ERR_ARG, "polarisation not finite");
  return PSF_OK;
}

// ---------------------------------------------------------------------------
// Eq. 13-14: layers of the Gibson-Lanni optical path, W/(2 pi) in cycles is
// sum_l t_l sqrt(n_l^2 - n_i^2 sin^2) / lambda.  Eq. 14 (as printed) fixes
// t_i = t_s + n_i (-t_s/n_s - t_g/n_g + t_g*/n_g* + t_i*/n_i*).
// ---------------------------------------------------------------------------
static double immersion_thickness(const psf_optics* o, double ts) {
  return ts + o->n_i * (-ts / o->n_s - o->t_g / o->n_g +
                        o->t_g_design / o->n_g_design +
                        o->t_i_design / o->n_i_design);
}

static GLLayers gl_layers(const psf_optics* o, double ts) {
  GLLayers g;
  g.n = 5;
  g.t[0] = ts;                              g.n_idx[0] = o->n_s;
  g.t[1] = immersion_thickness(o, ts);      g.n_idx[1] = o->n_i;
  g.t[2] = -o->t_i_design;                  g.n_idx[2] = o->n_i_design;
  g.t[3] = o->t_g;                          g.n_idx[3] = o->n_g;
  g.t[4] = -o->t_g_design;                  g.n_idx[4] = o->n_g_design;
  return g;
}

// On-axis (theta = 0) optical path of Eq. 13 as a0 + a1 t_s cycles: every
// layer contributes t_l n_l / lambda, and the thicknesses are affine in t_s.
void psf_axis_path_cycles(const psf_optics* o, double* a0, double* a1) {
  const GLLayers L0 = gl_layers(o, 0.0), L1 = gl_layers(o, 1.0);
  double s0 = 0.0, s1 = 0.0;
  for (int l = 0; l < L0.n; ++l) {
    s0 += L0.t[l] * L0.n_idx[l];
    s1 += (L1.t[l] - L0.t[l]) * L0.n_idx[l];
  }
  *a0 = s0 / o->lambda;
  *a1 = s1 / o->lambda;
}

// Layers with the same index share one root: t_a sqrt(n^2 - .) + t_b sqrt(n^2 - .)
// = (t_a + t_b) sqrt(n^2 - .).  Design layers equal to the actual ones cancel.
static GLLayers merge_layers(const GLLayers& in) {
  GLLayers g;
  g.n = 0;
  for (int l = 0; l < in.n; ++l) {
    int k = 0;
    while (k < g.n && g.n_idx[k] != in.n_idx[l]) ++k;
    if (k == g.n) {
      g.n_idx[g.n] = in.n_idx[l];
      g.t[g.n++] = in.t[l];
    } else {
      g.t[k] += in.t[l];
    }
  }
  int w = 0;
  for (int l = 0; l < g.n; ++l)
    if (g.t[l] != 0.0) {
      g.t[w] = g.t[l];
      g.n_idx[w++] = g.n_idx[l];
    }
  g.n = w;
  return g;
}

// ---------------------------------------------------------------------------
// Eq. 15, Noll ordering: j -> (n, m), m > 0 cosine, m < 0 sine.
// ---------------------------------------------------------------------------
static void noll_nm(int j, int* n_out, int* m_out) {
  int n = 0;
  while ((n + 1) * (n + 2) / 2 < j) ++n;
  const int k = j - n * (n + 1) / 2 - 1;
  const int am = (n % 2 == 0) ? 2 * ((k + 1) / 2) : 2 * (k / 2) + 1;
  *n_out = n;
  *m_out = am == 0 ? 0 : ((j % 2 == 0) ? am : -am);
}

static double fact(int n) {
  double f = 1;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// Radial polynomial coefficients of sqrt(norm) R_n^|m|: out[k] multiplies rho^k.
static void zernike_radial_coeffs(int n, int am, double* out) {
  for (int k = 0; k <= kZernMaxOrder; ++k) out[k] = 0;
  const double norm = am == 0 ? sqrt(n + 1.0) : sqrt(2.0 * (n + 1.0));
  for (int s = 0; s <= (n - am) / 2; ++s) {
    const double c = ((s % 2) ? -1.0 : 1.0) * fact(n - s) /
                     (fact(s) * fact((n + am) / 2 - s) * fact((n - am) / 2 - s));
    out[n - 2 * s] += norm * c;
  }
}

static ZernPoly zernike_poly(const double* c, int n_zern) {
  ZernPoly z;
  memset(&z, 0, sizeof(z));
  z.max_m = -1;
  double rc[kZernMaxOrder + 1];
  for (int j = 1; j <= n_zern; ++j) {
    if (c[j - 1] == 0.0) continue;
    int n, m;
    noll_nm(j, &n, &m);
    const int am = m < 0 ? -m : m;
    zernike_radial_coeffs(n, am, rc);
    for (int k = 0; k <= kZernMaxOrder; ++k) {
      if (m >= 0)
        z.c[am][k] += c[j - 1] * rc[k];
      else
        z.s[am][k] += c[j - 1] * rc[k];
    }
    if (am > z.max_m) z.max_m = am;
    if (n > z.deg) z.deg = n;
  }
  return z;
}

// ---------------------------------------------------------------------------
// Gauss-Legendre nodes on [-1, 1] by Newton's method on P_n (three-term
// recurrence), weights 2 / ((1 - x^2) P_n'(x)^2).
// ---------------------------------------------------------------------------
static void gauss_legendre_compute(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double r = cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = r;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * r * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double pn = n == 1 ? r : p1;
      const double pm = n == 1 ? 1.0 : p0;
      dp = n * (r * pn - pm) / (r * r - 1.0);
      const double dr = pn / dp;
      r -= dr;
      if (fabs(dr) < 1e-16) break;
    }
    x[i] = -r;
    x[n - 1 - i] = r;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - r * r) * dp * dp);
  }
}

// The rule depends on n alone: computed once per n (the Newton iterations
// cost a few hundred microseconds of host time at 200 nodes) and kept.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  static std::mutex mu;
  static std::map<int, std::pair<std::vector<double>, std::vector<double>>> rules;
  std::lock_guard<std::mutex> lock(mu);
  auto it = rules.find(n);
  if (it == rules.end()) {
    std::vector<double> xs, ws;
    gauss_legendre_compute(n, xs, ws);
    it = rules.emplace(n, std::make_pair(std::move(xs), std::move(ws))).first;
  }
  x = it->second.first;
  w = it->second.second;
}

// ---------------------------------------------------------------------------
// Workspace carving
// ---------------------------------------------------------------------------
struct Carver {
  char* base;
  size_t off;
  explicit Carver(void* b) : base((char*)b), off(kStatusBytes) {}
  template <class T>
  T* take(size_t n) {
    off = align_up(off, 256);
    T* p = base ? (T*)(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

// ===========================================================================
// Fourier strategy
// ===========================================================================
static int fourier_zchunk(int N, int nx, int ny, int nz) {
  // per-chunk pupil + stage-1 buffers up to 1 GB and 256 planes (longer
  // launches: 6.52 ms per 128-plane stack against 6.77 ms in 64 MB chunks)
  const double per_z = 3.0 * 8.0 * ((double)N * N + (double)ny * N);
  int zc = (int)(1024.0 * 1048576.0 / per_z);
  if (zc < 1) zc = 1;
  if (zc > 256) zc = 256;
  if (zc > nz) zc = nz;
  (void)nx;
  return zc;
}

struct FourierLayout {
  NodeTable nodes;
  float2* zz;
  float2 *Ax, *Ay;
  float2 *P, *U;       // FP32 path
  TcOperands tc;       // split-precision path, unfolded contraction
  TcFoldOperands fold; // split-precision path, symmetry-folded contraction
  bool fold_path;
  float2* czt_words;   // chirp-Z path: x tables | y tables
  size_t czt_wx, czt_wy;
  float2* T;           // chirp-Z stage-1 output [zc][3][ny][N]
  int zc;
  size_t bytes;
};

static int czt_fits(int N, int nx, int ny) { return czt_length(N, nx) && czt_length(N, ny); }

static int czt_zchunk(int N, int ny, int nz) {
  // stage-1 output of a chunk up to 1 GB and 256 planes: longer launches
  // fill the GPU better than an L2-sized chunk (256^2 -> 512^2 x 128 planes:
  // 1.54 ms as one chunk against 1.76 ms in 16-plane chunks of 48 MB)
  const double per_z = 3.0 * 8.0 * (double)ny * N;
  int zc = (int)(1024.0 * 1048576.0 / per_z);
  if (zc < 1) zc = 1;
  if (zc > 256) zc = 256;
  if (zc > nz) zc = nz;
  return zc;
}

// The split precisions run the symmetry-folded contractions (a quarter of the
// multiply-adds of the unfolded 2x2-block form); PSF_TC_FOLD=0 in the
// environment selects the unfolded form (same discrete sums, other rounding).
static bool fold_enabled() {
  const char* e = getenv("PSF_TC_FOLD");
  return !(e && e[0] == '0');
}

// max_planes caps the z-chunk (the call shortens its chunks to fit a smaller
// workspace than psf_fourier_workspace_size() asks for)
static FourierLayout fourier_layout(void* ws, int N, const psf_grid* g,
                                    int precision, int max_planes = 1 << 30) {
  FourierLayout L;
  memset(&L, 0, sizeof(L));
  Carver c(ws);
  const size_t NN = (size_t)N * N;
  L.nodes.amp = c.take<float>(6 * NN);
  L.nodes.wfr = c.take<float>(NN);
  L.nodes.kh = c.take<float>(NN);
  L.nodes.kl = c.take<float>(NN);
  L.nodes.rad = c.take<double>(kNodeRad * node_rad_count(N));
  L.zz = c.take<float2>(g->nz);
  auto capped = [&](int zc) { return zc < max_planes ? zc : (max_planes > 1 ? max_planes : 1); };
  L.zc = capped(fourier_zchunk(N, g->nx, g->ny, g->nz));
  if (precision == PSF_PREC_FP32_CHIRPZ) {
    L.czt_wx = czt_dir_words(N, g->nx);
    L.czt_wy = czt_dir_words(N, g->ny);
    L.czt_words = c.take<float2>(L.czt_wx + L.czt_wy);
    L.zc = capped(czt_zchunk(N, g->ny, g->nz));
    L.T = c.take<float2>((size_t)L.zc * 3 * g->ny * N);
  } else if (precision == PSF_PREC_FP32) {
    L.Ax = c.take<float2>((size_t)g->nx * N);
    L.Ay = c.take<float2>((size_t)g->ny * N);
    L.P = c.take<float2>((size_t)L.zc * 3 * NN);
    L.U = c.take<float2>((size_t)L.zc * 3 * g->ny * N);
  } else if (fold_enabled()) {
    L.fold_path = true;
    const int eb = precision == PSF_PREC_SPLIT_TF32 || precision == PSF_PREC_TF32 ? 4 : 2;
    L.zc = capped(tc_fold_zchunk(N, g->nx, g->ny, g->nz, eb));
    tc_fold_carve(c.base, &c.off, N, g->nx, g->ny, L.zc, &L.fold, eb);
  } else {
    L.zc = capped(tc_fourier_zchunk(N, g->nx, g->ny, g->nz));
    tc_fourier_carve(c.base, &c.off, N, g->nx, g->ny, L.zc, &L.tc);
  }
  L.bytes = align_up(c.off, 256);
  return L;
}

static int check_fourier_args(const psf_optics* opt, int N, const psf_grid* g,
                              int precision) {
  int r = check_optics(opt);
  if (r) return r;
  if (N < 2 || N > 4096) return fail(PSF_ERR_ARG, "n_pupil %d outside [2, 4096]", N);
  if (!g) return fail(PSF_ERR_ARG, "grid is NULL");
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || g->nx > 16384 || g->ny > 16384)
    return fail(PSF_ERR_ARG, "grid sizes must be in [1, 16384] (nz >= 1)");
  if (!finite_pos(g->dx) || !finite_pos(g->dy))
    return fail(PSF_ERR_ARG, "pixel pitch must be finite and > 0");
  if (!g->z) return fail(PSF_ERR_ARG, "grid z list is NULL");
  for (int i = 0; i < g->nz; ++i)
    if (!isfinite(g->z[i]) || fabs(g->z[i]) > 1e4)
      return fail(PSF_ERR_ARG, "z[%d] not finite or beyond 1e4 um", i);
  if (precision != PSF_PREC_FP32 && precision != PSF_PREC_SPLIT_FP16 &&
      precision != PSF_PREC_SPLIT_BF16 && precision != PSF_PREC_FP32_CHIRPZ &&
      precision != PSF_PREC_SPLIT_TF32 && precision != PSF_PREC_TF32)
    return fail(PSF_ERR_PRECISION, "unknown precision mode %d", precision);
  if ((precision == PSF_PREC_SPLIT_TF32 || precision == PSF_PREC_TF32) && !fold_enabled())
    return fail(PSF_ERR_PRECISION, "the TF32 modes run on the folded contraction only");
  if (precision == PSF_PREC_FP32_CHIRPZ) {
    if (!czt_length(N, g->nx) || !czt_length(N, g->ny))
      return fail(PSF_ERR_PRECISION, "chirp-Z: n_pupil + n_out - 1 = %d exceeds %d",
                  N + (g->nx > g->ny ? g->nx : g->ny) - 1, kCztMaxL);
  } else if (precision != PSF_PREC_FP32) {
    const char* why = tc_fourier_supported(N, g->nx, g->ny);
    if (why) return fail(PSF_ERR_PRECISION, "split precision: %s", why);
  }
  return PSF_OK;
}

static NodeParams node_params(const psf_optics* opt, int N, const double* zern,
                              int n_zern, const float* phase_map) {
  NodeParams p;
  memset(&p, 0, sizeof(p));
  p.N = N;
  p.s_max = opt->NA / opt->n_i;
  p.inv_lambda = 1.0 / opt->lambda;
  p.n_i = opt->n_i;
  p.gl = merge_layers(gl_layers(opt, opt->depth));
  p.apodize = opt->apodize;
  p.s_env = opt->s_env;
  for (int i = 0; i < 4; ++i) p.pol[i] = opt->pol[i];
  p.zp = zernike_poly(zern, n_zern);
  p.phase_map = phase_map;
  p.model = (opt->flags & PSF_SCALAR) ? 1 : ((opt->flags & PSF_FRESNEL) ? 2 : 0);
  p.n_s = opt->n_s;
  p.n_g = opt->n_g;
  return p;
}

// Output buffers may be device memory or pinned host memory (page-locked
// and registered with CUDA): the kernels then store through its device alias
// over the host link (the Fourier split path streams chunk copies instead,
// see psf_fourier_vectorial).  Host memory that is not registered is
// rejected (the device could not reach it); the check runs on the host
// before any launch.
static bool is_pinned_host(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost && a.devicePointer != nullptr;
}

static int resolve_output(void** p, const char* what) {
  if (!*p) return PSF_OK;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, *p) != cudaSuccess) {
    cudaGetLastError();
    return fail(PSF_ERR_ARG, "%s: not a pointer CUDA knows", what);
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return PSF_OK;
  if (a.type == cudaMemoryTypeHost && a.devicePointer) {
    *p = a.devicePointer;
    return PSF_OK;
  }
  return fail(PSF_ERR_ARG,
              "%s: host memory that is not pinned (use device memory or pinned host memory)",
              what);
}

// Workspace of the Fourier forward with one plane per z-chunk (the least
// psf_fourier_vectorial() runs with; the no-alloc entry point checks it).
size_t fourier_min_workspace_size(const psf_optics* opt, int n_pupil, const psf_grid* grid,
                                  int precision) {
  if (check_fourier_args(opt, n_pupil, grid, precision)) return 0;
  return fourier_layout(nullptr, n_pupil, grid, precision, 1).bytes;
}

// Z_j at the pupil centre (rho = 0) for Noll j = 1 .. n_zern (Eq. 15,
// RMS normalisation): sqrt(n + 1) (-1)^(n/2) for m = 0, 0 otherwise.
void psf_axis_zernike(int n_zern, double* z0) {
  for (int j = 1; j <= n_zern; ++j) {
    int n, m;
    noll_nm(j, &n, &m);
    z0[j - 1] = m == 0 ? sqrt(n + 1.0) * (((n / 2) & 1) ? -1.0 : 1.0) : 0.0;
  }
}

}  // namespace psf

using namespace psf;

extern "C" {

int psf_version(void) { return 100; }

const char* psf_last_error(void) { return g_err; }

int psf_workspace_status(const void* workspace, void* stream) {
  if (!workspace) return fail(PSF_ERR_ARG, "workspace is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) return cuda_check("stream sync");
  int st = 0;
  if (cudaMemcpy(&st, workspace, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return cuda_check("status read");
  return st;
}

size_t psf_fourier_workspace_size(const psf_optics* opt, int n_pupil,
                                  const psf_grid* grid, int precision) {
  if (grid) precision = resolve_fourier_precision(n_pupil, grid->nx, grid->ny, precision);
  if (check_fourier_args(opt, n_pupil, grid, precision)) return 0;
  if (fourier_envelope(opt, n_pupil, precision)) return 0;
  return fourier_layout(nullptr, n_pupil, grid, precision).bytes;
}

int psf_fourier_vectorial(const psf_optics* opt, int n_pupil,
                          const psf_grid* grid, const double* zernike,
                          int n_zern, const float* phase_map, int precision,
                          float* intensity, void* fields, void* workspace,
                          size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  if (grid) precision = resolve_fourier_precision(n_pupil, grid->nx, grid->ny, precision);
  int r = check_fourier_args(opt, n_pupil, grid, precision);
  if (r) return r;
  if ((r = fourier_envelope(opt, n_pupil, precision))) return r;
  if (n_zern < 0 || n_zern > 66) return fail(PSF_ERR_ARG, "n_zern %d outside [0, 66]", n_zern);
  if (n_zern > 0 && !zernike) return fail(PSF_ERR_ARG, "zernike is NULL");
  for (int j = 0; j < n_zern; ++j)
    if (!isfinite(zernike[j])) return fail(PSF_ERR_ARG, "zernike[%d] not finite", j);
  if (!intensity) return fail(PSF_ERR_ARG, "intensity is NULL");
  if (!workspace) return fail(PSF_ERR_WORKSPACE, "workspace is NULL");
  const int N = n_pupil;
  // the longest z-chunk the workspace holds (down to one plane)
  int max_planes = 1 << 30;
  FourierLayout L = fourier_layout(nullptr, N, grid, precision);
  while (ws_bytes < L.bytes && L.zc > 1) {
    max_planes = L.zc / 2;
    L = fourier_layout(nullptr, N, grid, precision, max_planes);
  }
  if (ws_bytes < L.bytes)
    return fail(PSF_ERR_WORKSPACE, "workspace %zu bytes < %zu needed (one plane per chunk)",
                ws_bytes, L.bytes);
  // A pinned host intensity (without fields) on the tensor-core path is
  // streamed: the stack is computed in eight z-chunks into a device staging
  // area behind the chunk layout, and each chunk is copied to the host while
  // the next is computed (256^2 pupil, 512^2 x 128 stack, host wall time per
  // call: compute + bulk copy 1.36 ms, streamed in 2 / 4 / 8 chunks 1.12 /
  // 0.98 / 0.92 ms; the device-to-host link moves about 190 GB/s).
  // Otherwise (or when the workspace has no room for the staging area) the
  // kernels store through the host memory's device alias.
  float* host_out = nullptr;
  float* stage = nullptr;
  const bool tc_path = precision == PSF_PREC_SPLIT_FP16 || precision == PSF_PREC_SPLIT_BF16 ||
                       precision == PSF_PREC_SPLIT_TF32 || precision == PSF_PREC_TF32;
  if (tc_path && !fields && is_pinned_host(intensity) && tc_host_streaming_available()) {
    const int chunks = 8;
    int zs = (grid->nz + chunks - 1) / chunks;
    if (zs > max_planes) zs = max_planes;
    if (zs < 1) zs = 1;
    FourierLayout Ls = fourier_layout(nullptr, N, grid, precision, zs);
    const size_t off = align_up(Ls.bytes, 256);
    const size_t stage_bytes = 2 * (size_t)Ls.zc * grid->nx * grid->ny * sizeof(float);
    if (ws_bytes >= off + stage_bytes) {
      max_planes = zs;
      host_out = intensity;
      stage = (float*)((char*)workspace + off);
    }
  }
  L = fourier_layout(workspace, N, grid, precision, max_planes);
  if (!host_out && (r = resolve_output((void**)&intensity, "intensity"))) return r;
  if ((r = resolve_output(&fields, "fields"))) return r;
  cudaStream_t s = (cudaStream_t)stream;

  std::vector<float2> zz(grid->nz);
  for (int i = 0; i < grid->nz; ++i) {
    const f2x v = split_double(grid->z[i]);
    zz[i] = make_float2(v.hi, v.lo);
  }
  cudaMemsetAsync(workspace, 0, sizeof(int), s);
  upload_async(L.zz, zz.data(), zz.size() * sizeof(float2), s);
  if ((r = cuda_check("workspace init"))) return r;

  NodeParams np = node_params(opt, N, zernike, n_zern, phase_map);
  {
    TimingScope ts(kTimeSetup, s);
    launch_node_table(np, L.nodes, s);
  }
  const double f = opt->NA / opt->lambda;   // k s_max / (2 pi)
  const double ds = 2.0 * (opt->NA / opt->n_i) / N;
  const float scale = (float)(ds * ds / (2.0 * kPi));
  if (precision == PSF_PREC_FP32_CHIRPZ) {
    // tables of both directions; the Eq. 8 prefactor C ds^2 = -i ds^2 / (2 pi)
    // rides on the x post-chirp (stage 2 zooms along x)
    std::vector<float2> words(L.czt_wx + L.czt_wy);
    czt_build_dir(N, grid->nx, f, grid->dx, 0.0, -ds * ds / (2.0 * kPi), words.data());
    czt_build_dir(N, grid->ny, f, grid->dy, 1.0, 0.0, words.data() + L.czt_wx);
    upload_async(L.czt_words, words.data(), words.size() * sizeof(float2), s);
    if ((r = cuda_check("chirp-Z tables"))) return r;
    const CztDir cx = czt_dir_view(L.czt_words, N, grid->nx);
    const CztDir cy = czt_dir_view(L.czt_words + L.czt_wx, N, grid->ny);
    for (int z0 = 0; z0 < grid->nz; z0 += L.zc) {
      const int nzc = grid->nz - z0 < L.zc ? grid->nz - z0 : L.zc;
      {
        TimingScope ts(kTimeStage1, s);
        launch_czt_stage1(L.nodes, N, L.zz, z0, nzc, cx, cy, grid->ny, L.T, s);
      }
      float2* fz = fields ? (float2*)fields + (size_t)z0 * 3 * grid->nx * grid->ny : nullptr;
      {
        TimingScope ts(kTimeStage2, s);
        launch_czt_stage2(L.T, N, grid->nx, grid->ny, nzc, cx,
                          intensity + (size_t)z0 * grid->nx * grid->ny, fz, s);
      }
    }
  } else if (precision == PSF_PREC_FP32) {
    {
      TimingScope ts(kTimeSetup, s);
      launch_twiddle(N, grid->nx, grid->dx, f, L.Ax, s);
    }
    {
      TimingScope ts(kTimeSetup, s);
      launch_twiddle(N, grid->ny, grid->dy, f, L.Ay, s);
    }
    for (int z0 = 0; z0 < grid->nz; z0 += L.zc) {
      const int nzc = grid->nz - z0 < L.zc ? grid->nz - z0 : L.zc;
      {
        TimingScope ts(kTimePupil, s);
        launch_pupil_z_f32(L.nodes, N, L.zz, z0, nzc, L.P, s);
      }
      {
        TimingScope ts(kTimeStage1, s);
        launch_stage1_f32(L.Ay, L.P, L.U, N, grid->ny, nzc, s);
      }
      float2* fz = fields ? (float2*)fields + (size_t)z0 * 3 * grid->nx * grid->ny : nullptr;
      {
        TimingScope ts(kTimeStage2, s);
        launch_stage2_f32(L.Ax, L.U, intensity + (size_t)z0 * grid->nx * grid->ny,
                          fz, N, grid->nx, grid->ny, nzc, scale, s);
      }
    }
  } else if (L.fold_path) {
    r = tc_fold_forward(L.fold, L.nodes, L.zz, N, grid->nx, grid->ny, grid->dx, grid->dy,
                        grid->nz, L.zc, f, scale, tc_pupil_amplitude_bound(np), precision,
                        host_out ? stage : intensity, (float2*)fields, host_out,
                        (int*)workspace, s);
    if (r) return fail(r, "split-precision (folded) launch failed");
  } else {
    r = tc_fourier_forward(L.tc, L.nodes, L.zz, N, grid->nx, grid->ny, grid->dx,
                           grid->dy, grid->nz, L.zc, f, scale,
                           tc_pupil_amplitude_bound(np), precision,
                           host_out ? stage : intensity, (float2*)fields, host_out,
                           (int*)workspace, s);
    if (r) return fail(r, "split-precision launch failed");
  }
  return cuda_check("psf_fourier_vectorial launch");
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Backward (adjoint of Eq. 8), FP32 contractions, per-z recomputation.
// ---------------------------------------------------------------------------
struct BackwardLayout {
  NodeTable nodes;
  float2* zz;
  float2 *Ax, *Ay, *AxH, *AyH;
  float2 *P, *U, *RT, *V, *Gh;
  float* gW;
  float* loss_part;
  int zc, n_part;
  TcBwdOperands tc;      // split-precision path
  float* Zt;             // [n_zern][N][N] Zernike basis (once per call)
  double* zpart;         // partial sums of the Zernike gradient
  size_t bytes;
};

// max_planes: planes per chunk the split path may use (whole groups of
// pupils share one pass; 128 unless the caller's workspace holds more)
static BackwardLayout backward_layout(void* ws, int N, const psf_grid* g,
                                      int precision = PSF_PREC_FP32, int n_zern = 66,
                                      int max_planes = 128) {
  BackwardLayout L;
  memset(&L, 0, sizeof(L));
  Carver c(ws);
  const size_t NN = (size_t)N * N;
  L.Zt = c.take<float>((size_t)n_zern * NN);
  L.nodes.amp = c.take<float>(6 * NN);
  L.nodes.wfr = c.take<float>(NN);
  L.nodes.kh = c.take<float>(NN);
  L.nodes.kl = c.take<float>(NN);
  L.nodes.rad = c.take<double>(kNodeRad * node_rad_count(N));
  L.zz = c.take<float2>(g->nz);
  if (precision != PSF_PREC_FP32) {
    L.zc = tc_fourier_bwd_zchunk(N, g->nx, g->ny, g->nz, max_planes);
    tc_fourier_bwd_carve(c.base, &c.off, N, g->nx, g->ny, g->nz, L.zc, &L.tc);
    L.zpart = (double*)c.take<char>(tc_zernike_parts_bytes(N, n_zern, L.tc.group));
    L.bytes = align_up(c.off, 256);
    return L;
  }
  L.zpart = (double*)c.take<char>(zernike_grad_part_bytes(n_zern, 1));
  // per-z: P, Gh [3][N][N], U [3][ny][N], RT [3][ny][nx], V [3][N][ny]
  const double per_z = 3.0 * 8.0 * (2.0 * NN + 2.0 * g->ny * N + (double)g->ny * g->nx);
  int zc = (int)(96.0 * 1048576.0 / per_z);
  zc = zc < 1 ? 1 : (zc > 32 ? 32 : zc);
  if (zc > g->nz) zc = g->nz;
  L.zc = zc;
  L.Ax = c.take<float2>((size_t)g->nx * N);
  L.Ay = c.take<float2>((size_t)g->ny * N);
  L.AxH = c.take<float2>((size_t)g->nx * N);
  L.AyH = c.take<float2>((size_t)g->ny * N);
  L.P = c.take<float2>((size_t)zc * 3 * NN);
  L.Gh = c.take<float2>((size_t)zc * 3 * NN);
  L.U = c.take<float2>((size_t)zc * 3 * g->ny * N);
  L.RT = c.take<float2>((size_t)zc * 3 * g->ny * g->nx);
  L.V = c.take<float2>((size_t)zc * 3 * N * g->ny);
  L.gW = c.take<float>(NN);
  L.n_part = g->nz * stage2_tiles(g->nx, g->ny);
  L.loss_part = c.take<float>((size_t)L.n_part);
  L.bytes = align_up(c.off, 256);
  return L;
}

static ZernBasis zernike_basis(int n_zern) {
  ZernBasis zb;
  memset(&zb, 0, sizeof(zb));
  zb.n_zern = n_zern;
  for (int j = 1; j <= n_zern; ++j) {
    int n, m;
    noll_nm(j, &n, &m);
    zb.m[j - 1] = m;
    zb.deg[j - 1] = n;
    zernike_radial_coeffs(n, m < 0 ? -m : m, zb.rc[j - 1]);
  }
  return zb;
}

extern "C" size_t psf_fourier_backward_workspace_size(const psf_optics* opt,
                                                       int n_pupil,
                                                       const psf_grid* grid,
                                                       int precision) {
  if (grid)
    precision = resolve_fourier_backward_precision(n_pupil, grid->nx, grid->ny, precision);
  if (check_fourier_args(opt, n_pupil, grid, precision)) return 0;
  if (precision == PSF_PREC_FP32_CHIRPZ || precision == PSF_PREC_SPLIT_TF32 ||
      precision == PSF_PREC_TF32)
    return 0;
  if (precision != PSF_PREC_FP32 && tc_fourier_bwd_supported(n_pupil, grid->nx, grid->ny))
    return 0;
  return backward_layout(nullptr, n_pupil, grid, precision).bytes;
}

extern "C" size_t psf_fourier_backward_workspace_size_batch(const psf_optics* opt,
                                                             int n_pupil, const psf_grid* grid,
                                                             int precision, int batch) {
  const size_t base = psf_fourier_backward_workspace_size(opt, n_pupil, grid, precision);
  if (base == 0 || batch < 1) return 0;
  precision = resolve_fourier_backward_precision(n_pupil, grid->nx, grid->ny, precision);
  const long long planes = (long long)batch * grid->nz;
  return backward_layout(nullptr, n_pupil, grid, precision, 66,
                         (int)(planes < 2048 ? planes : 2048)).bytes;
}

extern "C" int psf_fourier_vectorial_backward(
    const psf_optics* opt, int n_pupil, const psf_grid* grid, int batch,
    const double* zernike, int n_zern, const float* phase_map, int precision,
    const float* target, const float* grad_intensity, float* loss,
    float* grad_phase_map, float* grad_zernike, void* workspace,
    size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  if (grid)
    precision = resolve_fourier_backward_precision(n_pupil, grid->nx, grid->ny, precision);
  int r = check_fourier_args(opt, n_pupil, grid, precision);
  if (r) return r;
  if (precision == PSF_PREC_FP32_CHIRPZ || precision == PSF_PREC_SPLIT_TF32 ||
      precision == PSF_PREC_TF32)
    return fail(PSF_ERR_PRECISION, "the chirp-Z and TF32 modes are forward only");
  if (precision != PSF_PREC_FP32) {
    if (const char* why = tc_fourier_bwd_supported(n_pupil, grid->nx, grid->ny))
      return fail(PSF_ERR_ARG, "%s", why);
  }
  if (batch < 1) return fail(PSF_ERR_ARG, "batch must be >= 1");
  if (n_zern < 0 || n_zern > 66) return fail(PSF_ERR_ARG, "n_zern %d outside [0, 66]", n_zern);
  if (n_zern > 0 && !zernike) return fail(PSF_ERR_ARG, "zernike is NULL");
  for (long long j = 0; j < (long long)batch * n_zern; ++j)
    if (!isfinite(zernike[j])) return fail(PSF_ERR_ARG, "zernike[%lld] not finite", j);
  if (!target && !grad_intensity)
    return fail(PSF_ERR_ARG, "one of target / grad_intensity is required");
  if (loss && !target) return fail(PSF_ERR_ARG, "loss needs a target");
  if (!grad_phase_map && !grad_zernike && !loss)
    return fail(PSF_ERR_ARG, "no output requested");
  if (!workspace) return fail(PSF_ERR_WORKSPACE, "workspace is NULL");
  const int N = n_pupil;
  // the largest chunk (up to the whole batch, 2048 planes) the workspace holds
  int max_planes = (long long)batch * grid->nz < 2048 ? batch * grid->nz : 2048;
  while (max_planes > 128 &&
         backward_layout(nullptr, N, grid, precision, 66, max_planes).bytes > ws_bytes)
    max_planes = max_planes / 2 > 128 ? max_planes / 2 : 128;
  BackwardLayout L = backward_layout(workspace, N, grid, precision, 66, max_planes);
  if (ws_bytes < L.bytes)
    return fail(PSF_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, L.bytes);
  cudaStream_t s = (cudaStream_t)stream;
  const int nx = grid->nx, ny = grid->ny, nz = grid->nz;
  const size_t NN = (size_t)N * N, vox = (size_t)nz * nx * ny;

  std::vector<float2> zz(nz);
  for (int i = 0; i < nz; ++i) {
    const f2x v = split_double(grid->z[i]);
    zz[i] = make_float2(v.hi, v.lo);
  }
  cudaMemsetAsync(workspace, 0, sizeof(int), s);
  upload_async(L.zz, zz.data(), zz.size() * sizeof(float2), s);
  const double f = opt->NA / opt->lambda;
  const double ds = 2.0 * (opt->NA / opt->n_i) / N;
  const float scale = (float)(ds * ds / (2.0 * kPi));
  if (precision != PSF_PREC_FP32) {
    // tensor-core adjoint (split precision), one pupil at a time
    const ZernBasis zb = zernike_basis(n_zern);
    {
      TimingScope ts(kTimeSetup, s);
      if ((r = tc_fourier_bwd_setup(L.tc, N, nx, ny, grid->dx, grid->dy, f, precision, s)))
        return fail(r, "split-precision adjoint setup failed");
    }
    // groups of pupils share one pass over their planes (flat over (pupil, z));
    // the node table (amplitudes, defocus factors, Gibson-Lanni phase) is
    // common to all pupils, their phases differ by sum_j c_j Z_j + W_0
    const int gp = L.tc.group;
    const NodeParams np0 = node_params(opt, N, nullptr, 0, nullptr);
    const double amp_bound = tc_pupil_amplitude_bound(np0);   // phase-independent
    {
      TimingScope ts(kTimeSetup, s);
      launch_node_table(np0, L.nodes, s);        // L.nodes.wfr = Gibson-Lanni phase
      if (n_zern > 0) launch_zernike_table(zb, N, L.Zt, s);
    }
    for (int b0 = 0; b0 < batch; b0 += gp) {
      const int nb = batch - b0 < gp ? batch - b0 : gp;
      if (n_zern > 0)
        upload_async(L.tc.coef, zernike + (size_t)b0 * n_zern,
                        (size_t)nb * n_zern * sizeof(double), s);
      {
        TimingScope ts(kTimeSetup, s);
        tc_group_phase(L.tc, L.nodes.wfr, L.Zt, L.tc.coef, n_zern,
                       phase_map ? phase_map + (size_t)b0 * NN : nullptr, N, nb, s);
      }
      const float* Tb = target ? target + (size_t)b0 * vox : nullptr;
      const float* Gb = grad_intensity ? grad_intensity + (size_t)b0 * vox : nullptr;
      float* gWb = grad_phase_map ? grad_phase_map + (size_t)b0 * NN : L.tc.gW;
      r = tc_fourier_backward(L.tc, L.nodes, L.zz, N, nx, ny, nz, nb, L.zc, scale, amp_bound,
                              precision, Tb, Gb, gWb, loss ? loss + b0 : nullptr, L.Zt,
                              n_zern, L.zpart,
                              grad_zernike ? grad_zernike + (size_t)b0 * n_zern : nullptr,
                              (int*)workspace, s);
      if (r) return fail(r, "split-precision adjoint launch failed");
    }
    return cuda_check("psf_fourier_vectorial_backward launch");
  }
  launch_twiddle(N, nx, grid->dx, f, L.Ax, s);
  launch_twiddle(N, ny, grid->dy, f, L.Ay, s);
  launch_twiddle_adj(N, nx, grid->dx, f, L.AxH, s);
  launch_twiddle_adj(N, ny, grid->dy, f, L.AyH, s);
  const ZernBasis zb = zernike_basis(n_zern);
  if (grad_zernike) launch_zernike_table(zb, N, L.Zt, s);
  const int tiles = stage2_tiles(nx, ny);

  for (int b = 0; b < batch; ++b) {
    NodeParams np = node_params(opt, N, zernike ? zernike + (size_t)b * n_zern : nullptr,
                                n_zern, phase_map ? phase_map + (size_t)b * NN : nullptr);
    launch_node_table(np, L.nodes, s);
    cudaMemsetAsync(L.gW, 0, NN * sizeof(float), s);
    const float* Tb = target ? target + (size_t)b * vox : nullptr;
    const float* Gb = grad_intensity ? grad_intensity + (size_t)b * vox : nullptr;
    for (int z0 = 0; z0 < nz; z0 += L.zc) {
      const int nzc = nz - z0 < L.zc ? nz - z0 : L.zc;
      const size_t zoff = (size_t)z0 * nx * ny;
      launch_pupil_z_f32(L.nodes, N, L.zz, z0, nzc, L.P, s);
      launch_stage1_f32(L.Ay, L.P, L.U, N, ny, nzc, s);
      TimingScope ts(kTimeAdjoint, s);
      launch_stage2_adjsrc_f32(L.Ax, L.U, Tb ? Tb + zoff : nullptr,
                               Gb ? Gb + zoff : nullptr, L.RT,
                               L.loss_part + (size_t)z0 * tiles, N, nx, ny, nzc,
                               scale, s);
      // V[p][b] = sum_a conj(Ax[a][p]) R[a][b]    (M = N, N = ny, K = nx)
      launch_cgemm_nt_f32(L.AxH, 0, L.RT, (long long)ny * nx, L.V,
                          (long long)N * ny, N, ny, nx, nzc * 3, s);
      // Gh[p][q] = sum_b V[p][b] conj(Ay[b][q])   (M = N, N = N, K = ny)
      launch_cgemm_nt_f32(L.V, (long long)N * ny, L.AyH, 0, L.Gh, (long long)NN,
                          N, N, ny, nzc * 3, s);
      launch_grad_accum(L.Gh, L.P, L.gW, (int)NN, nzc, s);
    }
    if (loss) launch_sum_partials(L.loss_part, L.n_part, loss + b, s);
    if (grad_phase_map)
      cudaMemcpyAsync(grad_phase_map + (size_t)b * NN, L.gW, NN * sizeof(float),
                      cudaMemcpyDeviceToDevice, s);
    if (grad_zernike)
      launch_zernike_grad(zb, N, L.Zt, L.gW, 1, L.zpart, grad_zernike + (size_t)b * n_zern, s);
  }
  return cuda_check("psf_fourier_vectorial_backward launch");
}

// ===========================================================================
// Bessel strategy
// ===========================================================================
struct BesselLayout {
  double* theta_tab;     // (10 + kMaxM0 + 6) x n_theta doubles
  float* kappa;          // 2 x n_theta floats
  float* Bt;
  float2* BtC;           // complex J_n operand (Fresnel weights), FP32 path
  EmitterTable et;
  int* slice_em;
  float2* zz;
  float2* prof;
  int* pix_i0;
  float* pix_f;
  float* pix_g;
  float4* qtab;
  TcBessel tc;           // split-precision operands
  size_t bytes;
};

// complex_g: the model's angular weights are complex (Fresnel coefficients)
static bool bessel_complex_g(const psf_optics* base) {
  return (base->flags & PSF_FRESNEL) && !(base->flags & PSF_SCALAR);
}

static BesselLayout bessel_layout(void* ws, int n_em, int n_slices, int n_theta,
                                  int n_r, int nx, int ny, bool own_profiles,
                                  int precision, bool complex_g, bool fp32_bt = false) {
  BesselLayout L;
  memset(&L, 0, sizeof(L));
  Carver c(ws);
  L.theta_tab = c.take<double>((size_t)(10 + kMaxM0 + 6) * n_theta);
  L.kappa = c.take<float>(2 * (size_t)n_theta);
  if (precision == PSF_PREC_FP32 || (fp32_bt && !complex_g))
    L.Bt = c.take<float>((size_t)3 * n_r * n_theta);
  if (precision == PSF_PREC_FP32 || (fp32_bt && complex_g))
    L.BtC = c.take<float2>((size_t)3 * n_r * n_theta);
  if (precision != PSF_PREC_FP32)
    tc_bessel_carve(c.base, &c.off, n_theta, n_r, n_slices, complex_g, &L.tc);
  L.et.amp = c.take<float>((size_t)n_em * n_theta);
  L.et.wfr = c.take<float>((size_t)n_em * n_theta);
  L.et.valid = c.take<int>(n_em);
  L.slice_em = c.take<int>(n_slices);
  L.zz = c.take<float2>(n_slices);
  if (own_profiles) L.prof = c.take<float2>((size_t)n_slices * 3 * n_r);
  L.pix_i0 = c.take<int>((size_t)nx * ny);
  L.pix_f = c.take<float>((size_t)nx * ny);
  L.pix_g = c.take<float>((size_t)nx * ny);
  L.qtab = c.take<float4>((size_t)(nx / 2) * (ny / 2) + 1);
  L.bytes = align_up(c.off, 256);
  return L;
}

static int check_bessel_args(const psf_optics* base, int n_em, int n_slices,
                             int n_theta, int n_r, int nx, int ny, int precision) {
  int r = check_optics(base);
  if (r) return r;
  if (n_em < 1) return fail(PSF_ERR_ARG, "n_emitters must be >= 1");
  if (n_slices < 0) return fail(PSF_ERR_ARG, "n_slices must be >= 0");
  if (n_theta < 2 || n_theta > 880) return fail(PSF_ERR_ARG, "n_theta %d outside [2, 880]", n_theta);
  if (n_r < 2 || n_r > 4096) return fail(PSF_ERR_ARG, "n_r %d outside [2, 4096]", n_r);
  if (nx < 1 || ny < 1 || nx > 16384 || ny > 16384)
    return fail(PSF_ERR_ARG, "nx, ny must be in [1, 16384]");
  if (precision != PSF_PREC_FP32 && precision != PSF_PREC_SPLIT_FP16 &&
      precision != PSF_PREC_SPLIT_BF16)
    return fail(PSF_ERR_PRECISION, "unknown precision mode %d", precision);
  return PSF_OK;
}

extern "C" size_t psf_bessel_workspace_size(const psf_optics* base, int n_em,
                                            int n_slices, int n_theta, int n_r,
                                            int nx, int ny, int precision) {
  precision = resolve_spherical_precision(n_theta, precision);
  if (check_bessel_args(base, n_em, n_slices, n_theta, n_r, nx, ny, precision)) return 0;
  if (spherical_envelope(base, n_theta, precision)) return 0;
  return bessel_layout(nullptr, n_em, n_slices, n_theta, n_r, nx, ny, true,
                       precision, bessel_complex_g(base)).bytes;
}

// Host-side tables of one Bessel call and the setup launches shared by the
// forward and the adjoint: per-theta FP64 table, J_n operand, per-emitter
// integrand table, slice map and pixel table.
struct BesselRun {
  BesselParams bp;
  ThetaTable tt;
  double max_w;
  double g_max;          // max |g_n(theta_j)| over orders and nodes
  bool split;
};

static int bessel_prepare(const psf_optics* base, int n_em, const double* depth,
                          const double* zernike, int n_zern, const float* phase_theta,
                          const int* z_offsets, const double* z, int n_slices,
                          int n_theta, int n_r, int nx, int ny, double dx, double dy,
                          int precision, bool fp32_operand, BesselLayout& L,
                          void* workspace, BesselRun* R, cudaStream_t s) {
  int r;
  // Per-theta FP64 table: GL nodes on [0, theta_max]; W_GL affine in t_s.
  const double s_max = base->NA / base->n_i;
  const double th_max = asin(s_max);
  std::vector<double> gx, gw;
  gauss_legendre(n_theta, gx, gw);
  std::vector<double> tab((size_t)(10 + kMaxM0 + 6) * n_theta, 0.0);
  std::vector<float> kap(2 * (size_t)n_theta);
  double* T_th = tab.data();
  double* T_w = T_th + n_theta;
  double* T_s = T_w + n_theta;
  double* T_c = T_s + n_theta;
  double* T_are = T_c + n_theta;
  double* T_aim = T_are + n_theta;
  double* T_bre = T_aim + n_theta;
  double* T_bim = T_bre + n_theta;
  double* T_amp = T_bim + n_theta;
  double* T_zm0 = T_amp + 2 * n_theta;   // slot 9 unused (alignment)
  double* T_g = T_zm0 + (size_t)kMaxM0 * n_theta;   // [3][re, im][n_theta]
  const bool scalar = (base->flags & PSF_SCALAR) != 0;
  const bool fresnel = !scalar && (base->flags & PSF_FRESNEL) != 0;
  const GLLayers L0 = gl_layers(base, 0.0), L1 = gl_layers(base, 1.0);
  BesselParams& bp = R->bp;
  memset(&bp, 0, sizeof(bp));
  int m0_j[kMaxM0], n_m0 = 0;
  unsigned long long mask[2] = {0, 0};
  for (int j = 1; j <= n_zern; ++j) {
    int n, m;
    noll_nm(j, &n, &m);
    if (m == 0) {
      if (n_m0 < kMaxM0) m0_j[n_m0++] = j;
    } else {
      mask[(j - 1) >> 6] |= 1ULL << ((j - 1) & 63);
    }
  }
  for (int j = 0; j < n_theta; ++j) {
    const double th = 0.5 * th_max * (gx[j] + 1.0);
    const double st = sin(th), ct = cos(th);
    T_th[j] = th;
    T_w[j] = 0.5 * th_max * gw[j];
    T_s[j] = st;
    T_c[j] = ct;
    // W/(2 pi) = sum_l t_l(t_s) sqrt(n_l^2 - n_i^2 s^2)/lambda, t_l affine in t_s
    double a_re = 0, a_im = 0, b_re = 0, b_im = 0;
    for (int l = 0; l < 5; ++l) {
      const double arg = L0.n_idx[l] * L0.n_idx[l] - (base->n_i * st) * (base->n_i * st);
      const double root = sqrt(fabs(arg)) / base->lambda;
      const double tb = L0.t[l], ta = L1.t[l] - L0.t[l];
      if (arg >= 0) {
        a_re += ta * root;
        b_re += tb * root;
      } else {
        a_im += ta * root;
        b_im += tb * root;
      }
    }
    T_are[j] = a_re;
    T_aim[j] = a_im;
    T_bre[j] = b_re;
    T_bim[j] = b_im;
    double amp = base->apodize ? sqrt(ct) : 1.0;
    if (base->s_env > 0) amp *= exp(-(st * st) / (base->s_env * base->s_env));
    T_amp[j] = amp;
    const double rho = st / s_max;
    for (int q = 0; q < n_m0; ++q) {
      int n, m;
      noll_nm(m0_j[q], &n, &m);
      double rc[kZernMaxOrder + 1];
      zernike_radial_coeffs(n, 0, rc);
      double v = 0;
      for (int k = kZernMaxOrder; k >= 0; --k) v = v * rho + rc[k];
      T_zm0[(size_t)q * n_theta + j] = v;
    }
    const f2x kv = split_double(base->n_i * ct / base->lambda);
    kap[j] = kv.hi;
    kap[n_theta + j] = kv.lo;
    // angular weights g_n of the model (Eq. 11; Eq. 6-7 with Fresnel; Eq. 5)
    dcplx g[3];
    if (scalar) {
      g[0] = {2.0 * st, 0.0};
      g[1] = g[2] = {0.0, 0.0};
    } else if (fresnel) {
      dcplx qs, qp;
      fresnel_q(base->n_s, base->n_g, base->n_i, st, qs, qp);
      g[0] = st * (qs + ct * qp);
      g[1] = (st * st) * qp;
      g[2] = st * (ct * qp - qs);
    } else {
      g[0] = {st * (1.0 + ct), 0.0};
      g[1] = {st * st, 0.0};
      g[2] = {st * (ct - 1.0), 0.0};
    }
    for (int n = 0; n < 3; ++n) {
      T_g[(size_t)(2 * n) * n_theta + j] = g[n].re;
      T_g[(size_t)(2 * n + 1) * n_theta + j] = g[n].im;
    }
  }
  ThetaTable& tt = R->tt;
  tt.theta = L.theta_tab;
  tt.w = L.theta_tab + n_theta;
  tt.sin_t = tt.w + n_theta;
  tt.cos_t = tt.sin_t + n_theta;
  tt.a_re = tt.cos_t + n_theta;
  tt.a_im = tt.a_re + n_theta;
  tt.b_re = tt.a_im + n_theta;
  tt.b_im = tt.b_re + n_theta;
  tt.amp0 = tt.b_im + n_theta;
  tt.zm0 = tt.amp0 + 2 * n_theta;
  tt.g = tt.zm0 + (size_t)kMaxM0 * n_theta;
  tt.kh = L.kappa;
  tt.kl = L.kappa + n_theta;

  bp.n_theta = n_theta;
  bp.n_r = n_r;
  bp.nx = nx;
  bp.ny = ny;
  bp.n_em = n_em;
  bp.n_slices = n_slices;
  bp.n_zern = n_zern;
  bp.k = 2.0 * kPi * base->n_i / base->lambda;
  bp.r_max = sqrt(0.25 * (nx - 1) * (nx - 1) * dx * dx + 0.25 * (ny - 1) * (ny - 1) * dy * dy);
  bp.dr = bp.r_max / (n_r - 1);
  bp.dx = dx;
  bp.dy = dy;
  bp.n_m0 = n_m0;
  for (int q = 0; q < n_m0; ++q) bp.m0_j[q] = m0_j[q];
  bp.nonaxis_mask[0] = mask[0];
  bp.nonaxis_mask[1] = mask[1];
  bp.project = (base->flags & PSF_PROJECT_AXISYMMETRIC) ? 1 : 0;
  for (int i = 0; i < 4; ++i) bp.pol[i] = base->pol[i];
  if (scalar) {                 // Eq. 5 rides on channel x of Eq. 10
    bp.pol[0] = 1.0;
    bp.pol[1] = bp.pol[2] = bp.pol[3] = 0.0;
  }
  bp.complex_g = fresnel ? 1 : 0;

  cudaMemsetAsync(workspace, 0, sizeof(int), s);
  upload_async(L.theta_tab, tab.data(), tab.size() * sizeof(double), s);
  upload_async(L.kappa, kap.data(), kap.size() * sizeof(float), s);
  if ((r = cuda_check("workspace init"))) return r;

  R->split = !fp32_operand && precision != PSF_PREC_FP32;
  const bool split = R->split;
  double max_w = 0.0, g_max = 0.0;
  for (int j = 0; j < n_theta; ++j) max_w = fmax(max_w, T_w[j]);
  for (int n = 0; n < 3; ++n)
    for (int j = 0; j < n_theta; ++j)
      g_max = fmax(g_max, hypot(T_g[(size_t)(2 * n) * n_theta + j],
                                T_g[(size_t)(2 * n + 1) * n_theta + j]));
  R->max_w = max_w;
  R->g_max = g_max;
  {
    TimingScope ts(kTimeSetup, s);
    if (split)
      tc_bessel_jmat(bp, tt, max_w, precision, L.tc, s);
    else if (bp.complex_g)
      launch_bessel_jmat_complex(bp, tt, L.BtC, s);
    else
      launch_bessel_jmat(bp, tt, L.Bt, s);
  }
  if (split) cudaMemsetAsync(L.tc.amp_max, 0, sizeof(unsigned), s);
  {
    TimingScope ts(kTimeSetup, s);
    launch_bessel_emitters(bp, tt, depth, n_zern > 0 ? zernike : nullptr, phase_theta,
                           L.et, (int*)workspace, split ? L.tc.amp_max : nullptr, s);
  }
  if (n_slices > 0) {
    // slices no emitter claims keep emitter -1 and are skipped
    cudaMemsetAsync(L.slice_em, 0xFF, (size_t)n_slices * sizeof(int), s);
    {
      TimingScope ts(kTimeSetup, s);
      launch_slice_map(bp, z_offsets, z, L.slice_em, L.zz, (int*)workspace, s);
    }
    {
      TimingScope ts(kTimeSetup, s);
      launch_pixel_table(bp, L.pix_i0, L.pix_f, L.pix_g, s);
    }
  }
  return cuda_check("Bessel setup launch");
}

static int check_bessel_call(const psf_optics* base, int n_em, const double* depth,
                             const double* zernike, int n_zern, const int* z_offsets,
                             const double* z, int n_slices, int n_theta, int n_r, int nx,
                             int ny, double dx, double dy, int precision) {
  int r = check_bessel_args(base, n_em, n_slices, n_theta, n_r, nx, ny, precision);
  if (r) return r;
  if (!finite_pos(dx) || !finite_pos(dy)) return fail(PSF_ERR_ARG, "pixel pitch must be > 0");
  if (n_zern < 0 || n_zern > 66) return fail(PSF_ERR_ARG, "n_zern %d outside [0, 66]", n_zern);
  if (!depth || !z_offsets || (n_slices > 0 && !z) || (n_zern > 0 && !zernike))
    return fail(PSF_ERR_ARG, "depth / z_offsets / z / zernike pointer is NULL");
  return PSF_OK;
}

extern "C" int psf_bessel_vectorial(const psf_optics* base, int n_em,
                                    const double* depth, const double* zernike,
                                    int n_zern, const float* phase_theta,
                                    const int* z_offsets, const double* z, int n_slices,
                                    int n_theta, int n_r, int nx, int ny, double dx,
                                    double dy, int precision, float* intensity,
                                    void* profiles, void* workspace,
                                    size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  precision = resolve_spherical_precision(n_theta, precision);
  int r = check_bessel_call(base, n_em, depth, zernike, n_zern, z_offsets, z, n_slices,
                            n_theta, n_r, nx, ny, dx, dy, precision);
  if (r) return r;
  if ((r = spherical_envelope(base, n_theta, precision))) return r;
  if (!intensity && !profiles && n_slices > 0)
    return fail(PSF_ERR_ARG, "intensity and profiles are both NULL");
  if (!workspace) return fail(PSF_ERR_WORKSPACE, "workspace is NULL");
  BesselLayout L = bessel_layout(workspace, n_em, n_slices, n_theta, n_r, nx, ny,
                                 profiles == nullptr, precision, bessel_complex_g(base));
  if (ws_bytes < L.bytes)
    return fail(PSF_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, L.bytes);
  if ((r = resolve_output((void**)&intensity, "intensity")) ||
      (r = resolve_output(&profiles, "profiles")))
    return r;
  if (profiles) L.prof = (float2*)profiles;
  cudaStream_t s = (cudaStream_t)stream;
  BesselRun R;
  r = bessel_prepare(base, n_em, depth, zernike, n_zern, phase_theta, z_offsets, z,
                     n_slices, n_theta, n_r, nx, ny, dx, dy, precision, false, L,
                     workspace, &R, s);
  if (r) return r;
  const BesselParams& bp = R.bp;
  if (n_slices > 0) {
    if (R.split) {
      r = tc_bessel_contract(bp, R.tt, L.et, L.slice_em, L.zz, R.max_w, R.g_max, precision,
                             L.tc, L.prof, (int*)workspace, s);
      if (r) return fail(r, "split-precision Bessel contraction launch failed");
    } else if (bp.complex_g) {
      TimingScope ts(kTimeBesselRadial, s);
      launch_bessel_profiles_f32c(bp, R.tt, L.BtC, L.et, L.slice_em, L.zz, L.prof, s);
    } else {
      TimingScope ts(kTimeBesselRadial, s);
      launch_bessel_profiles_f32(bp, R.tt, L.Bt, L.et, L.slice_em, L.zz, L.prof, s);
    }
    if (!intensity) {
      // profiles only: no radial -> Cartesian epilogue
    } else if (bessel_mirror_fit(nx, ny, n_r) && ((uintptr_t)intensity & 15) == 0) {
      {
        TimingScope ts(kTimeSetup, s);
        launch_quarter_table(bp, L.qtab, s);
      }
      TimingScope ts(kTimeBesselEpilogue, s);
      launch_bessel_intensity_mirror(bp, L.prof, L.slice_em, L.et.valid, L.qtab,
                                     intensity, s);
    } else {
      TimingScope ts(kTimeBesselEpilogue, s);
      launch_bessel_intensity(bp, L.prof, L.slice_em, L.et.valid, L.pix_i0,
                              L.pix_f, L.pix_g, intensity, s);
    }
  }
  return cuda_check("psf_bessel_vectorial launch");
}

// ---------------------------------------------------------------------------
// Bessel adjoint
// ---------------------------------------------------------------------------
struct BesselBwdLayout {
  BesselLayout fwd;      // forward tables + FP32 J_n operand + own profiles
  float2* gF;            // [n_slices][n_theta]
  float* loss_slice;     // [n_slices]
  PixGroup* groups;      // [n_groups], cell-sorted
  int* cell_start;       // [n_r]
  int2* gpc;             // [n_groups] natural order: (sorted position, cell)
  float4* gfg;           // [n_groups] natural order: (f, gc, gs, 0)
  float* sorted_f;       // [n_groups]
  bool sorted_form;      // two-pass epilogue + tensor-core contraction
  TcBesselAdj tc;
  size_t bytes;
};

static size_t n_pix_groups(int nx, int ny) {
  return (size_t)((nx + 1) / 2) * (size_t)((ny + 1) / 2);
}

static BesselBwdLayout bessel_bwd_layout(void* ws, int n_em, int n_slices, int n_theta,
                                         int n_r, int nx, int ny, int precision,
                                         bool complex_g) {
  BesselBwdLayout B;
  memset(&B, 0, sizeof(B));
  B.fwd = bessel_layout(ws, n_em, n_slices, n_theta, n_r, nx, ny, true, precision, complex_g,
                        true);
  Carver c(ws);
  c.off = B.fwd.bytes;
  B.gF = c.take<float2>((size_t)n_slices * n_theta);
  B.loss_slice = c.take<float>((size_t)n_slices + 1);
  B.groups = c.take<PixGroup>(n_pix_groups(nx, ny));
  B.cell_start = c.take<int>((size_t)n_r);
  B.gpc = c.take<int2>(n_pix_groups(nx, ny));
  B.gfg = c.take<float4>(n_pix_groups(nx, ny));
  B.sorted_f = c.take<float>(n_pix_groups(nx, ny));
  BesselParams q;
  memset(&q, 0, sizeof(q));
  q.nx = nx;
  q.ny = ny;
  q.n_r = n_r;
  B.sorted_form = bessel_adj_sorted_fits(q);
  if (B.sorted_form && precision != PSF_PREC_FP32)
    tc_bessel_adj_carve(c.base, &c.off, n_theta, n_r, n_slices, complex_g, &B.tc);
  B.bytes = align_up(c.off, 256);
  return B;
}

// Pixels grouped by shared radius (a pixel and its mirrors), sorted by
// interpolation cell with a stable counting sort: the adjoint visits every
// cell's pixels in this fixed order.  FP64 geometry, same rule as the forward
// pixel table.
struct PixTables {
  std::vector<PixGroup> sorted;    // cell-sorted groups
  std::vector<int> start;          // [n_r]
  std::vector<int2> pc;            // natural order: (sorted position, cell)
  std::vector<float4> fg;          // natural order: (f, gc, gs, 0)
  std::vector<float> sorted_f;
};

static void build_pix_groups(int nx, int ny, double dx, double dy, int n_r, double dr,
                             const double* pol, PixTables& T) {
  std::vector<PixGroup>& out = T.sorted;
  std::vector<int>& start = T.start;
  const int ha = (nx + 1) / 2, hb = (ny + 1) / 2;
  const double S1 = pol[0] * pol[0] + pol[1] * pol[1] - pol[2] * pol[2] - pol[3] * pol[3];
  const double S2 = 2.0 * (pol[0] * pol[2] + pol[1] * pol[3]);
  std::vector<PixGroup> g((size_t)ha * hb);
  std::vector<int> count(n_r, 0);
  for (int a = 0; a < ha; ++a)
    for (int b = 0; b < hb; ++b) {
      PixGroup& q = g[(size_t)a * hb + b];
      const double x = (a - 0.5 * (nx - 1)) * dx;
      const double y = (b - 0.5 * (ny - 1)) * dy;
      const double rho = sqrt(x * x + y * y);
      const double tt = dr > 0 ? rho / dr : 0.0;
      int c = (int)floor(tt);
      c = c < 0 ? 0 : (c > n_r - 2 ? n_r - 2 : c);
      q.cell = c;
      q.f = (float)(tt - c);
      double c2 = 1.0, s2 = 0.0;
      if (rho > 0) {
        c2 = (x * x - y * y) / (rho * rho);
        s2 = 2.0 * x * y / (rho * rho);
      }
      q.gc = (float)(S1 * c2);
      q.gs = (float)(S2 * s2);
      const int a2 = nx - 1 - a, b2 = ny - 1 - b;
      q.pix[0] = a * ny + b;
      q.pix[1] = a2 != a ? a2 * ny + b : -1;
      q.pix[2] = b2 != b ? a * ny + b2 : -1;
      q.pix[3] = (a2 != a && b2 != b) ? a2 * ny + b2 : -1;
      ++count[c];
    }
  start.assign(n_r, 0);
  for (int c = 1; c < n_r; ++c) start[c] = start[c - 1] + count[c - 1];
  out.resize(g.size());
  T.pc.resize(g.size());
  T.fg.resize(g.size());
  T.sorted_f.resize(g.size());
  std::vector<int> pos(start.begin(), start.end());
  for (size_t i = 0; i < g.size(); ++i) {
    const PixGroup& q = g[i];
    const int k = pos[q.cell]++;
    out[k] = q;
    T.pc[i] = make_int2(k, q.cell);
    T.fg[i] = make_float4(q.f, q.gc, q.gs, 0.f);
    T.sorted_f[k] = q.f;
  }
}

extern "C" size_t psf_bessel_backward_workspace_size(const psf_optics* base, int n_em,
                                                     int n_slices, int n_theta, int n_r,
                                                     int nx, int ny, int precision) {
  precision = resolve_bessel_backward_precision(precision);
  if (check_bessel_args(base, n_em, n_slices, n_theta, n_r, nx, ny, precision)) return 0;
  if (nx > 4096 || ny > 4096 || n_r > 4096) return 0;
  return bessel_bwd_layout(nullptr, n_em, n_slices, n_theta, n_r, nx, ny, precision,
                           bessel_complex_g(base)).bytes;
}

extern "C" int psf_bessel_vectorial_backward(
    const psf_optics* base, int n_em, const double* depth, const double* zernike,
    int n_zern, const float* phase_theta, const int* z_offsets, const double* z,
    int n_slices, int n_theta, int n_r, int nx, int ny, double dx, double dy,
    int precision, const float* target, const float* grad_intensity, float* loss,
    float* grad_phase_theta, float* grad_zernike, float* grad_depth, void* workspace,
    size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  precision = resolve_bessel_backward_precision(precision);
  int r = check_bessel_call(base, n_em, depth, zernike, n_zern, z_offsets, z, n_slices,
                            n_theta, n_r, nx, ny, dx, dy, precision);
  if (r) return r;
  if (nx > 4096 || ny > 4096)
    return fail(PSF_ERR_ARG, "the Bessel adjoint takes nx, ny <= 4096");
  if (n_slices > 0 && !target && !grad_intensity)
    return fail(PSF_ERR_ARG, "target and grad_intensity are both NULL");
  if (loss && !target) return fail(PSF_ERR_ARG, "loss needs a target");
  if (!workspace) return fail(PSF_ERR_WORKSPACE, "workspace is NULL");
  BesselBwdLayout B = bessel_bwd_layout(workspace, n_em, n_slices, n_theta, n_r, nx, ny,
                                        precision, bessel_complex_g(base));
  if (ws_bytes < B.bytes)
    return fail(PSF_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, B.bytes);
  BesselLayout& L = B.fwd;
  cudaStream_t s = (cudaStream_t)stream;
  BesselRun R;
  r = bessel_prepare(base, n_em, depth, zernike, n_zern, phase_theta, z_offsets, z,
                     n_slices, n_theta, n_r, nx, ny, dx, dy, precision, false, L, workspace,
                     &R, s);
  if (r) return r;
  const BesselParams& bp = R.bp;
  const bool split = R.split;
  if (split) {
    // the adjoint contraction takes the J_n operand unscaled in FP32 as well
    TimingScope ts(kTimeSetup, s);
    if (bp.complex_g)
      launch_bessel_jmat_complex(bp, R.tt, L.BtC, s);
    else
      launch_bessel_jmat(bp, R.tt, L.Bt, s);
  }
  // the adjoint contraction's operand: B^H with complex weights
  const float* adj_Bt = bp.complex_g ? nullptr : L.Bt;
  const float2* adj_BtC = bp.complex_g ? L.BtC : nullptr;
  if (n_slices > 0) {
    PixTables pt;
    build_pix_groups(nx, ny, dx, dy, n_r, bp.dr, bp.pol, pt);
    const size_t ng = pt.sorted.size();
    const bool sorted_form = B.sorted_form;
    const bool tc_adj = sorted_form && split;
    if (sorted_form) {
      upload_async(B.gpc, pt.pc.data(), ng * sizeof(int2), s);
      upload_async(B.gfg, pt.fg.data(), ng * sizeof(float4), s);
      upload_async(B.sorted_f, pt.sorted_f.data(), ng * sizeof(float), s);
    } else {
      upload_async(B.groups, pt.sorted.data(), ng * sizeof(PixGroup), s);
    }
    upload_async(B.cell_start, pt.start.data(), pt.start.size() * sizeof(int), s);
    // recompute the profiles (per-z recomputation: nothing of the forward is stored)
    if (split) {
      r = tc_bessel_contract(bp, R.tt, L.et, L.slice_em, L.zz, R.max_w, R.g_max, precision,
                             L.tc, L.prof, (int*)workspace, s);
      if (r) return fail(r, "split-precision Bessel contraction launch failed");
    } else if (bp.complex_g) {
      TimingScope ts(kTimeBesselRadial, s);
      launch_bessel_profiles_f32c(bp, R.tt, L.BtC, L.et, L.slice_em, L.zz, L.prof, s);
    } else {
      TimingScope ts(kTimeBesselRadial, s);
      launch_bessel_profiles_f32(bp, R.tt, L.Bt, L.et, L.slice_em, L.zz, L.prof, s);
    }
    {
      TimingScope ts(kTimeAdjoint, s);
      const float* src = target ? target : grad_intensity;
      const bool staged = sorted_form && bessel_adj_staged_fits(bp, src);
      if (tc_adj) {
        if (staged)
          launch_bessel_adj_epilogue_staged(bp, L.prof, L.slice_em, L.et.valid, B.gpc, B.gfg,
                                            B.sorted_f, B.cell_start, target,
                                            target ? nullptr : grad_intensity, B.loss_slice,
                                            B.tc.G_hi, B.tc.G_lo, B.tc.kp, (int*)workspace,
                                            s);
        else
          launch_bessel_adj_epilogue_sorted(bp, L.prof, L.slice_em, L.et.valid, B.gpc,
                                            B.gfg, B.sorted_f, B.cell_start, target,
                                            target ? nullptr : grad_intensity, B.loss_slice,
                                            B.tc.G_hi, B.tc.G_lo, B.tc.kp, s);
        r = tc_bessel_adj_contract(bp, adj_Bt, adj_BtC, B.tc, B.gF, (int*)workspace, s);
        if (r) return fail(r, "tensor-core adjoint contraction launch failed");
      } else if (sorted_form) {
        if (staged)
          launch_bessel_adj_epilogue_staged(bp, L.prof, L.slice_em, L.et.valid, B.gpc, B.gfg,
                                            B.sorted_f, B.cell_start, target,
                                            target ? nullptr : grad_intensity, B.loss_slice,
                                            nullptr, nullptr, 0, (int*)workspace, s);
        else
          launch_bessel_adj_epilogue_sorted(bp, L.prof, L.slice_em, L.et.valid, B.gpc,
                                            B.gfg, B.sorted_f, B.cell_start, target,
                                            target ? nullptr : grad_intensity, B.loss_slice,
                                            nullptr, nullptr, 0, s);
        launch_bessel_adj_contract(bp, adj_Bt, adj_BtC, L.prof, B.gF, s);
      } else {
        launch_bessel_adj_epilogue(bp, L.prof, L.slice_em, L.et.valid, B.groups,
                                   B.cell_start, target, target ? nullptr : grad_intensity,
                                   B.loss_slice, s);
        launch_bessel_adj_contract(bp, adj_Bt, adj_BtC, L.prof, B.gF, s);
      }
    }
  }
  {
    TimingScope ts(kTimeAdjoint, s);
    launch_bessel_adj_reduce(bp, R.tt, L.et, z_offsets, L.zz, B.gF,
                             (target && n_slices > 0) ? B.loss_slice : nullptr, loss,
                             grad_phase_theta, grad_zernike, grad_depth, s);
  }
  return cuda_check("psf_bessel_vectorial_backward launch");
}

// ===========================================================================
// Spherical strategy without axial symmetry: azimuthal harmonics of the
// pupil (Eq. 9 with the Jacobi-Anger expansion; the harmonics of Eq. 6).
// ===========================================================================
static int harm_n_phi(int m_max) {
  int p = 1;
  while (p < m_max + 1) p *= 2;
  return 4 * p;
}

struct HarmLayout {
  BesselLayout b;
  float2* cs;      // [n_phi] e^{2 pi i k / n_phi}
  float* Zr;       // [kHarmMaxNA][n_theta] N_j R_n^{|m|}(sin theta / s_max)
  float2* Pm;      // [n_em][2 m_max + 1][n_theta] pupil harmonics
  int* ord;        // [n_em] adaptive order M_e
  float2* Bh;      // [n_em][3][n_ord][n_theta]
  float* Jt;       // [m_max + 3][n_r][n_theta]
  float2* D;       // [chunk][n_theta]
  float2* prof;    // [chunk][3][n_ord][n_r]
  int* octcnt;     // [n_r] counting-sort scratch (square grids)
  OctPix* octab;   // [octant pixels] ordered by radius sample (square grids)
  TcHarm tc;       // split operands of the tensor-core contraction
  int chunk;
  size_t bytes;
};

// The split form takes FP16 parts only: hi + lo in BF16 keeps 16 mantissa
// bits, and on the parity cases the harmonic stacks then missed the 1e-5
// bound (2.9e-5).
static bool harm_split(int precision) { return precision == PSF_PREC_SPLIT_FP16; }

static HarmLayout harm_layout(void* ws, int n_em, int n_slices, int n_theta, int n_r,
                              int nx, int ny, int m_max, int precision) {
  const bool split = harm_split(precision);
  HarmLayout H;
  memset(&H, 0, sizeof(H));
  H.b = bessel_layout(ws, n_em, n_slices, n_theta, n_r, nx, ny, false, PSF_PREC_FP32, false);
  Carver c(ws);
  c.off = H.b.bytes;
  const int n_ord = 2 * m_max + 5;
  H.cs = c.take<float2>(harm_n_phi(m_max));
  H.Zr = c.take<float>((size_t)kHarmMaxNA * n_theta);
  H.Pm = c.take<float2>((size_t)n_em * (2 * m_max + 1) * n_theta);
  H.ord = c.take<int>((size_t)(n_em > 0 ? n_em : 1));
  H.Bh = c.take<float2>((size_t)n_em * 3 * n_ord * n_theta);
  H.Jt = split ? nullptr : c.take<float>((size_t)(m_max + 3) * n_r * n_theta);
  // profiles (and the split B operand) of a slice chunk up to 1 GB
  double per_slice = 8.0 * (3.0 * n_ord * n_r + n_theta);
  if (split) per_slice += 4.0 * 6.0 * n_ord * tc_bessel_kp(n_theta);
  // (measured on the 256-emitter workload: 1 GB 12.0 ms, 256 MB 12.0, 96 MB
  // 12.9, 48 MB 14.5: the epilogue does not gain from profiles left in L2)
  long long chunk = (long long)(1024.0 * 1048576.0 / per_slice);
  if (chunk > n_slices) chunk = n_slices;
  if (chunk > 65535) chunk = 65535;
  if (chunk < 1) chunk = 1;
  H.chunk = (int)chunk;
  H.D = c.take<float2>((size_t)chunk * n_theta);
  H.prof = c.take<float2>((size_t)chunk * 3 * n_ord * n_r);
  const long long h = (nx + 1) / 2;
  const long long npx = nx == ny ? h * (h + 1) / 2 : 0;   // used when also dx = dy
  H.octcnt = c.take<int>((size_t)n_r);
  H.octab = c.take<OctPix>((size_t)(npx > 0 ? npx : 1));
  if (split) {
    size_t off = c.off;
    tc_harm_carve((char*)ws, &off, n_theta, n_r, m_max, (int)chunk, &H.tc);
    c.off = off;
  }
  H.bytes = align_up(c.off, 256);
  return H;
}

extern "C" int psf_bessel_harmonic_order(const double* zernike, int n_em, int n_zern,
                                         double tol) {
  g_err[0] = 0;
  if (n_em < 0 || n_zern < 0 || n_zern > 66 || (n_em > 0 && n_zern > 0 && !zernike) ||
      !(tol > 0.0) || !(tol < 1.0))
    return fail(PSF_ERR_ARG, "psf_bessel_harmonic_order: bad arguments");
  int best = 0;
  for (int e = 0; e < n_em; ++e) {
    double alpha = 0.0;
    int d = 0;
    for (int j = 1; j <= n_zern; ++j) {
      const double c = zernike[(size_t)e * n_zern + j - 1];
      int n, m;
      noll_nm(j, &n, &m);
      if (m == 0 || c == 0.0) continue;
      if (!isfinite(c)) return fail(PSF_ERR_ARG, "zernike not finite");
      alpha += fabs(c) * sqrt(2.0 * (n + 1.0));
      d = abs(m) > d ? abs(m) : d;
    }
    if (d == 0) continue;
    // tail of e^{i W}: sum_{k > K} alpha^k / k! <= alpha^{K+1} / (K+1)! e^alpha
    int K = 0;
    double term = alpha;
    while (term * exp(alpha) > tol && K < 1000) {
      ++K;
      term *= alpha / (K + 1);
    }
    const int M = (K > 1 ? K : 1) * d;
    best = M > best ? M : best;
  }
  return best;
}

static int check_harm_args(const psf_optics* base, int m_max, int n_theta, int precision) {
  if (m_max < 0 || m_max > kHarmMaxM)
    return fail(PSF_ERR_ARG, "m_max %d outside [0, %d]", m_max, kHarmMaxM);
  if (precision != PSF_PREC_FP32 && !harm_split(precision))
    return fail(PSF_ERR_PRECISION, "harmonic path: precision %d is not FP32 or split FP16",
                precision);
  return spherical_envelope(base, n_theta, precision);
}

extern "C" size_t psf_bessel_harmonic_workspace_size(const psf_optics* base, int n_em,
                                                     int n_slices, int n_theta, int n_r,
                                                     int nx, int ny, int m_max,
                                                     int precision) {
  if (check_bessel_args(base, n_em, n_slices, n_theta, n_r, nx, ny, PSF_PREC_FP32)) return 0;
  precision = resolve_spherical_precision(n_theta, precision);
  if (check_harm_args(base, m_max, n_theta, precision)) return 0;
  return harm_layout(nullptr, n_em, n_slices, n_theta, n_r, nx, ny, m_max, precision).bytes;
}

extern "C" int psf_bessel_vectorial_harmonic(const psf_optics* base, int n_em,
                                             const double* depth, const double* zernike,
                                             int n_zern, const int* z_offsets, const double* z,
                                             int n_slices, int n_theta, int n_r, int nx,
                                             int ny, double dx, double dy, int m_max,
                                             double tail_tol, int precision,
                                             float* intensity, void* workspace,
                                             size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  int r = check_bessel_call(base, n_em, depth, zernike, n_zern, z_offsets, z, n_slices,
                            n_theta, n_r, nx, ny, dx, dy, PSF_PREC_FP32);
  if (r) return r;
  precision = resolve_spherical_precision(n_theta, precision);
  if ((r = check_harm_args(base, m_max, n_theta, precision))) return r;
  if (!(tail_tol >= 0.0 && tail_tol < 1.0))
    return fail(PSF_ERR_ARG, "tail_tol %g outside [0, 1)", tail_tol);
  if (!intensity && n_slices > 0) return fail(PSF_ERR_ARG, "intensity is NULL");
  if (!workspace) return fail(PSF_ERR_WORKSPACE, "workspace is NULL");
  HarmLayout H = harm_layout(workspace, n_em, n_slices, n_theta, n_r, nx, ny, m_max, precision);
  const bool split = harm_split(precision);
  const int bf16 = 0;
  if (ws_bytes < H.bytes)
    return fail(PSF_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, H.bytes);
  if ((r = resolve_output((void**)&intensity, "intensity"))) return r;
  cudaStream_t s = (cudaStream_t)stream;
  // the emitter table carries the axisymmetric part (m != 0 terms dropped
  // there; they enter through the harmonics)
  psf_optics b2 = *base;
  b2.flags |= PSF_PROJECT_AXISYMMETRIC;
  BesselRun R;
  r = bessel_prepare(&b2, n_em, depth, zernike, n_zern, nullptr, z_offsets, z, n_slices,
                     n_theta, n_r, nx, ny, dx, dy, PSF_PREC_FP32, false, H.b, workspace, &R, s);
  if (r) return r;
  const BesselParams& bp = R.bp;
  HarmParams hp;
  memset(&hp, 0, sizeof(hp));
  hp.n_theta = n_theta;
  hp.n_r = n_r;
  hp.nx = nx;
  hp.ny = ny;
  hp.n_em = n_em;
  hp.n_zern = n_zern;
  hp.m_max = m_max;
  hp.n_phi = harm_n_phi(m_max);
  hp.n_ord = 2 * m_max + 5;
  hp.k = bp.k;
  hp.dr = bp.dr;
  hp.r_max = bp.r_max;
  hp.dx = dx;
  hp.dy = dy;
  hp.tail_tol = tail_tol;
  // host tables: m != 0 Zernike radial values at the nodes, azimuth phasors
  const double s_max = base->NA / base->n_i;
  std::vector<double> gx, gw;
  gauss_legendre(n_theta, gx, gw);
  const double th_max = asin(s_max);
  std::vector<float> zr((size_t)kHarmMaxNA * n_theta, 0.f);
  for (int j = 1; j <= n_zern; ++j) {
    int n, m;
    noll_nm(j, &n, &m);
    if (m == 0) continue;
    const int q = hp.n_na++;
    hp.na_j[q] = j;
    hp.na_m[q] = abs(m);
    hp.na_cos[q] = m > 0 ? 1 : 0;
    double rc[kZernMaxOrder + 1];
    zernike_radial_coeffs(n, abs(m), rc);
    for (int t = 0; t < n_theta; ++t) {
      const double rho = sin(0.5 * th_max * (gx[t] + 1.0)) / s_max;
      double v = 0;
      for (int k = kZernMaxOrder; k >= 0; --k) v = v * rho + rc[k];
      zr[(size_t)q * n_theta + t] = (float)v;
    }
  }
  std::vector<float2> cs(hp.n_phi);
  for (int k = 0; k < hp.n_phi; ++k)
    cs[k] = make_float2((float)cos(2.0 * kPi * k / hp.n_phi), (float)sin(2.0 * kPi * k / hp.n_phi));
  // channel x kind coefficients for the model's Jones vector (p_x, p_y)
  const double pxr = bp.pol[0], pxi = bp.pol[1], pyr = bp.pol[2], pyi = bp.pol[3];
  auto set = [&](int c, int kind, double re, double im) {
    hp.coef[c][kind][0] = re;
    hp.coef[c][kind][1] = im;
  };
  // (p_x - i p_y) and (p_x + i p_y)
  const double am_r = pxr + pyi, am_i = pxi - pyr;
  const double ap_r = pxr - pyi, ap_i = pxi + pyr;
  set(0, 0, 0.5 * pxr, 0.5 * pxi);
  set(0, 1, 0.25 * am_r, 0.25 * am_i);
  set(0, 2, 0.25 * ap_r, 0.25 * ap_i);
  set(1, 0, 0.5 * pyr, 0.5 * pyi);
  // (-i p_x - p_y) / 4 and (i p_x - p_y) / 4
  set(1, 1, 0.25 * (pxi - pyr), 0.25 * (-pxr - pyi));
  set(1, 2, 0.25 * (-pxi - pyr), 0.25 * (pxr - pyi));
  set(2, 3, -0.5 * am_r, -0.5 * am_i);
  set(2, 4, -0.5 * ap_r, -0.5 * ap_i);
  upload_async(H.Zr, zr.data(), zr.size() * sizeof(float), s);
  upload_async(H.cs, cs.data(), cs.size() * sizeof(float2), s);
  if ((r = cuda_check("harmonic tables"))) return r;
  const float sA = split ? tc_harm_scale_a(R.max_w) : 1.f;
  {
    TimingScope ts(kTimeSetup, s);
    launch_harm_pupil(hp, R.tt, H.b.et, n_zern > 0 ? zernike : nullptr, H.Zr, H.cs, H.Pm,
                      H.ord, H.Bh, split ? H.tc.bh_max : nullptr, s);
  }
  {
    TimingScope ts(kTimeSetup, s);
    launch_harm_jtab(hp, R.tt, H.Jt, split ? &H.tc : nullptr, sA, bf16, s);
    launch_harm_octant_table(hp, H.octcnt, H.octab, s);
  }
  for (int s0 = 0; s0 < n_slices; s0 += H.chunk) {
    const int ns = n_slices - s0 < H.chunk ? n_slices - s0 : H.chunk;
    if (split) {
      {
        TimingScope ts(kTimeSetup, s);
        launch_harm_operands(hp, R.tt, H.Bh, H.b.slice_em, H.b.et.valid, H.ord, H.b.zz, s0,
                             ns, H.D, H.tc, sA, s);
      }
      TimingScope ts(kTimeBesselRadial, s);
      if ((r = tc_harm_contract(H.tc, n_theta, n_r, m_max, 3 * ns, precision, H.prof,
                                (int*)workspace, s)))
        return fail(r, "harmonic tensor-core contraction launch failed");
    } else {
      TimingScope ts(kTimeBesselRadial, s);
      launch_harm_profiles(hp, R.tt, H.Jt, H.Bh, H.b.slice_em, H.b.et.valid, H.ord,
                           H.b.zz, s0, ns, H.D, H.prof, s);
    }
    {
      TimingScope ts(kTimeBesselEpilogue, s);
      launch_harm_intensity(hp, H.prof, H.b.slice_em, H.b.et.valid, H.ord, H.octab, s0,
                            ns, intensity, s);
    }
  }
  return cuda_check("psf_bessel_vectorial_harmonic launch");
}
