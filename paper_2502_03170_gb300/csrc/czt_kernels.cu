// Chirp-Z (Bluestein) evaluation of the Fourier strategy's zoom DFTs: FP32
// shared-memory FFTs, two kernels per z-chunk (one per zoom direction).
//
// This file holds the host side (FFT length, FP64 tables); the kernels are
// in czt_stage1.cu and czt_stage2.cu, the FFT itself in czt_fft.cuh.
#include "czt_kernels.cuh"

#include <cmath>
#include <complex>
#include <vector>

namespace psf {

int czt_length(int N, int n) {
  const long long need = (long long)N + n - 1;
  int L = kCztMinL;
  while (L < need && L < kCztMaxL) L *= 2;
  return L >= need ? L : 0;
}

// ---------------------------------------------------------------------------
// Host tables (FP64).
// ---------------------------------------------------------------------------
static size_t pre_cyc_words(int N) { return (size_t)(N + 1) / 2; }

size_t czt_dir_words(int N, int n) {
  const int L = czt_length(N, n);
  return (size_t)kCztTw2 + kCztTwL + (size_t)L + (size_t)N + (size_t)n + pre_cyc_words(N);
}

// iterative radix-2 FFT, forward sign, FP64 (table building only)
static void fft_f64(std::vector<std::complex<double>>& a) {
  const size_t n = a.size();
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    const size_t h = len / 2;
    for (size_t k = 0; k < h; ++k) {
      const double ang = -2.0 * kPi * (double)k / (double)len;
      const std::complex<double> w(std::cos(ang), std::sin(ang));
      for (size_t i = 0; i < n; i += len) {
        const std::complex<double> u = a[i + k], v = a[i + k + h] * w;
        a[i + k] = u + v;
        a[i + k + h] = u - v;
      }
    }
  }
}

static double frac_cycles(double x) { return x - std::nearbyint(x); }

void czt_build_dir(int N, int n, double f, double d, double post_re, double post_im,
                   float2* w) {
  const int L = czt_length(N, n);
  const double beta = 2.0 * f * d / N;
  const double p0 = 0.5 * (N - 1), a0 = 0.5 * (n - 1);
  float2* tw2 = w;
  float2* twL = tw2 + kCztTw2;
  float2* Hc = twL + kCztTwL;
  float2* pre = Hc + L;
  float2* post = pre + N;
  float* pre_cyc = (float*)(post + n);
  // W_256^{k r} at k * 17 + r (k, r < 16; column 16 unused), W_L^j for j < 256
  for (int k = 0; k < 16; ++k)
    for (int r = 0; r < 17; ++r) {
      const double ang = -2.0 * kPi * (double)((k * r) % 256) / 256.0;
      tw2[k * 17 + r] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
  for (int j = 0; j < kCztTwL; ++j) {
    const double ang = -2.0 * kPi * (double)j / L;
    twL[j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  // h_m = e^{-i pi beta m^2} for m in [-(N-1), n-1], circularly placed
  std::vector<std::complex<double>> h(L, 0.0);
  for (int m = -(N - 1); m <= n - 1; ++m) {
    const double cyc = frac_cycles(0.5 * beta * ((double)m * (double)m));
    h[(m + L) % L] = std::polar(1.0, -2.0 * kPi * cyc);
  }
  fft_f64(h);
  for (int m = 0; m < L; ++m) {
    const std::complex<double> v = std::conj(h[m]) / (double)L;
    Hc[m] = make_float2((float)v.real(), (float)v.imag());
  }
  for (int p = 0; p < N; ++p) {
    const double cyc = frac_cycles(beta * (0.5 * (double)p * p - p * a0));
    pre_cyc[p] = (float)cyc;
    pre[p] = make_float2((float)std::cos(2.0 * kPi * cyc), (float)std::sin(2.0 * kPi * cyc));
  }
  const std::complex<double> sc(post_re, post_im);
  for (int a = 0; a < n; ++a) {
    const double cyc = frac_cycles(beta * (0.5 * (double)a * a - a * p0 + p0 * a0));
    const std::complex<double> v = sc * std::polar(1.0, 2.0 * kPi * cyc);
    post[a] = make_float2((float)v.real(), (float)v.imag());
  }
  if (N & 1) pre_cyc[N] = 0.f;
}

CztDir czt_dir_view(const float2* w, int N, int n) {
  CztDir d;
  d.L = czt_length(N, n);
  d.tw2 = w;
  d.twL = w + kCztTw2;
  d.Hc = d.twL + kCztTwL;
  d.pre = d.Hc + d.L;
  d.post = d.pre + N;
  d.pre_cyc = (const float*)(d.post + n);
  return d;
}

}  // namespace psf
