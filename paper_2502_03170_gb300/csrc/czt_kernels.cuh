// Chirp-Z (Bluestein) form of the Fourier strategy's zoom DFTs (Eq. 8 with
// the twiddle A[a][p] = exp(2 pi i f u_p x_a), f = NA / lambda).
//
// With u_p = (2p + 1 - N)/N, x_a = (a - (n-1)/2) d and beta = 2 f d / N the
// twiddle phase is beta (p - p0)(a - a0) cycles, p0 = (N-1)/2, a0 = (n-1)/2.
// Writing p a = (p^2 + a^2 - (a - p)^2) / 2 factors it as
//   A[a][p] = v_a w_p h_{a-p},
//   w_p = e^{2 pi i beta (p^2/2 - p a0)},
//   v_a = e^{2 pi i beta (a^2/2 - a p0 + p0 a0)},
//   h_m = e^{-i pi beta m^2},
// so sum_p A[a][p] x_p = v_a (g * h)_a with g_p = w_p x_p: a linear
// convolution over m = a - p in [-(N-1), n-1], evaluated as a circular one of
// length L >= N + n - 1 by FFTs:
//   y = IFFT(FFT(g) . FFT(h)) = conj(FFT(conj(FFT(g)) . Hc)),  Hc = conj(FFT(h)) / L.
// The same discrete sum as the dense matrix-DFT (Sec. 4: the chirp-Z route
// for arbitrary pixel size), in O(L log L) per line instead of O(N n).
#pragma once

#include "fourier_kernels.cuh"
#include "psf_common.cuh"

namespace psf {

constexpr int kCztMinL = 256;
constexpr int kCztMaxL = 4096;
constexpr int kCztTw2 = 16 * 17;   // W_256^{k r} at k * 17 + r
constexpr int kCztTwL = 256;       // W_L^j, j < 256

// FFT length for N inputs and n outputs: the smallest power of two
// >= max(256, N + n - 1); 0 if that exceeds 4096.
int czt_length(int N, int n);

// One zoom direction, device tables (FP64 on the host, stored as FP32).
struct CztDir {
  int L;                 // FFT length
  const float2* tw2;     // [16 * 17] W_256^{k r} at k * 17 + r (radix-16 pass)
  const float2* twL;     // [256] W_L^j (last pass), W_L = e^{-2 pi i / L}
  const float2* Hc;      // [L] conj(FFT_L(h placed circularly)) / L
  const float* pre_cyc;  // [N] frac(beta (p^2/2 - p a0)) in cycles
  const float2* pre;     // [N] e^{2 pi i pre_cyc}
  const float2* post;    // [n] v_a times a constant prefactor
};

// Host tables of one direction, in the device layout of CztDir, packed as
// float2 words: tw2 [272] | twL [256] | Hc [L] | pre [N] | post [n] |
// pre_cyc [N] floats (padded to whole float2 words); v_a is multiplied by
// the complex constant (post_re, post_im).
size_t czt_dir_words(int N, int n);
void czt_build_dir(int N, int n, double f, double d, double post_re, double post_im,
                   float2* host_words);
CztDir czt_dir_view(const float2* dev_words, int N, int n);

// Stage 1 for the z-chunk [z0, z0 + nzc): per channel c and pupil row p
// (contiguous in the node table), the zoom along y:
//   T[zc][c][b][p] = w^x_p sum_q A_y[b][q] P_c(p, q) e^{i k z cos}, b < ny,
// with the pupil field formed from the node table on the fly.
void launch_czt_stage1(NodeTable t, int N, const float2* zz, int z0, int nzc,
                       const CztDir& cx, const CztDir& cy, int ny, float2* T,
                       cudaStream_t s);

// Stage 2: per output column b, the zoom along x,
//   E_c[a][b] = v^x_a sum_p h^x_{a-p} T[zc][c][b][p]
// (the Eq. 8 prefactor C ds^2 is folded into v^x), I = sum_c |E_c|^2 into
// I[zc][a][b]; fields [zc][3][a][b] too when non-null.
void launch_czt_stage2(const float2* T, int N, int nx, int ny, int nzc,
                       const CztDir& cx, float* I, float2* fields, cudaStream_t s);

}  // namespace psf
