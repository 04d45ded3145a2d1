// Shared-memory FFT of the chirp-Z kernels (FP32, forward sign), two
// transforms per thread in lockstep.
//
// Length L = 16^2 R3 (R3 in {1, 2, 4, 8, 16}): T = L/16 threads per
// transform pair, 16 elements of each transform per thread in registers,
// Stockham (self-sorting) passes of radix 16, 16 and R3 with strides
// Ns = 1, 16, 256:
//   pass with radix R, stride Ns, for j in [0, L/R), k = j mod Ns:
//     a_r = in[j + r L/R] W_{Ns R}^{k r},  a = DFT_R(a),
//     out[(j - k) R + k + s Ns] = a_s.
// Thread t takes j = t in the radix-16 passes and j = t + T i in the last
// one, so it reads elements t + T r in the first pass and holds elements
// t + T r after the last one: consecutive FFTs and the pointwise product
// between them need no shared-memory round trip.
//
// The two transforms A and B of a thread are stored as c2 {re, im} with
// re = (Re A, Re B) and im = (Im A, Im B): every complex add, subtract and
// multiply is a packed FP32x2 operation on both transforms (add/sub/mul/fma
// .f32x2), and multiplying by -i is a register rename.  A shared element is
// the 16-byte (Re A, Re B, Im A, Im B).
//
// Bank layout: transform buffers are padded by one element per 16 (the
// radix-16 pass's stride-16 stores spread over the banks) and spaced so that
// the QL buffers interleaved in a warp fall on distinct banks; the radix-16
// twiddles W_256^{k r} sit at k * 17 + r, so the values of k in a warp read
// distinct banks; last-pass twiddles W_L^{j r} are powers of one loaded
// W_L^j (at most four products deep).
#pragma once

#include "czt_kernels.cuh"

namespace psf {
namespace czt {

// ---- packed FP32x2 arithmetic ----------------------------------------------
PSF_D unsigned long long pk(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
PSF_D float2 upk(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
PSF_D float2 add2(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
  return upk(r);
}
PSF_D float2 sub2(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
  return upk(r);
}
PSF_D float2 mul2(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
  return upk(r);
}
PSF_D float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)), "l"(pk(c)));
  return upk(r);
}
PSF_D float2 dup(float a) { return make_float2(a, a); }

// two complex numbers, transform A in .x and B in .y
struct c2 {
  float2 re, im;
};

PSF_D c2 ld(const float4& f) { return c2{make_float2(f.x, f.y), make_float2(f.z, f.w)}; }
PSF_D float4 st(const c2& a) { return make_float4(a.re.x, a.re.y, a.im.x, a.im.y); }
PSF_D c2 cadd(const c2& a, const c2& b) { return c2{add2(a.re, b.re), add2(a.im, b.im)}; }
PSF_D c2 csub(const c2& a, const c2& b) { return c2{sub2(a.re, b.re), sub2(a.im, b.im)}; }
// (c + i s) a, c and s compile-time constants
PSF_D c2 cmulk(const c2& a, float c, float s) {
  return c2{fma2(a.im, dup(-s), mul2(a.re, dup(c))), fma2(a.im, dup(c), mul2(a.re, dup(s)))};
}
PSF_D c2 mul_mi(const c2& a) { return c2{a.im, mul2(a.re, dup(-1.f))}; }   // -i a
// w a, w = wr + i wi the same for both transforms
PSF_D c2 cmulw(const c2& a, float2 w) {
  const float2 wr = dup(w.x), wi = dup(w.y);
  return c2{sub2(mul2(a.re, wr), mul2(a.im, wi)), fma2(a.re, wi, mul2(a.im, wr))};
}
// conj(a) h
PSF_D c2 conj_mulw(const c2& a, float2 h) {
  const float2 hr = dup(h.x), hi = dup(h.y);
  return c2{fma2(a.im, hi, mul2(a.re, hr)), sub2(mul2(a.re, hi), mul2(a.im, hr))};
}

// cos(pi/8), sin(pi/8), cos(pi/4)
constexpr float kC1 = 0.923879532511286756f;
constexpr float kS1 = 0.382683432365089772f;
constexpr float kC2 = 0.707106781186547524f;

PSF_D void dft4(c2& x0, c2& x1, c2& x2, c2& x3) {
  const c2 t0 = cadd(x0, x2), t1 = csub(x0, x2);
  const c2 t2 = cadd(x1, x3), d = csub(x1, x3);
  x0 = cadd(t0, t2);
  x2 = csub(t0, t2);
  x1 = c2{add2(t1.re, d.im), sub2(t1.im, d.re)};   // t1 + (-i) d
  x3 = c2{sub2(t1.re, d.im), add2(t1.im, d.re)};   // t1 - (-i) d
}

PSF_D void dft2(c2& x0, c2& x1) {
  const c2 t = x0;
  x0 = cadd(t, x1);
  x1 = csub(t, x1);
}

// 8 = 4 x 2: n = 2 n1 + n2, k = k1 + 4 k2
PSF_D void dft8(c2 (&x)[8]) {
  dft4(x[0], x[2], x[4], x[6]);
  dft4(x[1], x[3], x[5], x[7]);
  x[3] = cmulk(x[3], kC2, -kC2);
  x[5] = mul_mi(x[5]);
  x[7] = cmulk(x[7], -kC2, -kC2);
  dft2(x[0], x[1]);
  dft2(x[2], x[3]);
  dft2(x[4], x[5]);
  dft2(x[6], x[7]);
  c2 y[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) y[k] = x[2 * (k & 3) + (k >> 2)];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = y[k];
}

// 16 = 4 x 4: n = 4 n1 + n2, k = k1 + 4 k2.  The first stage (over n1, in
// slots 4 n1 + n2) knows that inputs n >= NIN are zero: NIN = 4 leaves one
// input per column, NIN = 8 two.
template <int NIN>
PSF_D void dft16(c2 (&x)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    if constexpr (NIN == 4) {
      const c2 a = x[n2];
      x[4 + n2] = a;
      x[8 + n2] = a;
      x[12 + n2] = a;
    } else if constexpr (NIN == 8) {
      const c2 a = x[n2], b = x[4 + n2];
      x[n2] = cadd(a, b);
      x[4 + n2] = c2{add2(a.re, b.im), sub2(a.im, b.re)};    // a - i b
      x[8 + n2] = csub(a, b);
      x[12 + n2] = c2{sub2(a.re, b.im), add2(a.im, b.re)};   // a + i b
    } else {
      static_assert(NIN == 16, "NIN");
      dft4(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
    }
  }
  // twiddles W_16^{n2 k1} on slot 4 k1 + n2
  x[5] = cmulk(x[5], kC1, -kS1);     // W^1
  x[9] = cmulk(x[9], kC2, -kC2);     // W^2
  x[13] = cmulk(x[13], kS1, -kC1);   // W^3
  x[6] = cmulk(x[6], kC2, -kC2);     // W^2
  x[10] = mul_mi(x[10]);             // W^4
  x[14] = cmulk(x[14], -kC2, -kC2);  // W^6
  x[7] = cmulk(x[7], kS1, -kC1);     // W^3
  x[11] = cmulk(x[11], -kC2, -kC2);  // W^6
  x[15] = cmulk(x[15], -kC1, kS1);   // W^9
  dft4(x[0], x[1], x[2], x[3]);
  dft4(x[4], x[5], x[6], x[7]);
  dft4(x[8], x[9], x[10], x[11]);
  dft4(x[12], x[13], x[14], x[15]);
  c2 y[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) y[k] = x[4 * (k & 3) + (k >> 2)];
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = y[k];
}

template <int R>
PSF_D void dft_small(c2 (&a)[R]) {
  if constexpr (R == 2) {
    dft2(a[0], a[1]);
  } else if constexpr (R == 4) {
    dft4(a[0], a[1], a[2], a[3]);
  } else if constexpr (R == 8) {
    dft8(a);
  } else {
    static_assert(R == 16, "radix");
    dft16<16>(a);
  }
}

// split of r for powers(): r = hi + (r - hi), both already computed
__host__ __device__ constexpr int pow_split(int r) {
  return (r & (r - 1)) == 0 ? r / 2 : (r >= 8 ? 8 : (r >= 4 ? 4 : 2));
}

// w[r] = w1^r for r < R, each at most four products from w1
template <int R>
PSF_D void powers(float2 w1, float2 (&w)[R]) {
  w[0] = make_float2(1.f, 0.f);
  if constexpr (R > 1) w[1] = w1;
#pragma unroll
  for (int r = 2; r < R; ++r) w[r] = cmul(w[pow_split(r)], w[r - pow_split(r)]);
}

PSF_D int pidx(int i) { return i + (i >> 4); }

// Shared layout of one FFT length: the tables (float2 words: tw2 | twL | Hc)
// then the transform-pair buffers of STRIDE 16-byte elements each; STRIDE
// = 8/QL (mod 8) elements, so the QL buffers interleaved in a quarter-warp
// fall on distinct banks.
template <int L_, int SLOTS_, int QL_>
struct Shape {
  static constexpr int L = L_;
  static constexpr int T = L / 16;
  static constexpr int R3 = L / 256;
  static constexpr int SLOTS = SLOTS_;             // transform pairs per CTA
  static constexpr int QL = QL_;                   // interleaved in a warp
  static constexpr int THREADS = SLOTS * T;
  static constexpr int STRIDE = L + L / 16 + (QL == 2 ? 4 : 0);
  static constexpr int TAB = kCztTw2 + kCztTwL + L;   // float2 words
  static constexpr int TAB4 = (TAB + 1) / 2;          // in 16-byte elements
  static constexpr size_t SMEM = 16 * ((size_t)TAB4 + (size_t)SLOTS * STRIDE);
  // Barrier group: the whole warps that hold the QL interleaved transform
  // pairs of one buffer set (threads [g GROUP, (g + 1) GROUP)); only they
  // exchange data through those buffers.
  static constexpr int GROUP = QL * T < 32 ? 32 : QL * T;
  static constexpr int GROUPS = THREADS / GROUP;
  static_assert(SLOTS % QL == 0, "slots");
  static_assert(THREADS % GROUP == 0 && GROUP % 32 == 0, "barrier group");
  static_assert(GROUPS <= 15, "named barriers 1..15");
};

// Synchronise the barrier group of the calling thread (named barrier
// 1 + group, GROUP threads, every one of which arrives): the transform
// buffers of different groups are independent, so the groups of a CTA run
// their FFT passes out of step.
template <class S>
PSF_D void group_sync() {
  if constexpr (S::GROUP == S::THREADS) {
    __syncthreads();
  } else if constexpr (S::GROUP == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)threadIdx.x / S::GROUP), "n"(S::GROUP)
                 : "memory");
  }
}

// inputs with r >= NIN are zero: NIN = smallest of {4, 8, 16} >= ceil(N / T)
template <class S>
inline int czt_nin(int N) {
  const int rows = (N + S::T - 1) / S::T;
  return rows <= 4 ? 4 : (rows <= 8 ? 8 : 16);
}

template <class S>
PSF_D void lane_split(int tid, int* slot, int* t) {
  const int ql = tid % S::QL;
  *t = (tid / S::QL) % S::T;
  *slot = (tid / (S::QL * S::T)) * S::QL + ql;
}

// Copy the tables of one direction into shared memory (all threads).
template <class S>
PSF_D void load_tables(const CztDir& d, float2* tab) {
  for (int i = threadIdx.x; i < S::TAB; i += S::THREADS)
    tab[i] = i < kCztTw2 ? d.tw2[i]
                         : (i < kCztTw2 + kCztTwL ? d.twL[i - kCztTw2]
                                                  : d.Hc[i - kCztTw2 - kCztTwL]);
}

// Forward DFT_L of the transform pair whose elements t + T r this thread
// holds in v[r] (zero for r >= NIN); on return v[r] = X[t + T r].  Every
// thread of a barrier group calls it together (it synchronises the group).
template <class S, int NIN>
PSF_D void fft_block(c2 (&v)[16], float4* buf, const float2* tab, int t) {
  constexpr int T = S::T, R3 = S::R3;
  const float2* tw2 = tab;
  const float2* twL = tab + kCztTw2;
  // pass 1: radix 16, Ns = 1
  dft16<NIN>(v);
  group_sync<S>();   // earlier readers of buf are done
#pragma unroll
  for (int s = 0; s < 16; ++s) buf[pidx(16 * t + s)] = st(v[s]);
  group_sync<S>();
  // pass 2: radix 16, Ns = 16
  const int k = t & 15;
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = ld(buf[pidx(t + T * r)]);
#pragma unroll
  for (int r = 1; r < 16; ++r) v[r] = cmulw(v[r], tw2[k * 17 + r]);
  dft16<16>(v);
  if constexpr (R3 == 1) {
    return;   // L = 256: v[s] = X[t + 16 s]
  } else {
    group_sync<S>();
    const int base = (t >> 4) * 256 + k;
#pragma unroll
    for (int s = 0; s < 16; ++s) buf[pidx(base + 16 * s)] = st(v[s]);
    group_sync<S>();
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = ld(buf[pidx(t + T * r)]);
    // pass 3: radix R3, Ns = 256; j = t + T i holds elements i + r (16/R3)
    constexpr int S3 = 16 / R3;
#pragma unroll
    for (int i = 0; i < S3; ++i) {
      float2 w[R3];
      powers<R3>(twL[t + T * i], w);
      c2 a[R3];
#pragma unroll
      for (int r = 0; r < R3; ++r) a[r] = r ? cmulw(v[i + r * S3], w[r]) : v[i];
      dft_small<R3>(a);
#pragma unroll
      for (int s = 0; s < R3; ++s) v[i + s * S3] = a[s];
    }
  }
}

// y = conj(FFT(conj(FFT(v)) . Hc)): the circular convolution with h
// (without the final conjugate, which the callers fold into the post-chirp).
template <class S, int NIN>
PSF_D void convolve(c2 (&v)[16], float4* buf, const float2* tab, int t) {
  const float2* Hc = tab + kCztTw2 + kCztTwL;
  fft_block<S, NIN>(v, buf, tab, t);
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = conj_mulw(v[r], Hc[t + S::T * r]);
  fft_block<S, 16>(v, buf, tab, t);
}

}  // namespace czt
}  // namespace psf
