// Shared device helpers of libpsf: extended-precision phase arithmetic,
// the workspace status word, and small math utilities.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/psf.h"

#define PSF_HD __host__ __device__ __forceinline__
#define PSF_D __device__ __forceinline__

namespace psf {

constexpr double kPi = 3.14159265358979323846;
constexpr int kStatusBytes = 256;   // workspace header holding the status word

// ---------------------------------------------------------------------------
// Status word at the start of every workspace.  A kernel that detects a
// device-side error records the first code and returns; it never traps.
// ---------------------------------------------------------------------------
PSF_D void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// ---------------------------------------------------------------------------
// Double-float ("float-float") numbers: value = hi + lo with |lo| <= ulp(hi)/2.
// Used for per-(node, z) defocus phases, where FP64 would run at 1/64 of the
// FP32 rate on this part.  Products use the exact FMA error term (Dekker's
// two-product with a fused multiply-add).
// ---------------------------------------------------------------------------
struct f2x { float hi, lo; };

PSF_HD f2x split_double(double v) {
  f2x r;
  r.hi = (float)v;
  r.lo = (float)(v - (double)r.hi);
  return r;
}

// Fractional part (in cycles, in [-0.5, 0.5]) of a*b + c where a, b are
// double-float and c a small float (|c| < 1).  Error ~ 1e-7 cycles for
// |a*b| < 2^10.
PSF_D float frac_mul_add(f2x a, f2x b, float c) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);                 // exact low part of a.hi*b.hi
  float t = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)); // remaining small terms
  float f = p - rintf(p);                         // exact: |p| < 2^23
  float s = (f + c) + t;
  return s - rintf(s);
}

// e^{2 pi i r} for r in cycles (any r; reduced first)
PSF_D float2 cis_cycles(float r) {
  r = r - rintf(r);
  float s, c;
  sincospif(2.0f * r, &s, &c);
  return make_float2(c, s);
}

PSF_HD float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

PSF_HD int ceil_div(int a, int b) { return (a + b - 1) / b; }
PSF_HD size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace psf
