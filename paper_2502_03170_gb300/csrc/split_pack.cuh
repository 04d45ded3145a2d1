// Split of two FP32 values into 16-bit hi + lo parts (x = hi + lo to about
// 2^-22 relative), packed as the pairs the split operands store: element a
// in the low half of each 32-bit word, b in the high half.  The packed
// conversions round each half to nearest exactly as the scalar ones do.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace psf {
namespace tc {

__device__ __forceinline__ void split2(float a, float b, int bf16, uint32_t& hi, uint32_t& lo) {
  if (bf16) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 f = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - f.x, b - f.y);
    hi = *(const uint32_t*)&h;
    lo = *(const uint32_t*)&l;
  } else {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 f = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - f.x, b - f.y);
    hi = *(const uint32_t*)&h;
    lo = *(const uint32_t*)&l;
  }
}

}  // namespace tc
}  // namespace psf
