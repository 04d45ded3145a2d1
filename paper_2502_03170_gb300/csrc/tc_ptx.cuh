// Inline-PTX building blocks of the tcgen05 / TMEM / TMA kernels: mbarrier
// waits with a device-time bound, TMA tile loads, shared-memory matrix
// descriptors, single-thread tcgen05.mma issue and commit, TMEM loads, and
// the hi + lo split of FP32 values into two 16-bit operands.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "psf_common.cuh"

namespace psf {
namespace tc {

constexpr uint32_t kSpinLimit = 1u << 28;          // backstop to the timer
constexpr uint64_t kTimeoutNs = 2000000000ull;     // 2 s of device time

// --------------------------------------------------------------------------
// PTX wrappers
// --------------------------------------------------------------------------
PSF_D uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

PSF_D void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

PSF_D void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
               "r"(bytes) : "memory");
}

PSF_D void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

PSF_D bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

PSF_D uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait: true when the phase completed; false after kTimeoutNs of
// device time or when another role already gave up (abort flag).
PSF_D bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                     int* status) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u) {
      if (*abort_flag) return false;
      if (global_ns() - t0 > kTimeoutNs || it > kSpinLimit) break;
    }
  }
  set_status(status, PSF_ERR_DEVICE_TIMEOUT);
  *abort_flag = 1;
  return false;
}

// Wait used while draining after an abort: bounded, no status change.
PSF_D void mbar_drain_wait(uint32_t bar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return;
    if ((it & 255u) == 255u && (global_ns() - t0 > kTimeoutNs || it > kSpinLimit)) return;
  }
}

// Contiguous global -> shared copy on the TMA engine (addresses 16-byte
// aligned, bytes a multiple of 16), completing on mbarrier `bar`.
PSF_D void bulk_load_1d(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"((uint64_t)src), "r"(bytes), "r"(bar)
      : "memory");
}

PSF_D void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                       uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

PSF_D void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                       int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major, SWZ-byte swizzle (128 B: layout
// code 2, 64 B: code 4), 8-row groups 8 * SWZ bytes apart (stride byte
// offset), descriptor version 1.
template <int SWZ>
PSF_D uint64_t smem_desc(uint32_t addr) {
  static_assert(SWZ == 64 || SWZ == 128, "64- or 128-byte swizzle");
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) |
         ((uint64_t)((8 * SWZ) >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)(SWZ == 128 ? 2 : 4) << 61);
}

PSF_D void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                   uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

PSF_D void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

PSF_D void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
PSF_D void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

PSF_D void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32"
      " {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15,"
      " %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31},"
      " [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
        "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
        "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]),
        "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Splits x into hi + lo of the 16-bit type; returns the two 16-bit patterns.
// hi + lo back to FP32.
PSF_D float unsplit16(uint16_t hi, uint16_t lo, int bf16) {
  if (bf16)
    return __bfloat162float(__ushort_as_bfloat16(hi)) +
           __bfloat162float(__ushort_as_bfloat16(lo));
  return __half2float(__ushort_as_half(hi)) + __half2float(__ushort_as_half(lo));
}

PSF_D void split16(float x, int bf16, uint16_t& hi, uint16_t& lo) {
  if (bf16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
  } else {
    const __half h = __float2half_rn(x);
    const __half l = __float2half_rn(x - __half2float(h));
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(l);
  }
}

// x rounded to TF32 (10 explicit mantissa bits, nearest, ties away), kept in
// an FP32 container as the tensor core reads it.
PSF_D float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Splits x into TF32 hi + lo (three-product form); with one pass lo is 0.
PSF_D void split_tf32(float x, int passes, uint32_t& hi, uint32_t& lo) {
  const float h = round_tf32(x);
  hi = __float_as_uint(h);
  lo = passes == 3 ? __float_as_uint(round_tf32(x - h)) : 0u;
}

// The same split of an FP64 value (hi rounded from x, lo from x - hi).
PSF_D void split16d(double v, int bf16, uint16_t& hi, uint16_t& lo) {
  if (bf16) {
    const __nv_bfloat16 h = __double2bfloat16(v);
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(__double2bfloat16(v - (double)__bfloat162float(h)));
  } else {
    const __half h = __double2half(v);
    hi = __half_as_ushort(h);
    lo = __half_as_ushort(__double2half(v - (double)__half2float(h)));
  }
}

}  // namespace tc
}  // namespace psf
