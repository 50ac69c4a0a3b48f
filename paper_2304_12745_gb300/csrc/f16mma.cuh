// Split-FP16 warp MMA helpers (m16n8k16, FP16 in, FP32 accumulate).
//
// A value x is carried as hi + lo with hi = fp16_rn(x) and lo = fp16_rn(x - hi):
// 11 + 11 significant bits, so a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi is
// resolved to about 2^-22 relative (the dropped a_lo b_lo and the rounding of lo),
// as long as x sits inside the FP16 range; callers scale each instance by powers
// of two so that it does.  One m16n8k16 covers twice the reduction length of the
// TF32 m16n8k8 at the same issue cost.
#pragma once

#include <cuda_fp16.h>

#include <cstdint>

namespace precode {

__device__ __forceinline__ uint32_t h2_bits(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }

// (x0, x1) -> hi, lo as FP16 pairs (x0 in the low half)
__device__ __forceinline__ void split_h2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(x0, x1);
  const float2 hf = __half22float2(h);
  hi = h2_bits(h);
  lo = h2_bits(__floats2half2_rn(x0 - hf.x, x1 - hf.y));
}

// The same split with its first conversion kept in program order among the
// other splits (volatile): in long unrolled loops that hold a large W in
// registers this stops the scheduler from computing many splits ahead of their
// MMAs (and spilling for it).
__device__ __forceinline__ void split_h2_ordered(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  uint32_t h;
  asm volatile("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(x1), "f"(x0));  // x0 in the low half
  const float2 hf = __half22float2(*reinterpret_cast<const __half2*>(&h));
  hi = h;
  lo = h2_bits(__floats2half2_rn(x0 - hf.x, x1 - hf.y));
}

__device__ __forceinline__ uint32_t neg_h2(uint32_t x) { return x ^ 0x80008000u; }

// d += a . b  (m16n8k16, row.col, FP16 in, FP32 accumulate)
__device__ __forceinline__ void mma_f16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                        uint32_t a3, uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

}  // namespace precode
