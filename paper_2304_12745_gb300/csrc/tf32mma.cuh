// Split-TF32 warp MMA helpers shared by the tensor-core solve kernels.
#pragma once

#include <cstdint>

namespace precode {

// x = hi + lo exactly: hi keeps the 10 explicit mantissa bits a TF32 operand
// carries (low 13 bits cleared), lo = x - hi is exact in FP32; the MMA reads
// lo's top TF32 bits, so a b is resolved to about 2^-21 relative.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = __float_as_uint(x) & 0xffffe000u;
  lo = __float_as_uint(x - __uint_as_float(hi));
}

// The same split with the masking step kept in program order among the other
// splits (volatile): in long unrolled loops that hold a large W in registers this
// stops the scheduler from computing many iterations' splits ahead of their MMAs
// (and spilling for it).
__device__ __forceinline__ void split_tf32_ordered(float x, uint32_t& hi, uint32_t& lo) {
  asm volatile("and.b32 %0, %1, 0xffffe000;" : "=r"(hi) : "r"(__float_as_uint(x)));
  lo = __float_as_uint(x - __uint_as_float(hi));
}

__device__ __forceinline__ uint32_t neg_bits(uint32_t x) { return x ^ 0x80000000u; }

// d += a . b  (m16n8k8, row.col, TF32 in, FP32 accumulate)
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

}  // namespace precode
