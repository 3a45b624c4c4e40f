// warp_mma.h -- warp-level tensor-core helpers (inline PTX mma.sync) and the
// operand splits of the split precisions, for kernels that keep their
// accumulators in registers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fno {
namespace wm {

// D += A (16x16, row) * B (16x8, col), BF16 in, FP32 accumulate
__device__ __forceinline__ void mma16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                      uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// D += A (16x8, row) * B (8x8, col), TF32 in, FP32 accumulate
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Round to TF32 (10 stored mantissa bits, nearest, ties away from zero) with
// integer operations: adding half a TF32 unit to the bit pattern carries into
// the kept bits exactly when the 13 dropped bits are at least half a unit,
// then the dropped bits are cleared (a carry out of the mantissa moves to the
// next binade; Inf and NaN keep their class).  This is the rounding of the
// cvt.rna.tf32.f32 instruction, which measured far slower on this GPU.  A TF32
// value is exact as BF16 hi + lo, so split BF16 products of rounded operands
// are TF32 products.
__device__ __forceinline__ uint32_t tf32_rna_bits(float x) {
  return (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
}
__device__ __forceinline__ float tf32_round(float x) { return __uint_as_float(tf32_rna_bits(x)); }
template <bool TF>
__device__ __forceinline__ float rnd(float x) {
  return TF ? tf32_round(x) : x;
}

// a = big + small with both parts TF32 (small carries the rounding residual)
__device__ __forceinline__ void tf32_split(float a, uint32_t& big, uint32_t& small) {
  big = tf32_rna_bits(a);
  small = tf32_rna_bits(a - __uint_as_float(big));
}

// The same split without rounding small: the tensor core reads only its TF32
// bits, so big.big + big.small + small.big carries an error below 2^-21 |a b|
// per product.
__device__ __forceinline__ void tf32_split_int(float a, uint32_t& big, uint32_t& small) {
  big = tf32_rna_bits(a);
  small = __float_as_uint(a - __uint_as_float(big));
}

// hi/lo BF16 split of two floats, packed in pairs (first value in the low half)
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

}  // namespace wm
}  // namespace fno
