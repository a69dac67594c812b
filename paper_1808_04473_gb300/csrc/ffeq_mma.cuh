// Split-precision operands and warp-level MMAs shared by the tensor-core
// contractions (ffeq_gram_tc.cu, ffeq_gram_stream.cu).
//
// An FP32 value x is split into hi + lo with hi = x rounded to the MMA type and
// lo = the remainder (x - hi, exact in FP32) rounded to the same type; a product
// then accumulates A_lo B_hi + A_hi B_lo + A_hi B_hi in FP32 (the lo*lo term is
// dropped):
//   TF32: 11-bit significands, hi + lo carries ~22 bits (mma m16n8k8);
//   BF16:  8-bit significands, hi + lo carries ~16 bits (mma m16n8k16);
//   FP16: 11-bit significands, hi + lo carries ~22 bits (mma m16n8k16), within
//         FP16's range: |x| below 65504, and lo loses bits once it falls under
//         the normal range (|x| below about 2^-3).
#pragma once

#include <cstdint>

namespace ffeq {

constexpr int kTf32x3 = 1;
constexpr int kBf16x3 = 2;
constexpr int kFp16x3 = 3;

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

// Two floats -> packed hi and lo pairs (element 0 in the low half, as the MMA
// fragments expect).
__device__ __forceinline__ void split_bf16(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x1), "f"(x0));
  const float h0 = __uint_as_float(hi << 16);
  const float h1 = __uint_as_float(hi & 0xffff0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(x1 - h1), "f"(x0 - h0));
}

__device__ __forceinline__ void split_f16(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x1), "f"(x0));
  float h0, h1;
  asm("{\n\t.reg .f16 l, h;\n\tmov.b32 {l, h}, %2;\n\tcvt.f32.f16 %0, l;\n\tcvt.f32.f16 %1, h;\n\t}"
      : "=f"(h0), "=f"(h1)
      : "r"(hi));
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(x1 - h1), "f"(x0 - h0));
}

template <int MODE>
__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  if constexpr (MODE == kFp16x3) split_f16(x0, x1, hi, lo);
  else split_bf16(x0, x1, hi, lo);
}

// Not volatile: the compiler may interleave MMAs on independent accumulators.
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_f16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// m16n8k16 in the split type of MODE (BF16 or FP16); TF32 is m16n8k8.
template <int MODE>
__device__ __forceinline__ void mma_any(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  if constexpr (MODE == kTf32x3) mma_tf32(c, a, b0, b1);
  else if constexpr (MODE == kFp16x3) mma_f16(c, a, b0, b1);
  else mma_bf16(c, a, b0, b1);
}

}  // namespace ffeq
