// Register-resident Gauss-Jordan sweep shared by the solve kernels.
//
// A group of UP lanes (UP a power of two <= 32) holds one Hermitian positive
// definite system [M | R]: lane i keeps row i in aug[0..W) with M in the first
// UP columns and R in the remaining W - UP.  Each step k scales the pivot row by
// 1/p_k, broadcasts it through shared memory (rowbuf, W complex, 16-byte
// aligned) and eliminates it from every other row; the row is rotated left by
// one so the pivot column is always aug[0] and the new inverse column lands in
// aug[W-1].  All register indices are compile-time constants while the step
// loop is a runtime loop.  On return, lane i holds row i of M^{-1} R in
// aug[0 .. W-UP) and row i of M^{-1} in aug[W-UP .. W).  The pivots p_k are the
// Schur complements of M (the squared diagonal of its Cholesky factor); the
// return value is the 1-based index of the first pivot that is not positive, or
// 0.  `writer` is false for lanes that must not write rowbuf (spare lanes).
#pragma once

#include "ffeq_device.cuh"

namespace ffeq {

template <int UP, int W>
__device__ __forceinline__ int gj_sweep_rotating(float2 (&aug)[W], float2* rowbuf, int i, bool writer) {
  static_assert(W % 2 == 0, "row width must be even");
  int fail = 0;
#pragma unroll 1
  for (int k = 0; k < UP; ++k) {
    const float piv = __shfl_sync(kFullMask, aug[0].x, k, UP);
    const bool ok = piv > 0.f;
    if (!ok && fail == 0) fail = k + 1;
    const float r = 1.f / (ok ? piv : 1.f);
    if (i == k && writer) {
      // Scaled pivot row in the rotated layout: [aug[1..W-1] * r, r].
#pragma unroll
      for (int j = 0; j < W; j += 2) {
        const float2 v0 = j + 1 < W ? cscale(aug[j + 1], r) : make_float2(r, 0.f);
        const float2 v1 = j + 2 < W ? cscale(aug[j + 2], r) : make_float2(r, 0.f);
        *reinterpret_cast<float4*>(rowbuf + j) = make_float4(v0.x, v0.y, v1.x, v1.y);
      }
    }
    __syncwarp();
    const float2 f = aug[0];
    if (i == k) {
#pragma unroll
      for (int j = 0; j < W; j += 2) {
        const float4 q = *reinterpret_cast<const float4*>(rowbuf + j);
        aug[j] = make_float2(q.x, q.y);
        aug[j + 1] = make_float2(q.z, q.w);
      }
    } else {
#pragma unroll
      for (int j = 0; j < W; j += 2) {
        const float4 q = *reinterpret_cast<const float4*>(rowbuf + j);
        aug[j] = j + 1 < W ? cfms(f, make_float2(q.x, q.y), aug[j + 1]) : make_float2(-f.x * r, -f.y * r);
        aug[j + 1] = j + 2 < W ? cfms(f, make_float2(q.z, q.w), aug[j + 2]) : make_float2(-f.x * r, -f.y * r);
      }
    }
    __syncwarp();
  }
  return fail;
}

}  // namespace ffeq
