// Soft-output helpers shared by the solve and refinement kernels.
#pragma once

#include <cmath>

#include "ffeq_device.cuh"

namespace ffeq {

// Max-log LLRs of one Gray-labelled PAM axis with H bits (labels and sign as in
// ffeq.h): for each bit, the squared distance to the nearest level carrying a 1
// minus that to the nearest level carrying a 0, over sigma^2 (times inv_s2 =
// 1/sigma^2, taken once per symbol).  A zero difference gives 0 (also when
// sigma^2 = 0); sigma^2 = +inf gives 0 (inv_s2 = 0); NaN propagates.
template <int H>
__device__ __forceinline__ void axis_llr(float x, float inv_s2, float scale, float* out) {
  constexpr int L = 1 << H;
  float m0[H], m1[H];
#pragma unroll
  for (int t = 0; t < H; ++t) m0[t] = m1[t] = INFINITY;
#pragma unroll
  for (int l = 0; l < L; ++l) {
    const float e = x - scale * static_cast<float>(2 * l - (L - 1));
    const float d = e * e;
    const int g = l ^ (l >> 1);
#pragma unroll
    for (int t = 0; t < H; ++t) {
      if ((g >> (H - 1 - t)) & 1) m1[t] = fminf(m1[t], d);
      else m0[t] = fminf(m0[t], d);
    }
  }
#pragma unroll
  for (int t = 0; t < H; ++t) {
    const float diff = m1[t] - m0[t];
    out[t] = diff == 0.f ? 0.f : diff * inv_s2;
  }
}

__device__ __forceinline__ void symbol_llr(float2 z, float s2, float scale, int h, float* out) {
  const float inv = isinf(s2) ? 0.f : rcp_approx(s2);   // s2 = 0: +inf; NaN stays NaN
  switch (h) {
    case 1: axis_llr<1>(z.x, inv, scale, out); axis_llr<1>(z.y, inv, scale, out + 1); break;
    case 2: axis_llr<2>(z.x, inv, scale, out); axis_llr<2>(z.y, inv, scale, out + 2); break;
    case 3: axis_llr<3>(z.x, inv, scale, out); axis_llr<3>(z.y, inv, scale, out + 3); break;
    default: axis_llr<4>(z.x, inv, scale, out); axis_llr<4>(z.y, inv, scale, out + 4); break;
  }
}

}  // namespace ffeq
