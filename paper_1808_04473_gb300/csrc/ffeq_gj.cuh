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

// a * b + c on both halves: one paired FP32 FMA (fma.rn.f32x2, sm_100 and
// later); each half rounds exactly like fmaf.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

// One element of the deferred-scaling elimination, shared by every sweep so
// that all lane layouts round identically:
//     new = base - g q       (complex; g = f / p_k, q the unscaled pivot row)
// as re: base.re - g.re q.re + g.im q.im, im: base.im - g.re q.im - g.im q.re.
__device__ __forceinline__ float2 gj_update(float2 g, float2 q, float2 base) {
  base.x = fmaf(-g.x, q.x, base.x);
  base.x = fmaf(g.y, q.y, base.x);
  base.y = fmaf(-g.x, q.y, base.y);
  base.y = fmaf(-g.y, q.x, base.y);
  return base;
}

// Gauss-Jordan sweep with deferred row scaling and paired FMAs.
//
// Same system and result layout as gj_sweep_rotating, held as separate real
// and imaginary planes re[W], im[W] (lane i = row i).  At step k the pivot row
// is broadcast UNSCALED (its pivot-column entry replaced by 1, the identity
// column it turns into) together with the pivot p_k, and every other row does
// new = base - g q with g = f / p_k (f its pivot-column entry; base its own
// value, or 0 in the pivot column); the pivot row itself keeps its values
// (g = 0, pivot column 1).  A row that has been the pivot row is thereby stored
// multiplied by its pivot p_i, which later eliminations preserve (they are
// linear in the row); the caller multiplies the entries it uses by the returned
// 1/p_i (`scale`).  This avoids scaling and copying the pivot row inside the loop
// (a divergent path), and with rows in planes each complex update is two paired
// FMAs on (column j, column j+1).  Two steps per loop trip (pivot columns 0 and
// 1), each with its own broadcast buffer (one warp barrier per step), followed
// by a rotation by two keep the pairs aligned.  rowbuf: 2 (2W + 4) floats, 16-byte
// aligned.  Returns the 1-based index of the first non-positive pivot, or 0.
template <int UP, int W>
__device__ __forceinline__ int gj_sweep_pairs(float (&re)[W], float (&im)[W], float* rowbuf, int i, bool writer,
                                              float& scale) {
  static_assert(W % 4 == 0 && UP % 2 == 0, "paired sweep needs W % 4 == 0 and even UP");
  constexpr int kBuf = 2 * W + 4;          // re plane, im plane, pivot (padded to 16 bytes)
  int fail = 0;
  float my_r = 1.f;
#pragma unroll 1
  for (int k = 0; k < UP; k += 2) {
    static_for<2>([&](auto sc) {
      constexpr int s = decltype(sc)::value;   // pivot column of this step
      float* buf = rowbuf + s * kBuf;
      const int kk = k + s;
      const bool me = i == kk;
      if (me && writer) {
#pragma unroll
        for (int j = 0; j < W; j += 4) {
          *reinterpret_cast<float4*>(buf + j) =
              make_float4(j + 0 == s ? 1.f : re[j + 0], j + 1 == s ? 1.f : re[j + 1], j + 2 == s ? 1.f : re[j + 2],
                          j + 3 == s ? 1.f : re[j + 3]);
          *reinterpret_cast<float4*>(buf + W + j) =
              make_float4(j + 0 == s ? 0.f : im[j + 0], j + 1 == s ? 0.f : im[j + 1], j + 2 == s ? 0.f : im[j + 2],
                          j + 3 == s ? 0.f : im[j + 3]);
        }
        buf[2 * W] = re[s];
      }
      __syncwarp();
      const float piv = buf[2 * W];
      const bool ok = piv > 0.f;
      if (!ok && fail == 0) fail = kk + 1;
      const float r = __frcp_rn(ok ? piv : 1.f);
      if (me) my_r = r;
      const float gr = me ? 0.f : re[s] * r;
      const float gi = me ? 0.f : im[s] * r;
      const float2 ngr = make_float2(-gr, -gr), pgi = make_float2(gi, gi), ngi = make_float2(-gi, -gi);
      const float dlt = me ? 1.f : 0.f;
      float nre[W], nim[W];
#pragma unroll
      for (int j = 0; j < W; j += 4) {
        const float4 qr = *reinterpret_cast<const float4*>(buf + j);
        const float4 qi = *reinterpret_cast<const float4*>(buf + W + j);
#pragma unroll
        for (int h = 0; h < 4; h += 2) {
          const int c = j + h;
          const float2 qrp = h == 0 ? make_float2(qr.x, qr.y) : make_float2(qr.z, qr.w);
          const float2 qip = h == 0 ? make_float2(qi.x, qi.y) : make_float2(qi.z, qi.w);
          const float2 br = make_float2(c == s ? dlt : re[c], c + 1 == s ? dlt : re[c + 1]);
          const float2 bi = make_float2(c == s ? 0.f : im[c], c + 1 == s ? 0.f : im[c + 1]);
          float2 tr = ffma2(ngr, qrp, br);
          tr = ffma2(pgi, qip, tr);
          float2 ti = ffma2(ngr, qip, bi);
          ti = ffma2(ngi, qrp, ti);
          // After the second step, rotate left by two (inverse columns to the end).
          const int d = s == 1 ? (c + W - 2) % W : c;
          nre[d] = tr.x;
          nre[d + 1] = tr.y;
          nim[d] = ti.x;
          nim[d + 1] = ti.y;
        }
      }
#pragma unroll
      for (int j = 0; j < W; ++j) {
        re[j] = nre[j];
        im[j] = nim[j];
      }
    });
  }
  __syncwarp();   // the buffers may be reused after the sweep
  scale = my_r;
  return fail;
}

}  // namespace ffeq
