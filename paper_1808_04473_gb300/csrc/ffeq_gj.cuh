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
// Same system and result layout as gj_sweep_rotating, held as pairs of
// adjacent columns: rp[m] = (re col 2m, re col 2m+1), ip[m] likewise for the
// imaginary parts (lane i = row i).  At step k the pivot row is broadcast
// UNSCALED (its pivot-column entry replaced by 1, the identity column it turns
// into) together with the pivot p_k, and every other row does new = base - g q
// with g = f / p_k (f its pivot-column entry; base its own value, or 0 in the
// pivot column); the pivot row itself keeps its values (g = 0, pivot column 1).
// A row that has been the pivot row is thereby stored multiplied by its pivot
// p_i, which later eliminations preserve (they are linear in the row); the
// caller multiplies the entries it uses by the returned 1/p_i (`scale`).  This
// avoids scaling and copying the pivot row inside the loop (a divergent path),
// and each complex update of a column pair is four paired FMAs (__ffma2_rn,
// sm_100 and later), rounding exactly like gj_update.  Two steps per loop trip
// (pivot columns 0 and 1: pair 0), each with its own broadcast buffer (one warp
// barrier per step), followed by a rotation by one pair keep register indices
// compile-time constants.  rowbuf: 2 (2W + 4) floats, 16-byte aligned.  Returns
// the 1-based index of the first non-positive pivot, or 0.
template <int UP, int W>
__device__ __forceinline__ int gj_sweep_pairs(float2 (&rp)[W / 2], float2 (&ip)[W / 2], float* rowbuf, int i,
                                              bool writer, float& scale) {
  static_assert(W % 4 == 0 && UP % 2 == 0, "paired sweep needs W % 4 == 0 and even UP");
  constexpr int NP = W / 2;                // column pairs
  constexpr int kBuf = 2 * W + 4;          // re plane, im plane, pivot (padded to 16 bytes)
  int fail = 0;
  float my_r = 1.f;
#pragma unroll 1
  for (int k = 0; k < UP; k += 2) {
    static_for<2>([&](auto sc) {
      constexpr int s = decltype(sc)::value;   // pivot column of this step (half s of pair 0)
      float* buf = rowbuf + s * kBuf;
      const int kk = k + s;
      const bool me = i == kk;
      const float fr = s == 0 ? rp[0].x : rp[0].y;
      const float fi = s == 0 ? ip[0].x : ip[0].y;
      if (me && writer) {
        const float2 r0 = s == 0 ? make_float2(1.f, rp[0].y) : make_float2(rp[0].x, 1.f);
        const float2 i0 = s == 0 ? make_float2(0.f, ip[0].y) : make_float2(ip[0].x, 0.f);
#pragma unroll
        for (int m = 0; m < NP; m += 2) {
          const float2 ra = m == 0 ? r0 : rp[m], ia = m == 0 ? i0 : ip[m];
          *reinterpret_cast<float4*>(buf + 2 * m) = make_float4(ra.x, ra.y, rp[m + 1].x, rp[m + 1].y);
          *reinterpret_cast<float4*>(buf + W + 2 * m) = make_float4(ia.x, ia.y, ip[m + 1].x, ip[m + 1].y);
        }
        buf[2 * W] = fr;
      }
      __syncwarp();
      const float piv = buf[2 * W];
      const bool ok = piv > 0.f;
      if (!ok && fail == 0) fail = kk + 1;
      const float r = __frcp_rn(ok ? piv : 1.f);
      if (me) my_r = r;
      const float gr = me ? 0.f : fr * r;
      const float gi = me ? 0.f : fi * r;
      const float2 ngr = make_float2(-gr, -gr), pgi = make_float2(gi, gi), ngi = make_float2(-gi, -gi);
      const float dlt = me ? 1.f : 0.f;
      float2 nr[NP], ni[NP];
#pragma unroll
      for (int m = 0; m < NP; m += 2) {
        const float4 qr = *reinterpret_cast<const float4*>(buf + 2 * m);
        const float4 qi = *reinterpret_cast<const float4*>(buf + W + 2 * m);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = m + h;   // pair index
          const float2 qrp = h == 0 ? make_float2(qr.x, qr.y) : make_float2(qr.z, qr.w);
          const float2 qip = h == 0 ? make_float2(qi.x, qi.y) : make_float2(qi.z, qi.w);
          float2 br = rp[c], bi = ip[c];
          if (c == 0) {
            if (s == 0) {
              br.x = dlt;
              bi.x = 0.f;
            } else {
              br.y = dlt;
              bi.y = 0.f;
            }
          }
          float2 tr = __ffma2_rn(ngr, qrp, br);
          tr = __ffma2_rn(pgi, qip, tr);
          float2 ti = __ffma2_rn(ngr, qip, bi);
          ti = __ffma2_rn(ngi, qrp, ti);
          // After the second step, rotate left by one pair (inverse columns to the end).
          const int d = s == 1 ? (c + NP - 1) % NP : c;
          nr[d] = tr;
          ni[d] = ti;
        }
      }
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        rp[m] = nr[m];
        ip[m] = ni[m];
      }
    });
  }
  __syncwarp();   // the buffers may be reused after the sweep
  scale = my_r;
  return fail;
}

// The same sweep (deferred scaling, two steps per trip, rotation by two, one
// broadcast buffer per step) on interleaved complex registers with scalar FMAs
// (gj_update), which rounds exactly like gj_sweep_pairs.  rowbuf: 2 (2W + 4)
// floats, 16-byte aligned.
template <int UP, int W>
__device__ __forceinline__ int gj_sweep_deferred(float2 (&aug)[W], float* rowbuf, int i, bool writer,
                                                 float& scale) {
  static_assert(W % 2 == 0 && UP % 2 == 0, "sweep needs even W and UP");
  constexpr int kBuf = 2 * W + 4;          // W complex, then the pivot (padded to 16 bytes)
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
        for (int j = 0; j < W; j += 2) {
          const float2 a = j == s ? make_float2(1.f, 0.f) : aug[j];
          const float2 b = j + 1 == s ? make_float2(1.f, 0.f) : aug[j + 1];
          *reinterpret_cast<float4*>(buf + 2 * j) = make_float4(a.x, a.y, b.x, b.y);
        }
        buf[2 * W] = aug[s].x;
      }
      __syncwarp();
      const float piv = buf[2 * W];
      const bool ok = piv > 0.f;
      if (!ok && fail == 0) fail = kk + 1;
      const float r = __frcp_rn(ok ? piv : 1.f);
      if (me) my_r = r;
      const float2 gg = me ? make_float2(0.f, 0.f) : make_float2(aug[s].x * r, aug[s].y * r);
      const float dlt = me ? 1.f : 0.f;
      float2 nw[W];
#pragma unroll
      for (int j = 0; j < W; j += 2) {
        const float4 q = *reinterpret_cast<const float4*>(buf + 2 * j);
        const float2 b0 = j == s ? make_float2(dlt, 0.f) : aug[j];
        const float2 b1 = j + 1 == s ? make_float2(dlt, 0.f) : aug[j + 1];
        const int d = s == 1 ? (j + W - 2) % W : j;   // after the second step, rotate left by two
        nw[d] = gj_update(gg, make_float2(q.x, q.y), b0);
        nw[d + 1] = gj_update(gg, make_float2(q.z, q.w), b1);
      }
#pragma unroll
      for (int j = 0; j < W; ++j) aug[j] = nw[j];
    });
  }
  __syncwarp();   // the buffers may be reused after the sweep
  scale = my_r;
  return fail;
}

}  // namespace ffeq
