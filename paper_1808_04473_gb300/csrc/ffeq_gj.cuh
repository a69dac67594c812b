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
      const float r = rcp_approx(ok ? piv : 1.f);
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

// complex helpers for the block step
__device__ __forceinline__ float2 gj_cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Gauss-Jordan sweep with 2 x 2 block pivots, deferred row scaling and paired
// FMAs.  Same system, result layout and pivot semantics as gj_sweep_pairs: the
// pivots reported are the sequential ones (the squared Cholesky diagonal).
//
// Two consecutive pivot steps k, k+1 (pivot columns 0 and 1: pair 0) are fused
// into one broadcast round: lanes k and k+1 publish their rows (pivot-column
// pair replaced by (1, 0) and (0, 1), the identity columns they turn into)
// together with the 2 x 2 pivot block P.  With p_a = P00, h = P10 / p_a and
// p_b = P11 - h P01 (the two sequential pivots), every lane applies
//     new = base - alpha q_k - beta q_k+1
// with, for the other lanes (f0, f1 their pivot-column entries, base pair 0 = 0),
//     g = f0 / p_a,  beta = (f1 - g P01) / p_b,  alpha = g - beta h;
// for lane k (base pair 0 = (1, 0)):   beta = P01 / p_b, alpha = -beta h;
// for lane k+1 (base pair 0 = (0, 1)): alpha = h, beta = 0,
// which is algebraically the sequential deferred-scaling sweep (pivot rows stay
// multiplied by their pivot; the caller scales by the returned 1/p_i).  One warp
// barrier per two pivots instead of two (two broadcast areas, alternating), and
// both pivot rows are stored by one instruction.  UP must be even.  rowbuf:
// 2 (4 W + 16) floats, 16-byte aligned.
template <int UP, int W>
__device__ __forceinline__ int gj_sweep_block2(float2 (&rp)[W / 2], float2 (&ip)[W / 2], float* rowbuf, int i,
                                               bool writer, float& scale) {
  static_assert(W % 4 == 0 && UP % 2 == 0, "block sweep needs W % 4 == 0 and even UP");
  constexpr int NP = W / 2;                // column pairs
  constexpr int kArea = 4 * W + 16;        // one broadcast area
  int fail = 0;
  float my_r = 1.f;
#pragma unroll 1
  for (int k = 0; k < UP; k += 2) {
    float* area = rowbuf + ((k >> 1) & 1) * kArea;
    float* qk = area;                        // [re plane W][im plane W] of row k
    float* qk1 = area + 2 * W;               // the same for row k + 1
    float* blk = area + 4 * W;               // P00, P01, P10, P11 (complex)
    const bool mk = i == k, mk1 = i == k + 1;
    if ((mk || mk1) && writer) {
      float* q = mk ? qk : qk1;
      const float2 r0 = mk ? make_float2(1.f, 0.f) : make_float2(0.f, 1.f);
#pragma unroll
      for (int m = 0; m < NP; m += 2) {
        const float2 ra = m == 0 ? r0 : rp[m], ia = m == 0 ? make_float2(0.f, 0.f) : ip[m];
        *reinterpret_cast<float4*>(q + 2 * m) = make_float4(ra.x, ra.y, rp[m + 1].x, rp[m + 1].y);
        *reinterpret_cast<float4*>(q + W + 2 * m) = make_float4(ia.x, ia.y, ip[m + 1].x, ip[m + 1].y);
      }
      // Row k: P00 = entry 0, P01 = entry 1; row k + 1: P10, P11.
      *reinterpret_cast<float4*>(blk + (mk ? 0 : 4)) = make_float4(rp[0].x, ip[0].x, rp[0].y, ip[0].y);
    }
    __syncwarp();
    const float4 b0 = *reinterpret_cast<const float4*>(blk);
    const float4 b1 = *reinterpret_cast<const float4*>(blk + 4);
    const float2 P01 = make_float2(b0.z, b0.w), P10 = make_float2(b1.x, b1.y), P11 = make_float2(b1.z, b1.w);
    const float pa = b0.x;
    const bool oka = pa > 0.f;
    const float ra = rcp_approx(oka ? pa : 1.f);
    const float2 h = make_float2(P10.x * ra, P10.y * ra);
    const float pb = P11.x - (h.x * P01.x - h.y * P01.y);
    const bool okb = pb > 0.f;
    const float rb = rcp_approx(okb ? pb : 1.f);
    if (fail == 0) {
      if (!oka) fail = k + 1;
      else if (!okb) fail = k + 2;
    }
    if (mk) my_r = ra;
    if (mk1) my_r = rb;
    float2 alpha, beta;
    {
      const float2 f0 = make_float2(rp[0].x, ip[0].x), f1 = make_float2(rp[0].y, ip[0].y);
      const float2 g = make_float2(f0.x * ra, f0.y * ra);
      const float2 gp = gj_cmul(P01, g);
      const float2 bt = make_float2((f1.x - gp.x) * rb, (f1.y - gp.y) * rb);
      const float2 bh = gj_cmul(bt, h);
      alpha = make_float2(g.x - bh.x, g.y - bh.y);
      beta = bt;
      if (mk) {
        beta = make_float2(P01.x * rb, P01.y * rb);
        const float2 t = gj_cmul(beta, h);
        alpha = make_float2(-t.x, -t.y);
      }
      if (mk1) {
        alpha = h;
        beta = make_float2(0.f, 0.f);
      }
    }
    const float2 nar = make_float2(-alpha.x, -alpha.x), pai = make_float2(alpha.y, alpha.y);
    const float2 nai = make_float2(-alpha.y, -alpha.y);
    const float2 nbr = make_float2(-beta.x, -beta.x), pbi = make_float2(beta.y, beta.y);
    const float2 nbi = make_float2(-beta.y, -beta.y);
    const float2 base0 = mk ? make_float2(1.f, 0.f) : (mk1 ? make_float2(0.f, 1.f) : make_float2(0.f, 0.f));
    float2 nr[NP], ni[NP];
#pragma unroll
    for (int m = 0; m < NP; m += 2) {
      const float4 ar = *reinterpret_cast<const float4*>(qk + 2 * m);
      const float4 ai = *reinterpret_cast<const float4*>(qk + W + 2 * m);
      const float4 br = *reinterpret_cast<const float4*>(qk1 + 2 * m);
      const float4 bi = *reinterpret_cast<const float4*>(qk1 + W + 2 * m);
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int c = m + hh;
        const float2 akr = hh == 0 ? make_float2(ar.x, ar.y) : make_float2(ar.z, ar.w);
        const float2 aki = hh == 0 ? make_float2(ai.x, ai.y) : make_float2(ai.z, ai.w);
        const float2 bkr = hh == 0 ? make_float2(br.x, br.y) : make_float2(br.z, br.w);
        const float2 bki = hh == 0 ? make_float2(bi.x, bi.y) : make_float2(bi.z, bi.w);
        const float2 baser = c == 0 ? base0 : rp[c];
        const float2 basei = c == 0 ? make_float2(0.f, 0.f) : ip[c];
        // re: base - a.re qk.re + a.im qk.im - b.re qk1.re + b.im qk1.im
        float2 tr = __ffma2_rn(nar, akr, baser);
        tr = __ffma2_rn(pai, aki, tr);
        tr = __ffma2_rn(nbr, bkr, tr);
        tr = __ffma2_rn(pbi, bki, tr);
        // im: base - a.re qk.im - a.im qk.re - b.re qk1.im - b.im qk1.re
        float2 ti = __ffma2_rn(nar, aki, basei);
        ti = __ffma2_rn(nai, akr, ti);
        ti = __ffma2_rn(nbr, bki, ti);
        ti = __ffma2_rn(nbi, bkr, ti);
        const int d = (c + NP - 1) % NP;   // rotate left by one pair (inverse columns to the end)
        nr[d] = tr;
        ni[d] = ti;
      }
    }
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      rp[m] = nr[m];
      ip[m] = ni[m];
    }
  }
  __syncwarp();   // the areas may be reused after the sweep
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
      const float r = rcp_approx(ok ? piv : 1.f);
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

// One lane's part of an L-MMSE solve on a group of UP lanes (lane i = user i,
// U = UP): mrow holds row i of the Hermitian G as loaded by the caller; rho is
// added to its diagonal, the group runs the sweep (column pairs for UP <= 16,
// 2 x 2 block pivots for UP = 32) and the lane is left with row i of
// A = (G + rho I)^{-1} in arow (natural column order, scaled by 1/p_i), A_ii in
// Ai and G_ii in gii.  Returns the sweep's failure index (0: all pivots
// positive).  Every kernel that solves from a D tile goes through this, so the
// separate and the fused launches round identically.
template <int UP>
__device__ __forceinline__ int gj_solve_row(float2 (&mrow)[UP], float rho, float* rowbuf, int i, bool writer,
                                            float2 (&arow)[UP], float& Ai, float& gii) {
  constexpr int NP = UP / 2;
  gii = 0.f;
#pragma unroll
  for (int j = 0; j < UP; ++j) {
    if (j == i) {
      gii = mrow[j].x;
      mrow[j] = make_float2(mrow[j].x + rho, 0.f);
    }
  }
  float2 rp[NP], ip[NP];
#pragma unroll
  for (int m = 0; m < NP; ++m) {
    rp[m] = make_float2(mrow[2 * m].x, mrow[2 * m + 1].x);
    ip[m] = make_float2(mrow[2 * m].y, mrow[2 * m + 1].y);
  }
  float rs = 1.f;
  int fail;
  if constexpr (UP >= 32) {
    fail = gj_sweep_block2<UP, UP>(rp, ip, rowbuf, i, writer, rs);
  } else {
    fail = gj_sweep_pairs<UP, UP>(rp, ip, rowbuf, i, writer, rs);
  }
  Ai = 1.f;
#pragma unroll
  for (int j = 0; j < UP; ++j) {
    arow[j] = make_float2((j % 2 ? rp[j / 2].y : rp[j / 2].x) * rs, (j % 2 ? ip[j / 2].y : ip[j / 2].x) * rs);
    if (j == i) Ai = arow[j].x;
  }
  return fail;
}

// z = sum_j arow[j] rhs[j] over j = 0 .. UP-1 (rhs 16-byte aligned): one
// right-hand side of the solved system, as four real FMA chains in j order,
//   P = (sum a_re y_re, sum a_re y_im),  Q = (sum a_im y_re, sum a_im y_im),
//   z = (P.re - Q.im, P.im + Q.re).
// gj_row_dot_pairs computes the same chains two at a time with paired FMAs and
// gives the same bits.
template <int UP>
__device__ __forceinline__ float2 gj_row_dot(const float2 (&arow)[UP], const float2* rhs) {
  float2 P = make_float2(0.f, 0.f), Q = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < UP; j += 2) {
    const float4 y2 = *reinterpret_cast<const float4*>(rhs + j);
    P.x = fmaf(arow[j].x, y2.x, P.x);
    P.y = fmaf(arow[j].x, y2.y, P.y);
    Q.x = fmaf(arow[j].y, y2.x, Q.x);
    Q.y = fmaf(arow[j].y, y2.y, Q.y);
    P.x = fmaf(arow[j + 1].x, y2.z, P.x);
    P.y = fmaf(arow[j + 1].x, y2.w, P.y);
    Q.x = fmaf(arow[j + 1].y, y2.z, Q.x);
    Q.y = fmaf(arow[j + 1].y, y2.w, Q.y);
  }
  return make_float2(__fsub_rn(P.x, Q.y), __fadd_rn(P.y, Q.x));
}

// The row of A held as duplicated pairs for gj_row_dot_pairs: are[j] =
// (Re a_j, Re a_j), aim[j] = (Im a_j, Im a_j).
template <int UP>
__device__ __forceinline__ void gj_row_split(const float2 (&arow)[UP], float2 (&are)[UP], float2 (&aim)[UP]) {
#pragma unroll
  for (int j = 0; j < UP; ++j) {
    are[j] = make_float2(arow[j].x, arow[j].x);
    aim[j] = make_float2(arow[j].y, arow[j].y);
  }
}

// gj_row_dot on the duplicated pairs: P += (a_re, a_re) * (y_re, y_im) and
// Q += (a_im, a_im) * (y_re, y_im) are one paired FMA each (__ffma2_rn rounds
// each half as fmaf would), half the FMA instructions of the scalar form.
template <int UP>
__device__ __forceinline__ float2 gj_row_dot_pairs(const float2 (&are)[UP], const float2 (&aim)[UP],
                                                   const float2* rhs) {
  float2 P = make_float2(0.f, 0.f), Q = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < UP; j += 2) {
    const float4 y2 = *reinterpret_cast<const float4*>(rhs + j);
    const float2 y0 = make_float2(y2.x, y2.y), y1 = make_float2(y2.z, y2.w);
    P = __ffma2_rn(are[j], y0, P);
    Q = __ffma2_rn(aim[j], y0, Q);
    P = __ffma2_rn(are[j + 1], y1, P);
    Q = __ffma2_rn(aim[j + 1], y1, Q);
  }
  return make_float2(__fsub_rn(P.x, Q.y), __fadd_rn(P.y, Q.x));
}

}  // namespace ffeq
