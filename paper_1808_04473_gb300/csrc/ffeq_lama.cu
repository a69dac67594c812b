// LAMA equalization (Sec. III-B, Algorithm 1) for the PD and FD architectures.
//
// Input: the workspace D written by the contraction (per subcarrier and cluster
// c: G_c[u][v] = D[v][u], y_c^MRC(n)_u = D[U+n][u]; PD is the case of one
// cluster holding G and y^MRC).  One group of UP lanes (UP = U padded to 8/16/32)
// runs the algorithm for one (subcarrier, cluster, received vector): lane i is
// user i and keeps row i of the normalized Gram matrix in registers.  In the
// paper's normalization (channel entries of variance 1/B; a cluster of S_c
// antennas is the system H_c / sqrt(S_c)) the cluster's pair is scaled by
// kappa = 1/S_c, with N0 kappa and beta_c = U kappa.  Each iteration
//     z   = y^MRC + (I - G) s + v                (the matrix-vector product reads s
//                                                 from the group's shared-memory copy,
//                                                 real and imaginary planes, four entries
//                                                 per 128-bit broadcast load, paired FMAs)
//     tau = N0 + beta phi
//     s'  = F(z, tau),  phi' = <G(z, tau)>      (posterior mean / variance of the
//                                                 equiprobable square-QAM prior, Eq. F;
//                                                 <.> a butterfly sum over the U lanes)
//     v'  = beta phi' / tau (z - s)
// and after T iterations the group leaves z^T with sigma_c^2 = tau^T.  The CTA
// holds every cluster of NB received vectors of one subcarrier and fuses them
// per user with the weights of Lemma 1 (Eq. fusionrule, opt_fusion): the
// per-cluster variance is shared by the users, so z = sum_c z_c / sigma_c^2 /
// sum_c 1/sigma_c^2 and sigma^2 = 1 / sum_c 1/sigma_c^2 (Thm. 3); PD is C = 1.
// The epilogue writes z, sigma^2 per (subcarrier, symbol, user) and the LLRs.
// Every lane of a warp runs the same T iterations (shuffles and __syncwarp use
// the full mask);
// groups past the last symbol or cluster work on clamped inputs and write nothing.
#include <cmath>

#include "ffeq_device.cuh"
#include "ffeq_epilogue.cuh"
#include "ffeq_internal.h"

namespace ffeq {
namespace {

// Posterior mean and variance of both PAM axes of a square-QAM symbol at once
// (x = (re, im); levels a_m = (2m - L + 1) d, L = 2^HB, equiprobable) under
// Gaussian noise of variance tau/2 per axis:
// p(a_m | x) ~ exp(-(x - a_m)^2 / tau) = 2^(-(x - a_m)^2 log2(e) / tau).
// Exponents are taken relative to the nearest level a0, and the moments about
// a0, so that a sharp posterior on an outer level keeps its small variance.
// The two axes run as the halves of paired FP32 operations (__ffma2_rn and
// friends, sm_100+), each half rounding as the scalar operation would.
// inv_d = 1/d; l2t = log2(e) / tau (both once per call site, not per level).
template <int HB>
__device__ __forceinline__ void pam_posterior2(float2 x, float l2t, float d, float inv_d, float2& mean, float2& var) {
  constexpr int L = 1 << HB;
  // Nearest level index: round((x/d + L - 1) / 2), clamped to [0, L).
  const float2 t = __fmul2_rn(__ffma2_rn(x, make_float2(inv_d, inv_d), make_float2(L - 1.f, L - 1.f)),
                              make_float2(0.5f, 0.5f));
  const float2 q = make_float2(fminf(fmaxf(rintf(t.x), 0.f), L - 1.f), fminf(fmaxf(rintf(t.y), 0.f), L - 1.f));
  const float2 a0 = __fmul2_rn(__ffma2_rn(q, make_float2(2.f, 2.f), make_float2(1.f - L, 1.f - L)),
                               make_float2(d, d));
  const float2 r0 = __ffma2_rn(a0, make_float2(-1.f, -1.f), x);          // x - a0
  const float2 ne0 = __fmul2_rn(r0, make_float2(-r0.x, -r0.y));           // -(x - a0)^2
  const float2 nl2t = make_float2(-l2t, -l2t);
  const float2 na0 = make_float2(-a0.x, -a0.y);
  float2 sw = make_float2(0.f, 0.f), s1 = sw, s2 = sw;
#pragma unroll
  for (int m = 0; m < L; ++m) {
    const float a = (2.f * static_cast<float>(m) - static_cast<float>(L - 1)) * d;
    const float2 e = __fadd2_rn(x, make_float2(-a, -a));                  // x - a
    const float2 u = __fmul2_rn(__ffma2_rn(e, e, ne0), nl2t);             // ((x-a0)^2 - e^2) l2t <= 0
    const float2 w = make_float2(ex2_approx(u.x), ex2_approx(u.y));       // 1 at a0
    const float2 da = __fadd2_rn(make_float2(a, a), na0);
    sw = __fadd2_rn(sw, w);
    s1 = __ffma2_rn(w, da, s1);
    s2 = __ffma2_rn(__fmul2_rn(w, da), da, s2);
  }
  const float2 r = make_float2(rcp_approx(sw.x), rcp_approx(sw.y));   // sw >= 1
  const float2 m1 = __fmul2_rn(s1, r);
  mean = __fadd2_rn(a0, m1);
  const float2 v2 = __ffma2_rn(make_float2(-m1.x, -m1.y), m1, __fmul2_rn(s2, r));
  var = make_float2(fmaxf(v2.x, 0.f), fmaxf(v2.y, 0.f));
}

// The batch kernel's body: one CTA's share of a subcarrier, NB received vectors
// from n0 on, every cluster -- the computation of lama_kernel below, line for
// line, on per-unit sizes and pointers (lama_kernel keeps its own copy: the
// uniform kernel calling this body measured 2% slower, 124.8 against 122.4 us
// for the B = 256, U = 16, C = 8, 1200 x 14 FD launch, with the same bits).  Pointers are this subcarrier's (D [Ceff][U + NS][U], z and sigma^2
// [NS][U], LLRs [NS][U][bits], info [Ceff]); S is the antennas of the calling
// thread's cluster.  live = false: the CTA's subcarrier is past the end (inputs
// clamped in bounds, nothing written).
struct LamaUnit {
  const float2* D;
  float2* z;
  float* s2;
  float* llr;
  int* info;
  int U, NS, Ceff, NB, n0, S, iters, bits;
  float N0, Es, d;
  bool live;
};

template <int UP, int HB>
__device__ __forceinline__ void lama_block(const LamaUnit& w, unsigned char* smem) {
  const int U = w.U, NS = w.NS, Ceff = w.Ceff, NB = w.NB, n0 = w.n0;
  const int g = threadIdx.x / UP, i = threadIdx.x % UP;
  const int ngroups = Ceff * NB;
  const int ngroups_pad = static_cast<int>(blockDim.x) / UP;   // groups of the last warp's padding lanes included
  const int c = g % Ceff, nb = g / Ceff;
  const int n = n0 + nb;
  const bool valid = g < ngroups && n < NS && w.live;
  const int cc = g < ngroups ? c : 0;
  const int nc = valid ? n : n0;
  const bool real = i < U;
  const int ic = real ? i : 0;

  // s of every group, double-buffered by iteration parity, as planes of real
  // and imaginary parts: [2][ngroups_pad][2][UP] floats.
  float* sbuf = reinterpret_cast<float*>(smem);
  float2* Fz = reinterpret_cast<float2*>(sbuf + 4 * ngroups_pad * UP);   // [ngroups][UP]
  float* Wt = reinterpret_cast<float*>(Fz + ngroups * UP);               // [ngroups]
  float* const sb0 = sbuf + 2 * g * UP;
  float* const sb1 = sbuf + 2 * (ngroups_pad + g) * UP;

  const int S = w.S;
  const float kap = S > 0 ? 1.f / static_cast<float>(S) : 0.f;
  const float beta = static_cast<float>(U) * kap;
  const float n0n = S > 0 ? w.N0 * kap : 1.f;     // an empty cluster: any tau > 0, weight 0 below
  const float2* Dg = w.D + static_cast<size_t>(cc) * static_cast<size_t>(U + NS) * U;
  // Row i of kappa G_c as pairs of adjacent columns: (re j, re j+1), (im j, im j+1).
  float2 gre[UP / 2], gim[UP / 2];
#pragma unroll
  for (int j = 0; j < UP; j += 2) {
    const float2 v0 = Dg[(j < U ? j : 0) * U + ic], v1 = Dg[(j + 1 < U ? j + 1 : 0) * U + ic];
    const float2 g0 = (real && j < U) ? cscale(v0, kap) : make_float2(0.f, 0.f);
    const float2 g1 = (real && j + 1 < U) ? cscale(v1, kap) : make_float2(0.f, 0.f);
    gre[j / 2] = make_float2(g0.x, g1.x);
    gim[j / 2] = make_float2(g0.y, g1.y);
  }
  const float2 yv = real ? cscale(Dg[(U + nc) * U + ic], kap) : make_float2(0.f, 0.f);
  const float d = w.d;
  const float inv_d = 1.f / d;
  const float invU = 1.f / static_cast<float>(U);
  constexpr float kLog2e = 1.4426950408889634f;

  float2 s = make_float2(0.f, 0.f), v = make_float2(0.f, 0.f), z;
  float phi = w.Es, tau;
  for (int t = 1;; ++t) {
    // z = y + s - G s + v.  A group lies within one warp: __syncwarp orders this
    // iteration's stores before the loads, and the buffer written next iteration
    // is the other one (the one after that is only written once every lane has
    // passed the next __syncwarp, i.e. finished these loads).
    float* cur = (t & 1) ? sb1 : sb0;
    cur[i] = s.x;
    cur[UP + i] = s.y;
    __syncwarp();
    // (G s)_i = sum_j G_ij s_j: four paired partial sums over even / odd j,
    // Re = sum g_re s_re - sum g_im s_im, Im = sum g_re s_im + sum g_im s_re.
    float2 rr = make_float2(0.f, 0.f), ii = rr, ri = rr, ir = rr;
#pragma unroll
    for (int j = 0; j < UP; j += 4) {
      const float4 sr = *reinterpret_cast<const float4*>(cur + j);
      const float4 si = *reinterpret_cast<const float4*>(cur + UP + j);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2 sr2 = h ? make_float2(sr.z, sr.w) : make_float2(sr.x, sr.y);
        const float2 si2 = h ? make_float2(si.z, si.w) : make_float2(si.x, si.y);
        rr = __ffma2_rn(gre[j / 2 + h], sr2, rr);
        ii = __ffma2_rn(gim[j / 2 + h], si2, ii);
        ri = __ffma2_rn(gre[j / 2 + h], si2, ri);
        ir = __ffma2_rn(gim[j / 2 + h], sr2, ir);
      }
    }
    const float2 gs = make_float2((rr.x + rr.y) - (ii.x + ii.y), (ri.x + ri.y) + (ir.x + ir.y));
    z = __fadd2_rn(__fadd2_rn(__fadd2_rn(yv, s), make_float2(-gs.x, -gs.y)), v);
    tau = fmaf(beta, phi, n0n);
    if (t >= w.iters) break;
    const float inv_tau = rcp_approx(tau);
    const float l2t = kLog2e * inv_tau;
    float2 mean, var;
    pam_posterior2<HB>(z, l2t, d, inv_d, mean, var);
    float gsum = real ? var.x + var.y : 0.f;
#pragma unroll
    for (int o = UP / 2; o > 0; o >>= 1) gsum += __shfl_xor_sync(kFullMask, gsum, o, UP);
    const float phin = gsum * invU;
    const float f = beta * phin * inv_tau;
    v = __fmul2_rn(__fadd2_rn(z, make_float2(-s.x, -s.y)), make_float2(f, f));
    s = mean;
    phi = phin;
  }

  if (g < ngroups) {
    const float wc = S > 0 ? 1.f / tau : 0.f;
    Fz[g * UP + i] = cscale(z, wc);
    if (i == 0) Wt[g] = wc;
    if (valid && i == 0 && w.info) w.info[c] = 0;
  }
  __syncthreads();

  // ---- per (symbol, user) of this CTA: fuse over the clusters, write the outputs
  const int hb = w.bits / 2;
  for (int e = threadIdx.x; e < NB * U; e += blockDim.x) {
    const int b = e / U, u = e - b * U;
    const int nn = n0 + b;
    if (nn >= NS || !w.live) break;
    float2 nm = make_float2(0.f, 0.f);
    float dn = 0.f;
    for (int k = 0; k < Ceff; ++k) {
      nm = cadd(nm, Fz[(b * Ceff + k) * UP + u]);
      dn += Wt[b * Ceff + k];
    }
    float2 zz = make_float2(0.f, 0.f);
    float s2 = INFINITY;
    if (dn > 0.f) {
      const float rr = 1.f / dn;
      zz = cscale(nm, rr);
      s2 = rr;
    }
    const size_t zi = static_cast<size_t>(nn) * U + u;
    w.z[zi] = zz;
    w.s2[zi] = s2;
    if (w.bits) symbol_llr(zz, s2, w.d, hb, w.llr + zi * w.bits);
  }
}

template <int UP, int HB>
__global__ void __maxnreg__(UP == 32 ? 128 : 64) lama_kernel(const SolveParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int U = p.U, NS = p.n_sym, Ceff = p.Ceff, NB = p.spc;   // spc: received vectors per CTA
  const int nblk = (NS + NB - 1) / NB;
  const int sc = blockIdx.x / nblk;
  const int n0 = (blockIdx.x - sc * nblk) * NB;
  const int g = threadIdx.x / UP, i = threadIdx.x % UP;
  const int ngroups = Ceff * NB;
  const int ngroups_pad = static_cast<int>(blockDim.x) / UP;   // groups of the last warp's padding lanes included
  const int c = g % Ceff, nb = g / Ceff;
  const int n = n0 + nb;
  const bool valid = g < ngroups && n < NS && sc < p.n_sc;
  const int cc = g < ngroups ? c : 0;
  const int nc = valid ? n : n0;
  const int scc = sc < p.n_sc ? sc : p.n_sc - 1;
  const bool real = i < U;
  const int ic = real ? i : 0;

  // s of every group, double-buffered by iteration parity, as planes of real
  // and imaginary parts: [2][ngroups_pad][2][UP] floats.
  float* sbuf = reinterpret_cast<float*>(smem);
  float2* Fz = reinterpret_cast<float2*>(sbuf + 4 * ngroups_pad * UP);   // [ngroups][UP]
  float* Wt = reinterpret_cast<float*>(Fz + ngroups * UP);               // [ngroups]
  float* const sb0 = sbuf + 2 * g * UP;
  float* const sb1 = sbuf + 2 * (ngroups_pad + g) * UP;

  // Wait for the contraction grid (programmatic dependent launch).
  asm volatile("griddepcontrol.wait;" ::: "memory");

  const int S = p.cl_size[cc];
  const float kap = S > 0 ? 1.f / static_cast<float>(S) : 0.f;
  const float beta = static_cast<float>(U) * kap;
  const float n0n = S > 0 ? p.N0 * kap : 1.f;     // an empty cluster: any tau > 0, weight 0 below
  const float2* Dg = p.D + (static_cast<size_t>(scc) * Ceff + cc) * static_cast<size_t>(U + NS) * U;
  // Row i of kappa G_c as pairs of adjacent columns: (re j, re j+1), (im j, im j+1).
  float2 gre[UP / 2], gim[UP / 2];
#pragma unroll
  for (int j = 0; j < UP; j += 2) {
    const float2 v0 = Dg[(j < U ? j : 0) * U + ic], v1 = Dg[(j + 1 < U ? j + 1 : 0) * U + ic];
    const float2 g0 = (real && j < U) ? cscale(v0, kap) : make_float2(0.f, 0.f);
    const float2 g1 = (real && j + 1 < U) ? cscale(v1, kap) : make_float2(0.f, 0.f);
    gre[j / 2] = make_float2(g0.x, g1.x);
    gim[j / 2] = make_float2(g0.y, g1.y);
  }
  const float2 yv = real ? cscale(Dg[(U + nc) * U + ic], kap) : make_float2(0.f, 0.f);
  const float d = p.llr_scale;
  const float inv_d = 1.f / d;
  const float invU = 1.f / static_cast<float>(U);
  constexpr float kLog2e = 1.4426950408889634f;

  float2 s = make_float2(0.f, 0.f), v = make_float2(0.f, 0.f), z;
  float phi = p.Es, tau;
  for (int t = 1;; ++t) {
    // z = y + s - G s + v.  A group lies within one warp: __syncwarp orders this
    // iteration's stores before the loads, and the buffer written next iteration
    // is the other one (the one after that is only written once every lane has
    // passed the next __syncwarp, i.e. finished these loads).
    float* cur = (t & 1) ? sb1 : sb0;
    cur[i] = s.x;
    cur[UP + i] = s.y;
    __syncwarp();
    // (G s)_i = sum_j G_ij s_j: four paired partial sums over even / odd j,
    // Re = sum g_re s_re - sum g_im s_im, Im = sum g_re s_im + sum g_im s_re.
    float2 rr = make_float2(0.f, 0.f), ii = rr, ri = rr, ir = rr;
#pragma unroll
    for (int j = 0; j < UP; j += 4) {
      const float4 sr = *reinterpret_cast<const float4*>(cur + j);
      const float4 si = *reinterpret_cast<const float4*>(cur + UP + j);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float2 sr2 = h ? make_float2(sr.z, sr.w) : make_float2(sr.x, sr.y);
        const float2 si2 = h ? make_float2(si.z, si.w) : make_float2(si.x, si.y);
        rr = __ffma2_rn(gre[j / 2 + h], sr2, rr);
        ii = __ffma2_rn(gim[j / 2 + h], si2, ii);
        ri = __ffma2_rn(gre[j / 2 + h], si2, ri);
        ir = __ffma2_rn(gim[j / 2 + h], sr2, ir);
      }
    }
    const float2 gs = make_float2((rr.x + rr.y) - (ii.x + ii.y), (ri.x + ri.y) + (ir.x + ir.y));
    z = __fadd2_rn(__fadd2_rn(__fadd2_rn(yv, s), make_float2(-gs.x, -gs.y)), v);
    tau = fmaf(beta, phi, n0n);
    if (t >= p.lama_iters) break;
    const float inv_tau = rcp_approx(tau);
    const float l2t = kLog2e * inv_tau;
    float2 mean, var;
    pam_posterior2<HB>(z, l2t, d, inv_d, mean, var);
    float gsum = real ? var.x + var.y : 0.f;
#pragma unroll
    for (int o = UP / 2; o > 0; o >>= 1) gsum += __shfl_xor_sync(kFullMask, gsum, o, UP);
    const float phin = gsum * invU;
    const float f = beta * phin * inv_tau;
    v = __fmul2_rn(__fadd2_rn(z, make_float2(-s.x, -s.y)), make_float2(f, f));
    s = mean;
    phi = phin;
  }

  if (g < ngroups) {
    const float w = S > 0 ? 1.f / tau : 0.f;
    Fz[g * UP + i] = cscale(z, w);
    if (i == 0) Wt[g] = w;
    if (valid && i == 0 && p.info) p.info[static_cast<size_t>(sc) * Ceff + c] = 0;
  }
  __syncthreads();

  // ---- per (symbol, user) of this CTA: fuse over the clusters, write the outputs
  const int hb = p.llr_bits / 2;
  for (int e = threadIdx.x; e < NB * U; e += blockDim.x) {
    const int b = e / U, u = e - b * U;
    const int nn = n0 + b;
    if (nn >= NS || sc >= p.n_sc) break;
    float2 nm = make_float2(0.f, 0.f);
    float dn = 0.f;
    for (int k = 0; k < Ceff; ++k) {
      nm = cadd(nm, Fz[(b * Ceff + k) * UP + u]);
      dn += Wt[b * Ceff + k];
    }
    float2 zz = make_float2(0.f, 0.f);
    float s2 = INFINITY;
    if (dn > 0.f) {
      const float rr = 1.f / dn;
      zz = cscale(nm, rr);
      s2 = rr;
    }
    const size_t zi = (static_cast<size_t>(sc) * NS + nn) * U + u;
    p.z[zi] = zz;
    p.sigma2[zi] = s2;
    if (p.llr_bits) symbol_llr(zz, s2, p.llr_scale, hb, p.llr + zi * p.llr_bits);
  }
}

// Uneven batch: one CTA per unit (subcarrier of an instance), whose descriptor
// gives the sizes, scalars and offsets (each checked against the batch's
// extents; a unit that fails is skipped and sets FFEQ_ERR_INVALID_ARG in the
// status word).  The CTA takes the unit's received vectors NB at a time, NB =
// threads / (Ceff UP), clusters of B / Ceff antennas; sigma^2 per received
// vector ([NS][U] at s2_off).
template <int UP, int HB>
__global__ void __maxnreg__(UP == 32 ? 128 : 64) lama_batch_kernel(const SolveParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int j = blockIdx.x;
  if (j >= p.n_desc) return;
  const BatchDesc d = p.desc[j];
  const int U = d.U, NS = d.n_sym, Ceff = d.Ceff, B = d.B;
  const long long lanes = static_cast<long long>(Ceff) * UP;
  bool ok = U >= 1 && U <= UP && NS >= 1 && NS <= kNsymMax && Ceff >= 1 && Ceff <= kMaxClusters && B >= Ceff &&
            B % Ceff == 0 && lanes <= static_cast<long long>(blockDim.x) && d.N0 > 0.f && d.Es > 0.f &&
            d.llr_scale > 0.f && p.llr_bits > 0;
  if (ok) {
    const long long mat = static_cast<long long>(U + NS) * U, per = static_cast<long long>(NS) * U;
    ok = span_ok(d.d_off, Ceff * mat, p.lim.d) && span_ok(d.z_off, per, p.lim.z) && span_ok(d.s2_off, per, p.lim.s2) &&
         span_ok(d.llr_off, per * p.llr_bits, p.lim.llr) && (!p.info || span_ok(d.info_off, Ceff, p.lim.info));
  }
  if (!ok) {
    if (threadIdx.x == 0 && p.status) atomicExch(p.status, FFEQ_ERR_INVALID_ARG);
    return;
  }
  LamaUnit w;
  w.D = p.D + d.d_off;
  w.z = p.z + d.z_off;
  w.s2 = p.sigma2 + d.s2_off;
  w.llr = p.llr + d.llr_off;
  w.info = p.info ? p.info + d.info_off : nullptr;
  w.U = U;
  w.NS = NS;
  w.Ceff = Ceff;
  w.NB = static_cast<int>(blockDim.x / lanes);
  w.S = B / Ceff;
  w.iters = p.lama_iters;
  w.bits = p.llr_bits;
  w.N0 = d.N0;
  w.Es = d.Es;
  w.d = d.llr_scale;
  w.live = true;
  for (int n0 = 0; n0 < NS; n0 += w.NB) {
    w.n0 = n0;
    lama_block<UP, HB>(w, smem);
    __syncthreads();   // the next vectors reuse the shared areas
  }
}

template <int UP, int HB>
cudaError_t launch_lama_up(const SolveParams& p, cudaStream_t stream) {
  const int ngroups = p.Ceff * p.spc;
  const int threads = ((ngroups * UP + 31) / 32) * 32;
  const int ngroups_pad = threads / UP;
  const size_t smem = static_cast<size_t>(4 * ngroups_pad) * UP * sizeof(float) +
                      static_cast<size_t>(ngroups) * UP * sizeof(float2) + static_cast<size_t>(ngroups) * 4;
  const int nblk = (p.n_sym + p.spc - 1) / p.spc;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(p.n_sc) * nblk);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, lama_kernel<UP, HB>, p);
}

template <int UP>
cudaError_t launch_lama_bits(const SolveParams& p, cudaStream_t stream) {
  switch (p.llr_bits) {
    case 2: return launch_lama_up<UP, 1>(p, stream);
    case 4: return launch_lama_up<UP, 2>(p, stream);
    case 6: return launch_lama_up<UP, 3>(p, stream);
    default: return launch_lama_up<UP, 4>(p, stream);
  }
}

template <int UP, int HB>
cudaError_t launch_lama_batch_up(const SolveParams& p, cudaStream_t stream) {
  const int ngp = p.threads / UP;   // lane groups of a CTA (each unit uses Ceff * NB of them)
  const size_t smem = static_cast<size_t>(4 * ngp) * UP * sizeof(float) +
                      static_cast<size_t>(ngp) * UP * sizeof(float2) + static_cast<size_t>(ngp) * 4;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(p.n_desc));
  cfg.blockDim = dim3(p.threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, lama_batch_kernel<UP, HB>, p);
}

template <int UP>
cudaError_t launch_lama_batch_bits(const SolveParams& p, cudaStream_t stream) {
  switch (p.llr_bits) {
    case 2: return launch_lama_batch_up<UP, 1>(p, stream);
    case 4: return launch_lama_batch_up<UP, 2>(p, stream);
    case 6: return launch_lama_batch_up<UP, 3>(p, stream);
    default: return launch_lama_batch_up<UP, 4>(p, stream);
  }
}

}  // namespace

// Uneven batch (p.U = the group's users padding, p.threads a multiple of 32 of
// at least Ceff * UP for every unit, p.desc / p.n_desc the group's units).
cudaError_t launch_lama_batch(const SolveParams& p, cudaStream_t stream) {
  if (p.n_desc <= 0) return cudaSuccess;
  if (p.threads < 32 || p.threads > 512 || p.threads % 32 || p.threads % p.U) return cudaErrorInvalidValue;
  switch (p.U) {
    case 8: return launch_lama_batch_bits<8>(p, stream);
    case 16: return launch_lama_batch_bits<16>(p, stream);
    case 32: return launch_lama_batch_bits<32>(p, stream);
    default: return cudaErrorInvalidValue;
  }
}

// Received vectors per CTA: the groups of all clusters of NB vectors, at most
// 256 lanes, with NB chosen so that the blocks of one subcarrier split n_sym evenly.
int lama_symbols_per_cta(int U, int Ceff, int n_sym) {
  const int lanes = Ceff * padded_users(U);
  int nbmax = 256 / lanes;
  if (nbmax < 1) nbmax = 1;
  const int nblk = (n_sym + nbmax - 1) / nbmax;
  return (n_sym + nblk - 1) / nblk;
}

cudaError_t launch_lama(const SolveParams& p_in, cudaStream_t stream) {
  SolveParams p = p_in;
  p.spc = lama_symbols_per_cta(p.U, p.Ceff, p.n_sym);
  switch (padded_users(p.U)) {
    case 8: return launch_lama_bits<8>(p, stream);
    case 16: return launch_lama_bits<16>(p, stream);
    default: return launch_lama_bits<32>(p, stream);
  }
}

}  // namespace ffeq
