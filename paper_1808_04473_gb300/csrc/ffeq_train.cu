// Differentiable FD equalization: forward with per-cluster regularizers and
// free fusion weights, and its hand-written adjoint.
//
// Forward (per subcarrier k, cluster c; n_sym right-hand sides):
//   X_c = (G_c + rho_c I)^{-1} B_c,  B_c = H_c^H Y_c       (L-MMSE, Sec. III-A, with rho_c free)
//   z_u = sum_c nu[c][u] X_c[u]                            (Eq. fusionrule with free weights)
// Adjoint of a real loss with g_z = dL/dRe z + i dL/dIm z:
//   G_x,c = diag(nu_c) G_z,   G_b,c = (G_c + rho_c I)^{-1} G_x,c
//   dL/dH_c   = Y_c G_b^H - H_c W_c,   W_c = G_b X_c^H + X_c G_b^H
//   dL/dY_c   = H_c G_b
//   dL/drho_c = -sum_k Re tr(G_b^H X_c),  dL/dnu[c][u] = sum_k sum_n Re(conj(g_z,u,n) X_c,u,n)
// (dX = M^{-1}(dB - dM X), dM = dH^H H + H^H dH + drho I, dB = dH^H Y + H^H dY.)
// The factorization is recomputed in the backward pass (a Gauss-Jordan sweep on
// [G_c + rho_c I | G_x,c]); the forward keeps the local Gram matrices and the
// local estimates X_c in the workspace.
//
// Every sweep is the paired-FMA Gauss-Jordan sweep with deferred scaling of
// ffeq_gj.cuh on the augmented row [G_c + rho I | R] of UP + NR columns, NR the
// right-hand-side columns rounded up from n_sym (4 when n_sym <= 4, else 16),
// so a one-symbol problem does not sweep 16 columns of padding.
//
// Workspace: D [n_sc][C][U+n_sym][U] (contraction output, as ffeq_equalize),
// X [n_sc][C][n_sym][U], Gb [n_sc][C][n_sym][U], W [n_sc][C][U][U] (complex) and
// per-subcarrier partial sums P [n_sc][C][1+U] (float).
#include <cmath>

#include "ffeq_device.cuh"
#include "ffeq_gj.cuh"
#include "ffeq_internal.h"

namespace ffeq {
namespace {

// Right-hand-side columns of the augmented sweep for n_sym symbols.
inline int rhs_columns(int n_sym) { return n_sym <= 4 ? 4 : kNsymMax; }

template <int UP, int NR>
struct TrainLayout {
  static constexpr int kW = UP + NR;              // augmented row width
  static constexpr int kRow = 2 * kW + 4;         // the sweep's two pivot-row buffers (float2 units)
  // Per group: pivot-row buffers + two [NR][UP] blocks.
  static constexpr int kGroup = kRow + 2 * NR * UP + 8;
};

// Row i of [G_c + rho I | R] from the workspace D (padding: identity / zero), as
// pairs of adjacent columns (rp: re of columns 2m, 2m + 1; ip: im).  rhs(n)
// supplies R[i][n] for n < NS.
template <int UP, int NR, typename Rhs>
__device__ __forceinline__ void load_row(float2 (&rp)[(UP + NR) / 2], float2 (&ip)[(UP + NR) / 2],
                                         const float2* Dg, int U, int NS, int i, bool valid, float rho, Rhs rhs) {
  constexpr int W = UP + NR;
  const int ic = i < U ? i : 0;
  float2 aug[W];
#pragma unroll
  for (int j = 0; j < UP; ++j) aug[j] = Dg[(j < U ? j : 0) * U + ic];
#pragma unroll
  for (int j = 0; j < UP; ++j) {
    const bool real = valid && i < U && j < U;
    float2 v = real ? aug[j] : make_float2(i == j ? 1.f : 0.f, 0.f);
    if (real && i == j) v = make_float2(v.x + rho, 0.f);
    aug[j] = v;
  }
#pragma unroll
  for (int n = 0; n < NR; ++n) aug[UP + n] = (n < NS && valid && i < U) ? rhs(n) : make_float2(0.f, 0.f);
#pragma unroll
  for (int m = 0; m < W / 2; ++m) {
    rp[m] = make_float2(aug[2 * m].x, aug[2 * m + 1].x);
    ip[m] = make_float2(aug[2 * m].y, aug[2 * m + 1].y);
  }
}

// Column t of the swept row (after the sweep: t < NR the solution for right-hand
// side t, NR + j column j of the inverse), times the deferred scale 1 / p_i.
template <int W>
__device__ __forceinline__ float2 swept(const float2 (&rp)[W / 2], const float2 (&ip)[W / 2], int t, float rs) {
  return make_float2((t % 2 ? rp[t / 2].y : rp[t / 2].x) * rs, (t % 2 ? ip[t / 2].y : ip[t / 2].x) * rs);
}

// Forward: one CTA per subcarrier, one group of UP lanes per cluster.
template <int UP, int NR>
__global__ void __launch_bounds__(512) train_forward_kernel(const TrainParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  using Lay = TrainLayout<UP, NR>;
  constexpr int W = Lay::kW;
  const int U = p.U, NS = p.n_sym, C = p.C;
  const int g = threadIdx.x / UP, i = threadIdx.x % UP;
  const int k = blockIdx.x;
  const int gm = g < C ? g : C - 1;
  const bool valid = g < C;
  float2* rowbuf = reinterpret_cast<float2*>(smem + 16) + gm * Lay::kGroup;
  float2* F = rowbuf + Lay::kRow;              // [NR][UP]: nu * X of this cluster
  int* fail_any = reinterpret_cast<int*>(smem);
  if (threadIdx.x == 0) *fail_any = 0;
  __syncthreads();

  const size_t matSize = static_cast<size_t>(U + NS) * U;
  const float2* Dg = p.D + (static_cast<size_t>(k) * C + gm) * matSize;
  float2 rp[W / 2], ip[W / 2];
  const float rho = p.rho_c[gm];
  load_row<UP, NR>(rp, ip, Dg, U, NS, i, valid, rho, [&](int n) { return Dg[(U + n) * U + i]; });
  float rs = 1.f;
  const int fail = gj_sweep_pairs<UP, W>(rp, ip, reinterpret_cast<float*>(rowbuf), i, valid, rs);
  if (valid && i == 0 && fail) atomicOr(fail_any, 1);

  const float w = (valid && i < U) ? p.nu[gm * U + i] : 0.f;
  if (valid && i < U) {
    float2* Xk = p.X + (static_cast<size_t>(k) * C + gm) * NS * U;
#pragma unroll
    for (int n = 0; n < NR; ++n) {
      if (n < NS) {
        const float2 x = swept<W>(rp, ip, n, rs);
        Xk[n * U + i] = x;
        F[n * UP + i] = cscale(x, w);
      }
    }
  }
  __syncthreads();
  const bool bad = *fail_any != 0;
  for (int e = threadIdx.x; e < U * NS; e += blockDim.x) {
    const int u = e % U, n = e / U;
    float2 acc = make_float2(0.f, 0.f);
    for (int c = 0; c < C; ++c)
      acc = cadd(acc, (reinterpret_cast<float2*>(smem + 16) + c * Lay::kGroup + Lay::kRow)[n * UP + u]);
    p.z[(static_cast<size_t>(k) * NS + n) * U + u] = bad ? make_float2(NAN, NAN) : acc;
  }
}

// Backward, per cluster: G_b = (G_c + rho_c I)^{-1} diag(nu_c) G_z, the partial
// sums of dL/drho_c and dL/dnu[c][.] for this subcarrier, and W_c.
template <int UP, int NR>
__global__ void __launch_bounds__(512) train_backward_solve_kernel(const TrainParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  using Lay = TrainLayout<UP, NR>;
  constexpr int W = Lay::kW;
  const int U = p.U, NS = p.n_sym, C = p.C;
  const int g = threadIdx.x / UP, i = threadIdx.x % UP;
  const int k = blockIdx.x;
  const int gm = g < C ? g : C - 1;
  const bool valid = g < C;
  float2* rowbuf = reinterpret_cast<float2*>(smem + 16) + gm * Lay::kGroup;
  float2* Gs = rowbuf + Lay::kRow;              // [NR][UP]  G_b of this cluster
  float2* Xs = Gs + NR * UP;                    // [NR][UP]  X of this cluster

  const size_t matSize = static_cast<size_t>(U + NS) * U;
  const float2* Dg = p.D + (static_cast<size_t>(k) * C + gm) * matSize;
  const float2* gz = p.gz + static_cast<size_t>(k) * NS * U;
  const float w = (valid && i < U) ? p.nu[gm * U + i] : 0.f;
  float2 rp[W / 2], ip[W / 2];
  load_row<UP, NR>(rp, ip, Dg, U, NS, i, valid, p.rho_c[gm], [&](int n) { return cscale(gz[n * U + i], w); });
  float rs = 1.f;
  gj_sweep_pairs<UP, W>(rp, ip, reinterpret_cast<float*>(rowbuf), i, valid, rs);

  // Row i of G_b; X row i from the forward pass.
  const size_t off = (static_cast<size_t>(k) * C + gm) * NS * U;
  float2 gb[NR], x[NR];
  float prho = 0.f, pnu = 0.f;
#pragma unroll
  for (int n = 0; n < NR; ++n) {
    gb[n] = swept<W>(rp, ip, n, rs);
    x[n] = (n < NS && valid && i < U) ? p.X[off + n * U + i] : make_float2(0.f, 0.f);
    const float2 gzv = (n < NS && valid && i < U) ? gz[n * U + i] : make_float2(0.f, 0.f);
    if (n < NS) {
      prho -= gb[n].x * x[n].x + gb[n].y * x[n].y;          // Re(conj(G_b) X)
      pnu += gzv.x * x[n].x + gzv.y * x[n].y;               // Re(conj(g_z) X)
    }
  }
#pragma unroll
  for (int o = UP / 2; o > 0; o >>= 1) prho += __shfl_xor_sync(kFullMask, prho, o, UP);
  float* P = p.P + (static_cast<size_t>(k) * C + gm) * (1 + U);
  if (valid) {
    if (i == 0) P[0] = prho;
    if (i < U) P[1 + i] = pnu;
  }
  if (valid && i < U) {
#pragma unroll
    for (int n = 0; n < NR; ++n) {
      if (n < NS) {
        p.Gb[off + n * U + i] = gb[n];
        Gs[n * UP + i] = gb[n];
        Xs[n * UP + i] = x[n];
      }
    }
  }
  __syncwarp();
  // W row i: W[i][v] = sum_n G_b[i][n] conj(X[v][n]) + X[i][n] conj(G_b[v][n]).
  if (valid && i < U) {
    float2* Wk = p.Wm + (static_cast<size_t>(k) * C + gm) * U * U + i * U;
    for (int v = 0; v < U; ++v) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int n = 0; n < NR; ++n) {
        if (n < NS) {
          const float2 xv = Xs[n * UP + v], gv = Gs[n * UP + v];
          // G_b[i] conj(X[v]) + X[i] conj(G_b[v])
          acc = cfma(gb[n], make_float2(xv.x, -xv.y), acc);
          acc = cfma(x[n], make_float2(gv.x, -gv.y), acc);
        }
      }
      Wk[v] = acc;
    }
  }
}

// Adjoint through the optimal-weight rule (the FD estimate ffeq_equalize
// computes with unbiased pairs: Lemma 1's weights from diag(A_c) and mu),
// per subcarrier, from the contraction output D and dL/dz.  With M_c = G_c +
// rho I, A_c = M_c^{-1}, X_c = A_c B_c, a_c = diag(A_c), w_c = 1 / a_c,
// D_u = sum_c (w_{c,u} - rho) and z_u = sum_c w_{c,u} X_{c,u} / D_u (Eq. fusionrule
// with nu = mu / (N0 a) / sum, N0 cancelled):
//   G_x = diag(w_c / D) G_z,   G_b = A_c G_x,
//   q_u = -Re(sum_n conj(g_z,u,n) (X_{c,u,n} - z_{u,n})) / (D_u a_{c,u}^2),
//   W_c = X_c G_b^H + G_b X_c^H + 2 A_c diag(q) A_c,
// after which train_backward_contract_kernel forms dL/dH_c = Y_c G_b^H - H_c W_c
// and dL/dY_c = H_c G_b.  (dz_u = sum_c (w dX + (X - z) dw) / D with dw = -da / a^2,
// dX = A (dB - dM X), da_u = -[A dM A]_uu.)  One CTA per subcarrier, one group of
// UP lanes per cluster; lane i = user i.  The sweep runs on [M_c | B_c] and
// leaves row i of X_c and of A_c.  A user no cluster can see (D_u <= 0) has
// z = 0 and contributes nothing.  A subcarrier with a system that is not
// positive definite gets NaN gradients.
template <int UP, int NR>
struct OptimalLayout {
  static constexpr int kW = UP + NR;
  static constexpr int kRow = 2 * kW + 4;   // the sweep's pivot-row buffers; then row broadcasts of A
  // Per group: pivot-row buffers, X [NR][UP], G_x then G_b [NR][UP], and q
  // (UP floats as UP / 2 complex).
  static constexpr int kGroup = kRow + 2 * NR * UP + UP / 2 + 8;
};

template <int UP, int NR>
__global__ void __launch_bounds__(512) train_optimal_solve_kernel(const TrainParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  using Lay = OptimalLayout<UP, NR>;
  constexpr int W = Lay::kW;
  const int U = p.U, NS = p.n_sym, C = p.C;
  const int g = threadIdx.x / UP, i = threadIdx.x % UP;
  const int k = blockIdx.x;
  const int gm = g < C ? g : C - 1;
  const bool valid = g < C;
  int* fail_any = reinterpret_cast<int*>(smem);
  float* wv = reinterpret_cast<float*>(smem + 16);                       // [C][UP]: w_{c,u}
  float2* grp = reinterpret_cast<float2*>(smem + 16 + ((static_cast<size_t>(C) * UP * 4 + 15) / 16) * 16);
  float2* rowbuf = grp + gm * Lay::kGroup;
  float2* Xs = rowbuf + Lay::kRow;            // [NR][UP]
  float2* Gs = Xs + NR * UP;                  // [NR][UP]
  float* qv = reinterpret_cast<float*>(Gs + NR * UP);   // [UP]
  if (threadIdx.x == 0) *fail_any = 0;
  __syncthreads();

  const size_t matSize = static_cast<size_t>(U + NS) * U;
  const float2* Dg = p.D + (static_cast<size_t>(k) * C + gm) * matSize;
  const float rho = p.rho;
  float2 rp[W / 2], ip[W / 2];
  load_row<UP, NR>(rp, ip, Dg, U, NS, i, valid, rho, [&](int n) { return Dg[(U + n) * U + i]; });
  float rs = 1.f;
  const int fail = gj_sweep_pairs<UP, W>(rp, ip, reinterpret_cast<float*>(rowbuf), i, valid, rs);
  if (valid && i == 0 && fail) atomicOr(fail_any, 1);
  // Row i of X_c and of A_c.
  float2 xr[NR], ar[UP];
#pragma unroll
  for (int n = 0; n < NR; ++n) xr[n] = swept<W>(rp, ip, n, rs);
#pragma unroll
  for (int j = 0; j < UP; ++j) ar[j] = swept<W>(rp, ip, NR + j, rs);
  float a = 1.f;
#pragma unroll
  for (int j = 0; j < UP; ++j)
    if (j == i) a = ar[j].x;
  const bool real = valid && i < U;
  const float w = real ? 1.f / a : 0.f;
  if (valid) {
    wv[gm * UP + i] = real ? w : rho;         // padding users: w - rho = 0
#pragma unroll
    for (int n = 0; n < NR; ++n) Xs[n * UP + i] = (real && n < NS) ? xr[n] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const bool bad = *fail_any != 0;
  // D_u and z_u over the clusters in a fixed order (every group for its own users).
  float Du = 0.f;
  for (int cc = 0; cc < C; ++cc) Du += wv[cc * UP + i] - rho;
  const bool seen = Du > 0.f;
  const float invD = seen ? 1.f / Du : 0.f;
  const float2* gzk = p.gz + static_cast<size_t>(k) * NS * U;
  float qn = 0.f;                                 // sum_n Re(conj(g_z) (X - z))
#pragma unroll
  for (int n = 0; n < NR; ++n) {
    if (n < NS) {
      float2 num = make_float2(0.f, 0.f);
      for (int cc = 0; cc < C; ++cc) {
        const float2 xc = (grp + cc * Lay::kGroup + Lay::kRow)[n * UP + i];
        const float wc = wv[cc * UP + i];
        num = make_float2(fmaf(wc, xc.x, num.x), fmaf(wc, xc.y, num.y));
      }
      const float2 zn = cscale(num, invD);
      const float2 gzv = real ? gzk[n * U + i] : make_float2(0.f, 0.f);
      qn = fmaf(gzv.x, xr[n].x - zn.x, fmaf(gzv.y, xr[n].y - zn.y, qn));
      if (valid) Gs[n * UP + i] = cscale(gzv, w * invD);   // G_x
    }
  }
  if (valid) qv[i] = (real && seen) ? -qn * invD * w * w : 0.f;   // 1 / a^2 = w^2
  __syncwarp();
  // G_b row i = sum_j A_ij G_x[j].
  float2 gb[NR];
#pragma unroll
  for (int n = 0; n < NR; ++n) {
    float2 acc = make_float2(0.f, 0.f);
    if (n < NS) {
#pragma unroll
      for (int j = 0; j < UP; ++j) acc = cfma(ar[j], Gs[n * UP + j], acc);
    }
    gb[n] = bad ? make_float2(NAN, NAN) : acc;
  }
  __syncwarp();
  const size_t off = (static_cast<size_t>(k) * C + gm) * NS * U;
  if (valid) {
#pragma unroll
    for (int n = 0; n < NR; ++n) {
      if (n < NS) {
        Gs[n * UP + i] = gb[n];
        if (real) p.Gb[off + n * U + i] = gb[n];
      }
    }
  }
  // W row i, column v: sum_n (G_b[i][n] conj(X[v][n]) + X[i][n] conj(G_b[v][n]))
  // + 2 sum_j A_ij q_j A_jv, with row v of A broadcast by lane v (A_jv = conj(A_vj)).
  float2* Wk = p.Wm + (static_cast<size_t>(k) * C + gm) * U * U + static_cast<size_t>(i) * U;
  for (int v = 0; v < U; ++v) {
    __syncwarp();
    if (valid && i == v) {
#pragma unroll
      for (int j = 0; j < UP; ++j) rowbuf[j] = ar[j];
    }
    __syncwarp();
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int n = 0; n < NR; ++n) {
      if (n < NS) {
        const float2 xv = Xs[n * UP + v], gv = Gs[n * UP + v];
        acc = cfma(gb[n], make_float2(xv.x, -xv.y), acc);
        acc = cfma(xr[n], make_float2(gv.x, -gv.y), acc);
      }
    }
    float2 ext = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < UP; ++j) {
      const float2 av = rowbuf[j];                                     // A_vj
      ext = cfma(cscale(ar[j], qv[j]), make_float2(av.x, -av.y), ext);
    }
    if (real) Wk[v] = bad ? make_float2(NAN, NAN) : make_float2(fmaf(2.f, ext.x, acc.x), fmaf(2.f, ext.y, acc.y));
  }
}

// Fused forms for FP32 plans whose subcarrier fits in shared memory: one CTA per
// subcarrier stages H_k and Y_k antenna by antenna, each antenna's row laid out
// like a row of the sweep, W = UP + NR columns (H[0..U)[b], zeros up to UP,
// Y[0..n_sym)[b], zeros up to W) held as a plane of real parts then a plane of
// imaginary parts, and lane i of group c forms row i of [G_c + rho_c I | R]
// itself, in the sweep's column pairs, with two paired FMAs per complex
// product and no column guards:
//   G_c[i][j] = sum_{b in c} conj(H[i][b]) H[j][b],   B_c[i][n] = sum_{b in c} conj(H[i][b]) Y[n][b]
// (Sec. II-C, the contraction of the separate path in antenna order), so the
// local Gram matrices never go through the workspace: the forward pass forms
// them for its sweep, the backward pass forms them again (the factorization is
// recomputed, not stored) and, with H and Y still staged, forms the gradients
// of H and Y in the same CTA from the low-rank form of W:
//   sum_v H[v][b] W[v][u] = sum_n (H X)_n[b] conj(G_b[n][u]) + (H G_b)_n[b] conj(X[n][u]),
//   dL/dH[u][b] = sum_n (Y[n][b] - (H X)_n[b]) conj(G_b[n][u]) - dL/dY[n][b] conj(X[n][u]),
//   dL/dY[n][b] = (H G_b)_n[b] = sum_u H[u][b] G_b[n][u],
// which needs neither W nor G_b in the workspace.
template <int UP, int NR>
struct FusedTrainLayout {
  static constexpr int kW = UP + NR;   // columns of a staged row (a multiple of 4)
  // Bytes: flags, the staged rows (B rows of 2 kW floats), the groups.
  __host__ __device__ static size_t staged(int B) { return static_cast<size_t>(B) * 2 * kW * sizeof(float); }
  __host__ __device__ static size_t bytes(int B, int C) {
    return 16 + staged(B) + static_cast<size_t>(C) * TrainLayout<UP, NR>::kGroup * sizeof(float2);
  }
};

// Stage H_k [U][B] and Y_k [NS][B] into the planar rows (every thread): 4-byte
// asynchronous copies, coalesced on the global side and all in flight at once,
// and zeros in the padding columns; completed (and made visible to the CTA) by
// the caller's stage_wait.
template <int UP, int NR>
__device__ __forceinline__ void stage_rows(const float2* Hk, const float2* Yk, int U, int NS, int B, float* Wf) {
  constexpr int W = UP + NR;
  for (int r = 0; r < U + NS; ++r) {
    const float2* src = r < U ? Hk + static_cast<size_t>(r) * B : Yk + static_cast<size_t>(r - U) * B;
    const int col = r < U ? r : UP + (r - U);
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
      float* dst = Wf + b * 2 * W + col;
      const float* s = reinterpret_cast<const float*>(src + b);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(s) : "memory");
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst + W)), "l"(s + 1) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  const int pad = (UP - U) + (NR - NS);   // zero columns [U, UP) and [UP + NS, W)
  for (int e = threadIdx.x; e < B * pad; e += blockDim.x) {
    const int b = e / pad, q = e - b * pad;
    const int col = q < UP - U ? U + q : UP + NS + (q - (UP - U));
    Wf[b * 2 * W + col] = 0.f;
    Wf[b * 2 * W + W + col] = 0.f;
  }
}

__device__ __forceinline__ void stage_wait() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
}

// Antennas [b0, b1) of cluster c.
__device__ __forceinline__ void cluster_range(const TrainParams& p, int c, int& b0, int& b1) {
  if (p.cl_uniform) {
    const int S = p.B / p.C;
    b0 = c * S;
    b1 = b0 + S;
  } else {
    b0 = p.cl_off[c];
    b1 = p.cl_off[c + 1];
  }
}

// Row i of [G_c + rho I | R] formed from the staged rows in the sweep's column
// pairs (rp[m]: real parts of columns 2m, 2m + 1; ip[m]: imaginary parts):
// columns [0, MC) accumulate conj(H[i][b]) times the staged row of every
// antenna b of the cluster, MC = W with the right-hand sides B_c (WITH_Y), else
// MC = UP and R[i][n] = rhs(n).  Each half of a pair rounds as cfma_conj would.
// Padding rows and groups past the clusters are identity rows with zero
// right-hand sides.
template <int UP, int NR, bool WITH_Y, typename Rhs>
__device__ __forceinline__ void form_row(float2 (&rp)[(UP + NR) / 2], float2 (&ip)[(UP + NR) / 2], const float* Wf,
                                         int U, int NS, int b0, int b1, int i, bool valid, float rho, Rhs rhs) {
  constexpr int W = UP + NR;
  constexpr int MC = WITH_Y ? W : UP;
#pragma unroll
  for (int m = 0; m < W / 2; ++m) rp[m] = ip[m] = make_float2(0.f, 0.f);
  const bool live = valid && i < U;
  if (live) {
    for (int b = b0; b < b1; ++b) {
      const float* wr = Wf + b * 2 * W;   // real parts, then imaginary parts
      const float hr = wr[i], hi = wr[W + i];
      const float2 hr2 = make_float2(hr, hr), hi2 = make_float2(hi, hi), nhi2 = make_float2(-hi, -hi);
#pragma unroll
      for (int c4 = 0; c4 < MC; c4 += 4) {
        const float4 re = *reinterpret_cast<const float4*>(wr + c4);
        const float4 im = *reinterpret_cast<const float4*>(wr + W + c4);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int m = c4 / 2 + h;
          const float2 r2 = h ? make_float2(re.z, re.w) : make_float2(re.x, re.y);
          const float2 i2 = h ? make_float2(im.z, im.w) : make_float2(im.x, im.y);
          rp[m] = __ffma2_rn(hr2, r2, rp[m]);    // Re conj(h) w = h_re w_re + h_im w_im
          rp[m] = __ffma2_rn(hi2, i2, rp[m]);
          ip[m] = __ffma2_rn(hr2, i2, ip[m]);    // Im conj(h) w = h_re w_im - h_im w_re
          ip[m] = __ffma2_rn(nhi2, r2, ip[m]);
        }
      }
    }
  }
  // The diagonal (G_ii real, plus rho); identity rows for padding lanes.
#pragma unroll
  for (int j = 0; j < UP; ++j) {
    float re = j % 2 ? rp[j / 2].y : rp[j / 2].x;
    float im = j % 2 ? ip[j / 2].y : ip[j / 2].x;
    if (!live) {
      re = i == j ? 1.f : 0.f;
      im = 0.f;
    } else if (j == i) {
      re += rho;
      im = 0.f;
    }
    if (j % 2) {
      rp[j / 2].y = re;
      ip[j / 2].y = im;
    } else {
      rp[j / 2].x = re;
      ip[j / 2].x = im;
    }
  }
  if constexpr (!WITH_Y) {
#pragma unroll
    for (int n = 0; n < NR; ++n) {
      const float2 v = (live && n < NS) ? rhs(n) : make_float2(0.f, 0.f);
      const int j = UP + n;
      if (j % 2) {
        rp[j / 2].y = v.x;
        ip[j / 2].y = v.y;
      } else {
        rp[j / 2].x = v.x;
        ip[j / 2].x = v.y;
      }
    }
  }
}

// Fused forward: the local Gram matrices, the sweep, X_c to the workspace and
// z = sum_c nu_c X_c (fixed cluster order).
template <int UP, int NR>
__global__ void __launch_bounds__(512) train_forward_fused_kernel(const TrainParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  using Lay = TrainLayout<UP, NR>;
  constexpr int W = Lay::kW;
  const int U = p.U, NS = p.n_sym, C = p.C, B = p.B;
  const int g = threadIdx.x / UP, i = threadIdx.x % UP;
  const int k = blockIdx.x;
  const int gm = g < C ? g : C - 1;
  const bool valid = g < C;
  int* fail_any = reinterpret_cast<int*>(smem);
  float* Wf = reinterpret_cast<float*>(smem + 16);
  float2* groups = reinterpret_cast<float2*>(smem + 16 + FusedTrainLayout<UP, NR>::staged(B));
  float2* rowbuf = groups + gm * Lay::kGroup;
  float2* F = rowbuf + Lay::kRow;              // [NR][UP]: nu * X of this cluster
  if (threadIdx.x == 0) *fail_any = 0;
  stage_rows<UP, NR>(p.H + static_cast<size_t>(k) * U * B, p.y + static_cast<size_t>(k) * NS * B, U, NS, B, Wf);
  stage_wait();

  int b0, b1;
  cluster_range(p, gm, b0, b1);
  float2 rp[W / 2], ip[W / 2];
  form_row<UP, NR, true>(rp, ip, Wf, U, NS, b0, b1, i, valid, p.rho_c[gm], [](int) { return make_float2(0.f, 0.f); });
  float rs = 1.f;
  const int fail = gj_sweep_pairs<UP, W>(rp, ip, reinterpret_cast<float*>(rowbuf), i, valid, rs);
  if (valid && i == 0 && fail) atomicOr(fail_any, 1);

  const float w = (valid && i < U) ? p.nu[gm * U + i] : 0.f;
  if (valid && i < U) {
    float2* Xk = p.X + (static_cast<size_t>(k) * C + gm) * NS * U;
#pragma unroll
    for (int n = 0; n < NR; ++n) {
      if (n < NS) {
        const float2 x = swept<W>(rp, ip, n, rs);
        Xk[n * U + i] = x;
        F[n * UP + i] = cscale(x, w);
      }
    }
  }
  __syncthreads();
  const bool bad = *fail_any != 0;
  for (int e = threadIdx.x; e < U * NS; e += blockDim.x) {
    const int u = e % U, n = e / U;
    float2 acc = make_float2(0.f, 0.f);
    for (int c = 0; c < C; ++c) acc = cadd(acc, (groups + c * Lay::kGroup + Lay::kRow)[n * UP + u]);
    p.z[(static_cast<size_t>(k) * NS + n) * U + u] = bad ? make_float2(NAN, NAN) : acc;
  }
}

// Fused backward: G_b from the recomputed factorization of [G_c + rho_c I |
// diag(nu_c) G_z], the partial sums of dL/drho_c and dL/dnu[c][.] (X_c from the
// forward pass), then the gradients of H and Y per antenna from the staged rows
// (the low-rank form above; sums over users and symbols in a fixed order).
template <int UP, int NR>
__global__ void __launch_bounds__(512) train_backward_fused_kernel(const TrainParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  using Lay = TrainLayout<UP, NR>;
  constexpr int W = Lay::kW;
  const int U = p.U, NS = p.n_sym, C = p.C, B = p.B;
  const int g = threadIdx.x / UP, i = threadIdx.x % UP;
  const int k = blockIdx.x;
  const int gm = g < C ? g : C - 1;
  const bool valid = g < C;
  float* Wf = reinterpret_cast<float*>(smem + 16);
  float2* groups = reinterpret_cast<float2*>(smem + 16 + FusedTrainLayout<UP, NR>::staged(B));
  float2* rowbuf = groups + gm * Lay::kGroup;
  float2* Gs = rowbuf + Lay::kRow;              // [NR][UP]  G_b of this cluster
  float2* Xs = Gs + NR * UP;                    // [NR][UP]  X of this cluster
  stage_rows<UP, NR>(p.H + static_cast<size_t>(k) * U * B, p.y + static_cast<size_t>(k) * NS * B, U, NS, B, Wf);
  stage_wait();

  int b0, b1;
  cluster_range(p, gm, b0, b1);
  const float2* gz = p.gz + static_cast<size_t>(k) * NS * U;
  const float w = (valid && i < U) ? p.nu[gm * U + i] : 0.f;
  float2 rp[W / 2], ip[W / 2];
  form_row<UP, NR, false>(rp, ip, Wf, U, NS, b0, b1, i, valid, p.rho_c[gm],
                          [&](int n) { return cscale(gz[n * U + i], w); });
  float rs = 1.f;
  gj_sweep_pairs<UP, W>(rp, ip, reinterpret_cast<float*>(rowbuf), i, valid, rs);

  const bool live = valid && i < U;
  const size_t off = (static_cast<size_t>(k) * C + gm) * NS * U;
  float prho = 0.f, pnu = 0.f;
#pragma unroll
  for (int n = 0; n < NR; ++n) {
    if (n < NS) {
      const float2 gb = live ? swept<W>(rp, ip, n, rs) : make_float2(0.f, 0.f);
      const float2 x = live ? p.X[off + n * U + i] : make_float2(0.f, 0.f);
      const float2 gzv = live ? gz[n * U + i] : make_float2(0.f, 0.f);
      prho -= gb.x * x.x + gb.y * x.y;          // Re(conj(G_b) X)
      pnu += gzv.x * x.x + gzv.y * x.y;         // Re(conj(g_z) X)
      if (valid) {
        Gs[n * UP + i] = gb;
        Xs[n * UP + i] = x;
      }
    }
  }
#pragma unroll
  for (int o = UP / 2; o > 0; o >>= 1) prho += __shfl_xor_sync(kFullMask, prho, o, UP);
  float* P = p.P + (static_cast<size_t>(k) * C + gm) * (1 + U);
  if (valid) {
    if (i == 0) P[0] = prho;
    if (i < U) P[1 + i] = pnu;
  }
  __syncthreads();

  // Per antenna b of cluster c: (H X)_n, (H G_b)_n = dL/dY[n][b], then dL/dH[.][b].
  float2* gHk = p.gH + static_cast<size_t>(k) * U * B;
  float2* gyk = p.gy + static_cast<size_t>(k) * NS * B;
  const int S = p.cl_uniform ? B / C : 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    int c = 0;
    if (p.cl_uniform) {
      c = b / S;
    } else {
      while (c + 1 < C && b >= p.cl_off[c + 1]) ++c;
    }
    const float2* Gc = groups + c * Lay::kGroup + Lay::kRow;
    const float2* Xc = Gc + NR * UP;
    const float* wr = Wf + b * 2 * W;
    float2 hx[NR], hg[NR];
#pragma unroll
    for (int n = 0; n < NR; ++n) hx[n] = hg[n] = make_float2(0.f, 0.f);
    for (int v = 0; v < U; ++v) {
      const float2 h = make_float2(wr[v], wr[W + v]);
#pragma unroll
      for (int n = 0; n < NR; ++n) {
        if (n < NS) {
          hx[n] = cfma(h, Xc[n * UP + v], hx[n]);
          hg[n] = cfma(h, Gc[n * UP + v], hg[n]);
        }
      }
    }
#pragma unroll
    for (int n = 0; n < NR; ++n) {
      if (n < NS) {
        hx[n] = csub(make_float2(wr[UP + n], wr[W + UP + n]), hx[n]);   // Y[n][b] - (H X)_n[b]
        gyk[static_cast<size_t>(n) * B + b] = hg[n];
      }
    }
    for (int u = 0; u < U; ++u) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int n = 0; n < NR; ++n) {
        if (n < NS) {
          acc = cfma_conj(Gc[n * UP + u], hx[n], acc);    // conj(G_b[n][u]) (Y - H X)_n
          acc = cfms_bconj(hg[n], Xc[n * UP + u], acc);   // - dL/dY[n][b] conj(X[n][u])
        }
      }
      gHk[static_cast<size_t>(u) * B + b] = acc;
    }
  }
}

// Fused adjoint through the optimal weights (FP32 plans whose subcarrier fits):
// the rows of [M_c | B_c] formed from the staged H and Y as in the fused
// training kernels, the sweep's rows of X_c and A_c, the weights, z, q, G_x and
// G_b of train_optimal_solve_kernel, row i of A_c kept in shared memory, and the
// gradients per antenna from the low-rank part of W_c and its full-rank term:
//   sum_v H[v][b] W_c[v][u] = sum_n (H X)_n conj(G_b[n][u]) + (H G_b)_n conj(X[n][u])
//                             + 2 sum_w (H A)_w q_w A[w][u],  (H A)_w = sum_v H[v][b] A[v][w],
// so neither D nor W_c nor G_b goes through the workspace.
template <int UP, int NR>
struct OptimalFusedLayout {
  static constexpr int kG = OptimalLayout<UP, NR>::kGroup + UP * UP;   // per group, + A [UP][UP]
  __host__ __device__ static size_t wv_bytes(int C) { return ((static_cast<size_t>(C) * UP * 4 + 15) / 16) * 16; }
  __host__ __device__ static size_t bytes(int B, int C) {
    return 16 + wv_bytes(C) + FusedTrainLayout<UP, NR>::staged(B) + static_cast<size_t>(C) * kG * sizeof(float2);
  }
};

template <int UP, int NR>
__global__ void __launch_bounds__(512) train_optimal_fused_kernel(const TrainParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  using Lay = OptimalLayout<UP, NR>;
  using FL = OptimalFusedLayout<UP, NR>;
  constexpr int W = Lay::kW;
  const int U = p.U, NS = p.n_sym, C = p.C, B = p.B;
  const int g = threadIdx.x / UP, i = threadIdx.x % UP;
  const int k = blockIdx.x;
  const int gm = g < C ? g : C - 1;
  const bool valid = g < C;
  int* fail_any = reinterpret_cast<int*>(smem);
  float* wv = reinterpret_cast<float*>(smem + 16);                       // [C][UP]: w_{c,u}
  float* Wf = reinterpret_cast<float*>(smem + 16 + FL::wv_bytes(C));
  float2* grp = reinterpret_cast<float2*>(smem + 16 + FL::wv_bytes(C) + FusedTrainLayout<UP, NR>::staged(B));
  float2* rowbuf = grp + gm * FL::kG;
  float2* Xs = rowbuf + Lay::kRow;            // [NR][UP]
  float2* Gs = Xs + NR * UP;                  // [NR][UP]
  float* qv = reinterpret_cast<float*>(Gs + NR * UP);   // [UP]
  float2* As = rowbuf + Lay::kGroup;          // [UP][UP]: row v of A_c at v UP
  if (threadIdx.x == 0) *fail_any = 0;
  stage_rows<UP, NR>(p.H + static_cast<size_t>(k) * U * B, p.y + static_cast<size_t>(k) * NS * B, U, NS, B, Wf);
  stage_wait();

  int b0, b1;
  cluster_range(p, gm, b0, b1);
  const float rho = p.rho;
  float2 rp[W / 2], ip[W / 2];
  form_row<UP, NR, true>(rp, ip, Wf, U, NS, b0, b1, i, valid, rho, [](int) { return make_float2(0.f, 0.f); });
  float rs = 1.f;
  const int fail = gj_sweep_pairs<UP, W>(rp, ip, reinterpret_cast<float*>(rowbuf), i, valid, rs);
  if (valid && i == 0 && fail) atomicOr(fail_any, 1);
  // Row i of X_c and of A_c.
  float2 xr[NR], ar[UP];
#pragma unroll
  for (int n = 0; n < NR; ++n) xr[n] = swept<W>(rp, ip, n, rs);
#pragma unroll
  for (int j = 0; j < UP; ++j) ar[j] = swept<W>(rp, ip, NR + j, rs);
  float a = 1.f;
#pragma unroll
  for (int j = 0; j < UP; ++j)
    if (j == i) a = ar[j].x;
  const bool real = valid && i < U;
  const float w = real ? 1.f / a : 0.f;
  if (valid) {
    wv[gm * UP + i] = real ? w : rho;         // padding users: w - rho = 0
#pragma unroll
    for (int n = 0; n < NR; ++n) Xs[n * UP + i] = (real && n < NS) ? xr[n] : make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < UP; ++j) As[i * UP + j] = ar[j];
  }
  __syncthreads();
  const bool bad = *fail_any != 0;
  // D_u and z_u over the clusters in a fixed order (every group for its own users).
  float Du = 0.f;
  for (int cc = 0; cc < C; ++cc) Du += wv[cc * UP + i] - rho;
  const bool seen = Du > 0.f;
  const float invD = seen ? 1.f / Du : 0.f;
  const float2* gzk = p.gz + static_cast<size_t>(k) * NS * U;
  float qn = 0.f;                                 // sum_n Re(conj(g_z) (X - z))
#pragma unroll
  for (int n = 0; n < NR; ++n) {
    if (n < NS) {
      float2 num = make_float2(0.f, 0.f);
      for (int cc = 0; cc < C; ++cc) {
        const float2 xc = (grp + cc * FL::kG + Lay::kRow)[n * UP + i];
        const float wc = wv[cc * UP + i];
        num = make_float2(fmaf(wc, xc.x, num.x), fmaf(wc, xc.y, num.y));
      }
      const float2 zn = cscale(num, invD);
      const float2 gzv = real ? gzk[n * U + i] : make_float2(0.f, 0.f);
      qn = fmaf(gzv.x, xr[n].x - zn.x, fmaf(gzv.y, xr[n].y - zn.y, qn));
      if (valid) Gs[n * UP + i] = cscale(gzv, w * invD);   // G_x
    }
  }
  if (valid) qv[i] = (real && seen) ? -qn * invD * w * w : 0.f;   // 1 / a^2 = w^2
  __syncwarp();
  // G_b row i = sum_j A_ij G_x[j].
  float2 gb[NR];
#pragma unroll
  for (int n = 0; n < NR; ++n) {
    float2 acc = make_float2(0.f, 0.f);
    if (n < NS) {
#pragma unroll
      for (int j = 0; j < UP; ++j) acc = cfma(ar[j], Gs[n * UP + j], acc);
    }
    gb[n] = bad ? make_float2(NAN, NAN) : acc;
  }
  __syncwarp();
  if (valid) {
#pragma unroll
    for (int n = 0; n < NR; ++n)
      if (n < NS) Gs[n * UP + i] = real ? gb[n] : make_float2(0.f, 0.f);
  }
  __syncthreads();

  // Per antenna b of cluster c: (H X)_n, (H G_b)_n = dL/dY[n][b], (H A)_w, then dL/dH[.][b].
  float2* gHk = p.gH + static_cast<size_t>(k) * U * B;
  float2* gyk = p.gy + static_cast<size_t>(k) * NS * B;
  const int S = p.cl_uniform ? B / C : 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    int c = 0;
    if (p.cl_uniform) {
      c = b / S;
    } else {
      while (c + 1 < C && b >= p.cl_off[c + 1]) ++c;
    }
    const float2* base = grp + c * FL::kG;
    const float2* Xc = base + Lay::kRow;
    const float2* Gc = Xc + NR * UP;
    const float* qc = reinterpret_cast<const float*>(Gc + NR * UP);
    const float2* Ac = base + Lay::kGroup;
    const float* wr = Wf + b * 2 * W;
    float2 hx[NR], hg[NR], ha[UP];
#pragma unroll
    for (int n = 0; n < NR; ++n) hx[n] = hg[n] = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < UP; ++j) ha[j] = make_float2(0.f, 0.f);
    for (int v = 0; v < U; ++v) {
      const float2 h = make_float2(wr[v], wr[W + v]);
#pragma unroll
      for (int n = 0; n < NR; ++n) {
        if (n < NS) {
          hx[n] = cfma(h, Xc[n * UP + v], hx[n]);
          hg[n] = cfma(h, Gc[n * UP + v], hg[n]);
        }
      }
#pragma unroll
      for (int j = 0; j < UP; ++j) ha[j] = cfma(h, Ac[v * UP + j], ha[j]);
    }
#pragma unroll
    for (int j = 0; j < UP; ++j) ha[j] = cscale(ha[j], 2.f * qc[j]);   // 2 q_w (H A)_w
#pragma unroll
    for (int n = 0; n < NR; ++n) {
      if (n < NS) {
        hx[n] = csub(make_float2(wr[UP + n], wr[W + UP + n]), hx[n]);   // Y[n][b] - (H X)_n[b]
        gyk[static_cast<size_t>(n) * B + b] = hg[n];
      }
    }
    for (int u = 0; u < U; ++u) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int n = 0; n < NR; ++n) {
        if (n < NS) {
          acc = cfma_conj(Gc[n * UP + u], hx[n], acc);    // conj(G_b[n][u]) (Y - H X)_n
          acc = cfms_bconj(hg[n], Xc[n * UP + u], acc);   // - dL/dY[n][b] conj(X[n][u])
        }
      }
#pragma unroll
      for (int j = 0; j < UP; ++j)
        if (j < U) acc = cfms(ha[j], Ac[j * UP + u], acc);   // - 2 sum_w (H A)_w q_w A[w][u]
      gHk[static_cast<size_t>(u) * B + b] = acc;
    }
  }
}

// Backward contraction, per subcarrier (G_b and W of its clusters staged in
// shared memory):
//   dL/dH[u][b] = sum_n Y[n][b] conj(G_b[n][u]) - sum_v H[v][b] W[v][u]
//   dL/dY[n][b] = sum_u H[u][b] G_b[n][u]
// A work item of dL/dH is one antenna b and kUq users (kUq independent
// accumulators, so the dependent chains overlap); its column of H is read from
// HBM coalesced over b (the items of one antenna share it through L1).  Antenna
// b belongs to cluster b / S, or to the cluster whose offsets hold it.
constexpr int kUq = 4;

template <int UP>
__global__ void __launch_bounds__(256) train_backward_contract_kernel(const TrainParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int U = p.U, NS = p.n_sym, C = p.C, B = p.B, S = B / C;
  const int k = blockIdx.x;
  float2* Gs = reinterpret_cast<float2*>(smem);            // [C][NS][U]
  float2* Ws = Gs + static_cast<size_t>(C) * NS * U;       // [C][U][U]
  const float2* Gk = p.Gb + static_cast<size_t>(k) * C * NS * U;
  const float2* Wk = p.Wm + static_cast<size_t>(k) * C * U * U;
  for (int e = threadIdx.x; e < C * NS * U; e += blockDim.x) Gs[e] = Gk[e];
  for (int e = threadIdx.x; e < C * U * U; e += blockDim.x) Ws[e] = Wk[e];
  __syncthreads();
  const float2* Hk = p.H + static_cast<size_t>(k) * U * B;
  const float2* Yk = p.y + static_cast<size_t>(k) * NS * B;
  float2* gHk = p.gH + static_cast<size_t>(k) * U * B;
  float2* gyk = p.gy + static_cast<size_t>(k) * NS * B;
  auto cluster_of = [&](int b) {
    if (p.cl_uniform) return b / S;
    int c = 0;
    while (c + 1 < C && b >= p.cl_off[c + 1]) ++c;
    return c;
  };
  const int nq = (U + kUq - 1) / kUq;
  for (int e = threadIdx.x; e < B * nq; e += blockDim.x) {
    const int b = e % B, u0 = (e / B) * kUq;
    const int c = cluster_of(b);
    const float2* Gc = Gs + static_cast<size_t>(c) * NS * U;
    const float2* Wc = Ws + static_cast<size_t>(c) * U * U;
    float2 acc[kUq];
#pragma unroll
    for (int q = 0; q < kUq; ++q) acc[q] = make_float2(0.f, 0.f);
    for (int n = 0; n < NS; ++n) {
      const float2 yv = Yk[static_cast<size_t>(n) * B + b];
#pragma unroll
      for (int q = 0; q < kUq; ++q)
        if (u0 + q < U) acc[q] = cfma_conj(Gc[n * U + u0 + q], yv, acc[q]);   // Y[n][b] conj(G_b[n][u])
    }
#pragma unroll
    for (int v = 0; v < UP; ++v) {
      if (v < U) {
        const float2 hv = Hk[static_cast<size_t>(v) * B + b];
#pragma unroll
        for (int q = 0; q < kUq; ++q)
          if (u0 + q < U) acc[q] = cfms(hv, Wc[v * U + u0 + q], acc[q]);          // - H[v][b] W[v][u]
      }
    }
#pragma unroll
    for (int q = 0; q < kUq; ++q)
      if (u0 + q < U) gHk[static_cast<size_t>(u0 + q) * B + b] = acc[q];
  }
  for (int e = threadIdx.x; e < B * NS; e += blockDim.x) {
    const int b = e % B, n = e / B;
    const float2* Gc = Gs + static_cast<size_t>(cluster_of(b)) * NS * U;
    float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < UP; u += 2) {
      if (u < U) acc0 = cfma(Hk[static_cast<size_t>(u) * B + b], Gc[n * U + u], acc0);
      if (u + 1 < U) acc1 = cfma(Hk[static_cast<size_t>(u + 1) * B + b], Gc[n * U + u + 1], acc1);
    }
    gyk[static_cast<size_t>(n) * B + b] = cadd(acc0, acc1);
  }
}

// dL/drho_c and dL/dnu[c][u]: fixed-order sums of the per-subcarrier partials
// (block j reduces column j of P [n_sc][C * (1 + U)]).
__global__ void __launch_bounds__(256) train_reduce_kernel(const TrainParams p) {
  __shared__ float red[256];
  const int U = p.U, C = p.C, J = C * (1 + U);
  const int j = blockIdx.x;
  float acc = 0.f;
  for (int k = threadIdx.x; k < p.n_sc; k += blockDim.x) acc += p.P[static_cast<size_t>(k) * J + j];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int c = j / (1 + U), q = j % (1 + U);
    if (q == 0) p.grho[c] = red[0];
    else p.gnu[c * U + q - 1] = red[0];
  }
}

template <typename K>
cudaError_t set_smem(K kernel, size_t smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                    static_cast<int>(smem));
  return cudaSuccess;
}

template <int UP, int NR>
size_t train_smem_up(int C) {
  return 16 + static_cast<size_t>(C) * TrainLayout<UP, NR>::kGroup * sizeof(float2);
}

template <int UP>
cudaError_t launch_contract_up(const TrainParams& p, cudaStream_t st) {
  const size_t smem2 = (static_cast<size_t>(p.C) * p.n_sym * p.U + static_cast<size_t>(p.C) * p.U * p.U) *
                       sizeof(float2);
  const cudaError_t e = set_smem(train_backward_contract_kernel<UP>, smem2);
  if (e != cudaSuccess) return e;
  train_backward_contract_kernel<UP><<<p.n_sc, 256, smem2, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_contract(const TrainParams& p, cudaStream_t st) {
  switch (padded_users(p.U)) {
    case 8: return launch_contract_up<8>(p, st);
    case 16: return launch_contract_up<16>(p, st);
    default: return launch_contract_up<32>(p, st);
  }
}

template <int UP, int NR>
cudaError_t launch_forward_up(const TrainParams& p, cudaStream_t st) {
  const int threads = ((p.C * UP + 31) / 32) * 32;
  const size_t smem = train_smem_up<UP, NR>(p.C);
  cudaError_t e = set_smem(train_forward_kernel<UP, NR>, smem);
  if (e != cudaSuccess) return e;
  train_forward_kernel<UP, NR><<<p.n_sc, threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <int UP, int NR>
cudaError_t launch_backward_up(const TrainParams& p, cudaStream_t st) {
  const int threads = ((p.C * UP + 31) / 32) * 32;
  const size_t smem = train_smem_up<UP, NR>(p.C);
  cudaError_t e = set_smem(train_backward_solve_kernel<UP, NR>, smem);
  if (e != cudaSuccess) return e;
  train_backward_solve_kernel<UP, NR><<<p.n_sc, threads, smem, st>>>(p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_contract(p, st)) != cudaSuccess) return e;
  train_reduce_kernel<<<p.C * (1 + p.U), 256, 0, st>>>(p);
  return cudaGetLastError();
}

template <int UP, int NR>
cudaError_t launch_forward_fused_up(const TrainParams& p, cudaStream_t st) {
  const int threads = ((p.C * UP + 31) / 32) * 32;
  const size_t smem = FusedTrainLayout<UP, NR>::bytes(p.B, p.C);
  cudaError_t e = set_smem(train_forward_fused_kernel<UP, NR>, smem);
  if (e != cudaSuccess) return e;
  train_forward_fused_kernel<UP, NR><<<p.n_sc, threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <int UP, int NR>
cudaError_t launch_backward_fused_up(const TrainParams& p, cudaStream_t st) {
  const int threads = ((p.C * UP + 31) / 32) * 32;
  const size_t smem = FusedTrainLayout<UP, NR>::bytes(p.B, p.C);
  cudaError_t e = set_smem(train_backward_fused_kernel<UP, NR>, smem);
  if (e != cudaSuccess) return e;
  train_backward_fused_kernel<UP, NR><<<p.n_sc, threads, smem, st>>>(p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  train_reduce_kernel<<<p.C * (1 + p.U), 256, 0, st>>>(p);
  return cudaGetLastError();
}

template <int UP, int NR>
cudaError_t launch_optimal_fused_up(const TrainParams& p, cudaStream_t st) {
  const int threads = ((p.C * UP + 31) / 32) * 32;
  const size_t smem = OptimalFusedLayout<UP, NR>::bytes(p.B, p.C);
  cudaError_t e = set_smem(train_optimal_fused_kernel<UP, NR>, smem);
  if (e != cudaSuccess) return e;
  train_optimal_fused_kernel<UP, NR><<<p.n_sc, threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <int UP, int NR>
size_t optimal_smem_up(int C) {
  return 16 + ((static_cast<size_t>(C) * UP * 4 + 15) / 16) * 16 +
         static_cast<size_t>(C) * OptimalLayout<UP, NR>::kGroup * sizeof(float2);
}

template <int UP, int NR>
cudaError_t launch_optimal_up(const TrainParams& p, cudaStream_t st) {
  const int threads = ((p.C * UP + 31) / 32) * 32;
  const size_t smem = optimal_smem_up<UP, NR>(p.C);
  cudaError_t e = set_smem(train_optimal_solve_kernel<UP, NR>, smem);
  if (e != cudaSuccess) return e;
  train_optimal_solve_kernel<UP, NR><<<p.n_sc, threads, smem, st>>>(p);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return launch_contract(p, st);
}

}  // namespace

// Dispatch on (padded users, right-hand-side columns of the sweep).
#define FFEQ_TRAIN_DISPATCH(call)                                             \
  switch (padded_users(p.U) * 100 + rhs_columns(p.n_sym)) {                   \
    case 804: return call<8, 4>(p, st);                                       \
    case 816: return call<8, kNsymMax>(p, st);                                \
    case 1604: return call<16, 4>(p, st);                                     \
    case 1616: return call<16, kNsymMax>(p, st);                              \
    case 3204: return call<32, 4>(p, st);                                     \
    default: return call<32, kNsymMax>(p, st);                                \
  }

size_t train_smem_bytes(int U, int C) {
  // The widest form (n_sym > 4) bounds every problem with these U and C.
  switch (padded_users(U)) {
    case 8: return train_smem_up<8, kNsymMax>(C);
    case 16: return train_smem_up<16, kNsymMax>(C);
    default: return train_smem_up<32, kNsymMax>(C);
  }
}

cudaError_t launch_train_forward(const TrainParams& p, cudaStream_t st) { FFEQ_TRAIN_DISPATCH(launch_forward_up) }

cudaError_t launch_train_backward(const TrainParams& p, cudaStream_t st) { FFEQ_TRAIN_DISPATCH(launch_backward_up) }

bool train_fused_fits(int U, int n_sym, int B, int C) {
  const bool wide = rhs_columns(n_sym) > 4;
  size_t bytes;
  switch (padded_users(U)) {
    case 8: bytes = wide ? FusedTrainLayout<8, kNsymMax>::bytes(B, C) : FusedTrainLayout<8, 4>::bytes(B, C); break;
    case 16: bytes = wide ? FusedTrainLayout<16, kNsymMax>::bytes(B, C) : FusedTrainLayout<16, 4>::bytes(B, C); break;
    default: bytes = wide ? FusedTrainLayout<32, kNsymMax>::bytes(B, C) : FusedTrainLayout<32, 4>::bytes(B, C); break;
  }
  return bytes <= 227 * 1024;
}

cudaError_t launch_train_forward_fused(const TrainParams& p, cudaStream_t st) {
  FFEQ_TRAIN_DISPATCH(launch_forward_fused_up)
}

cudaError_t launch_train_backward_fused(const TrainParams& p, cudaStream_t st) {
  FFEQ_TRAIN_DISPATCH(launch_backward_fused_up)
}

size_t train_optimal_smem_bytes(int U, int C) {
  switch (padded_users(U)) {
    case 8: return optimal_smem_up<8, kNsymMax>(C);
    case 16: return optimal_smem_up<16, kNsymMax>(C);
    default: return optimal_smem_up<32, kNsymMax>(C);
  }
}

cudaError_t launch_train_optimal_backward(const TrainParams& p, cudaStream_t st) {
  FFEQ_TRAIN_DISPATCH(launch_optimal_up)
}

bool train_optimal_fused_fits(int U, int n_sym, int B, int C) {
  const bool wide = rhs_columns(n_sym) > 4;
  size_t bytes;
  switch (padded_users(U)) {
    case 8: bytes = wide ? OptimalFusedLayout<8, kNsymMax>::bytes(B, C) : OptimalFusedLayout<8, 4>::bytes(B, C); break;
    case 16: bytes = wide ? OptimalFusedLayout<16, kNsymMax>::bytes(B, C) : OptimalFusedLayout<16, 4>::bytes(B, C); break;
    default: bytes = wide ? OptimalFusedLayout<32, kNsymMax>::bytes(B, C) : OptimalFusedLayout<32, 4>::bytes(B, C); break;
  }
  return bytes <= 227 * 1024;
}

cudaError_t launch_train_optimal_backward_fused(const TrainParams& p, cudaStream_t st) {
  FFEQ_TRAIN_DISPATCH(launch_optimal_fused_up)
}

#undef FFEQ_TRAIN_DISPATCH

}  // namespace ffeq
