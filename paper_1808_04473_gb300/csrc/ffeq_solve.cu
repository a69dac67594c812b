// Central / local L-MMSE solve, optimal fusion and soft outputs (FP32).
//
// Input: the workspace written by the contraction kernel, one matrix
// D = [G ; (y^MRC)^T] of (U + n_sym) x U complex per (subcarrier, cluster):
// G[u][v] = D[v][u], y^MRC_u(n) = D[U+n][u].  Column i of D is therefore row i of
// the augmented system [G + rho I | y^MRC] (rho = N0/Es, Sec. III-A), up to the
// added rho.  One group of UP lanes (UP = U padded to 8/16/32; lane i = user i)
// keeps its row in registers and runs a Gauss-Jordan sweep: at step k the pivot
// row is scaled by 1/p_k, broadcast through shared memory, and eliminated from
// every other row, while the pivot column is replaced by the inverse.  After U
// steps the left block holds A = (G + rho I)^{-1} and the right block holds
// z = A y^MRC for all n_sym right-hand sides.  The pivots p_k are the Schur
// complements of the Hermitian positive definite matrix, i.e. the squared
// diagonal of its Cholesky factor: a pivot that is not positive marks a failed
// factorization at the same index k.  Every lane does the same (U + n_sym)
// complex updates per step (no triangular idle lanes).
//
// A CTA holds the C clusters of one subcarrier (FD) or several subcarriers (PD)
// and fuses per user with the optimal weights (Eq. fusionrule, Lemma 1):
//     z_u = sum_c (z_{c,u}/A_{c,uu}) / sum_c (g_{c,u}/A_{c,uu}),
//     sigma_u^2 = N0 / sum_c (g_{c,u}/A_{c,uu})             (Thm. 3)
// with g = mu = 1 - rho A_uu (unbiased pairs) or g = 1 (literal pairs); this is
// nu_c = sigma_c^-2 / sum sigma^-2 with sigma_c^2 = N0 A/g, written so that N0
// cancels from the weights (N0 = 0, zero forcing, needs no special case).  PD
// is the case C = 1.  The epilogue writes z, sigma^2 and max-log LLRs.
// The ZF equalizer of Sec. III-A is this sweep with rho = 0 and g = 1; MRC
// needs no inversion and has its own kernel (mrc_fuse_kernel) with the same
// fusion areas and epilogue.
#include <cmath>

#include "ffeq_device.cuh"
#include "ffeq_epilogue.cuh"
#include "ffeq_gj.cuh"
#include "ffeq_internal.h"

namespace ffeq {
namespace {

template <int UP>
struct SolveLayout {
  // Per matrix: pivot-row broadcast buffer (UP + kNsymMax complex), fusion
  // numerators [kNsymMax][UP] complex and denominators [UP] floats; padded so
  // consecutive matrices start 64 bytes apart modulo 128.
  // (two broadcast buffers of 2W + 4 floats for the paired sweep, W = UP + kNsymMax;
  // two areas of 4 UP + 16 floats for the block sweep on the matrix)
  static constexpr int kRowPairs = 2 * (UP + kNsymMax) + 4;
  static constexpr int kRowBlock = 4 * UP + 16;
  static constexpr int kRow = kRowPairs > kRowBlock ? kRowPairs : kRowBlock;
  static constexpr int kNum = kNsymMax * UP;
  static constexpr int kMat = ((kRow + kNum + UP / 2 + 15) / 16) * 16 + 8;   // float2 units
};

// Per-descriptor fields the batch epilogue needs, cached in shared memory.
struct EpiDesc {
  long long z_off, s2_off, llr_off;
  int U, NS, Ceff, out0, slot0;
  float s2s, llr_scale;   // variance scale (N0; Es for MRC, whose denominators are Es / sigma_c^2)
  int pad;
};
constexpr int kEpiCacheBytes = kTileSlots * static_cast<int>(sizeof(EpiDesc));

// Outputs of an uneven-batch tile: the tile's descriptors are read once into
// shared memory (in parallel) with the prefix sums of their outputs and matrix
// slots, then every output (descriptor j, symbol n, user u) is one work item:
// sum descriptor j's Ceff slots (contiguous, in tile order) and write z, sigma^2
// and LLRs at its offsets.  zflag [kTileSlots][UP] (MRC, or nullptr): users of
// descriptor j fused with the N0 -> 0 limit weights, whose variance is 0.
template <int UP>
__device__ void batch_epilogue(const SolveParams& p, const float2* base, const int* fail, int nslot,
                               EpiDesc* cache, int* ndesc, const int* zflag = nullptr) {
  using Lay = SolveLayout<UP>;
  const SolveTile tile = p.tiles[blockIdx.x];
  const int bits = p.llr_bits, hb = bits / 2;
  const int count = tile.first >= 0 && tile.count > 0 ? (tile.count < kTileSlots ? tile.count : kTileSlots) : 0;
  for (int j = threadIdx.x; j < count; j += blockDim.x) {
    EpiDesc e{};
    e.U = -1;   // invalid unless set below
    if (tile.first + j < p.n_desc) {
      const BatchDesc& d = p.desc[tile.first + j];
      e.z_off = d.z_off;
      e.s2_off = d.s2_off;
      e.llr_off = d.llr_off;
      e.U = d.U;
      e.NS = d.n_sym;
      e.Ceff = d.Ceff;
      e.s2s = p.equalizer == FFEQ_MRC ? d.Es : d.N0;
      e.llr_scale = d.llr_scale;
    }
    cache[j] = e;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // Prefix sums; the tile ends at the first descriptor that fails its checks.
    int out = 0, slot0 = 0, n = 0;
    for (; n < count; ++n) {
      EpiDesc& e = cache[n];
      const int U = e.U, NS = e.NS, Ceff = e.Ceff, per = U * NS;
      const bool ok = U >= 1 && U <= UP && NS >= 1 && NS <= kNsymMax && Ceff >= 1 && Ceff <= kTileSlots &&
                      slot0 + Ceff <= kTileSlots && slot0 + Ceff <= nslot && span_ok(e.z_off, per, p.lim.z) &&
                      span_ok(e.s2_off, U, p.lim.s2) &&
                      (!bits || span_ok(e.llr_off, static_cast<long long>(per) * bits, p.lim.llr));
      if (!ok) {
        if (p.status) atomicExch(p.status, FFEQ_ERR_INVALID_ARG);
        break;
      }
      e.out0 = out;
      e.slot0 = slot0;
      out += per;
      slot0 += Ceff;
    }
    ndesc[0] = n;
    ndesc[1] = out;
  }
  __syncthreads();
  const int nd = ndesc[0], total = ndesc[1];
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    int j = 0;
    while (j + 1 < nd && cache[j + 1].out0 <= e) ++j;
    const EpiDesc& d = cache[j];
    const int U = d.U, Ceff = d.Ceff;
    const int r = e - d.out0;
    const int n = r / U, u = r - n * U;
    float2 nm = make_float2(0.f, 0.f);
    float dn = 0.f;
    for (int cc = 0; cc < Ceff; ++cc) {
      const float2* Lm = base + (d.slot0 + cc) * Lay::kMat + Lay::kRow;
      nm = cadd(nm, Lm[n * UP + u]);
      dn += reinterpret_cast<const float*>(Lm + Lay::kNum)[u];
    }
    float2 zz;
    float s2;
    if (fail[j]) {
      zz = make_float2(NAN, NAN);
      s2 = NAN;
    } else if (dn > 0.f) {
      const float rr = rcp_approx(dn);
      zz = cscale(nm, rr);
      s2 = (zflag && zflag[j * UP + u]) ? 0.f : d.s2s * rr;
    } else {
      zz = make_float2(0.f, 0.f);
      s2 = INFINITY;
    }
    p.z[d.z_off + r] = zz;
    if (n == 0) p.sigma2[d.s2_off + u] = s2;
    if (bits) symbol_llr(zz, s2, d.llr_scale, hb, p.llr + d.llr_off + static_cast<long long>(r) * bits);
  }
}

// Outputs of a uniform problem, per subcarrier of this CTA: every (symbol, user)
// sums the Ceff fusion numerators and denominators of its subcarrier and writes
// z = num / den, sigma^2 = s2_scale / den (s2_scale = N0 for the solve, whose
// denominators are g / A_uu; Es for MRC, whose are Es / sigma_c^2) and the LLRs.
// zflag [spc][UP] (MRC, or nullptr): users fused with the N0 -> 0 limit weights,
// whose variance is 0.
template <int UP>
__device__ __forceinline__ void uniform_epilogue(const SolveParams& p, const float2* base, const int* fail_sc,
                                                 int sc0, int U, int NS, int Ceff, float s2_scale,
                                                 const int* zflag = nullptr) {
  using Lay = SolveLayout<UP>;
  const int spc = p.spc;
  const int per = U * NS;   // uniform problem: every group has the problem's sizes
  const int bits = p.llr_bits, hb = bits / 2;
  for (int e = threadIdx.x; e < spc * per; e += blockDim.x) {
    const int s = e / per, r = e - s * per;
    const int n = r / U, u = r - n * U;
    const int k = sc0 + s;
    if (k >= p.n_sc) break;
    float2 nm = make_float2(0.f, 0.f);
    float dn = 0.f;
    for (int cc = 0; cc < Ceff; ++cc) {
      const float2* Lm = base + (s * Ceff + cc) * Lay::kMat + Lay::kRow;
      nm = cadd(nm, Lm[n * UP + u]);
      dn += reinterpret_cast<const float*>(Lm + Lay::kNum)[u];
    }
    float2 zz;
    float s2;
    if (fail_sc[s]) {
      zz = make_float2(NAN, NAN);
      s2 = NAN;
    } else if (dn > 0.f) {
      const float rr = rcp_approx(dn);
      zz = cscale(nm, rr);
      s2 = (zflag && zflag[s * UP + u]) ? 0.f : s2_scale * rr;
    } else {
      zz = make_float2(0.f, 0.f);
      s2 = INFINITY;
    }
    const size_t zi = (static_cast<size_t>(k) * NS + n) * U + u;
    p.z[zi] = zz;
    if (n == 0) p.sigma2[static_cast<size_t>(k) * U + u] = s2;
    if (bits) symbol_llr(zz, s2, p.llr_scale, hb, p.llr + zi * bits);
  }
}

// LPR lanes per row: with LPR = 2 the two lanes of row i hold halves of its
// augmented row (columns [0, W/2) and [W/2, W)), halving the work per lane and
// step; the pivot column k < UP always lies in the first half.
// Uniform problems with one lane per row and up to 16 users: at most 64
// registers, so that 8 CTAs of 128 threads fit one SM (the FD throughput
// workload's 1200 subcarriers then run in one wave).
template <int UP, int LPR, bool BATCH>
constexpr int solve_min_blocks() {
  return (!BATCH && LPR == 1 && UP <= 16) ? 2 : 1;
}

template <int UP, int LPR, bool BATCH>
__global__ void __launch_bounds__(512, (solve_min_blocks<UP, LPR, BATCH>())) solve_fuse_kernel(const SolveParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  using Lay = SolveLayout<UP>;
  constexpr int GS = UP * LPR;                // lanes per matrix
  constexpr int W = UP + kNsymMax;            // augmented row width (RHS columns beyond n_sym unused)
  constexpr int WH = W / LPR;                 // columns per lane
  static_assert(UP <= WH, "pivot columns must lie in the first half of a row");
  const int spc = p.spc;
  constexpr bool batch = BATCH;
  const int nmat = batch ? static_cast<int>(blockDim.x) / GS : spc * p.Ceff;
  const int g = threadIdx.x / GS, gl = threadIdx.x % GS;
  const int i = gl % UP;
  const int h = LPR == 1 ? 0 : gl / UP;        // which half of the row this lane holds
  int* fail_sc = reinterpret_cast<int*>(smem);                       // [spc] or [tile count]
  // Batch mode: descriptor cache for the epilogue after the flags.
  float2* base = reinterpret_cast<float2*>(smem + 256 + (BATCH ? kEpiCacheBytes + 16 : 0));
  const int sc0 = blockIdx.x * spc;

  if (threadIdx.x < 64) fail_sc[threadIdx.x] = 0;
  __syncthreads();

  // Wait for the contraction grid (programmatic dependent launch).
  asm volatile("griddepcontrol.wait;" ::: "memory");

  // ---- the system this lane group solves
  const int gm = g < nmat ? g : nmat - 1;       // spare lanes shadow the last matrix
  int U, NS, Ceff, scl, c, sc = 0;
  float rho;
  bool valid;
  const float2* Dg;
  int* info_at = nullptr;
  if constexpr (!batch) {
    U = p.U; NS = p.n_sym; Ceff = p.Ceff; rho = p.rho;
    scl = gm / Ceff; c = gm % Ceff;
    sc = sc0 + scl;
    valid = g < nmat && sc < p.n_sc;
    const size_t matSize = static_cast<size_t>(U + NS) * U;
    Dg = p.D + (static_cast<size_t>(valid ? sc : 0) * Ceff + c) * matSize;
    if (p.info) info_at = p.info + static_cast<size_t>(sc) * Ceff + c;
  } else {
    // Slot g of this tile: cluster c of its descriptor j (map checked against the tile and the buffers).
    const SolveTile tile = p.tiles[blockIdx.x];
    const unsigned m = g < kTileSlots ? p.slot_map[static_cast<size_t>(blockIdx.x) * kTileSlots + g] : 0xffffu;
    const int j = static_cast<int>(m >> 8);
    c = static_cast<int>(m & 0xffu);
    scl = j;
    const int dj = tile.first + j;
    valid = m != 0xffffu && j < tile.count && j < kTileSlots && tile.first >= 0 && dj < p.n_desc;
    const BatchDesc* d = valid ? p.desc + dj : p.desc;
    U = d->U; NS = d->n_sym; Ceff = d->Ceff; rho = d->rho;
    valid = valid && U >= 1 && U <= UP && NS >= 1 && NS <= kNsymMax && Ceff >= 1 && Ceff <= kTileSlots && c < Ceff;
    const long long matSize = valid ? static_cast<long long>(U + NS) * U : 0;
    valid = valid && span_ok(d->d_off, Ceff * matSize, p.lim.d) &&
            (!p.info || span_ok(d->info_off, Ceff, p.lim.info));
    if (!valid) {
      U = UP; NS = 1; Ceff = 1; c = 0; rho = 1.f;
      if (m != 0xffffu && gl == 0 && p.status) atomicExch(p.status, FFEQ_ERR_INVALID_ARG);
    }
    Dg = p.D + (valid ? d->d_off + c * matSize : 0);
    if (p.info && valid) info_at = p.info + d->info_off + c;
  }
  float2* rowbuf = base + gm * Lay::kMat;
  float2* Fz = rowbuf + Lay::kRow;
  float* Dn = reinterpret_cast<float*>(Fz + Lay::kNum);

  int fail = 0;
  if constexpr (LPR == 1) {
    // ---- row i of G + rho I in registers (padding: identity); the right-hand
    // sides y^MRC go straight to this system's shared block ys[n][u] (the fusion
    // terms overwrite it later).  Loads are unconditional where the address is
    // clamped in bounds, so they all issue before the first use.
    float2* ys = Fz;
    const int ic = i < U ? i : 0;
    float2 mrow[UP];
#pragma unroll
    for (int j = 0; j < UP; ++j) {
      const int row = j < U ? j : 0;
      if constexpr (batch) {
        mrow[j] = valid ? Dg[row * U + ic] : make_float2(0.f, 0.f);
      } else {
        mrow[j] = Dg[row * U + ic];   // invalid groups read subcarrier 0 (in bounds)
      }
    }
    if (g < nmat) {
#pragma unroll
      for (int n = 0; n < kNsymMax; ++n) {
        const bool real = valid && i < U && n < NS;
        float2 v = make_float2(0.f, 0.f);
        if constexpr (batch) {
          if (real) v = Dg[(U + n) * U + ic];
        } else {
          v = Dg[(real ? U + n : 0) * U + ic];
          if (!real) v = make_float2(0.f, 0.f);
        }
        ys[n * UP + i] = v;
      }
    }
    float gii = 1.f;
#pragma unroll
    for (int j = 0; j < UP; ++j) {
      const bool real = valid && i < U && j < U;
      float2 v = real ? mrow[j] : make_float2(j == i ? 1.f : 0.f, 0.f);
      if (j == i && real) {
        gii = v.x;
        v = make_float2(v.x + rho, 0.f);
      }
      mrow[j] = v;
    }
    // ---- Gauss-Jordan sweep on the matrix (paired form, ffeq_gj.cuh): row i of
    // A = (G + rho I)^{-1}, then z = A y^MRC per right-hand side.
    float2 rp[UP / 2], ip[UP / 2];
#pragma unroll
    for (int m = 0; m < UP / 2; ++m) {
      rp[m] = make_float2(mrow[2 * m].x, mrow[2 * m + 1].x);
      ip[m] = make_float2(mrow[2 * m].y, mrow[2 * m + 1].y);
    }
    float rs = 1.f;
    // 32 pivots: fuse pivot pairs (half the broadcast rounds); up to 16: the
    // sequential paired sweep is faster (measured).
    if constexpr (UP >= 32) {
      fail = gj_sweep_block2<UP, UP>(rp, ip, reinterpret_cast<float*>(rowbuf), i, g < nmat, rs);
    } else {
      fail = gj_sweep_pairs<UP, UP>(rp, ip, reinterpret_cast<float*>(rowbuf), i, g < nmat, rs);
    }
    float2 arow[UP];
    float Ai = 1.f;
#pragma unroll
    for (int j = 0; j < UP; ++j) {
      arow[j] = cscale(make_float2(j % 2 ? rp[j / 2].y : rp[j / 2].x, j % 2 ? ip[j / 2].y : ip[j / 2].x), rs);
      if (j == i) Ai = arow[j].x;
    }
    const float invA = rcp_approx(Ai);
    // mu = [A G]_ii = 1 - rho A_ii; a user the cluster cannot see (G_ii = 0) has
    // mu = 0 exactly, which the subtraction would only reach up to rounding.
    const float mu = gii == 0.f ? 0.f : fmaxf(1.f - rho * Ai, 0.f);
    bool store = false;
    size_t sys = 0;
    if constexpr (!batch) {
      store = p.Xs != nullptr;   // refinement follows: keep estimates and inverses
      sys = static_cast<size_t>(sc) * Ceff + c;
    }
    // z_n = sum_j A[i][j] y^MRC_j(n) in j order; after every lane of the warp has
    // read row n of ys, the fusion term z_n / A_ii replaces it ([n][u]: the
    // epilogue reads along u).
#pragma unroll
    for (int n = 0; n < kNsymMax; ++n) {
      float2 zn = make_float2(0.f, 0.f);
      if (n < NS) {
#pragma unroll
        for (int j = 0; j < UP; j += 2) {
          const float4 y2 = *reinterpret_cast<const float4*>(ys + n * UP + j);
          zn = cfma(arow[j], make_float2(y2.x, y2.y), zn);
          zn = cfma(arow[j + 1], make_float2(y2.z, y2.w), zn);
        }
      }
      __syncwarp();
      if (n < NS && g < nmat) {
        if (store) {
          if (valid && i < U) p.Xs[(sys * NS + n) * U + i] = zn;
        } else {
          ys[n * UP + i] = cscale(zn, invA);
        }
      }
    }
    if (store) {
      // Inverse stored transposed (row j = column j of A, coalesced over the lanes i).
      if (g < nmat && valid && i < U) {
#pragma unroll
        for (int j = 0; j < UP; ++j)
          if (j < U) p.As[(sys * U + j) * U + i] = arow[j];
        if (gl == 0) {
          p.fails[sys] = fail;
          if (info_at) *info_at = fail;
        }
      }
      return;   // the refinement kernel fuses and writes the outputs
    }
    if (g < nmat) {
      Dn[i] = (p.unbiased ? mu : 1.f) * invA;
      if (gl == 0 && valid) {
        if (info_at) *info_at = fail;
        if (fail) atomicOr(&fail_sc[scl], 1);
      }
    }
  } else {
    // ---- this lane's columns of row i of [G + rho I | y^MRC] (padding: identity, zero RHS)
    // Loads are unconditional (clamped to valid addresses) so they all issue before
    // the first use; padding values are selected afterwards.
    float2 aug[WH];
    const int ic = i < U ? i : 0;
  #pragma unroll
    for (int j = 0; j < WH; ++j) {
      const int col = h * WH + j;
      const int row = col < UP ? (col < U ? col : 0) : (col - UP < NS ? U + col - UP : 0);
      if constexpr (batch) {
        aug[j] = valid ? Dg[row * U + ic] : make_float2(0.f, 0.f);
      } else {
        aug[j] = Dg[row * U + ic];   // invalid groups read subcarrier 0 (in bounds)
      }
    }
    float gii = 1.f;
  #pragma unroll
    for (int j = 0; j < WH; ++j) {
      const int col = h * WH + j;
      const bool real = valid && i < U && (col < UP ? col < U : col - UP < NS);
      float2 v = real ? aug[j] : make_float2(col == i ? 1.f : 0.f, 0.f);
      if (col == i && real) {
        gii = v.x;
        v = make_float2(v.x + rho, 0.f);
      }
      aug[j] = v;
    }

      // ---- Gauss-Jordan sweep (deferred row scaling: every lane runs the same update)
      // Two lanes per row, columns in place: the same element update as the paired
      // form (gj_update), so both layouts give identical bits.
      float my_r = 1.f;
      static_for<UP>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        const float piv = __shfl_sync(kFullMask, aug[k].x, k, GS);
        const float2 f = make_float2(__shfl_sync(kFullMask, aug[k].x, i, GS), __shfl_sync(kFullMask, aug[k].y, i, GS));
        const bool ok = piv > 0.f;
        if (!ok && fail == 0) fail = k + 1;
        const float r = rcp_approx(ok ? piv : 1.f);
        const bool me = i == k;
        if (me) my_r = r;
        const float2 gg = me ? make_float2(0.f, 0.f) : make_float2(f.x * r, f.y * r);
        if (me && g < nmat) {
  #pragma unroll
          for (int j = 0; j < WH; j += 2)
            if (h * WH + j < UP + NS)
              *reinterpret_cast<float4*>(rowbuf + h * WH + j) =
                  make_float4((h == 0 && j == k) ? 1.f : aug[j].x, (h == 0 && j == k) ? 0.f : aug[j].y,
                              (h == 0 && j + 1 == k) ? 1.f : aug[j + 1].x, (h == 0 && j + 1 == k) ? 0.f : aug[j + 1].y);
        }
        __syncwarp();
        const float dlt = me ? 1.f : 0.f;
        const float2* rb = rowbuf + h * WH;
  #pragma unroll
        for (int j = 0; j < WH; j += 2) {
          if (h * WH + j < UP + NS) {
            const float4 q = *reinterpret_cast<const float4*>(rb + j);
            const float2 b0 = (h == 0 && j == k) ? make_float2(dlt, 0.f) : aug[j];
            const float2 b1 = (h == 0 && j + 1 == k) ? make_float2(dlt, 0.f) : aug[j + 1];
            aug[j] = gj_update(gg, make_float2(q.x, q.y), b0);
            aug[j + 1] = gj_update(gg, make_float2(q.z, q.w), b1);
          }
        }
        __syncwarp();
      });
      // Deferred scaling: row i times 1/p_i (both halves of row i recorded it at step i).
  #pragma unroll
      for (int j = 0; j < WH; ++j) aug[j] = cscale(aug[j], my_r);

    if constexpr (!batch) {
      if (p.Xs) {
        // Refinement follows: keep this system's estimates X [n][u] and its inverse
        // stored transposed (row j = column j of A, coalesced over the lanes i).
        if (g < nmat && valid && i < U) {
          const size_t sys = static_cast<size_t>(sc) * Ceff + c;
  #pragma unroll
          for (int j = 0; j < WH; ++j) {
            if constexpr (LPR == 1) {
              if (j >= kNsymMax && j - kNsymMax < U) p.As[(sys * U + (j - kNsymMax)) * U + i] = aug[j];
              if (j < NS) p.Xs[(sys * NS + j) * U + i] = aug[j];
            } else {
              const int col = h * WH + j;
              if (col < U) p.As[(sys * U + col) * U + i] = aug[j];
              if (col >= UP && col - UP < NS) p.Xs[(sys * NS + (col - UP)) * U + i] = aug[j];
            }
          }
          if (gl == 0) {
            p.fails[sys] = fail;
            if (info_at) *info_at = fail;
          }
        }
        return;   // the refinement kernel fuses and writes the outputs
      }
    }

    // ---- fusion terms of this matrix: A_ii on the first-half lane of row i
    // (column i before rotation; column kNsymMax + i after the rotating sweep)
    constexpr int kA = LPR == 1 ? kNsymMax : 0;   // first column of A in this lane's registers
    constexpr int kZ = LPR == 1 ? 0 : UP;         // first RHS column (global column index)
    float Ai = 1.f;
  #pragma unroll
    for (int j = 0; j < UP; ++j)
      if (j == i) Ai = aug[kA + j].x;
    Ai = __shfl_sync(kFullMask, Ai, i, GS);
    const float invA = rcp_approx(Ai);
    // mu = [A G]_ii = 1 - rho A_ii; a user the cluster cannot see (G_ii = 0) has
    // mu = 0 exactly, which the subtraction would only reach up to rounding.
    const float mu = gii == 0.f ? 0.f : fmaxf(1.f - rho * Ai, 0.f);
    if (g < nmat) {
  #pragma unroll
      for (int j = 0; j < WH; ++j) {
        const int n = h * WH + j - kZ;
        if (n >= 0 && n < NS && (LPR != 1 || j < kNsymMax))
          Fz[n * UP + i] = cscale(aug[j], invA);   // [n][u]: the epilogue reads along u
      }
      if (h == 0) Dn[i] = (p.unbiased ? mu : 1.f) * invA;
      if (gl == 0 && valid) {
        if (info_at) *info_at = fail;
        if (fail) atomicOr(&fail_sc[scl], 1);
      }
    }
  }
  __syncthreads();
  if constexpr (batch) {
    batch_epilogue<UP>(p, base, fail_sc, nmat, reinterpret_cast<EpiDesc*>(smem + 256),
                       reinterpret_cast<int*>(smem + 256 + kEpiCacheBytes));
    return;
  }

  uniform_epilogue<UP>(p, base, fail_sc, sc0, U, NS, Ceff, p.N0);
}

template <int UP, int LPR, bool BATCH>
cudaError_t launch_up(const SolveParams& p, cudaStream_t stream) {
  using Lay = SolveLayout<UP>;
  constexpr bool batch = BATCH;
  const int nmat = batch ? p.threads / (UP * LPR) : p.spc * p.Ceff;
  const int threads = batch ? p.threads : ((nmat * UP * LPR + 31) / 32) * 32;
  const size_t smem = 256 + (batch ? kEpiCacheBytes + 16 : 0) + static_cast<size_t>(nmat) * Lay::kMat * sizeof(float2);
  static int configured[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 64 && !configured[dev]) {
    err = cudaFuncSetAttribute(solve_fuse_kernel<UP, LPR, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    configured[dev] = 1;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(batch ? p.n_tiles : (p.n_sc + p.spc - 1) / p.spc);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, solve_fuse_kernel<UP, LPR, BATCH>, p);
}

// Solve / fusion / soft outputs for uniform problems whose users fill the lane
// group (U == UP: 8, 16 or 32), one lane per row.  The same computation as
// solve_fuse_kernel's one-lane path, specialized so that the sizes that shape
// the work are compile-time constants: every lane loads its row with fixed
// offsets from one column pointer (no padding rows, no clamped or selected
// addresses), the right-hand sides reach shared memory by asynchronous copies
// that overlap the sweep, and the epilogue walks (symbol, user) outputs with
// shifts and masks instead of runtime divisions.  Registers are not capped for
// occupancy: 96 per thread without spills, five 128-thread CTAs per SM (the FD
// throughput workload's 1200 CTAs in 1.6 waves) ran faster than a cap of 64
// with spills and one wave (FD 24.7 -> 23.1 us alone, and the concurrent
// PD + FD step 75.2 -> 70.7 us).
template <int UP>
__global__ void __launch_bounds__(512, 1) solve_full_kernel(const SolveParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  using Lay = SolveLayout<UP>;
  constexpr int U = UP;
  const int NS = p.n_sym, Ceff = p.Ceff, spc = p.spc;
  const int nmat = spc * Ceff;
  const int g = threadIdx.x / UP, i = threadIdx.x % UP;
  int* fail_sc = reinterpret_cast<int*>(smem);                     // [spc]
  float2* base = reinterpret_cast<float2*>(smem + 256);
  const int sc0 = blockIdx.x * spc;
  if (threadIdx.x < 64) fail_sc[threadIdx.x] = 0;
  __syncthreads();
  // Wait for the contraction grid (programmatic dependent launch).
  asm volatile("griddepcontrol.wait;" ::: "memory");

  const int gm = g < nmat ? g : nmat - 1;       // spare lanes shadow the last matrix
  const int scl = gm / Ceff, c = gm - scl * Ceff;
  const int sc = sc0 + scl;
  const bool live = g < nmat && sc < p.n_sc;
  const float rho = p.rho;
  const size_t mat = static_cast<size_t>(U + NS) * U;
  // Column i of this system's D: D[v][i] = G[i][v] (v < U), D[U + n][i] = y^MRC_i(n).
  const float2* Dg = p.D + (static_cast<size_t>(live ? sc : 0) * Ceff + c) * mat + i;
  float2* rowbuf = base + gm * Lay::kMat;
  float2* Fz = rowbuf + Lay::kRow;
  float* Dn = reinterpret_cast<float*>(Fz + Lay::kNum);

  // The right-hand sides [n][u] are one contiguous block of D with the layout
  // of the fusion area: copied global -> shared by the group's lanes in 16-byte
  // pieces (cp.async, no registers), completed before the product.
  if (g < nmat) {
    const char* src = reinterpret_cast<const char*>(Dg - i + U * U);
    const uint32_t dst = smem_u32(Fz);
    const int pieces = NS * U / 2;
    for (int e = i; e < pieces; e += UP)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16 * e), "l"(src + 16 * e) : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  float2 mrow[UP];
#pragma unroll
  for (int j = 0; j < UP; ++j) mrow[j] = Dg[j * U];
  // Lane i: row i of A = (G + rho I)^{-1} (natural column order) and A_ii.
  float2 arow[UP];
  float Ai, gii;
  const int fail = gj_solve_row<UP>(mrow, rho, reinterpret_cast<float*>(rowbuf), i, g < nmat, arow, Ai, gii);
  const float invA = rcp_approx(Ai);
  // mu = [A G]_ii = 1 - rho A_ii; a user the cluster cannot see (G_ii = 0) has
  // mu = 0 exactly, which the subtraction would only reach up to rounding.
  const float mu = gii == 0.f ? 0.f : fmaxf(1.f - rho * Ai, 0.f);
  const bool store = p.Xs != nullptr;   // refinement follows: keep estimates and inverses
  const size_t sys = static_cast<size_t>(sc) * Ceff + c;
  float2 are[UP], aim[UP];
  gj_row_split<UP>(arow, are, aim);
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();
  // z_n = sum_j A[i][j] y^MRC_j(n) in j order, two right-hand sides per round
  // (four independent paired-FMA chains per lane); after every lane of the warp
  // has read rows n and n + 1, the fusion terms z_n / A_ii replace them ([n][u]).
#pragma unroll
  for (int n = 0; n < kNsymMax; n += 2) {
    if (n < NS) {
      const float2 z0 = gj_row_dot_pairs<UP>(are, aim, Fz + n * UP);
      const float2 z1 = n + 1 < NS ? gj_row_dot_pairs<UP>(are, aim, Fz + (n + 1) * UP) : make_float2(0.f, 0.f);
      __syncwarp();
      if (g < nmat) {
        if (store) {
          if (live) {
            p.Xs[(sys * NS + n) * U + i] = z0;
            if (n + 1 < NS) p.Xs[(sys * NS + n + 1) * U + i] = z1;
          }
        } else {
          Fz[n * UP + i] = cscale(z0, invA);
          if (n + 1 < NS) Fz[(n + 1) * UP + i] = cscale(z1, invA);
        }
      }
    }
  }
  if (store) {
    // Inverse stored transposed (row j = column j of A, coalesced over the lanes i).
    if (live) {
#pragma unroll
      for (int j = 0; j < UP; ++j) p.As[(sys * U + j) * U + i] = make_float2(are[j].x, aim[j].x);
      if (i == 0) {
        p.fails[sys] = fail;
        if (p.info) p.info[sys] = fail;
      }
    }
    return;   // the refinement kernel fuses and writes the outputs
  }
  if (g < nmat) {
    Dn[i] = (p.unbiased ? mu : 1.f) * invA;
    if (i == 0 && live) {
      if (p.info) p.info[sys] = fail;
      if (fail) atomicOr(&fail_sc[scl], 1);
    }
  }
  __syncthreads();
  // ---- outputs: per subcarrier of this CTA, (symbol n, user u) = (e / UP, e % UP).
  const int per = UP * NS;
  const int bits = p.llr_bits, hb = bits / 2;
  for (int s = 0; s < spc; ++s) {
    const int k = sc0 + s;
    if (k >= p.n_sc) break;
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int n = e / UP, u = e % UP;
      float2 nm = make_float2(0.f, 0.f);
      float dn = 0.f;
      for (int cc = 0; cc < Ceff; ++cc) {
        const float2* Lm = base + (s * Ceff + cc) * Lay::kMat + Lay::kRow;
        nm = cadd(nm, Lm[n * UP + u]);
        dn += reinterpret_cast<const float*>(Lm + Lay::kNum)[u];
      }
      float2 zz;
      float s2;
      if (fail_sc[s]) {
        zz = make_float2(NAN, NAN);
        s2 = NAN;
      } else if (dn > 0.f) {
        const float rr = rcp_approx(dn);
        zz = cscale(nm, rr);
        s2 = p.N0 * rr;
      } else {
        zz = make_float2(0.f, 0.f);
        s2 = INFINITY;
      }
      const size_t zi = (static_cast<size_t>(k) * NS + n) * U + u;
      p.z[zi] = zz;
      if (n == 0) p.sigma2[static_cast<size_t>(k) * U + u] = s2;
      if (bits) symbol_llr(zz, s2, p.llr_scale, hb, p.llr + zi * bits);
    }
  }
}

template <int UP>
cudaError_t launch_full(const SolveParams& p, cudaStream_t stream) {
  using Lay = SolveLayout<UP>;
  const int nmat = p.spc * p.Ceff;
  const int threads = ((nmat * UP + 31) / 32) * 32;
  const size_t smem = 256 + static_cast<size_t>(nmat) * Lay::kMat * sizeof(float2);
  static int configured[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 64 && !configured[dev]) {
    err = cudaFuncSetAttribute(solve_full_kernel<UP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    configured[dev] = 1;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((p.n_sc + p.spc - 1) / p.spc);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, solve_full_kernel<UP>, p);
}

// Maximum-ratio combining (Sec. III-A) per (subcarrier, cluster), uniform
// problems: lane i of a group of UP lanes reads row i of G_c and forms
//   sigma_c^2 / Es = (rho G_ii + I_i) / G_ii^2,   I_i = sum_{j != i} |G_ij|^2,
// then leaves the fusion denominator w = Es / sigma_c^2 and the numerators
// w y^MRC_i(n) / G_ii in the areas the epilogue sums, so that z = sum_c (w z_c) /
// sum_c w (Eq. fusionrule, opt_fusion) and sigma^2 = Es / sum_c w (Thm. 3); PD
// (one cluster) is z = y^MRC_i / G_ii.  A user the cluster cannot see (G_ii = 0)
// gets w = 0.  With N0 = 0 a variance is exactly 0 where the user has no
// interference (I_i = 0: a single user, or channels of disjoint support); the
// weights are then those of the limit N0 -> 0, where such a cluster's
// Es / sigma_c^2 ~ G_ii Es / N0 outgrows every other: per user, the
// zero-interference clusters share the weight in proportion to G_ii, the others
// get 0, and the fused variance is 0.  No system is solved: info is 0.
template <int UP>
__global__ void __launch_bounds__(512) mrc_fuse_kernel(const SolveParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  using Lay = SolveLayout<UP>;
  int* fail_sc = reinterpret_cast<int*>(smem);
  float2* base = reinterpret_cast<float2*>(smem + 256);
  const int U = p.U, NS = p.n_sym, Ceff = p.Ceff;
  const int nmat = p.spc * Ceff;
  int* zflag = reinterpret_cast<int*>(base + nmat * Lay::kMat);   // [spc][UP]: some cluster has variance 0
  const int g = threadIdx.x / UP, i = threadIdx.x % UP;
  const int sc0 = blockIdx.x * p.spc;
  const bool noiseless = p.N0 == 0.f;
  if (threadIdx.x < 64) fail_sc[threadIdx.x] = 0;
  for (int t = threadIdx.x; t < p.spc * UP; t += blockDim.x) zflag[t] = 0;

  // Wait for the contraction grid (programmatic dependent launch).
  asm volatile("griddepcontrol.wait;" ::: "memory");

  const int c = g % Ceff, s = g / Ceff, sc = sc0 + s;
  const bool live = g < nmat && sc < p.n_sc && i < U;
  const float2* Dg = p.D + (static_cast<size_t>(live ? sc : 0) * Ceff + c) * static_cast<size_t>(U + NS) * U;
  float gii = 0.f, intf = 0.f;
  if (live) {
#pragma unroll
    for (int j = 0; j < UP; ++j) {
      if (j < U) {
        const float2 v = Dg[j * U + i];   // G_ij (conjugate symmetric)
        if (j == i) {
          gii = v.x;
        } else {
          intf = fmaf(v.x, v.x, fmaf(v.y, v.y, intf));
        }
      }
    }
    if (noiseless && gii > 0.f && intf == 0.f) atomicOr(&zflag[s * UP + i], 1);
  }
  __syncthreads();
  if (g < nmat) {
    float2* Fz = base + g * Lay::kMat + Lay::kRow;
    float* Dn = reinterpret_cast<float*>(Fz + Lay::kNum);
    float w = 0.f;
    if (live) {
      float zs = 0.f;
      if (gii > 0.f) {
        if (noiseless && zflag[s * UP + i]) {
          w = intf == 0.f ? gii : 0.f;          // the N0 -> 0 limit weights
        } else {
          const float den = fmaf(p.rho, gii, intf);
          w = den > 0.f ? gii * gii / den : 0.f;
        }
        zs = w / gii;
      }
      for (int n = 0; n < NS; ++n) Fz[n * UP + i] = cscale(Dg[(U + n) * U + i], zs);
      if (i == 0 && p.info) p.info[static_cast<size_t>(sc) * Ceff + c] = 0;
    }
    Dn[i] = w;
  }
  __syncthreads();
  uniform_epilogue<UP>(p, base, fail_sc, sc0, U, NS, Ceff, p.Es, zflag);
}

template <int UP>
cudaError_t launch_mrc_up(const SolveParams& p, cudaStream_t stream) {
  using Lay = SolveLayout<UP>;
  const int nmat = p.spc * p.Ceff;
  const int threads = ((nmat * UP + 31) / 32) * 32;
  const size_t smem = 256 + static_cast<size_t>(nmat) * Lay::kMat * sizeof(float2) +
                      static_cast<size_t>(p.spc) * UP * sizeof(int);
  static int configured[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 64 && !configured[dev]) {
    err = cudaFuncSetAttribute(mrc_fuse_kernel<UP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    configured[dev] = 1;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((p.n_sc + p.spc - 1) / p.spc);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, mrc_fuse_kernel<UP>, p);
}

// Maximum-ratio combining (Sec. III-A) for the tiles of an uneven batch: one
// group of UP lanes per local system, the descriptor and cluster of each slot
// decoded and checked as in solve_fuse_kernel's batch mode, the per-lane
// arithmetic of mrc_fuse_kernel (weight w = Es / sigma_c^2, numerators
// w y^MRC_i(n) / G_ii, the N0 -> 0 limit weights per descriptor with N0 = 0),
// and the batch epilogue with sigma^2 = Es / sum w (0 for the limit-weight users).
template <int UP>
__global__ void __launch_bounds__(512) mrc_batch_kernel(const SolveParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  using Lay = SolveLayout<UP>;
  int* fail_sc = reinterpret_cast<int*>(smem);                        // [tile count]: MRC never fails
  float2* base = reinterpret_cast<float2*>(smem + 256 + kEpiCacheBytes + 16);
  const int nmat = static_cast<int>(blockDim.x) / UP;
  int* zflag = reinterpret_cast<int*>(base + nmat * Lay::kMat);       // [kTileSlots][UP]
  const int g = threadIdx.x / UP, i = threadIdx.x % UP;
  if (threadIdx.x < 64) fail_sc[threadIdx.x] = 0;
  for (int t = threadIdx.x; t < kTileSlots * UP; t += blockDim.x) zflag[t] = 0;
  __syncthreads();
  // Wait for the contraction grid (programmatic dependent launch).
  asm volatile("griddepcontrol.wait;" ::: "memory");

  const SolveTile tile = p.tiles[blockIdx.x];
  const unsigned m = g < kTileSlots ? p.slot_map[static_cast<size_t>(blockIdx.x) * kTileSlots + g] : 0xffffu;
  const int j = static_cast<int>(m >> 8);
  const int c = static_cast<int>(m & 0xffu);
  const int dj = tile.first + j;
  bool valid = m != 0xffffu && j < tile.count && j < kTileSlots && tile.first >= 0 && dj < p.n_desc;
  const BatchDesc* d = valid ? p.desc + dj : p.desc;
  const int U = d->U, NS = d->n_sym, Ceff = d->Ceff;
  valid = valid && U >= 1 && U <= UP && NS >= 1 && NS <= kNsymMax && Ceff >= 1 && Ceff <= kTileSlots && c < Ceff;
  const long long matSize = valid ? static_cast<long long>(U + NS) * U : 0;
  valid = valid && span_ok(d->d_off, Ceff * matSize, p.lim.d) &&
          (!p.info || span_ok(d->info_off, Ceff, p.lim.info));
  if (!valid && m != 0xffffu && i == 0 && p.status) atomicExch(p.status, FFEQ_ERR_INVALID_ARG);
  const float2* Dg = p.D + (valid ? d->d_off + c * matSize : 0);
  const bool live = valid && i < U;
  const bool noiseless = valid && d->N0 == 0.f;
  const float rho = valid ? d->rho : 0.f;
  float gii = 0.f, intf = 0.f;
  if (live) {
    for (int jj = 0; jj < U; ++jj) {
      const float2 v = Dg[jj * U + i];   // G_i,jj (conjugate symmetric)
      if (jj == i) {
        gii = v.x;
      } else {
        intf = fmaf(v.x, v.x, fmaf(v.y, v.y, intf));
      }
    }
    if (noiseless && gii > 0.f && intf == 0.f) atomicOr(&zflag[j * UP + i], 1);
  }
  __syncthreads();
  if (g < nmat) {
    float2* Fz = base + g * Lay::kMat + Lay::kRow;
    float* Dn = reinterpret_cast<float*>(Fz + Lay::kNum);
    float w = 0.f;
    if (live) {
      float zs = 0.f;
      if (gii > 0.f) {
        if (noiseless && zflag[j * UP + i]) {
          w = intf == 0.f ? gii : 0.f;          // the N0 -> 0 limit weights
        } else {
          const float den = fmaf(rho, gii, intf);
          w = den > 0.f ? gii * gii / den : 0.f;
        }
        zs = w / gii;
      }
      for (int n = 0; n < NS; ++n) Fz[n * UP + i] = cscale(Dg[(U + n) * U + i], zs);
      if (i == 0 && p.info) p.info[d->info_off + c] = 0;
    }
    Dn[i] = w;
  }
  __syncthreads();
  batch_epilogue<UP>(p, base, fail_sc, nmat, reinterpret_cast<EpiDesc*>(smem + 256),
                     reinterpret_cast<int*>(smem + 256 + kEpiCacheBytes), zflag);
}

template <int UP>
cudaError_t launch_mrc_batch(const SolveParams& p, cudaStream_t stream) {
  const size_t smem = solve_batch_smem_bytes(UP, 1, p.threads, FFEQ_MRC);
  static int configured[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 64 && !configured[dev]) {
    err = cudaFuncSetAttribute(mrc_batch_kernel<UP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    configured[dev] = 1;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.n_tiles);
  cfg.blockDim = dim3(p.threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, mrc_batch_kernel<UP>, p);
}

}  // namespace

// PD (one system per subcarrier) with 8 < U < 16: a full warp per system (two
// lanes per row) and 4 subcarriers per CTA, for more warps in flight; PD with
// U = 8, 16 or 32 (solve_full_kernel): 2 subcarriers per CTA, one lane per row
// (measured faster than two lanes per row: half the instructions per system);
// FD: the C systems of one subcarrier in one CTA, UP lanes each.
static int lanes_per_row(int U, int Ceff) { return (Ceff == 1 && padded_users(U) == 16 && U != 16) ? 2 : 1; }

int solve_subcarriers_per_cta(int U, int Ceff) {
  if (Ceff != 1) return 1;
  if (padded_users(U) == U) return 2;
  return 128 / (padded_users(U) * lanes_per_row(U, Ceff));
}

size_t solve_smem_bytes(int U, int Ceff) {
  const int spc = solve_subcarriers_per_cta(U, Ceff);
  const int nmat = spc * Ceff;
  size_t per = 0;
  switch (padded_users(U)) {
    case 8: per = SolveLayout<8>::kMat; break;
    case 16: per = SolveLayout<16>::kMat; break;
    default: per = SolveLayout<32>::kMat; break;
  }
  return 256 + static_cast<size_t>(nmat) * per * sizeof(float2);
}

cudaError_t launch_solve(const SolveParams& p, cudaStream_t stream) {
  if (p.equalizer == FFEQ_MRC) {
    switch (padded_users(p.U)) {
      case 8: return launch_mrc_up<8>(p, stream);
      case 16: return launch_mrc_up<16>(p, stream);
      default: return launch_mrc_up<32>(p, stream);
    }
  }
  const int UP = padded_users(p.U);
  if (p.U == UP && lanes_per_row(p.U, p.Ceff) == 1) {   // users fill the lane group
    switch (UP) {
      case 8: return launch_full<8>(p, stream);
      case 16: return launch_full<16>(p, stream);
      default: return launch_full<32>(p, stream);
    }
  }
  switch (UP) {
    case 8: return launch_up<8, 1, false>(p, stream);
    case 16: return lanes_per_row(p.U, p.Ceff) == 2 ? launch_up<16, 2, false>(p, stream)
                                                    : launch_up<16, 1, false>(p, stream);
    default: return launch_up<32, 1, false>(p, stream);
  }
}

cudaError_t launch_solve_batch(const SolveParams& p, int lpr, cudaStream_t stream) {
  if (p.equalizer == FFEQ_MRC) {
    if (lpr != 1) return cudaErrorInvalidValue;
    switch (p.U) {
      case 8: return launch_mrc_batch<8>(p, stream);
      case 16: return launch_mrc_batch<16>(p, stream);
      default: return launch_mrc_batch<32>(p, stream);
    }
  }
  switch (p.U) {
    case 8: return lpr == 2 ? launch_up<8, 2, true>(p, stream) : launch_up<8, 1, true>(p, stream);
    case 16: return lpr == 2 ? launch_up<16, 2, true>(p, stream) : launch_up<16, 1, true>(p, stream);
    default: return launch_up<32, 1, true>(p, stream);
  }
}

size_t solve_batch_smem_bytes(int UP, int lpr, int threads, int equalizer) {
  const int nmat = threads / (UP * lpr);
  size_t per = UP == 8 ? SolveLayout<8>::kMat : (UP == 16 ? SolveLayout<16>::kMat : SolveLayout<32>::kMat);
  const size_t zflags = equalizer == FFEQ_MRC ? static_cast<size_t>(kTileSlots) * UP * sizeof(int) : 0;
  return 256 + kEpiCacheBytes + 16 + static_cast<size_t>(nmat) * per * sizeof(float2) + zflags;
}

}  // namespace ffeq
