// Streamed local preprocessing (Sec. II-C) on the tensor cores: the contraction
// D_{k,c}[m][u] = sum_{b in cluster c} conj(H_k[u][b]) W_k[m][b], W_k = [H_k ; Y_k]
// of ffeq_gram.cuh, reorganised so that no warp ever waits for another one's
// partial sums.
//
// Work split.  A CTA holds several subcarriers at once (8 for U <= 16, 4 for
// U = 32).  Each subcarrier is owned by a team of 2 (or 4) MMA warps; each MMA
// warp owns a fixed set of output tiles (one 16-user m-tile times two or three
// 8-row n-tiles of W) and accumulates them in registers over the whole antenna
// range of a cluster (PD: all B antennas, the adder tree of Eq. fullMRC in the
// accumulators; FD: S = B/C antennas, then the cluster's tile is stored and the
// accumulators restart).  No split-K, no shared-memory reduction, no CTA-wide
// barrier after the prologue.  Besides the 16 MMA warps the CTA has converter
// warps (8 for U <= 16, one per team; 4 for U = 32): a converter warp issues its
// teams' copies (producer) and converts each landed slice (below), so the MMA
// warps only wait, load fragments, multiply and release.
//
// Staging.  A subcarrier streams through a private ring of `ring` (2 or 3)
// slices of 32 antennas; each slice is two 16-antenna blocks [H rows | y rows]
// x 128 bytes, written by tensor-map copies (cp.async.bulk.tensor, four per
// slice, 128-byte swizzle: 16-byte chunk j of row r lands at chunk j ^ (r mod
// 8), so that the 8 rows read by one ldmatrix phase fall in distinct bank
// groups) that complete on the slice's mbarrier ("full").  The converter
// refills a stage once the team's MMA warps have released it ("empty", one
// arrival per MMA warp).  Rows the copies never write (user slots >= U, symbol
// slots >= n_sym) are zeroed once; antennas past B arrive as zeros from the
// copies' bounds fill.
//
// Conversion.  Each landed slice is converted in place by its converter warp,
// one staged block row per lane at a time, half a row at a time: the 8 complex
// FP32 values of antennas 8h .. 8h+7 become four 16-bit planes (re hi, re lo,
// im hi, im lo; hi = x rounded to BF16 or FP16, lo = the rounded remainder),
// plane p in chunk 4h + p of the same row.  Every staged value is split once
// per subcarrier; a third mbarrier ("converted", one arrival after a warp
// barrier) hands the slice to the MMA warps.  The converter polls its teams
// without blocking, so the slices of one team never wait behind another's.
//
// Measured on the 1200 x 14, B = 256, U = 16 workload (BF16x3): one converter
// warp per four teams kept the MMA warps waiting (27-29 us per launch); one per
// team brings PD / FD to about 22.5 / 24.6 us, against 14.2 us for the copies
// alone.
//
// Arithmetic.  MMA operand A is H (16 users x 16 antennas), B is W (16 antennas
// x 8 rows), both fragments loaded with ldmatrix from the planes.  conj(h) w
// takes four real products, Re D = sum h_re w_re + h_im w_im and Im D = sum
// h_re w_im + (-h_im) w_re (the sign flipped on the A fragments, exact), each
// split as A_lo B_hi + A_hi B_lo + A_hi B_hi (the lo*lo term is dropped):
// twelve MMAs per tile and k-step into two accumulators (Re, Im).
//
// Fused form (one launch for a whole equalization, U = 8 or 16).  The same CTA
// also solves what its teams contract: a completed cluster tile D_c (G_c and
// y_c^MRC, Sec. II-C) goes from the team's MMA warps to a shared-memory handoff
// buffer (two per team, "tile full" / "tile free" mbarriers) instead of the
// workspace, and a solve group of U lanes per team (solve warps after the
// converter warps) runs the L-MMSE sweep on it (Sec. III-A; ZF is rho = 0),
// accumulates the Lemma 1 fusion terms of the subcarrier's clusters in cluster
// order (PD: the one central system), and writes z, sigma^2 (Thm. 3) and the
// max-log LLRs when the last cluster is in.  The solve of cluster c overlaps the
// contraction of cluster c + 1, and D never leaves the SM.  Per lane the
// arithmetic is that of the separate solve kernel (gj_solve_row, gj_row_dot and
// the same fusion order), so both launches give the same bits.
#include <cuda.h>

#include <cstdint>
#include <new>

#include "ffeq_device.cuh"
#include "ffeq_epilogue.cuh"
#include "ffeq_gj.cuh"
#include "ffeq_internal.h"
#include "ffeq_mma.cuh"

namespace ffeq {
namespace {

constexpr int kStreamWarps = 16;         // MMA warps of the full-size CTA (one CTA per SM)
constexpr int kStreamWarpsHalf = 8;      // MMA warps of the half-size CTA (two CTAs per SM)
constexpr int kStreamKsb = 2;            // 16-antenna blocks per slice (one per half-row conversion step)
constexpr int kStreamMaxRing = 3;
static_assert(kStreamKsb == 2, "one half-row conversion step per k-step of a slice");

template <int UP, int MW = kStreamWarps>
struct StreamShape {
  static constexpr int MT = UP <= 16 ? 1 : 2;       // 16-user m-tiles
  static constexpr int HR = 16 * MT;                // user row slots per block
  static constexpr int BR = HR + 16;                // rows per block (then n_sym <= 16 symbol slots)
  static constexpr int BLOCK = BR * 128;            // bytes per 16-antenna block (multiple of 1024)
  static constexpr int WPU = 2 * MT;                // warps per subcarrier
  static constexpr int UPC = MW / WPU;              // subcarriers in flight per CTA
  static constexpr int NTH = UP <= 16 ? 2 : 3;      // 8-row n-tiles of W per warp
  static constexpr int SLICE = kStreamKsb * BLOCK;
};

struct StreamParams {
  CUtensorMap map_h;   // H as [n_sc * U rows][2B floats], box 32 x U, 128-byte swizzle
  CUtensorMap map_y;   // y as [n_sc * n_sym rows][2B floats], box 32 x n_sym
  float2* D;
  int* status;
  int B, U, Ceff, n_sc, n_sym, ring;
  // Fused form only: outputs and scalars of the solve (as in SolveParams).
  float2* z;
  float* sigma2;
  float* llr;
  int* info;
  float rho, N0, llr_scale;
  int unbiased, llr_bits;
};

// Shared-memory areas of one team in the fused form: two handoff tiles of
// D_c [m][u] (m < U + n_sym <= UP + 16 rows of UP complex), the fusion
// numerators [n][u] of the subcarrier in progress, and the sweep's two
// broadcast buffers.
template <int UP>
struct FusedShape {
  static constexpr int MR = UP + kNsymMax;
  static constexpr int TILE = MR * UP;                        // float2 per handoff tile
  static constexpr int ACC = kNsymMax * UP;                   // float2
  static constexpr int ROWBUF = (2 * (2 * UP + 4) * 4 + 15) / 16 * 16;   // bytes
  static constexpr size_t TEAM = 2 * TILE * 8 + ACC * 8 + ROWBUF;
  static constexpr int WARPS = StreamShape<UP>::UPC * UP / 32;   // one lane group of UP lanes per team
  static_assert(UP <= 16, "the fused form holds one 8- or 16-lane group per team");
};

template <int UP, bool FUSED, int MW>
constexpr size_t stream_smem_bytes(int ring) {
  using Sh = StreamShape<UP, MW>;
  size_t b = 1024 + static_cast<size_t>(Sh::UPC) * ring * Sh::SLICE + 3 * Sh::UPC * kStreamMaxRing * 8;
  if constexpr (FUSED) b += 4 * Sh::UPC * 8 + 16 + Sh::UPC * FusedShape<UP>::TEAM;
  return b;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "l"(policy)
      : "memory");
}

__device__ __forceinline__ float4 lds128(uint32_t addr) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
  return v;
}

// Bounded wait on phase `parity` that lets the thread sleep in hardware until
// the phase completes (suspend-time hint of 1 us per try) instead of spinning on
// the issue slots; after kWaitTries tries (seconds) it records `code` and
// returns false.
constexpr int kWaitTries = 1 << 22;
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t* bar, uint32_t parity, int* status, int code) {
  for (int it = 0; it < kWaitTries; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(1000u)
        : "memory");
    if (ok) return true;
  }
  if (status) atomicExch(status, code);
  return false;
}

__device__ __forceinline__ void sts128(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}

// In-place conversion of half a staged row (antennas 8h .. 8h+7 of a block row,
// FP32 chunks 4h .. 4h+3): the 8 complex values become the four 16-bit planes
// of the split operands, plane p (re hi, re lo, im hi, im lo) in chunk 4h + p,
// the same 64 bytes (under the swizzle).  Load and convert are separate steps
// so that a warp can interleave them with its MMAs.
__device__ __forceinline__ void load_half(uint32_t row_addr, int r, int h, float4 (&q)[4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) q[j] = lds128(row_addr + (((4 * h + j) ^ (r & 7)) << 4));
}

template <int MODE>
__device__ __forceinline__ void store_half_planes(uint32_t row_addr, int r, int h, const float4 (&q)[4]) {
  uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    split_pair<MODE>(q[j].x, q[j].z, rh[j], rl[j]);
    split_pair<MODE>(q[j].y, q[j].w, ih[j], il[j]);
  }
  const int r7 = r & 7;
  sts128(row_addr + (((4 * h + 0) ^ r7) << 4), rh[0], rh[1], rh[2], rh[3]);
  sts128(row_addr + (((4 * h + 1) ^ r7) << 4), rl[0], rl[1], rl[2], rl[3]);
  sts128(row_addr + (((4 * h + 2) ^ r7) << 4), ih[0], ih[1], ih[2], ih[3]);
  sts128(row_addr + (((4 * h + 3) ^ r7) << 4), il[0], il[1], il[2], il[3]);
}

// Block row holding W row m (user rows first, then symbol rows); rows past the
// problem fall on a zeroed slot inside the block.
template <int UP>
__device__ __forceinline__ int w_row(int m, int U) {
  using Sh = StreamShape<UP>;
  const int r = m < U ? m : Sh::HR + m - U;
  return r < Sh::BR ? r : U;
}

// Per-lane ldmatrix row offsets (bytes within a block) of one warp, fixed for
// the whole kernel: A (16 users x 16 antennas; lanes 0-7 rows 0-7 / k 0-7, 8-15
// rows 8-15, then the same for k 8-15 -- the a0..a3 fragment order) and B (16
// antennas x 8 W rows per n-tile; lanes 0-7 k 0-7 and 8-15 k 8-15 of tile nt0
// -- b0, b1 -- and lanes 16-31 the same for tile nt0 + 1; a third tile with
// ldmatrix.x2).  Plane pl of antenna half h of block row r is chunk 4h + pl.
struct FragOffsets {
  uint32_t a[4], b[4], b3[4];
};

template <int UP>
__device__ __forceinline__ FragOffsets frag_offsets(int mt, int nt0, int nt_end, int U, int lane) {
  FragOffsets f;
  const int ar = 16 * mt + (lane & 7) + ((lane >> 3) & 1) * 8, ah = (lane >> 4) & 1;
  const int bh = (lane >> 3) & 1;
  const int nt = nt0 + (lane >> 4);
  const int br = w_row<UP>(8 * (nt < nt_end ? nt : nt0) + (lane & 7), U);
  const int n3 = nt0 + 2 < nt_end ? nt0 + 2 : nt0;
  const int br3 = w_row<UP>(8 * n3 + (lane & 7), U);
#pragma unroll
  for (int pl = 0; pl < 4; ++pl) {
    f.a[pl] = static_cast<uint32_t>(ar * 128 + (((4 * ah + pl) ^ (ar & 7)) << 4));
    f.b[pl] = static_cast<uint32_t>(br * 128 + (((4 * bh + pl) ^ (br & 7)) << 4));
    f.b3[pl] = static_cast<uint32_t>(br3 * 128 + (((4 * bh + pl) ^ (br3 & 7)) << 4));
  }
  return f;
}

// One 16-antenna k-step of one warp on converted planes.  conj(h) w takes four
// real products, Re D = sum h_re w_re + h_im w_im and Im D = sum h_re w_im +
// (-h_im) w_re (sign flipped in the A fragments), each split as A_lo B_hi +
// A_hi B_lo + A_hi B_hi: acc[j][0] += Re, acc[j][1] += Im of n-tile nt0 + j.
template <int UP, int MODE>
__device__ __forceinline__ void stream_kstep(uint32_t blk, const FragOffsets& f, int ntiles,
                                             float (&acc)[StreamShape<UP>::NTH][2][4]) {
  constexpr int NTH = StreamShape<UP>::NTH;
  uint32_t A[4][4];
#pragma unroll
  for (int pl = 0; pl < 4; ++pl) ldsm_x4(blk + f.a[pl], A[pl]);
  uint32_t Bf[4][NTH][2];
#pragma unroll
  for (int pl = 0; pl < 4; ++pl) {
    uint32_t r[4];
    ldsm_x4(blk + f.b[pl], r);
    Bf[pl][0][0] = r[0];
    Bf[pl][0][1] = r[1];
    Bf[pl][1][0] = r[2];
    Bf[pl][1][1] = r[3];
    if constexpr (NTH == 3) ldsm_x2(blk + f.b3[pl], Bf[pl][2][0], Bf[pl][2][1]);
  }
  uint32_t anim[2][4];                        // -h_im, lo and hi
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    anim[0][q] = A[3][q] ^ 0x80008000u;
    anim[1][q] = A[2][q] ^ 0x80008000u;
  }
  // Split products A_lo B_hi, A_hi B_lo, A_hi B_hi; the four accumulators of a
  // tile pair are each touched once per round of four MMAs.
#pragma unroll
  for (int prod = 0; prod < 3; ++prod) {
    const int pa = prod == 0 ? 1 : 0, pb = prod == 1 ? 1 : 0;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
#pragma unroll
      for (int j = 0; j < NTH; ++j) {
        if (j < ntiles) {
          if (half == 0) {
            mma_any<MODE>(acc[j][0], A[pa], Bf[pb][j][0], Bf[pb][j][1]);          // h_re w_re
            mma_any<MODE>(acc[j][1], A[pa], Bf[2 + pb][j][0], Bf[2 + pb][j][1]);  // h_re w_im
          } else {
            mma_any<MODE>(acc[j][0], A[2 + pa], Bf[2 + pb][j][0], Bf[2 + pb][j][1]);  // h_im w_im
            mma_any<MODE>(acc[j][1], anim[1 - pa], Bf[pb][j][0], Bf[pb][j][1]);       // -h_im w_re
          }
        }
      }
    }
  }
}

// Walks a team's slices in order: subcarrier k (slot, slot + nslots, ...),
// slice ks within it, ring stage s and the parity ph of that stage's use.
struct SliceCursor {
  int k, ks, s;
  uint32_t ph;
  __device__ __forceinline__ void next(int NC, int R, int nslots) {
    if (++ks == NC) {
      ks = 0;
      k += nslots;
    }
    if (++s == R) {
      s = 0;
      ph ^= 1u;
    }
  }
};

// Warp-specialized form.  MW MMA warps (teams as above; 16, or 8 for the
// half-size CTA of which two share an SM) and kConvWarps converter warps per CTA.  A converter warp owns UPC / kConvWarps
// teams: it issues their copies (producer), and as soon as a slice has landed
// it converts it in place to planes and signals the team (conv barrier, one
// arrival); the MMA warps only wait for converted slices, run ldmatrix and the
// MMAs, and release the slice (empty barrier, one arrival per MMA warp).  The
// converter polls its teams without blocking (a slice is converted only after
// it has been issued, a refill only after its gate has completed), so no wait
// depends on the order in which the teams progress; every wait is bounded.
template <int UP, int MW>
__host__ __device__ constexpr int conv_warps() { return StreamShape<UP, MW>::UPC; }   // one team per converter warp
template <int UP, bool FUSED>
__host__ __device__ constexpr int solve_warps() {
  if constexpr (FUSED) return FusedShape<UP>::WARPS;
  return 0;
}
template <int UP, bool FUSED, int MW>
__host__ __device__ constexpr int ws_threads() {
  return (MW + conv_warps<UP, MW>() + solve_warps<UP, FUSED>()) * 32;
}
constexpr long kConvPollLimit = 1L << 24;   // converter passes without progress before it gives up

// Solve warps of the fused form.  Solve warp sw holds 32 / UP lane groups; group
// `team` (lane i = user i) walks the team's subcarriers k = slot, slot + nslots,
// ... and their Ceff clusters in order, taking each cluster's tile from handoff
// buffer hq & 1: row i of G_c (D[j][i], j < U), the sweep (gj_solve_row), the
// right-hand sides (D rows U + n, read in place), then the tile goes back to the
// MMA warps.  The fusion numerators z_c,n / A_c,ii (Eq. fusionrule, Lemma 1) are
// summed in cluster order in the group's area (each lane owns its column), the
// denominators (g / A_c,ii, g = mu or 1) in a register; after the last cluster
// lane i writes user i's z, sigma^2 = N0 / den (Thm. 3) and LLRs, NaN for a
// subcarrier with a failed factorization.  A group whose team has no subcarrier
// left runs the sweep on an identity (its warp's other group may still be
// working) and writes nothing.  Every wait is bounded; a time-out ends the warp.
template <int UP>
__device__ __forceinline__ void fused_solve(const StreamParams& p, unsigned char* team_area, uint64_t* hfull,
                                            uint64_t* hfree, int sw, int lane) {
  using FS = FusedShape<UP>;
  const int gl = sw * 32 + lane;
  const int team = gl / UP, i = gl % UP;
  const int nslots = gridDim.x * StreamShape<UP>::UPC;
  const int NS = p.n_sym, Ceff = p.Ceff;
  unsigned char* area = team_area + team * FS::TEAM;
  const float2* tiles = reinterpret_cast<const float2*>(area);
  float2* acc = reinterpret_cast<float2*>(area + 2 * FS::TILE * 8);           // [n][UP]
  float* rowbuf = reinterpret_cast<float*>(area + 2 * FS::TILE * 8 + FS::ACC * 8);
  const float rho = p.rho;
  const int bits = p.llr_bits, hb = bits / 2;
  int hq = 0;
  for (int k = blockIdx.x + gridDim.x * team;; k += nslots) {
    const bool live = k < p.n_sc;
    if (!__any_sync(kFullMask, live)) return;
    bool failed = false;
    float dn = 0.f;
    for (int c = 0; c < Ceff; ++c) {
      const int b = hq & 1;
      bool ready = true;
      if (live) ready = mbar_wait_sleep(&hfull[team * 2 + b], (hq >> 1) & 1, p.status, FFEQ_ERR_TIMEOUT);
      if (!__all_sync(kFullMask, ready)) return;
      const float2* T = tiles + b * FS::TILE;
      float2 mrow[UP];
#pragma unroll
      for (int j = 0; j < UP; ++j) mrow[j] = live ? T[j * UP + i] : make_float2(j == i ? 1.f : 0.f, 0.f);
      float2 arow[UP];
      float Ai, gii;
      const int fail = gj_solve_row<UP>(mrow, rho, rowbuf, i, true, arow, Ai, gii);
      const float invA = rcp_approx(Ai);
      const float mu = gii == 0.f ? 0.f : fmaxf(1.f - rho * Ai, 0.f);
#pragma unroll
      for (int n = 0; n < kNsymMax; ++n) {
        if (n < NS) {
          const float2 zn = gj_row_dot<UP>(arow, T + (UP + n) * UP);
          if (live) {
            // The term is rounded on its own before the sum (no contraction
            // into an FMA), as when it is stored and summed by the separate kernel.
            const float2 prev = c == 0 ? make_float2(0.f, 0.f) : acc[n * UP + i];
            acc[n * UP + i] = cadd(prev, make_float2(__fmul_rn(zn.x, invA), __fmul_rn(zn.y, invA)));
          }
        }
      }
      __syncwarp();   // every lane of the group has read the tile
      if (live && i == 0) {
        mbar_arrive(&hfree[team * 2 + b]);
        if (p.info) p.info[static_cast<size_t>(k) * Ceff + c] = fail;
      }
      ++hq;
      dn += __fmul_rn(p.unbiased ? mu : 1.f, invA);
      failed = failed || fail != 0;
    }
    if (!live) continue;
    const float rr = rcp_approx(dn);
    for (int n = 0; n < NS; ++n) {
      float2 zz;
      float s2;
      if (failed) {
        zz = make_float2(NAN, NAN);
        s2 = NAN;
      } else if (dn > 0.f) {
        zz = cscale(acc[n * UP + i], rr);
        s2 = p.N0 * rr;
      } else {
        zz = make_float2(0.f, 0.f);
        s2 = INFINITY;
      }
      const size_t zi = (static_cast<size_t>(k) * NS + n) * UP + i;
      p.z[zi] = zz;
      if (n == 0) p.sigma2[static_cast<size_t>(k) * UP + i] = s2;
      if (bits) symbol_llr(zz, s2, p.llr_scale, hb, p.llr + zi * bits);
    }
  }
}

template <int UP, int MODE, bool FUSED, int MW>
__global__ void __launch_bounds__(ws_threads<UP, FUSED, MW>(), (MW == kStreamWarps ? 1 : 2))
    gram_ws_kernel(const __grid_constant__ StreamParams p) {
  using Sh = StreamShape<UP, MW>;
  using FS = FusedShape<UP <= 16 ? UP : 16>;
  constexpr int NTH = Sh::NTH;
  constexpr int kConvWarps = conv_warps<UP, MW>();
  constexpr int kWsThreads = ws_threads<UP, FUSED, MW>();
  constexpr int TPC = Sh::UPC / kConvWarps;       // teams per converter warp
  static_assert(Sh::UPC % kConvWarps == 0, "teams split evenly over the converter warps");
  static_assert(!FUSED || (UP <= 16 && MW == kStreamWarps), "fused form: 8 or 16 users, full-size CTA");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t ring0 = (raw + 1023u) & ~1023u;
  const int R = p.ring;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (ring0 - raw) + static_cast<size_t>(Sh::UPC) * R * Sh::SLICE);
  uint64_t* full_all = bars;                                      // [UPC][kStreamMaxRing]
  uint64_t* empty_all = bars + Sh::UPC * kStreamMaxRing;
  uint64_t* conv_all = bars + 2 * Sh::UPC * kStreamMaxRing;
  // Fused form: handoff barriers [UPC][2] (tile full: one arrival per MMA warp
  // of the team; tile free: one by the solve group), then the teams' areas.
  uint64_t* hfull = bars + 3 * Sh::UPC * kStreamMaxRing;
  uint64_t* hfree = hfull + 2 * Sh::UPC;
  unsigned char* team_area = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(hfree + 2 * Sh::UPC) + 15) & ~static_cast<uintptr_t>(15));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int U = p.U, NS = p.n_sym, B = p.B, Ceff = p.Ceff, S = B / Ceff, Mrows = U + NS;
  const int NC = (B + 16 * kStreamKsb - 1) / (16 * kStreamKsb);
  const int nslots = gridDim.x * Sh::UPC;
  const int nkb_last = (B - (NC - 1) * 16 * kStreamKsb + 15) / 16;

  // Zero the rows no copy writes; init the barriers.
  {
    const int zrows = (Sh::HR - U) + (16 - NS);
    const int nblk = Sh::UPC * R * kStreamKsb;
    for (int e = tid; e < nblk * zrows * 8; e += kWsThreads) {
      const int blk = e / (zrows * 8), rest = e - blk * zrows * 8;
      const int zr = rest >> 3, c16 = rest & 7;
      const int row = zr < Sh::HR - U ? U + zr : Sh::HR + NS + (zr - (Sh::HR - U));
      const uint32_t a = ring0 + static_cast<uint32_t>(blk * Sh::BLOCK + row * 128 + c16 * 16);
      asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(a), "r"(0u) : "memory");
    }
    if (tid < Sh::UPC * kStreamMaxRing) {
      mbar_init(&full_all[tid], 1);          // the copies of a slice
      mbar_init(&empty_all[tid], Sh::WPU);   // the team's MMA warps released it
      mbar_init(&conv_all[tid], 1);          // its converter warp converted it
    }
    if (FUSED && tid < 2 * Sh::UPC) {
      mbar_init(&hfull[tid], Sh::WPU);       // the team's MMA warps wrote the tile
      mbar_init(&hfree[tid], 1);             // the team's solve group is done with it
    }
    fence_mbar_init();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }

  if (FUSED && warp >= MW + kConvWarps) {
    if constexpr (FUSED) fused_solve<UP>(p, team_area, hfull, hfree, warp - MW - kConvWarps, lane);
  } else if (warp >= MW) {
    // ---------------- converter / producer warp
    const int cw = warp - MW;
    const uint64_t pol = l2_evict_first_policy();
    const uint32_t tx_full = static_cast<uint32_t>(kStreamKsb * 128 * Mrows);
    const uint32_t tx_last = static_cast<uint32_t>(nkb_last * 128 * Mrows);
    SliceCursor pc[TPC], cv[TPC];
    int issued[TPC], converted[TPC];
    for (int q = 0; q < TPC; ++q) {
      const int team = cw * TPC + q;
      const int slot = blockIdx.x + gridDim.x * team;
      pc[q] = SliceCursor{slot, 0, 0, 0u};
      cv[q] = pc[q];
      issued[q] = 0;
      converted[q] = 0;
    }
    auto issue = [&](int q) {   // lane 0
      const int team = cw * TPC + q;
      const SliceCursor& c = pc[q];
      const int nkb = c.ks == NC - 1 ? nkb_last : kStreamKsb;
      const uint32_t st = ring0 + static_cast<uint32_t>((team * R + c.s) * Sh::SLICE);
      uint64_t* fb = &full_all[team * kStreamMaxRing + c.s];
      mbar_arrive_expect_tx(fb, nkb == kStreamKsb ? tx_full : tx_last);
      for (int kb = 0; kb < nkb; ++kb) {
        const int x = 2 * 16 * (kStreamKsb * c.ks + kb);
        tma_load_2d(st + kb * Sh::BLOCK, &p.map_h, x, c.k * U, smem_u32(fb), pol);
        tma_load_2d(st + kb * Sh::BLOCK + Sh::HR * 128, &p.map_y, x, c.k * NS, smem_u32(fb), pol);
      }
    };
    if (lane == 0) {
      for (int q = 0; q < TPC; ++q)
        for (; issued[q] < R && pc[q].k < p.n_sc; ++issued[q]) {
          issue(q);
          pc[q].next(NC, R, nslots);
        }
    }
    long idle = 0;
    for (;;) {
      bool pending = false, progressed = false;
#pragma unroll
      for (int q = 0; q < TPC; ++q) {
        const int team = cw * TPC + q;
        // Refill every stage whose slice the team's MMA warps have released.
        if (lane == 0) {
          while (pc[q].k < p.n_sc && mbar_try_wait(&empty_all[team * kStreamMaxRing + pc[q].s], pc[q].ph ^ 1u)) {
            issue(q);
            pc[q].next(NC, R, nslots);
            ++issued[q];
            progressed = true;
          }
        }
        if (cv[q].k >= p.n_sc) continue;
        pending = true;
        // Convert the next slice once it has been issued and has landed.
        const int iss = __shfl_sync(kFullMask, issued[q], 0);
        if (converted[q] >= iss) continue;
        const bool landed = mbar_try_wait(&full_all[team * kStreamMaxRing + cv[q].s], cv[q].ph);
        if (!__all_sync(kFullMask, landed)) continue;
        const int nkb = cv[q].ks == NC - 1 ? nkb_last : kStreamKsb;
        const uint32_t st = ring0 + static_cast<uint32_t>((team * R + cv[q].s) * Sh::SLICE);
        for (int e = lane; e < nkb * Mrows; e += 32) {
          const int kbt = e / Mrows, rr = e - kbt * Mrows;
          const int row = rr < U ? rr : Sh::HR + (rr - U);
          const uint32_t addr = st + static_cast<uint32_t>(kbt * Sh::BLOCK + row * 128);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float4 v[4];
            load_half(addr, row, h, v);
            store_half_planes<MODE>(addr, row, h, v);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&conv_all[team * kStreamMaxRing + cv[q].s]);
        cv[q].next(NC, R, nslots);
        ++converted[q];
        progressed = true;
      }
      progressed = __any_sync(kFullMask, progressed);
      if (!pending) break;
      if (progressed) {
        idle = 0;
      } else if (++idle > kConvPollLimit) {
        if (lane == 0 && p.status) atomicExch(p.status, FFEQ_ERR_TIMEOUT);
        break;
      } else {
        __nanosleep(64);
      }
    }
    // Let the copies issued for slices nobody will convert any more land before
    // leaving (only after a time-out; a normal exit has none in flight).
    if (lane == 0) {
      for (int q = 0; q < TPC; ++q) {
        SliceCursor c = cv[q];
        for (int r = converted[q]; r < issued[q]; ++r) {
          mbar_wait_bounded(&full_all[(cw * TPC + q) * kStreamMaxRing + c.s], c.ph, nullptr, 0);
          c.next(NC, R, nslots);
        }
      }
    }
  } else {
    // ---------------- MMA warp
    const int team = warp / Sh::WPU, wi = warp % Sh::WPU;
    const int slot = blockIdx.x + gridDim.x * team;
    uint64_t* empty = empty_all + team * kStreamMaxRing;
    uint64_t* conv = conv_all + team * kStreamMaxRing;
    const uint32_t myring = ring0 + static_cast<uint32_t>(team * R * Sh::SLICE);
    const int g = lane >> 2, t = lane & 3;
    const int mt = wi % Sh::MT, half = wi / Sh::MT;
    const int NT = (Mrows + 7) / 8;
    const int nt0 = half * NTH;
    const int nt_end = min(NT, nt0 + NTH);
    const int ntiles = nt_end - nt0;
    const FragOffsets fo = frag_offsets<UP>(mt, nt0, nt_end, U, lane);
    const size_t mat = static_cast<size_t>(Mrows) * U;
    float acc[NTH][2][4];
#pragma unroll
    for (int j = 0; j < NTH; ++j)
#pragma unroll
      for (int o = 0; o < 2; ++o)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[j][o][q] = 0.f;
    int cl_left = S;
    float2* Dc = FUSED ? nullptr : p.D + static_cast<size_t>(slot) * Ceff * mat;
    int hq = 0;              // fused: tiles handed to the solve group so far
    bool aborted = false;
    SliceCursor cc{slot, 0, 0, 0u};
    while (cc.k < p.n_sc && !aborted) {
      const bool ready = mbar_wait_sleep(&conv[cc.s], cc.ph, p.status, FFEQ_ERR_TIMEOUT);
      if (!__all_sync(kFullMask, ready)) break;
      const int nkb = cc.ks == NC - 1 ? nkb_last : kStreamKsb;
      const uint32_t st = myring + static_cast<uint32_t>(cc.s * Sh::SLICE);
      for (int kb = 0; kb < nkb; ++kb) {
        stream_kstep<UP, MODE>(st + kb * Sh::BLOCK, fo, ntiles, acc);
        cl_left -= 16;
        if (cl_left <= 0) {
          // Cluster complete: D[k][c][m][u] for this warp's tiles, to the
          // workspace, or (fused) to the team's handoff tile hq & 1 once the
          // solve group has released that tile's previous cluster.
          float2* out = Dc;
          int ld = U;
          if constexpr (FUSED) {
            const int b = team * 2 + (hq & 1);
            const bool freed = mbar_wait_sleep(&hfree[b], ((hq >> 1) & 1) ^ 1u, p.status, FFEQ_ERR_TIMEOUT);
            if (!__all_sync(kFullMask, freed)) {
              aborted = true;
              break;
            }
            out = reinterpret_cast<float2*>(team_area + team * FS::TEAM) + (hq & 1) * FS::TILE;
            ld = UP;
          }
#pragma unroll
          for (int j = 0; j < NTH; ++j) {
            if (j < ntiles) {
#pragma unroll
              for (int q4 = 0; q4 < 4; ++q4) {
                const int u = 16 * mt + g + 8 * (q4 >> 1);
                const int m = 8 * (nt0 + j) + 2 * t + (q4 & 1);
                if (u < U && m < Mrows) out[m * ld + u] = make_float2(acc[j][0][q4], acc[j][1][q4]);
              }
            }
#pragma unroll
            for (int o = 0; o < 2; ++o)
#pragma unroll
              for (int q4 = 0; q4 < 4; ++q4) acc[j][o][q4] = 0.f;
          }
          if constexpr (FUSED) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&hfull[team * 2 + (hq & 1)]);
            ++hq;
          }
          cl_left = S;
          if constexpr (!FUSED) Dc += mat;
        }
      }
      if (aborted) break;
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[cc.s]);
      SliceCursor nc = cc;
      nc.next(NC, R, nslots);
      if (!FUSED && nc.ks == 0) Dc = p.D + static_cast<size_t>(nc.k) * Ceff * mat;   // next subcarrier
      cc = nc;
    }
  }
  // Let the dependent solve kernel start its launch while this grid drains, but
  // only once every warp of the CTA is done: the converter warps finish before
  // the MMA warps, and a solve grid launched on their signal parks its CTAs in
  // the shared memory this CTA leaves free, where waiting for this grid slowed it
  // (PD: 31 -> 52 us per call on the 1200 x 14, B = 256, U = 16 workload).
  __syncthreads();
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependency on the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {   // thread-safe one-time lookup
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(f);
    return nullptr;
  }();
  return fn;
}

// Rows of 2B floats (complex interleaved), 16-byte aligned base and row stride;
// boxes of 32 floats (16 antennas, 128 bytes) by box_rows rows, 128-byte swizzle,
// zeros past the row end.
bool encode_rows(CUtensorMap* map, const void* base, long long rows, int B, int box_rows) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[2] = {static_cast<cuuint64_t>(2) * B, static_cast<cuuint64_t>(rows)};
  const cuuint64_t strides[1] = {static_cast<cuuint64_t>(B) * 8};
  const cuuint32_t box[2] = {32, static_cast<cuuint32_t>(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int UP, int MODE, bool FUSED, int MW = kStreamWarps>
cudaError_t launch_stream_up(const StreamParams& sp, cudaStream_t stream) {
  static int configured[64] = {0};
  static int num_sms[64] = {0};
  constexpr int kMaxRing = FUSED ? kGramFusedRing : kStreamMaxRing;
  constexpr int kPerSm = MW == kStreamWarps ? 1 : 2;   // CTAs that share an SM
  static_assert(kPerSm * stream_smem_bytes<UP, FUSED, MW>(kMaxRing) <= 227 * 1024, "shared memory of an SM");
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 64 && !configured[dev]) {
    err = cudaFuncSetAttribute(gram_ws_kernel<UP, MODE, FUSED, MW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(stream_smem_bytes<UP, FUSED, MW>(kMaxRing)));
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    configured[dev] = 1;
  }
  if (sp.ring < 2 || sp.ring > kMaxRing) return cudaErrorInvalidValue;
  const int slots = (dev < 64 ? num_sms[dev] : 152) * kPerSm;
  constexpr int UPC = StreamShape<UP, MW>::UPC;
  const int need = (sp.n_sc + UPC - 1) / UPC;
  const int grid = need < slots ? need : slots;
  gram_ws_kernel<UP, MODE, FUSED, MW>
      <<<grid, ws_threads<UP, FUSED, MW>(), stream_smem_bytes<UP, FUSED, MW>(sp.ring), stream>>>(sp);
  return cudaGetLastError();
}

}  // namespace

// Maps of the last kEntries input pairs of a plan (the plan fixes every size,
// so the addresses of H and y identify the maps).
struct TensorMapCache {
  static constexpr int kEntries = 16;
  struct Entry {
    CUtensorMap mh, my;
    const void* H = nullptr;
    const void* y = nullptr;
  };
  Entry e[kEntries];
  int next = 0;
};

TensorMapCache* tensor_map_cache_create() { return new (std::nothrow) TensorMapCache; }
void tensor_map_cache_destroy(TensorMapCache* cache) { delete cache; }

bool gram_stream_eligible(int precision, int B, int U, int n_sym, int Ceff) {
  if (precision != FFEQ_BF16X3 && precision != FFEQ_FP16X3) return false;
  if (U < 1 || U > 32 || n_sym < 1 || n_sym > 16 || B < 2 || B % 2 != 0 || Ceff < 1 || B % Ceff != 0) return false;
  return Ceff == 1 || (B / Ceff) % 16 == 0;
}

// Tensor maps (from the plan's cache where the inputs were seen before) and
// the contraction fields of the streamed launch.
static bool stream_params(const GramParams& p, StreamParams& sp) {
  TensorMapCache* c = p.map_cache;
  int hit = -1;
  if (c)
    for (int q = 0; q < TensorMapCache::kEntries; ++q)
      if (c->e[q].H == p.H && c->e[q].y == p.y) hit = q;
  if (hit >= 0) {
    sp.map_h = c->e[hit].mh;
    sp.map_y = c->e[hit].my;
  } else {
    if (!encode_rows(&sp.map_h, p.H, static_cast<long long>(p.n_sc) * p.U, p.B, p.U) ||
        !encode_rows(&sp.map_y, p.y, static_cast<long long>(p.n_sc) * p.n_sym, p.B, p.n_sym))
      return false;
    if (c) {
      TensorMapCache::Entry& e = c->e[c->next];
      e.mh = sp.map_h;
      e.my = sp.map_y;
      e.H = p.H;
      e.y = p.y;
      c->next = (c->next + 1) % TensorMapCache::kEntries;
    }
  }
  sp.D = p.D;
  sp.status = p.status;
  sp.B = p.B;
  sp.U = p.U;
  sp.Ceff = p.Ceff;
  sp.n_sc = p.n_sc;
  sp.n_sym = p.n_sym;
  // The next slice is converted while the current one is consumed: two slices at least.
  sp.ring = p.stages < 2 ? 2 : (p.stages > kStreamMaxRing ? kStreamMaxRing : p.stages);
  return true;
}

template <int MW>
cudaError_t launch_stream_mw(const StreamParams& sp, int precision, int UP, cudaStream_t stream) {
  const bool f16 = precision == FFEQ_FP16X3;
  switch (UP) {
    case 8:
      return f16 ? launch_stream_up<8, kFp16x3, false, MW>(sp, stream)
                 : launch_stream_up<8, kBf16x3, false, MW>(sp, stream);
    case 16:
      return f16 ? launch_stream_up<16, kFp16x3, false, MW>(sp, stream)
                 : launch_stream_up<16, kBf16x3, false, MW>(sp, stream);
    default:
      return f16 ? launch_stream_up<32, kFp16x3, false, MW>(sp, stream)
                 : launch_stream_up<32, kBf16x3, false, MW>(sp, stream);
  }
}

cudaError_t launch_gram_stream(const GramParams& p, int precision, cudaStream_t stream) {
  if (p.n_sc == 0) return cudaSuccess;
  StreamParams sp{};
  if (!stream_params(p, sp)) return cudaErrorInvalidValue;
  if (p.variant == kGramStreamHalf) return launch_stream_mw<kStreamWarpsHalf>(sp, precision, padded_users(p.U), stream);
  const bool f16 = precision == FFEQ_FP16X3;
  switch (padded_users(p.U)) {
    case 8:
      return f16 ? launch_stream_up<8, kFp16x3, false>(sp, stream) : launch_stream_up<8, kBf16x3, false>(sp, stream);
    case 16:
      return f16 ? launch_stream_up<16, kFp16x3, false>(sp, stream) : launch_stream_up<16, kBf16x3, false>(sp, stream);
    default:
      return f16 ? launch_stream_up<32, kFp16x3, false>(sp, stream) : launch_stream_up<32, kBf16x3, false>(sp, stream);
  }
}

bool gram_fused_eligible(int precision, int B, int U, int n_sym, int Ceff) {
  return (U == 8 || U == 16) && gram_stream_eligible(precision, B, U, n_sym, Ceff);
}

cudaError_t launch_gram_fused(const GramParams& p, const SolveParams& s, int precision, cudaStream_t stream) {
  if (p.n_sc == 0) return cudaSuccess;
  if (!gram_fused_eligible(precision, p.B, p.U, p.n_sym, p.Ceff) || !p.cl_uniform || !s.z || !s.sigma2 ||
      (s.llr_bits && !s.llr))
    return cudaErrorInvalidValue;
  StreamParams sp{};
  if (!stream_params(p, sp)) return cudaErrorInvalidValue;
  sp.D = nullptr;
  sp.ring = kGramFusedRing;
  sp.z = s.z;
  sp.sigma2 = s.sigma2;
  sp.llr = s.llr_bits ? s.llr : nullptr;
  sp.info = s.info;
  sp.rho = s.rho;
  sp.N0 = s.N0;
  sp.llr_scale = s.llr_scale;
  sp.unbiased = s.unbiased;
  sp.llr_bits = s.llr_bits;
  const bool f16 = precision == FFEQ_FP16X3;
  if (p.U == 8)
    return f16 ? launch_stream_up<8, kFp16x3, true>(sp, stream) : launch_stream_up<8, kBf16x3, true>(sp, stream);
  return f16 ? launch_stream_up<16, kFp16x3, true>(sp, stream) : launch_stream_up<16, kBf16x3, true>(sp, stream);
}

}  // namespace ffeq
