// Streamed local preprocessing (Sec. II-C) on the tensor cores: the contraction
// D_{k,c}[m][u] = sum_{b in cluster c} conj(H_k[u][b]) W_k[m][b], W_k = [H_k ; Y_k]
// of ffeq_gram.cuh, reorganised so that no warp ever waits for another one's
// partial sums.
//
// Work split.  A CTA of 16 warps holds several subcarriers at once (8 for
// U <= 16, 4 for U = 32).  Each subcarrier is owned by a team of 2 (or 4) warps;
// each warp owns a fixed set of output tiles (one 16-user m-tile times two or
// three 8-row n-tiles of W) and accumulates them in registers over the whole
// antenna range of a cluster (PD: all B antennas, the adder tree of Eq.
// fullMRC in the accumulators; FD: S = B/C antennas, then the cluster's tile is
// stored and the accumulators restart).  No split-K, no shared-memory
// reduction, no CTA-wide barrier after the prologue.
//
// Staging.  A subcarrier streams through a private ring of `ring` (2 or 3)
// slices of 32 antennas; each slice is two 16-antenna blocks [H rows | y rows]
// x 128 bytes, written by tensor-map copies (cp.async.bulk.tensor, four per
// slice, 128-byte swizzle: 16-byte chunk j of row r lands at chunk j ^ (r mod
// 8), so that the 8 rows read by one ldmatrix phase fall in distinct bank
// groups) that complete on the slice's mbarrier.  Lane 0 of the team's first
// warp refills a slice once every warp of the team has released it (a second
// mbarrier).  Rows the copies never write (user slots >= U, symbol slots >=
// n_sym) are zeroed once; antennas past B arrive as zeros from the copies'
// bounds fill.
//
// Conversion.  Each landed slice is converted in place by the team's threads,
// one staged block row each, half a row at a time: the 8 complex FP32 values
// of antennas 8h .. 8h+7 become four 16-bit planes (re hi, re lo, im hi, im lo;
// hi = x rounded to BF16 or FP16, lo = the rounded remainder), plane p in chunk
// 4h + p of the same row.  Every staged value is split once per subcarrier.  A
// third mbarrier tells the team that a slice's planes
// are complete (one arrival per warp, after a warp barrier).  The conversion of slice i + 1 is interleaved with the MMAs of
// slice i in every warp (software pipelining), so the split arithmetic and the
// tensor pipe overlap instead of taking turns.
//
// Arithmetic.  MMA operand A is H (16 users x 16 antennas), B is W (16 antennas
// x 8 rows), both fragments loaded with ldmatrix from the planes.  conj(h) w
// takes four real products, Re D = sum h_re w_re + h_im w_im and Im D = sum
// h_re w_im + (-h_im) w_re (the sign flipped on the A fragments, exact), each
// split as A_lo B_hi + A_hi B_lo + A_hi B_hi (the lo*lo term is dropped):
// twelve MMAs per tile and k-step into two accumulators (Re, Im).
#include <cuda.h>

#include <cstdint>

#include "ffeq_device.cuh"
#include "ffeq_internal.h"
#include "ffeq_mma.cuh"

namespace ffeq {
namespace {

constexpr int kStreamWarps = 16;
constexpr int kStreamKsb = 2;            // 16-antenna blocks per slice (one per half-row conversion step)
constexpr int kStreamMaxRing = 3;
static_assert(kStreamKsb == 2, "one half-row conversion step per k-step of a slice");

template <int UP>
struct StreamShape {
  static constexpr int MT = UP <= 16 ? 1 : 2;       // 16-user m-tiles
  static constexpr int HR = 16 * MT;                // user row slots per block
  static constexpr int BR = HR + 16;                // rows per block (then n_sym <= 16 symbol slots)
  static constexpr int BLOCK = BR * 128;            // bytes per 16-antenna block (multiple of 1024)
  static constexpr int WPU = 2 * MT;                // warps per subcarrier
  static constexpr int UPC = kStreamWarps / WPU;    // subcarriers in flight per CTA
  static constexpr int NTH = UP <= 16 ? 2 : 3;      // 8-row n-tiles of W per warp
  static constexpr int SLICE = kStreamKsb * BLOCK;
};

struct StreamParams {
  CUtensorMap map_h;   // H as [n_sc * U rows][2B floats], box 32 x U, 128-byte swizzle
  CUtensorMap map_y;   // y as [n_sc * n_sym rows][2B floats], box 32 x n_sym
  float2* D;
  int* status;
  int B, U, Ceff, n_sc, n_sym, ring;
};

template <int UP>
constexpr size_t stream_smem_bytes(int ring) {
  using Sh = StreamShape<UP>;
  return 1024 + static_cast<size_t>(Sh::UPC) * ring * Sh::SLICE + 3 * Sh::UPC * kStreamMaxRing * 8;
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

template <int UP, int MODE>
__global__ void __launch_bounds__(kStreamWarps * 32, 1) gram_stream_kernel(const __grid_constant__ StreamParams p) {
  using Sh = StreamShape<UP>;
  constexpr int NTH = Sh::NTH;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t ring0 = (raw + 1023u) & ~1023u;   // swizzled copies want 1024-byte aligned blocks
  const int R = p.ring;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (ring0 - raw) + static_cast<size_t>(Sh::UPC) * R * Sh::SLICE);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int team = warp / Sh::WPU, wi = warp % Sh::WPU;
  uint64_t* full = bars + team * kStreamMaxRing;
  uint64_t* empty = bars + (Sh::UPC + team) * kStreamMaxRing;
  uint64_t* conv = bars + (2 * Sh::UPC + team) * kStreamMaxRing;
  const uint32_t myring = ring0 + static_cast<uint32_t>(team * R * Sh::SLICE);
  const int U = p.U, NS = p.n_sym, B = p.B, Ceff = p.Ceff, S = B / Ceff, Mrows = U + NS;
  const int NC = (B + 16 * kStreamKsb - 1) / (16 * kStreamKsb);   // slices per subcarrier
  const int slot = blockIdx.x + gridDim.x * team, nslots = gridDim.x * Sh::UPC;

  // Zero the rows no copy writes, in every block of the ring; init the barriers.
  {
    const int zrows = (Sh::HR - U) + (16 - NS);
    const int nblk = Sh::UPC * R * kStreamKsb;
    for (int e = tid; e < nblk * zrows * 8; e += kStreamWarps * 32) {
      const int blk = e / (zrows * 8), rest = e - blk * zrows * 8;
      const int zr = rest >> 3, c16 = rest & 7;
      const int row = zr < Sh::HR - U ? U + zr : Sh::HR + NS + (zr - (Sh::HR - U));
      const uint32_t a = ring0 + static_cast<uint32_t>(blk * Sh::BLOCK + row * 128 + c16 * 16);
      asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(a), "r"(0u) : "memory");
    }
    if (tid < Sh::UPC * kStreamMaxRing) {
      mbar_init(&bars[tid], 1);                                         // full: the copies
      mbar_init(&bars[Sh::UPC * kStreamMaxRing + tid], Sh::WPU);        // empty: one arrival per warp
      mbar_init(&bars[2 * Sh::UPC * kStreamMaxRing + tid], Sh::WPU);   // converted: one arrival per warp
    }
    fence_mbar_init();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
  }
  const uint64_t pol = l2_evict_first_policy();
  const bool producer = wi == 0 && lane == 0;
  const int nkb_last = (B - (NC - 1) * 16 * kStreamKsb + 15) / 16;   // 16-antenna blocks of the last slice
  const uint32_t tx_full = static_cast<uint32_t>(kStreamKsb * 128 * Mrows);
  const uint32_t tx_last = static_cast<uint32_t>(nkb_last * 128 * Mrows);
  // Copies of the slice under cursor c into its stage (lane 0 of warp 0 only).
  auto issue = [&](const SliceCursor& c) {
    const int nkb = c.ks == NC - 1 ? nkb_last : kStreamKsb;
    const uint32_t st = myring + static_cast<uint32_t>(c.s * Sh::SLICE);
    const uint32_t bar = smem_u32(&full[c.s]);
    mbar_arrive_expect_tx(&full[c.s], nkb == kStreamKsb ? tx_full : tx_last);
    for (int kb = 0; kb < nkb; ++kb) {
      const int x = 2 * 16 * (kStreamKsb * c.ks + kb);
      tma_load_2d(st + kb * Sh::BLOCK, &p.map_h, x, c.k * U, bar, pol);
      tma_load_2d(st + kb * Sh::BLOCK + Sh::HR * 128, &p.map_y, x, c.k * NS, bar, pol);
    }
  };
  SliceCursor pc{slot, 0, 0, 0u};       // next slice to copy (producer lane)
  int issued = 0;                        // slices copied so far (producer lane)
  if (producer) {
    for (; issued < R && pc.k < p.n_sc; ++issued) {
      issue(pc);
      pc.next(NC, R, nslots);
    }
  }
  __syncwarp();
  // The slice `issued` goes into the stage of slice issued - R once every warp
  // of the team has released that one (phase pc.ph ^ 1 of the stage's empty
  // barrier; the barrier cannot run a further phase ahead before this copy).
  auto refill_ready = [&]() { return mbar_try_wait(&empty[pc.s], pc.ph ^ 1u); };

  const int g = lane >> 2, t = lane & 3;
  const int mt = wi % Sh::MT, half = wi / Sh::MT;
  // Bounded chance for the copies already issued (at most R - 1 slices after
  // the one under c) to land before the warp leaves.
  auto drain = [&](SliceCursor c) {
    if (!producer) return;
    for (int q = 1; q < R; ++q) {
      c.next(NC, R, nslots);
      if (c.k >= p.n_sc) break;
      mbar_wait_bounded(&full[c.s], c.ph, nullptr, 0);
    }
  };
  const int NT = (Mrows + 7) / 8;
  const int nt0 = half * NTH;
  const int nt_end = min(NT, nt0 + NTH);
  const int ntiles = nt_end - nt0;                 // may be <= 0: the warp only converts
  const FragOffsets fo = frag_offsets<UP>(mt, nt0, nt_end, U, lane);
  float acc[NTH][2][4];
#pragma unroll
  for (int j = 0; j < NTH; ++j)
#pragma unroll
    for (int o = 0; o < 2; ++o)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[j][o][q] = 0.f;
  // This thread's conversion task, the same in every slice: one block row
  // (rows U .. HR-1 and symbol slots >= n_sym are never loaded and stay zero).
  // A team has at least kStreamKsb * (U + n_sym) threads, so one task at most.
  const int ce = wi * 32 + lane;
  const int ckb = ce / Mrows, crr = ce - ckb * Mrows;
  const int crow = crr < U ? crr : Sh::HR + (crr - U);
  const uint32_t coff = static_cast<uint32_t>(ckb * Sh::BLOCK + crow * 128);
  const bool ctask_full = ce < kStreamKsb * Mrows, ctask_last = ce < nkb_last * Mrows;
  // Output position of this warp's tiles: c0 (user g, row 2t), c1 (g, 2t+1),
  // c2 (g+8, 2t), c3 (g+8, 2t+1) of each n-tile.
  const size_t mat = static_cast<size_t>(Mrows) * U;

  // Prologue: planes of slice 0.
  SliceCursor cc{slot, 0, 0, 0u};       // slice being consumed
  if (cc.k < p.n_sc) {
    const bool landed = mbar_wait_sleep(&full[0], 0u, p.status, FFEQ_ERR_TIMEOUT);
    if (!__all_sync(kFullMask, landed)) {
      drain(cc);
      return;
    }
    if (NC == 1 ? ctask_last : ctask_full) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float4 q[4];
        load_half(myring + coff, crow, h, q);
        store_half_planes<MODE>(myring + coff, crow, h, q);
      }
    }
    // Order the plane writes before the copy that later refills the slice; the
    // warp barrier makes every lane's writes part of lane 0's release.
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0) mbar_arrive(&conv[0]);
  }
  int cl_left = S;                       // antennas left in the current cluster
  float2* Dc = p.D + static_cast<size_t>(slot) * Ceff * mat;

  // Slice i: its planes are complete (every thread of the team arrived on
  // conv); the MMAs of its k-steps are interleaved with this thread's
  // conversion of slice i + 1 (one half-row per k-step), so that the split
  // arithmetic and the tensor pipe overlap within each warp.
  for (int i = 0; cc.k < p.n_sc; ++i) {
    const bool converted = mbar_wait_sleep(&conv[cc.s], cc.ph, p.status, FFEQ_ERR_TIMEOUT);
    if (!__all_sync(kFullMask, converted)) {
      drain(cc);
      return;
    }
    SliceCursor nc = cc;
    nc.next(NC, R, nslots);
    const bool has_next = nc.k < p.n_sc;
    // The next slice must have been copied before anyone waits for it: a refill
    // the producer deferred becomes a (bounded) blocking wait here.
    bool ok = true;
    if (producer && has_next && issued <= i + 1) {
      ok = mbar_wait_sleep(&empty[pc.s], pc.ph ^ 1u, p.status, FFEQ_ERR_TIMEOUT);
      if (ok) {
        issue(pc);
        pc.next(NC, R, nslots);
        ++issued;
      } else {
        drain(cc);
      }
    }
    if (!__shfl_sync(kFullMask, ok, 0)) return;
    if (has_next) {
      const bool landed = mbar_wait_sleep(&full[nc.s], nc.ph, p.status, FFEQ_ERR_TIMEOUT);
      if (!__all_sync(kFullMask, landed)) {
        drain(cc);
        return;
      }
    }
    const bool conv_now = has_next && (nc.ks == NC - 1 ? ctask_last : ctask_full);
    const uint32_t caddr = myring + static_cast<uint32_t>(nc.s * Sh::SLICE) + coff;
    const int nkb = cc.ks == NC - 1 ? nkb_last : kStreamKsb;
    const uint32_t st = myring + static_cast<uint32_t>(cc.s * Sh::SLICE);
#pragma unroll
    for (int kb = 0; kb < kStreamKsb; ++kb) {
      float4 q[4];
      if (conv_now) load_half(caddr, crow, kb, q);
      if (kb < nkb) {
        stream_kstep<UP, MODE>(st + kb * Sh::BLOCK, fo, ntiles, acc);
        cl_left -= 16;
        if (cl_left <= 0) {
          // Cluster complete: D[k][c][m][u] for this warp's tiles.
#pragma unroll
          for (int j = 0; j < NTH; ++j) {
            if (j < ntiles) {
#pragma unroll
              for (int q4 = 0; q4 < 4; ++q4) {
                const int u = 16 * mt + g + 8 * (q4 >> 1);
                const int m = 8 * (nt0 + j) + 2 * t + (q4 & 1);
                if (u < U && m < Mrows) Dc[m * U + u] = make_float2(acc[j][0][q4], acc[j][1][q4]);
              }
            }
#pragma unroll
            for (int o = 0; o < 2; ++o)
#pragma unroll
              for (int q4 = 0; q4 < 4; ++q4) acc[j][o][q4] = 0.f;
          }
          cl_left = S;
          Dc += mat;
        }
      }
      if (conv_now) store_half_planes<MODE>(caddr, crow, kb, q);
    }
    if (has_next) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv[nc.s]);
    }
    if (nc.ks == 0) Dc = p.D + static_cast<size_t>(nc.k) * Ceff * mat;   // next subcarrier
    // Release slice i.  The producer refills every stage whose slice all warps
    // have released, without waiting for the other warps (a refill that is not
    // ready yet is tried again after the next slice).
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[cc.s]);
    if (producer) {
      while (pc.k < p.n_sc && issued <= i + R && refill_ready()) {
        issue(pc);
        pc.next(NC, R, nslots);
        ++issued;
      }
    }
    __syncwarp();
    cc = nc;
  }
  // Let the dependent solve kernel start its launch while this grid drains.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependency on the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
    looked = true;
  }
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

template <int UP, int MODE>
cudaError_t launch_stream_up(const StreamParams& sp, cudaStream_t stream) {
  static int configured[64] = {0};
  static int num_sms[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 64 && !configured[dev]) {
    err = cudaFuncSetAttribute(gram_stream_kernel<UP, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               static_cast<int>(stream_smem_bytes<UP>(kStreamMaxRing)));
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    configured[dev] = 1;
  }
  const int sms = dev < 64 ? num_sms[dev] : 152;
  const int need = (sp.n_sc + StreamShape<UP>::UPC - 1) / StreamShape<UP>::UPC;
  const int grid = need < sms ? need : sms;
  gram_stream_kernel<UP, MODE><<<grid, kStreamWarps * 32, stream_smem_bytes<UP>(sp.ring), stream>>>(sp);
  return cudaGetLastError();
}

}  // namespace

bool gram_stream_eligible(int precision, int B, int U, int n_sym, int Ceff) {
  if (precision != FFEQ_BF16X3 && precision != FFEQ_FP16X3) return false;
  if (U < 1 || U > 32 || n_sym < 1 || n_sym > 16 || B < 2 || B % 2 != 0 || Ceff < 1 || B % Ceff != 0) return false;
  return Ceff == 1 || (B / Ceff) % 16 == 0;
}

cudaError_t launch_gram_stream(const GramParams& p, int precision, cudaStream_t stream) {
  if (p.n_sc == 0) return cudaSuccess;
  StreamParams sp{};
  if (!encode_rows(&sp.map_h, p.H, static_cast<long long>(p.n_sc) * p.U, p.B, p.U) ||
      !encode_rows(&sp.map_y, p.y, static_cast<long long>(p.n_sc) * p.n_sym, p.B, p.n_sym))
    return cudaErrorInvalidValue;
  sp.D = p.D;
  sp.status = p.status;
  sp.B = p.B;
  sp.U = p.U;
  sp.Ceff = p.Ceff;
  sp.n_sc = p.n_sc;
  sp.n_sym = p.n_sym;
  // The next slice is converted while the current one is consumed: two slices at least.
  sp.ring = p.stages < 2 ? 2 : (p.stages > kStreamMaxRing ? kStreamMaxRing : p.stages);
  const bool f16 = precision == FFEQ_FP16X3;
  switch (padded_users(p.U)) {
    case 8: return f16 ? launch_stream_up<8, kFp16x3>(sp, stream) : launch_stream_up<8, kBf16x3>(sp, stream);
    case 16: return f16 ? launch_stream_up<16, kFp16x3>(sp, stream) : launch_stream_up<16, kBf16x3>(sp, stream);
    default: return f16 ? launch_stream_up<32, kFp16x3>(sp, stream) : launch_stream_up<32, kBf16x3>(sp, stream);
  }
}

}  // namespace ffeq
