// Local preprocessing (Sec. II-C) on the tensor cores with split-precision
// operands: the complex contraction D = H_c^H [H_c ; Y_c] of the persistent
// kernel in ffeq_gram.cuh, written as one real GEMM per cluster and computed
// with warp-level mma.sync.
//
// Real form.  For conj(h) w with h = H[u][b], w = W[m][b] (W = [H; Y] rows),
// Gauss's three real products per block of antennas
//   T1 = sum w_re h_re,  T2 = sum w_im h_im,  T3 = sum (w_re + w_im)(h_re - h_im)
// give Re D = T1 + T2 and Im D = T3 - T1 + T2, i.e. three real GEMMs
// C_q = A_q B_q with rows m of A_q from W and columns u of B_q from H.  The
// fragments of all three are formed in registers from the same staged values,
// so every staged element is read from shared memory once per warp and never
// rewritten.
//
// Split precision.  Each FP32 operand x is split in registers into hi + lo
// (hi = x rounded to the MMA type, lo = the rounded remainder) and the product
// accumulates A_lo B_hi + A_hi B_lo + A_hi B_hi in FP32 (the lo*lo term is
// dropped):
//   kTf32x3: mma.m16n8k8 TF32 (11-bit significands: hi+lo carries ~22 bits);
//   kBf16x3: mma.m16n8k16 BF16 (8-bit significands: hi+lo carries ~16 bits);
//   kFp16x3: mma.m16n8k16 FP16 (11-bit significands, FP16's range).
#include <cstdint>

#include "ffeq_gram.cuh"
#include "ffeq_mma.cuh"

namespace ffeq {
namespace {

// Complex value of row `row` at antenna a, zero outside [.., k1).
__device__ __forceinline__ float2 ld(const float2* __restrict__ row, int a, int k1) {
  return a < k1 ? row[a] : make_float2(0.f, 0.f);
}

// Antennas a and a+1 (a even, rows 16-byte aligned when vec): one 16-byte load.
__device__ __forceinline__ void ld2(const float2* __restrict__ row, int a, int k1, bool vec, float2& v0, float2& v1) {
  if (vec && a + 1 < k1) {
    const float4 q = *reinterpret_cast<const float4*>(row + a);
    v0 = make_float2(q.x, q.y);
    v1 = make_float2(q.z, q.w);
  } else {
    v0 = ld(row, a, k1);
    v1 = ld(row, a + 1, k1);
  }
}

// One warp: rows [16 mtile, 16 mtile + 16) of D over antennas [k0, k1) (H rows
// then Y rows; rows >= Mrows read row 0 and are dropped), NX = UP/8 tiles of 8
// users for the real parts (x) and NX for the imaginary parts (r).
template <int UP, int MODE, typename Out>
__device__ __forceinline__ void tc_tiles(const float2* __restrict__ Ws, int RS, int Mrows, int U, int k0, int k1,
                                         bool vec, int lane, int mtile, Out out) {
  constexpr int NX = UP / 8;
  constexpr int MTMAX = 1;                       // one 16-row m-tile per call
  constexpr int KB = MODE == kTf32x3 ? 8 : 16;   // antennas per MMA k-step pair (re, im)
  const int MT = 1;
  const int mbase = mtile * 16;
  const int g = lane >> 2, t = lane & 3;

  // Gauss's three-product complex multiply: with T1 = A_re B_re, T2 = A_im B_im and
  // T3 = (A_re + A_im)(B_re - B_im), Re D = T1 + T2 and Im D = T3 - T1 + T2.
  // acc[i][3j + q] holds T_{q+1} of user tile j.
  float acc[MTMAX][3 * NX][4];
#pragma unroll
  for (int i = 0; i < MTMAX; ++i)
#pragma unroll
    for (int j = 0; j < 3 * NX; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

  const float2* arow[MTMAX][2];
#pragma unroll
  for (int i = 0; i < MTMAX; ++i)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = mbase + i * 16 + g + 8 * h;
      arow[i][h] = Ws + (m < Mrows ? m : 0) * RS;
    }
  const float2* brow[NX];
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    const int u = j * 8 + g;
    brow[j] = Ws + (u < U ? u : 0) * RS;
  }
  // Pair loads need an even start: true for even cluster starts with even rows.
  const bool v2 = vec && ((k0 & 1) == 0);

  for (int a0 = k0; a0 < k1; a0 += KB) {
    // B fragments: re, im and re - im parts, hi and lo.
    uint32_t bre_h[NX][2], bre_l[NX][2], bim_h[NX][2], bim_l[NX][2], bd_h[NX][2], bd_l[NX][2];
#pragma unroll
    for (int j = 0; j < NX; ++j) {
      if constexpr (MODE == kTf32x3) {
        const float2 v0 = ld(brow[j], a0 + t, k1), v1 = ld(brow[j], a0 + t + 4, k1);
        split_tf32(v0.x, bre_h[j][0], bre_l[j][0]);
        split_tf32(v1.x, bre_h[j][1], bre_l[j][1]);
        split_tf32(v0.y, bim_h[j][0], bim_l[j][0]);
        split_tf32(v1.y, bim_h[j][1], bim_l[j][1]);
        split_tf32(v0.x - v0.y, bd_h[j][0], bd_l[j][0]);
        split_tf32(v1.x - v1.y, bd_h[j][1], bd_l[j][1]);
      } else {
        float2 v0, v1, v2_, v3;
        ld2(brow[j], a0 + 2 * t, k1, v2, v0, v1);
        ld2(brow[j], a0 + 8 + 2 * t, k1, v2, v2_, v3);
        split_pair<MODE>(v0.x, v1.x, bre_h[j][0], bre_l[j][0]);
        split_pair<MODE>(v2_.x, v3.x, bre_h[j][1], bre_l[j][1]);
        split_pair<MODE>(v0.y, v1.y, bim_h[j][0], bim_l[j][0]);
        split_pair<MODE>(v2_.y, v3.y, bim_h[j][1], bim_l[j][1]);
        split_pair<MODE>(v0.x - v0.y, v1.x - v1.y, bd_h[j][0], bd_l[j][0]);
        split_pair<MODE>(v2_.x - v2_.y, v3.x - v3.y, bd_h[j][1], bd_l[j][1]);
      }
    }
#pragma unroll
    for (int i = 0; i < MTMAX; ++i) {
      if (i < MT) {
        uint32_t are_h[4], are_l[4], aim_h[4], aim_l[4], as_h[4], as_l[4];
        if constexpr (MODE == kTf32x3) {
          // a0: (g, t)  a1: (g+8, t)  a2: (g, t+4)  a3: (g+8, t+4)
          float2 w[4];
          w[0] = ld(arow[i][0], a0 + t, k1);
          w[1] = ld(arow[i][1], a0 + t, k1);
          w[2] = ld(arow[i][0], a0 + t + 4, k1);
          w[3] = ld(arow[i][1], a0 + t + 4, k1);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            split_tf32(w[q].x, are_h[q], are_l[q]);
            split_tf32(w[q].y, aim_h[q], aim_l[q]);
            split_tf32(w[q].x + w[q].y, as_h[q], as_l[q]);
          }
        } else {
          // a0: (g, 2t..2t+1)  a1: (g+8, 2t..)  a2: (g, 8+2t..)  a3: (g+8, 8+2t..)
          float2 w0[4], w1[4];
          ld2(arow[i][0], a0 + 2 * t, k1, v2, w0[0], w1[0]);
          ld2(arow[i][1], a0 + 2 * t, k1, v2, w0[1], w1[1]);
          ld2(arow[i][0], a0 + 8 + 2 * t, k1, v2, w0[2], w1[2]);
          ld2(arow[i][1], a0 + 8 + 2 * t, k1, v2, w0[3], w1[3]);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            split_pair<MODE>(w0[q].x, w1[q].x, are_h[q], are_l[q]);
            split_pair<MODE>(w0[q].y, w1[q].y, aim_h[q], aim_l[q]);
            split_pair<MODE>(w0[q].x + w0[q].y, w1[q].x + w1[q].y, as_h[q], as_l[q]);
          }
        }
        // Issue order: one split product (A_lo B_hi, A_hi B_lo, A_hi B_hi) at a
        // time over every accumulator tile, so consecutive MMAs never wait on
        // each other.
#pragma unroll
        for (int prod = 0; prod < 3; ++prod) {
          const uint32_t(&ar)[4] = prod == 0 ? are_l : are_h;
          const uint32_t(&ai)[4] = prod == 0 ? aim_l : aim_h;
          const uint32_t(&as)[4] = prod == 0 ? as_l : as_h;
#pragma unroll
          for (int j = 0; j < NX; ++j) {
            mma_any<MODE>(acc[i][3 * j], ar, prod == 1 ? bre_l[j][0] : bre_h[j][0],
                          prod == 1 ? bre_l[j][1] : bre_h[j][1]);
            mma_any<MODE>(acc[i][3 * j + 1], ai, prod == 1 ? bim_l[j][0] : bim_h[j][0],
                          prod == 1 ? bim_l[j][1] : bim_h[j][1]);
            mma_any<MODE>(acc[i][3 * j + 2], as, prod == 1 ? bd_l[j][0] : bd_h[j][0],
                          prod == 1 ? bd_l[j][1] : bd_h[j][1]);
          }
        }
      }
    }
  }
  // c0: (g, 2t)  c1: (g, 2t+1)  c2: (g+8, 2t)  c3: (g+8, 2t+1): each lane owns the
  // users pair (2t, 2t+1) of rows g and g+8 -- one 16-byte store per row.
#pragma unroll
  for (int i = 0; i < MTMAX; ++i) {
    if (i < MT) {
#pragma unroll
      for (int j = 0; j < NX; ++j) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int m = mbase + i * 16 + g + 8 * h;
          const int u = j * 8 + 2 * t;
          if (m < Mrows && u < U) {
            const float* t1 = acc[i][3 * j];
            const float* t2 = acc[i][3 * j + 1];
            const float* t3 = acc[i][3 * j + 2];
            const int q0 = 2 * h, q1 = 2 * h + 1;
            out(m, u, make_float2(t1[q0] + t2[q0], t3[q0] - t1[q0] + t2[q0]),
                make_float2(t1[q1] + t2[q1], t3[q1] - t1[q1] + t2[q1]), u + 1 < U);
          }
        }
      }
    }
  }
}

template <int MODE, int WARPS = 16, int MINB = 1>
struct TensorSplit {
  static constexpr bool kPrep = false;
  static constexpr bool kDense = true;
  static constexpr int kWarps = WARPS;
  static constexpr int kMinBlocks = MINB;
  static constexpr bool kSplitM = true;
  template <int UP, typename Out>
  __device__ __forceinline__ static void run(const float2* __restrict__ Ws, int RS, int Mrows, int U, int k0,
                                             int k1, bool vec, int lane, int mt, Out out) {
    tc_tiles<UP, MODE>(Ws, RS, Mrows, U, k0, k1, vec, lane, mt, out);
  }
};

// ---------------------------------------------------------------------------
// Pre-split BF16x3.  The staged FP32 rows of a unit are converted once, by all
// warps, into four BF16 planes [plane][row][PS]: re hi, re lo, im hi, im lo
// (hi = x rounded to BF16, lo = the rounded remainder), cluster segments
// padded with zeros to whole 16-antenna k-steps (presplit_seg).  Fragments then
// come straight from the planes with ldmatrix: rows m of W = [H; Y] are the A
// operand (16 x 16 tile: one ldmatrix.x4 per plane), rows u < U of the same
// planes the B operand (two 8-user tiles per ldmatrix.x4).  The complex
// product conj(h) w takes four real products,
//   Re D = sum w_re h_re + w_im h_im,   Im D = sum w_im h_re + w_re (-h_im),
// each split as A_lo B_hi + A_hi B_lo + A_hi B_hi (the lo*lo term is dropped),
// with -h_im formed by flipping the BF16 sign bits (exact).  Compared with
// splitting in registers per fragment, every staged element is converted once
// per unit instead of once per warp that reads it, and a k-step costs 8-12
// ldmatrix + 12 NX mma instead of ~160 load/convert instructions.

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r0), "=r"(r1) : "r"(addr));
}

struct TensorSplitPre {
  static constexpr bool kPrep = true;
  static constexpr bool kDense = true;
  static constexpr int kWarps = 16;
  static constexpr int kMinBlocks = 1;
  static constexpr bool kSplitM = true;

  // Rows [0, Mrows) of the stage -> planes; four antennas per thread item.
  __device__ __forceinline__ static void prep(const float2* __restrict__ Ws, int RS, int Mrows, int B, int Ceff,
                                              uint16_t* __restrict__ planes, int PS, int SP, int tid, int nthr) {
    const int S = B / Ceff;
    const int qpc = SP / 4;              // quads per cluster segment (with padding)
    const int quads = Ceff * qpc;
    const int plane = Mrows * PS;
    for (int e = tid; e < Mrows * quads; e += nthr) {
      const int m = e / quads, qq = e - m * quads;
      const int c = qq / qpc, a = (qq - c * qpc) * 4;
      uint2 rh = make_uint2(0u, 0u), rl = rh, ih = rh, il = rh;
      if (a < S) {
        const float4* src = reinterpret_cast<const float4*>(Ws + m * RS + c * S + a);
        const float4 v01 = src[0], v23 = src[1];
        split_bf16(v01.x, v01.z, rh.x, rl.x);
        split_bf16(v23.x, v23.z, rh.y, rl.y);
        split_bf16(v01.y, v01.w, ih.x, il.x);
        split_bf16(v23.y, v23.w, ih.y, il.y);
      }
      const int off = m * PS + c * SP + a;
      *reinterpret_cast<uint2*>(planes + off) = rh;
      *reinterpret_cast<uint2*>(planes + plane + off) = rl;
      *reinterpret_cast<uint2*>(planes + 2 * plane + off) = ih;
      *reinterpret_cast<uint2*>(planes + 3 * plane + off) = il;
    }
  }

  // One warp: rows [16 mt, 16 mt + 16) of D over plane columns [k0, k1) (whole
  // 16-steps), all UP users in NX = UP/8 tiles.
  template <int UP, typename Out>
  __device__ __forceinline__ static void run(const uint16_t* __restrict__ planes, int PS, int Mrows, int U, int k0,
                                             int k1, int lane, int mt, Out out) {
    constexpr int NX = UP / 8;
    constexpr int NB = (NX + 1) / 2;     // ldmatrix loads per plane for the B tiles
    const uint32_t pbytes = static_cast<uint32_t>(Mrows * PS) * 2u;
    // A: lane -> matrix lane/8 (rows +8 for odd, k +8 for the upper two), row lane%8.
    const int ar = 16 * mt + (lane & 7) + ((lane >> 3) & 1) * 8;
    const uint32_t a_base = smem_u32(planes + (ar < Mrows ? ar : 0) * PS + ((lane >> 4) & 1) * 8);
    // B: lane -> users 16 jb + (lane/16)*8 + lane%8, k +8 for odd matrices.
    uint32_t b_base[NB];
#pragma unroll
    for (int jb = 0; jb < NB; ++jb) {
      const int bn = jb * 16 + ((lane >> 4) & 1) * 8 + (lane & 7);
      b_base[jb] = smem_u32(planes + (bn < U ? bn : 0) * PS + ((lane >> 3) & 1) * 8);
    }
    float are[NX][4], aim[NX][4];
#pragma unroll
    for (int j = 0; j < NX; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) are[j][q] = aim[j][q] = 0.f;

    for (int k = k0; k < k1; k += 16) {
      const uint32_t kb = static_cast<uint32_t>(k) * 2u;
      uint32_t A[4][4];                  // plane: re hi, re lo, im hi, im lo
#pragma unroll
      for (int pl = 0; pl < 4; ++pl) ldsm_x4(a_base + pl * pbytes + kb, A[pl][0], A[pl][1], A[pl][2], A[pl][3]);
      uint32_t Bf[4][NX][2];
#pragma unroll
      for (int pl = 0; pl < 4; ++pl) {
#pragma unroll
        for (int jb = 0; jb < NB; ++jb) {
          if (2 * jb + 1 < NX) {
            ldsm_x4(b_base[jb] + pl * pbytes + kb, Bf[pl][2 * jb][0], Bf[pl][2 * jb][1], Bf[pl][2 * jb + 1][0],
                    Bf[pl][2 * jb + 1][1]);
          } else {
            ldsm_x2(b_base[jb] + pl * pbytes + kb, Bf[pl][2 * jb][0], Bf[pl][2 * jb][1]);
          }
        }
      }
      // Split products, issued one split term at a time over all accumulators.
#pragma unroll
      for (int prod = 0; prod < 3; ++prod) {
        const int ah = prod == 0 ? 1 : 0;      // A_lo B_hi, A_hi B_lo, A_hi B_hi
        const int bh = prod == 1 ? 1 : 0;
#pragma unroll
        for (int j = 0; j < NX; ++j) {
          const uint32_t nb0 = Bf[2 + bh][j][0] ^ 0x80008000u, nb1 = Bf[2 + bh][j][1] ^ 0x80008000u;
          mma_bf16(are[j], A[0 + ah], Bf[0 + bh][j][0], Bf[0 + bh][j][1]);   // w_re h_re
          mma_bf16(aim[j], A[2 + ah], Bf[0 + bh][j][0], Bf[0 + bh][j][1]);   // w_im h_re
          mma_bf16(are[j], A[2 + ah], Bf[2 + bh][j][0], Bf[2 + bh][j][1]);   // w_im h_im
          mma_bf16(aim[j], A[0 + ah], nb0, nb1);                             // w_re (-h_im)
        }
      }
    }
    // c0: (g, 2t)  c1: (g, 2t+1)  c2: (g+8, 2t)  c3: (g+8, 2t+1)
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < NX; ++j) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = 16 * mt + g + 8 * h;
        const int u = j * 8 + 2 * t;
        if (m < Mrows && u < U)
          out(m, u, make_float2(are[j][2 * h], aim[j][2 * h]), make_float2(are[j][2 * h + 1], aim[j][2 * h + 1]),
              u + 1 < U);
      }
    }
  }
};

template <int MODE, int WARPS, int MINB>
cudaError_t launch_mode(const GramParams& p, size_t smem, cudaStream_t stream) {
  switch (padded_users(p.U)) {
    case 8: return launch_gram_up<8, TensorSplit<MODE, WARPS, MINB>>(p, smem, stream);
    case 16: return launch_gram_up<16, TensorSplit<MODE, WARPS, MINB>>(p, smem, stream);
    default: return launch_gram_up<32, TensorSplit<MODE, WARPS, MINB>>(p, smem, stream);
  }
}

}  // namespace

GramCaps gram_tc_caps(int B, int U, int n_sym, int Ceff, int variant) {
  GramCaps c{};
  if (variant == kGram8x2) {
    gram_capacity<TensorSplit<kBf16x3, 8, 2>>(B, U, n_sym, Ceff, c.stage_elems, c.slot_elems, c.slots);
  } else if (variant == kGram4x3) {
    gram_capacity<TensorSplit<kBf16x3, 4, 3>>(B, U, n_sym, Ceff, c.stage_elems, c.slot_elems, c.slots);
  } else {
    gram_capacity<TensorSplit<kBf16x3>>(B, U, n_sym, Ceff, c.stage_elems, c.slot_elems, c.slots);
  }
  if (variant == kGramPresplit) c.plane_bytes = 4 * (U + n_sym) * presplit_row(B, Ceff) * 2;
  return c;
}

cudaError_t launch_gram_tc(const GramParams& p, int precision, cudaStream_t stream) {
  if (p.variant == kGramStream || p.variant == kGramStreamHalf) return launch_gram_stream(p, precision, stream);
  const size_t smem = gram_smem_bytes(p);
  if (precision == FFEQ_FP16X3) return launch_mode<kFp16x3, 16, 1>(p, smem, stream);   // the 16-warp shape only
  if (precision == FFEQ_BF16X3 && p.variant == kGramPresplit && p.plane_bytes > 0) {
    switch (padded_users(p.U)) {
      case 8: return launch_gram_up<8, TensorSplitPre>(p, smem, stream);
      case 16: return launch_gram_up<16, TensorSplitPre>(p, smem, stream);
      default: return launch_gram_up<32, TensorSplitPre>(p, smem, stream);
    }
  }
  if (p.variant == kGram8x2) {
    return precision == FFEQ_TF32X3 ? launch_mode<kTf32x3, 8, 2>(p, smem, stream)
                                    : launch_mode<kBf16x3, 8, 2>(p, smem, stream);
  }
  if (p.variant == kGram4x3) {
    return precision == FFEQ_TF32X3 ? launch_mode<kTf32x3, 4, 3>(p, smem, stream)
                                    : launch_mode<kBf16x3, 4, 3>(p, smem, stream);
  }
  return precision == FFEQ_TF32X3 ? launch_mode<kTf32x3, 16, 1>(p, smem, stream)
                                  : launch_mode<kBf16x3, 16, 1>(p, smem, stream);
}

}  // namespace ffeq
