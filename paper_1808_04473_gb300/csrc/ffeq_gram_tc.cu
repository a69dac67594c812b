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
//   kBf16x3: mma.m16n8k16 BF16 (8-bit significands: hi+lo carries ~16 bits).
#include <cstdint>

#include "ffeq_gram.cuh"

namespace ffeq {
namespace {

constexpr int kTf32x3 = 1;
constexpr int kBf16x3 = 2;

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

// Two floats -> bf16x2 hi and lo (element 0 in the low half, as the MMA expects).
__device__ __forceinline__ void split_bf16(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x1), "f"(x0));
  const float h0 = __uint_as_float(hi << 16);
  const float h1 = __uint_as_float(hi & 0xffff0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(x1 - h1), "f"(x0 - h0));
}

// Not volatile: the compiler may interleave MMAs on independent accumulators.
__device__ __forceinline__ void mma_tf32(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <int MODE>
__device__ __forceinline__ void mma_any(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  if constexpr (MODE == kTf32x3) mma_tf32(c, a, b0, b1);
  else mma_bf16(c, a, b0, b1);
}

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
        split_bf16(v0.x, v1.x, bre_h[j][0], bre_l[j][0]);
        split_bf16(v2_.x, v3.x, bre_h[j][1], bre_l[j][1]);
        split_bf16(v0.y, v1.y, bim_h[j][0], bim_l[j][0]);
        split_bf16(v2_.y, v3.y, bim_h[j][1], bim_l[j][1]);
        split_bf16(v0.x - v0.y, v1.x - v1.y, bd_h[j][0], bd_l[j][0]);
        split_bf16(v2_.x - v2_.y, v3.x - v3.y, bd_h[j][1], bd_l[j][1]);
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
            split_bf16(w0[q].x, w1[q].x, are_h[q], are_l[q]);
            split_bf16(w0[q].y, w1[q].y, aim_h[q], aim_l[q]);
            split_bf16(w0[q].x + w0[q].y, w1[q].x + w1[q].y, as_h[q], as_l[q]);
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

template <int MODE>
struct TensorSplit {
  static constexpr int kWarps = 16;
  static constexpr bool kSplitM = true;
  template <int UP, typename Out>
  __device__ __forceinline__ static void run(const float2* __restrict__ Ws, int RS, int Mrows, int U, int k0,
                                             int k1, bool vec, int lane, int mt, Out out) {
    tc_tiles<UP, MODE>(Ws, RS, Mrows, U, k0, k1, vec, lane, mt, out);
  }
};

template <int MODE>
cudaError_t launch_mode(const GramParams& p, size_t smem, cudaStream_t stream) {
  switch (padded_users(p.U)) {
    case 8: return launch_gram_up<8, TensorSplit<MODE>>(p, smem, stream);
    case 16: return launch_gram_up<16, TensorSplit<MODE>>(p, smem, stream);
    default: return launch_gram_up<32, TensorSplit<MODE>>(p, smem, stream);
  }
}

}  // namespace

void gram_tc_capacity(int B, int U, int n_sym, int Ceff, int& stage_elems, int& slot_elems, int& slots) {
  gram_capacity<TensorSplit<kBf16x3>>(B, U, n_sym, Ceff, stage_elems, slot_elems, slots);
}

cudaError_t launch_gram_tc(const GramParams& p, int precision, cudaStream_t stream) {
  const size_t smem = gram_smem_bytes(p);
  return precision == FFEQ_TF32X3 ? launch_mode<kTf32x3>(p, smem, stream) : launch_mode<kBf16x3>(p, smem, stream);
}

}  // namespace ffeq
