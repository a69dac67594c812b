// Local preprocessing (Sec. II-C) in FP32 on the CUDA cores: the warp-tiled
// complex contraction D = H_c^H [H_c ; Y_c] of the persistent kernel in
// ffeq_gram.cuh, plus the sizing shared by all contraction variants.
#include "ffeq_gram.cuh"

namespace ffeq {

__device__ int g_device_status = 0;

namespace {


// Accumulate this lane's 4x4 tiles of D over antennas [k0, k1).  Tile t covers
// rows m = mg + NMG*i and users u = ug + NUG*j: the lanes of a warp read
// consecutive shared-memory rows, whose stride (B+2 complex) shifts the bank by
// 16 bytes per row, so the loads never conflict.  out(m, u, value) stores.
template <int UP, typename Out>
__device__ __forceinline__ void simt_tiles(const float2* __restrict__ Ws, int RS, int Mrows, int U, int k0,
                                               int k1, bool vec, int lane, Out out) {
  constexpr int NUG = UP / 4;
  const int NMG = (Mrows + 3) / 4;
  for (int t = lane; t < NMG * NUG; t += 32) {
    const int ug = t % NUG, mg = t / NUG;
    const float2* ur[4];
    const float2* mr[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int u = ug + NUG * j;
      ur[j] = Ws + (u < U ? u : 0) * RS;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = mg + NMG * i;
      mr[i] = Ws + (m < Mrows ? m : 0) * RS;
    }
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

    int k = k0;
    if (vec) {
      if ((k & 1) && k < k1) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = cfma_conj(ur[j][k], mr[i][k], acc[i][j]);
        ++k;
      }
#pragma unroll 2
      for (; k + 1 < k1; k += 2) {
        float4 a[4], w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) a[j] = *reinterpret_cast<const float4*>(ur[j] + k);
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = *reinterpret_cast<const float4*>(mr[i] + k);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j] = cfma_conj(make_float2(a[j].x, a[j].y), make_float2(w[i].x, w[i].y), acc[i][j]);
            acc[i][j] = cfma_conj(make_float2(a[j].z, a[j].w), make_float2(w[i].z, w[i].w), acc[i][j]);
          }
      }
    }
    for (; k < k1; ++k) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = cfma_conj(ur[j][k], mr[i][k], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int m = mg + NMG * i, u = ug + NUG * j;
        if (m < Mrows && u < U) out(m, u, acc[i][j], acc[i][j], false);
      }
  }
}

// Contraction policy for gram_kernel: CUDA-core FP32 (MINB CTAs per SM).
template <int MINB>
struct SimtFp32 {
  static constexpr int kWarps = 8;
  static constexpr int kMinBlocks = MINB;
  static constexpr bool kSplitM = false;
  static constexpr bool kPrep = false;
  static constexpr bool kDense = false;
  template <int UP, typename Out>
  __device__ __forceinline__ static void run(const float2* __restrict__ Ws, int RS, int Mrows, int U, int k0,
                                             int k1, bool vec, int lane, int /*mt*/, Out out) {
    simt_tiles<UP>(Ws, RS, Mrows, U, k0, k1, vec, lane, out);
  }
};

}  // namespace

int padded_users(int U) { return U <= 8 ? 8 : (U <= 16 ? 16 : 32); }

bool gram_presplit_eligible(int precision, int B, int Ceff) {
  return precision == FFEQ_BF16X3 && B % 4 == 0 && Ceff > 0 && B % Ceff == 0 && (B / Ceff) % 4 == 0;
}

size_t gram_smem_budget(int variant) {
  // CTAs per SM share 228 KB, less 1 KB reserved per CTA.
  if (variant == kGram8x2) return 113 * 1024;
  if (variant == kGram4x3) return 75 * 1024;
  return kGramSmemBudget;
}

GramCaps gram_instance_caps(int precision, int B, int U, int n_sym, int Ceff, int variant) {
  if (precision == FFEQ_FP32) {
    GramCaps c{};
    if (variant == kGram8x2 || variant == kGram4x3)
      gram_capacity<SimtFp32<2>>(B, U, n_sym, Ceff, c.stage_elems, c.slot_elems, c.slots);
    else
      gram_capacity<SimtFp32<1>>(B, U, n_sym, Ceff, c.stage_elems, c.slot_elems, c.slots);
    return c;
  }
  return gram_tc_caps(B, U, n_sym, Ceff, variant);
}

int gram_stages_fit_bytes(size_t stage_elems, size_t fixed_bytes, bool bulk, size_t budget) {
  return gram_stages_fit(stage_elems, fixed_bytes, bulk, budget);
}

int gram_stages(int precision, int B, int U, int n_sym, int Ceff, bool bulk) {
  const GramCaps c = gram_instance_caps(precision, B, U, n_sym, Ceff, kGram16);
  return gram_stages_fit(c.stage_elems, static_cast<size_t>(c.slots) * c.slot_elems * 8, bulk);
}

bool gram_configure(GramParams& p, int precision, int variant, int stages) {
  p.n_units = p.n_sc;
  p.desc = nullptr;
  p.queue = nullptr;
  p.UP = padded_users(p.U);
  p.lim = BatchLimits{};
  p.grid_cap = 0;
  const bool stream_ok = p.cl_uniform && gram_stream_eligible(precision, p.B, p.U, p.n_sym, p.Ceff);
  // Default: the streamed shape where it applies (16-byte aligned inputs),
  // else 16 warps.
  if (variant == kGramAuto) variant = stream_ok && p.bulk ? kGramStream : kGram16;
  if (variant < kGram16 || variant > kGramVariantMax) return false;
  if (variant == kGramFused) {
    // The contraction of the fused shape is the streamed one with a ring of 2
    // (what ffeq_local_preprocess runs; ffeq_equalize fuses the solve into it).
    if (!stream_ok || !gram_fused_eligible(precision, p.B, p.U, p.n_sym, p.Ceff)) return false;
    if (stages != 0 && stages != kGramFusedRing) return false;
    variant = kGramStream;
    stages = kGramFusedRing;
  }
  if (variant == kGram4x3 && precision == FFEQ_FP32) return false;   // CUDA-core shapes: 16 (8 warps) and 8x2
  if (precision == FFEQ_FP16X3 && variant != kGram16 && variant != kGramStream && variant != kGramStreamHalf)
    return false;
  if (variant == kGramPresplit && (!p.cl_uniform || !gram_presplit_eligible(precision, p.B, p.Ceff))) return false;
  if ((variant == kGramStream || variant == kGramStreamHalf) && !stream_ok) return false;
  if (variant != kGramStream && variant != kGramStreamHalf && stages > kGramMaxStages) return false;
  if (!p.bulk) {              // plain-load staging: one stage, no pre-split planes, no tensor maps
    if (variant == kGramPresplit || variant == kGramStream || variant == kGramStreamHalf) variant = kGram16;
    stages = 0;
  }
  if (variant == kGramStream || variant == kGramStreamHalf) {
    if (stages == 1) return false;          // the streamed shape converts one slice ahead
    p.stage_elems = p.slot_elems = p.n_slots = p.plane_bytes = 0;
    p.stages = stages > 0 ? stages : kGramStreamRing;
    p.variant = variant;
    return true;
  }
  const GramCaps c = gram_instance_caps(precision, p.B, p.U, p.n_sym, p.Ceff, variant);
  const int fit = gram_stages_fit(c.stage_elems, static_cast<size_t>(c.slots) * c.slot_elems * 8 + c.plane_bytes,
                                  p.bulk != 0, gram_smem_budget(variant));
  if (fit < 1 || stages > fit) return false;
  p.stage_elems = c.stage_elems;
  p.slot_elems = c.slot_elems;
  p.n_slots = c.slots;
  p.plane_bytes = c.plane_bytes;
  p.stages = stages > 0 ? stages : fit;
  p.variant = variant;
  return true;
}

cudaError_t launch_gram_fp32(const GramParams& p, cudaStream_t stream) {
  const size_t smem = gram_smem_bytes(p);
  if (p.variant == kGram8x2) {
    switch (padded_users(p.U)) {
      case 8: return launch_gram_up<8, SimtFp32<2>>(p, smem, stream);
      case 16: return launch_gram_up<16, SimtFp32<2>>(p, smem, stream);
      default: return launch_gram_up<32, SimtFp32<2>>(p, smem, stream);
    }
  }
  switch (padded_users(p.U)) {
    case 8: return launch_gram_up<8, SimtFp32<1>>(p, smem, stream);
    case 16: return launch_gram_up<16, SimtFp32<1>>(p, smem, stream);
    default: return launch_gram_up<32, SimtFp32<1>>(p, smem, stream);
  }
}

int* device_status_ptr() {
  static SymbolAddressCache cache;
  cudaError_t e = cudaSuccess;
  void* p = cached_symbol_address(
      cache, [](void** out) { return cudaGetSymbolAddress(out, g_device_status); }, &e);
  return static_cast<int*>(p);
}

}  // namespace ffeq
