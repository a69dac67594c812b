// Persistent local-preprocessing kernel skeleton shared by the CUDA-core and
// tensor-core contractions (see ffeq_gram_fp32.cu and ffeq_gram_tc.cu).
//
// For every subcarrier k and antenna cluster c (Sec. II-C) the contraction
//     D_{k,c}[m][u] = sum_{b in cluster c} conj(H_k[u][b]) * W_k[m][b],
//     W_k = [H_k ; Y_k]  (rows 0..U-1: channel rows, rows U..U+n_sym-1: receive rows)
// gives the local Gram matrix G_c[u][v] = D[v][u] (v < U) and the local MRC
// outputs y_c^MRC[u] = D[U+n][u] for OFDM symbol n.  PD sums all clusters (the
// adder tree of Eq. fullMRC) on chip as a split-K reduction over the warps of
// the CTA; FD keeps one D per cluster.  D goes to the workspace
// [n_sc][Ceff][U + n_sym][U] complex, Ceff = C (FD) or 1 (PD).
//
// One CTA per SM walks subcarriers b, b + gridDim.x, ...; the U + n_sym rows of
// B complex of each are staged into shared memory on a per-stage mbarrier, up
// to three subcarriers ahead of the contraction: densely with two cp.async.bulk
// copies (the H block, the y block) for the tensor-core contractions, with row
// stride B + 2 and one copy per row for the CUDA-core one.  Clusters are B / C
// antennas each, or of the sizes given to the plan (offsets cl_off).  The
// default tensor-core shape is the streamed kernel of ffeq_gram_stream.cu.
#pragma once

#include "ffeq_device.cuh"
#include "ffeq_internal.h"

namespace ffeq {

constexpr int kGramHeaderBytes = 128;
constexpr int kGramMaxStages = 3;
constexpr size_t kGramSmemBudget = 227 * 1024;

// Work items of one subcarrier: (cluster c, K-part p, m-tile mt).  A contraction
// policy either covers all rows of D per item (kSplitM = false: nM = 1) or one
// 16-row m-tile per item (nM = ceil(Mrows/16)).  K-parts split each cluster's
// antennas when there are fewer items than warps; their partial sums meet in
// shared-memory slots (one per cluster and part) and are reduced in a fixed
// order, so the result does not depend on scheduling.
struct GramSplit {
  int nM, P, slots;
};

__host__ __device__ inline GramSplit gram_split(int Ceff, int Mrows, int warps, bool splitM) {
  GramSplit g;
  g.nM = splitM ? (Mrows + 15) / 16 : 1;
  const int base = Ceff * g.nM;
  g.P = base >= warps ? 1 : warps / base;
  g.slots = g.P > 1 ? Ceff * g.P : 0;
  return g;
}

// Pre-split planes: each cluster's S antennas padded to SP = 16 * ceil(S / 16)
// (whole 16-antenna k-steps, zero-filled), a row holds the Ceff segments plus 8
// elements, so that rows are 16-byte aligned and ldmatrix reads of 8 rows fall
// in distinct bank groups (the row stride is an odd multiple of 16 bytes).
__host__ __device__ inline int presplit_seg(int B, int Ceff) { return ((B / Ceff + 15) / 16) * 16; }
__host__ __device__ inline int presplit_row(int B, int Ceff) { return Ceff * presplit_seg(B, Ceff) + 8; }

// One unit of work: a subcarrier of a uniform problem, or one descriptor of an
// uneven batch (sizes and pointers from the descriptor, checked against the
// group's shared-memory capacities and the buffers' extents).
struct GramUnit {
  int B, U, NS, Ceff;
  bool ok;
  const float2* H;
  const float2* y;
  float2* D;
};

template <bool BATCH>
__device__ __forceinline__ GramUnit gram_unit(const GramParams& p, int t, int warps, bool splitM, bool dense) {
  GramUnit u;
  if constexpr (BATCH) {
    const BatchDesc& d = p.desc[t];
    u.B = d.B; u.U = d.U; u.NS = d.n_sym; u.Ceff = d.Ceff;
    const int Mrows = u.U + u.NS;
    // (d_off even: the paired float4 stores below need 16-byte aligned rows.)
    bool ok = (d.d_off & 1) == 0 && u.U >= 1 && u.U <= p.UP && u.NS >= 1 && u.NS <= kNsymMax && u.B >= 1 && u.B <= (1 << 20) &&
              u.Ceff >= 1 &&
              u.B % u.Ceff == 0 && Mrows * (dense ? u.B : u.B + 2) <= p.stage_elems;
    if (ok) {
      const GramSplit sp = gram_split(u.Ceff, Mrows, warps, splitM);
      ok = sp.slots <= p.n_slots && (sp.slots == 0 || Mrows * (p.UP + 1) <= p.slot_elems) &&
           span_ok(d.h_off, static_cast<long long>(u.U) * u.B, p.lim.h) &&
           span_ok(d.y_off, static_cast<long long>(u.NS) * u.B, p.lim.y) &&
           span_ok(d.d_off, static_cast<long long>(u.Ceff) * Mrows * u.U, p.lim.d) &&
           (!p.bulk || ((u.B & 1) == 0 && (d.h_off & 1) == 0 && (d.y_off & 1) == 0)) &&
           (p.plane_bytes == 0 ||
            ((u.B & 3) == 0 && ((u.B / u.Ceff) & 3) == 0 &&
             4ll * Mrows * presplit_row(u.B, u.Ceff) * 2 <= static_cast<long long>(p.plane_bytes)));
    }
    u.ok = ok;
    u.H = p.H + d.h_off; u.y = p.y + d.y_off; u.D = p.D + d.d_off;
  } else {
    u.B = p.B; u.U = p.U; u.NS = p.n_sym; u.Ceff = p.Ceff;
    u.ok = true;
    u.H = p.H + static_cast<size_t>(t) * p.U * p.B;
    u.y = p.y + static_cast<size_t>(t) * p.n_sym * p.B;
    u.D = p.D + static_cast<size_t>(t) * p.Ceff * (p.U + p.n_sym) * p.U;
  }
  return u;
}

// Stage a unit's U + n_sym rows into `dst`, completing on `bar`.
// DENSE (row stride B): the unit's H rows and y rows are each contiguous in
// global memory, so two cp.async.bulk copies move them (issued by lane 0; each
// bulk copy has a fixed issue cost, and one per row would serialize the refill).
// Otherwise (row stride B + 2, so that consecutive rows shift by 16 bytes of bank
// offset for the CUDA-core contraction): one copy per row, spread over the lanes.
// A unit that failed its checks completes the phase with a plain arrive.
template <bool DENSE>
__device__ __forceinline__ void issue_rows(const GramUnit& w, float2* dst, uint64_t* bar, int lane) {
  if (!w.ok) {
    if (lane == 0) mbar_arrive(bar);
    return;
  }
  const int U = w.U, B = w.B, NS = w.NS;
  // H and y are read once: evict them first, keeping the workspace this kernel
  // writes in L2 for the solve kernel that reads it next.
  const uint64_t pol = l2_evict_first_policy();
  const uint32_t hb = static_cast<uint32_t>(U) * B * 8u, yb = static_cast<uint32_t>(NS) * B * 8u;
  if constexpr (DENSE) {
    if (lane == 0) {
      mbar_arrive_expect_tx(bar, hb + yb);
      bulk_g2s_hint(dst, w.H, hb, bar, pol);
      bulk_g2s_hint(dst + static_cast<size_t>(U) * B, w.y, yb, bar, pol);
    }
  } else {
    const int Mrows = U + NS, RS = B + 2;
    if (lane == 0) mbar_arrive_expect_tx(bar, hb + yb);
    __syncwarp();
    for (int r = lane; r < Mrows; r += 32) {
      const float2* src = r < U ? w.H + static_cast<size_t>(r) * B : w.y + static_cast<size_t>(r - U) * B;
      bulk_g2s_hint(dst + r * RS, src, static_cast<uint32_t>(B) * 8u, bar, pol);
    }
  }
}

// Row stride of a staged unit for contraction policy C.
template <class C>
__host__ __device__ constexpr int stage_row_stride(int B) {
  return C::kDense ? B : B + 2;
}

// Unit that follows unit t in slot order: static stride for uniform problems,
// the work queue (units sorted by decreasing cost on the host) for batches.
__device__ __forceinline__ int gram_next(const GramParams& p, int t, int nst) {
  if (p.queue) return nst * gridDim.x + atomicAdd(p.queue, 1);
  return t + nst * gridDim.x;
}

// Persistent: CTA b handles subcarriers b, b + gridDim.x, ...  With bulk
// staging, p.stages subcarriers are in flight per CTA: the loads of the next
// ones overlap the contraction of the current one.  Contract::run<UP> computes
// one warp's share of D over antennas [k0, k1) and hands each (m, u) entry to
// the output functor.
template <int UP, class Contract, bool BATCH>
__global__ void __launch_bounds__(Contract::kWarps * 32, Contract::kMinBlocks) gram_kernel(const GramParams p) {
  constexpr int kWarps = Contract::kWarps;
  constexpr int kThreads = kWarps * 32;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);                 // [p.stages]
  int* ring = reinterpret_cast<int*>(smem + 64);                      // unit of each stage
  constexpr int SU = UP + 1;
  const int nst = p.stages;
  float2* stage0 = reinterpret_cast<float2*>(smem + kGramHeaderBytes);
  const int stageSize = p.stage_elems;         // capacity of one stage (float2)
  float2* slots = stage0 + nst * stageSize;    // split-K partials (only when P > 1)
  const int slotSize = p.slot_elems;           // capacity of one partial slot (float2)
  // Pre-split planes (Contract::kPrep): [4][Mrows][PS] bf16 after the slots.
  uint16_t* planes = reinterpret_cast<uint16_t*>(slots + static_cast<size_t>(p.n_slots) * slotSize);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n_units = p.n_units;
  constexpr bool kSM = Contract::kSplitM;

  if (tid == 0) {
    for (int s = 0; s < nst; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
    for (int s = 0; s < nst; ++s) ring[s] = blockIdx.x + s * gridDim.x;
  }
  __syncthreads();
  // Prologue: fill the ring.
  if (p.bulk && warp == 0) {
    for (int s = 0; s < nst; ++s) {
      const int t = blockIdx.x + s * gridDim.x;
      if (t < n_units) {
        const GramUnit w = gram_unit<BATCH>(p, t, kWarps, kSM, Contract::kDense);
        if (!w.ok && lane == 0 && p.status) atomicExch(p.status, FFEQ_ERR_INVALID_ARG);
        issue_rows<Contract::kDense>(w, stage0 + s * stageSize, &full[s], lane);
      } else if (BATCH && lane == 0) {
        mbar_arrive(&full[s]);   // the batch loop reads the sentinel through this stage
      }
    }
  }

  for (int it = 0;; ++it) {
    const int s = it % nst;
    float2* Ws = stage0 + s * stageSize;
    if (!BATCH && blockIdx.x + it * gridDim.x >= n_units) break;   // uniform: nothing was staged
    if (p.bulk) {
      if (!mbar_wait_bounded(&full[s], (it / nst) & 1, p.status, FFEQ_ERR_TIMEOUT)) {
        // Give every copy still in flight a bounded chance to land, then leave.
        for (int q = 0; q < nst; ++q) mbar_wait_bounded(&full[q], ((it + q) / nst) & 1, nullptr, 0);
        return;
      }
    }
    // Batch: the unit handed out with this stage; uniform: static stride.
    const int t = BATCH ? ring[s] : blockIdx.x + it * gridDim.x;
    if (t >= n_units) break;
    const GramUnit w = gram_unit<BATCH>(p, t, kWarps, kSM, Contract::kDense);
    const int U = w.U, B = w.B, NS = w.NS, Ceff = w.Ceff;
    const int Mrows = U + NS, RS = stage_row_stride<Contract>(B), S = B / Ceff;
    const GramSplit sp = gram_split(Ceff, Mrows, kWarps, kSM);
    const int P = sp.P, nM = sp.nM;
    const int nItems = w.ok ? Ceff * P * nM : 0;
    const bool vec = (B & 1) == 0;
    const int matSize = Mrows * U;
    if (!p.bulk) {
      if (!w.ok && tid == 0 && p.status) atomicExch(p.status, FFEQ_ERR_INVALID_ARG);
      if (w.ok) {
        for (int e = tid; e < Mrows * B; e += kThreads) {
          const int r = e / B, b = e - r * B;
          Ws[r * RS + b] = r < U ? w.H[static_cast<size_t>(r) * B + b] : w.y[static_cast<size_t>(r - U) * B + b];
        }
      }
      __syncthreads();
    }
    // Issue the unit that follows into stage s (its data are no longer read).
    auto issue_next = [&]() {
      if constexpr (BATCH) {
        if (warp == 0) {
          const int tn = lane == 0 ? gram_next(p, t, nst) : 0;
          const int tnb = __shfl_sync(kFullMask, tn, 0);
          if (lane == 0) ring[s] = tnb;
          if (p.bulk) {
            if (tnb < n_units) {
              const GramUnit wn = gram_unit<BATCH>(p, tnb, kWarps, kSM, Contract::kDense);
              if (!wn.ok && lane == 0 && p.status) atomicExch(p.status, FFEQ_ERR_INVALID_ARG);
              issue_rows<Contract::kDense>(wn, Ws, &full[s], lane);
            } else if (lane == 0) {
              mbar_arrive(&full[s]);
            }
          }
        }
      } else {
        // Uniform: a unit past the end is never waited on, so no arrival is needed.
        const int tn = t + nst * gridDim.x;
        if (p.bulk && warp == 0 && tn < n_units)
          issue_rows<Contract::kDense>(gram_unit<BATCH>(p, tn, kWarps, kSM, Contract::kDense), Ws, &full[s], lane);
      }
    };
    int SP = 0, PS = 0;
    if constexpr (Contract::kPrep) {
      // Convert the staged rows once into hi/lo BF16 planes; the stage is then free.
      SP = presplit_seg(B, Ceff);
      PS = presplit_row(B, Ceff);
      if (w.ok) Contract::prep(Ws, RS, Mrows, B, Ceff, planes, PS, SP, tid, kThreads);
      __syncthreads();
      issue_next();
    }
    float2* Dk = w.D;
    for (int item = warp; item < nItems; item += kWarps) {
      const int mt = kSM ? item % nM : -1;
      const int rest = item / nM;
      const int part = rest % P, c = rest / P;
      int k0, k1;
      if constexpr (Contract::kPrep) {
        // Plane columns of cluster c, split at whole 16-antenna steps.
        const int nK = SP / 16;
        k0 = c * SP + ((part * nK) / P) * 16;
        k1 = c * SP + (((part + 1) * nK) / P) * 16;
      } else if (BATCH || p.cl_uniform) {
        k0 = c * S + (part * S) / P;
        k1 = c * S + ((part + 1) * S) / P;
      } else {
        // Clusters of their own sizes (Sec. II-B: B_c antennas for cluster c).
        const int cs = p.cl_off[c], Sc = p.cl_off[c + 1] - cs;
        k0 = cs + (part * Sc) / P;
        k1 = cs + ((part + 1) * Sc) / P;
      }
      auto contract = [&](auto&& out) {
        if constexpr (Contract::kPrep) {
          Contract::template run<UP>(planes, PS, Mrows, U, k0, k1, lane, mt, out);
        } else {
          Contract::template run<UP>(Ws, RS, Mrows, U, k0, k1, vec, lane, mt, out);
        }
      };
      if (P == 1) {
        float2* Dc = Dk + c * matSize;
        contract([&](int m, int u, float2 v0, float2 v1, bool has1) {
          float2* d = Dc + m * U + u;
          if (has1 && (U & 1) == 0) {
            *reinterpret_cast<float4*>(d) = make_float4(v0.x, v0.y, v1.x, v1.y);
          } else {
            d[0] = v0;
            if (has1) d[1] = v1;
          }
        });
      } else {
        float2* slot = slots + (c * P + part) * slotSize;
        contract([&](int m, int u, float2 v0, float2 v1, bool has1) {
          slot[m * SU + u] = v0;
          if (has1) slot[m * SU + u + 1] = v1;
        });
      }
    }
    __syncthreads();   // stage s / planes (and, with split K, the partial slots) complete; ring[s] read by all
    if constexpr (!Contract::kPrep) issue_next();
    if (P > 1 && w.ok) {
      // Fixed-order reduction of the K-parts, written coalesced to the workspace.
      for (int e = tid; e < Ceff * matSize; e += kThreads) {
        const int c = e / matSize, r = e - c * matSize;
        const int m = r / U, u = r - m * U;
        const float2* sl = slots + (c * P) * slotSize + m * SU + u;
        float2 v = sl[0];
        for (int q = 1; q < P; ++q) v = cadd(v, sl[q * slotSize]);
        Dk[e] = v;
      }
    }
    // Slots free for the next unit; batch without bulk staging: publishes ring[s].
    if ((P > 1 && w.ok) || (BATCH && !p.bulk)) __syncthreads();
  }
  // Let the dependent solve kernel start its launch while this grid drains.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Shared-memory capacity of one stage and of one partial slot (float2) for a
// problem of these sizes, and the number of slots its split needs.
template <class Contract>
void gram_capacity(int B, int U, int n_sym, int Ceff, int& stage_elems, int& slot_elems, int& slots) {
  const int Mrows = U + n_sym;
  const GramSplit sp = gram_split(Ceff, Mrows, Contract::kWarps, Contract::kSplitM);
  // Both rounded to an even count: stages and slots start 16-byte aligned.
  stage_elems = (Mrows * stage_row_stride<Contract>(B) + 1) & ~1;
  slot_elems = (Mrows * (padded_users(U) + 1) + 1) & ~1;
  slots = sp.slots;
}

// Stages that fit for the given capacities (0 when one unit does not fit).
inline int gram_stages_fit(size_t stage_elems, size_t slot_bytes_total, bool bulk,
                           size_t smem_budget = kGramSmemBudget) {
  const size_t stage = stage_elems * 8;
  if (slot_bytes_total + kGramHeaderBytes >= smem_budget) return 0;
  const size_t budget = smem_budget - kGramHeaderBytes - slot_bytes_total;
  if (stage > budget) return 0;
  const size_t fit = budget / stage;
  if (!bulk) return 1;
  return static_cast<int>(fit < kGramMaxStages ? fit : kGramMaxStages);
}

template <class Contract>
int gram_stages_for(int B, int U, int n_sym, int Ceff, bool bulk) {
  int st, sl, ns;
  gram_capacity<Contract>(B, U, n_sym, Ceff, st, sl, ns);
  return gram_stages_fit(st, static_cast<size_t>(ns) * sl * 8, bulk);
}

inline size_t gram_smem_bytes(const GramParams& p) {
  return kGramHeaderBytes + static_cast<size_t>(p.stages) * p.stage_elems * 8 +
         static_cast<size_t>(p.n_slots) * p.slot_elems * 8 + static_cast<size_t>(p.plane_bytes);
}

// Launch on min(n_sc, #SMs) persistent CTAs.
template <int UP, class Contract>
cudaError_t launch_gram_up(const GramParams& p, size_t smem, cudaStream_t stream) {
  static int configured[64] = {0};
  static int num_sms[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 64 && !configured[dev]) {
    err = cudaFuncSetAttribute(gram_kernel<UP, Contract, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               227 * 1024);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(gram_kernel<UP, Contract, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               227 * 1024);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    configured[dev] = 1;
  }
  const int sms = (dev < 64 ? num_sms[dev] : 152) * Contract::kMinBlocks;
  int grid = p.n_units < sms ? p.n_units : sms;
  if (p.grid_cap > 0 && grid > p.grid_cap) grid = p.grid_cap;
  if (p.desc) {
    gram_kernel<UP, Contract, true><<<grid, Contract::kWarps * 32, smem, stream>>>(p);
  } else {
    gram_kernel<UP, Contract, false><<<grid, Contract::kWarps * 32, smem, stream>>>(p);
  }
  return cudaGetLastError();
}


}  // namespace ffeq
