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
// B complex of each are staged into shared memory (row stride B + 2 complex)
// with one cp.async.bulk per row on a per-stage mbarrier, up to three
// subcarriers ahead of the contraction.
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

// Stage subcarrier k's U + n_sym rows into `dst` (row stride B + 2 complex),
// completing on `bar` (one cp.async.bulk per row; issued by one warp).
__device__ __forceinline__ void issue_rows(const GramParams& p, int k, float2* dst, uint64_t* bar, int lane) {
  const int U = p.U, B = p.B, NS = p.n_sym, Mrows = U + NS, RS = B + 2;
  const float2* Hk = p.H + static_cast<size_t>(k) * U * B;
  const float2* Yk = p.y + static_cast<size_t>(k) * NS * B;
  if (lane == 0) mbar_arrive_expect_tx(bar, static_cast<uint32_t>(Mrows) * B * 8u);
  __syncwarp();
  for (int r = lane; r < Mrows; r += 32) {
    const float2* src = r < U ? Hk + static_cast<size_t>(r) * B : Yk + static_cast<size_t>(r - U) * B;
    bulk_g2s(dst + r * RS, src, static_cast<uint32_t>(B) * 8u, bar);
  }
}

// Persistent: CTA b handles subcarriers b, b + gridDim.x, ...  With bulk
// staging, p.stages subcarriers are in flight per CTA: the loads of the next
// ones overlap the contraction of the current one.  Contract::run<UP> computes
// one warp's share of D over antennas [k0, k1) and hands each (m, u) entry to
// the output functor.
template <int UP, class Contract>
__global__ void __launch_bounds__(Contract::kWarps * 32, 1) gram_kernel(const GramParams p) {
  constexpr int kWarps = Contract::kWarps;
  constexpr int kThreads = kWarps * 32;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);                 // [p.stages]
  const int U = p.U, B = p.B, NS = p.n_sym;
  const int Mrows = U + NS, RS = B + 2, SU = UP + 1;
  const int nst = p.stages;
  float2* stage0 = reinterpret_cast<float2*>(smem + kGramHeaderBytes);
  const int stageSize = Mrows * RS;
  float2* slots = stage0 + nst * stageSize;    // split-K partials (only when P > 1)
  const int slotSize = Mrows * SU;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const int Ceff = p.Ceff;
  const int S = B / Ceff;
  const GramSplit sp = gram_split(Ceff, Mrows, kWarps, Contract::kSplitM);
  const int P = sp.P, nM = sp.nM;
  const int nItems = Ceff * P * nM;
  const bool vec = (B & 1) == 0;
  const int matSize = Mrows * U;

  if (tid == 0) {
    for (int s = 0; s < nst; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  // Prologue: fill the ring.
  if (p.bulk && warp == 0) {
    for (int s = 0; s < nst; ++s) {
      const int k = blockIdx.x + s * gridDim.x;
      if (k < p.n_sc) issue_rows(p, k, stage0 + s * stageSize, &full[s], lane);
    }
  }

  int it = 0;
  for (int k = blockIdx.x; k < p.n_sc; k += gridDim.x, ++it) {
    const int s = it % nst;
    float2* Ws = stage0 + s * stageSize;
    if (p.bulk) {
      if (!mbar_wait_bounded(&full[s], (it / nst) & 1, p.status, FFEQ_ERR_TIMEOUT)) {
        // Give every copy still in flight a bounded chance to land, then leave.
        for (int q = 0; q < nst; ++q) mbar_wait_bounded(&full[q], ((it + q) / nst) & 1, nullptr, 0);
        return;
      }
    } else {
      const float2* Hk = p.H + static_cast<size_t>(k) * U * B;
      const float2* Yk = p.y + static_cast<size_t>(k) * NS * B;
      for (int e = tid; e < Mrows * B; e += kThreads) {
        const int r = e / B, b = e - r * B;
        Ws[r * RS + b] = r < U ? Hk[static_cast<size_t>(r) * B + b] : Yk[static_cast<size_t>(r - U) * B + b];
      }
      __syncthreads();
    }
    float2* Dk = p.D + static_cast<size_t>(k) * Ceff * matSize;
    for (int item = warp; item < nItems; item += kWarps) {
      const int mt = Contract::kSplitM ? item % nM : -1;
      const int rest = item / nM;
      const int part = rest % P, c = rest / P;
      const int k0 = c * S + (part * S) / P, k1 = c * S + ((part + 1) * S) / P;
      if (P == 1) {
        float2* Dc = Dk + c * matSize;
        Contract::template run<UP>(Ws, RS, Mrows, U, k0, k1, vec, lane, mt,
                                   [&](int m, int u, float2 v0, float2 v1, bool has1) {
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
        Contract::template run<UP>(Ws, RS, Mrows, U, k0, k1, vec, lane, mt,
                                   [&](int m, int u, float2 v0, float2 v1, bool has1) {
                                     slot[m * SU + u] = v0;
                                     if (has1) slot[m * SU + u + 1] = v1;
                                   });
      }
    }
    __syncthreads();   // stage s (and, with split K, the partial slots) complete
    if (p.bulk && warp == 0) {
      const int kn = k + nst * gridDim.x;
      if (kn < p.n_sc) issue_rows(p, kn, Ws, &full[s], lane);
    }
    if (P > 1) {
      // Fixed-order reduction of the K-parts, written coalesced to the workspace.
      for (int e = tid; e < Ceff * matSize; e += kThreads) {
        const int c = e / matSize, r = e - c * matSize;
        const int m = r / U, u = r - m * U;
        const float2* sl = slots + (c * P) * slotSize + m * SU + u;
        float2 v = sl[0];
        for (int q = 1; q < P; ++q) v = cadd(v, sl[q * slotSize]);
        Dk[e] = v;
      }
      __syncthreads();   // slots free for the next subcarrier
    }
  }
  // Let the dependent solve kernel start its launch while this grid drains.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Shared-memory stages that fit (0 when one subcarrier does not fit) and bytes.
template <class Contract>
int gram_stages_for(int B, int U, int n_sym, int Ceff, bool bulk) {
  const size_t Mrows = static_cast<size_t>(U) + n_sym;
  const size_t SU = static_cast<size_t>(padded_users(U)) + 1;
  const GramSplit sp = gram_split(Ceff, static_cast<int>(Mrows), Contract::kWarps, Contract::kSplitM);
  const size_t partials = static_cast<size_t>(sp.slots) * Mrows * SU * 8;
  const size_t stage = Mrows * (static_cast<size_t>(B) + 2) * 8;
  if (partials + kGramHeaderBytes >= kGramSmemBudget) return 0;
  const size_t budget = kGramSmemBudget - kGramHeaderBytes - partials;
  if (stage > budget) return 0;
  const size_t fit = budget / stage;
  if (!bulk) return 1;
  return static_cast<int>(fit < kGramMaxStages ? fit : kGramMaxStages);
}

template <class Contract>
size_t gram_smem_for(int B, int U, int n_sym, int Ceff, int stages) {
  const size_t Mrows = static_cast<size_t>(U) + n_sym;
  const size_t SU = static_cast<size_t>(padded_users(U)) + 1;
  const GramSplit sp = gram_split(Ceff, static_cast<int>(Mrows), Contract::kWarps, Contract::kSplitM);
  return kGramHeaderBytes + static_cast<size_t>(stages) * Mrows * (static_cast<size_t>(B) + 2) * 8 +
         static_cast<size_t>(sp.slots) * Mrows * SU * 8;
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
    err = cudaFuncSetAttribute(gram_kernel<UP, Contract>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    configured[dev] = 1;
  }
  const int sms = dev < 64 ? num_sms[dev] : 152;
  const int grid = p.n_sc < sms ? p.n_sc : sms;
  gram_kernel<UP, Contract><<<grid, Contract::kWarps * 32, smem, stream>>>(p);
  return cudaGetLastError();
}


}  // namespace ffeq
