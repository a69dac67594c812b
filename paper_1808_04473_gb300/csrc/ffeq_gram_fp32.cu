// Local preprocessing in FP32 on the CUDA cores: for every subcarrier k and
// antenna cluster c (Sec. II-C) the warp-tiled contraction
//
//     D_{k,c}[m][u] = sum_{b in cluster c} conj(H_k[u][b]) * W_k[m][b],
//     W_k = [H_k ; Y_k]  (rows 0..U-1: channel rows, rows U..U+n_sym-1: receive rows)
//
// gives the local Gram matrix G_c[u][v] = D[v][u] (v < U) and the local MRC
// outputs y_c^MRC[u] = D[U+n][u] for OFDM symbol n.  PD sums over all clusters
// (the adder tree of Eq. fullMRC) on chip, as a split-K reduction over the
// warps of the CTA; FD keeps one D per cluster.  D goes to the workspace,
// [n_sc][Ceff][U + n_sym][U] complex, Ceff = C (FD) or 1 (PD).
//
// One CTA per subcarrier: the U + n_sym rows of B complex are staged into
// shared memory with one cp.async.bulk per row on an mbarrier.
#include "ffeq_device.cuh"
#include "ffeq_internal.h"

namespace ffeq {

__device__ int g_device_status = 0;

namespace {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kHeaderBytes = 128;

// Accumulate this lane's 4x4 tiles of D over antennas [k0, k1).  Tile t covers
// rows m = mg + NMG*i and users u = ug + NUG*j: the lanes of a warp read
// consecutive shared-memory rows, whose stride (B+2 complex) shifts the bank by
// 16 bytes per row, so the loads never conflict.  out(m, u, value) stores.
template <int UP, typename Out>
__device__ __forceinline__ void contract_tiles(const float2* __restrict__ Ws, int RS, int Mrows, int U, int k0,
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
        if (m < Mrows && u < U) out(m, u, acc[i][j]);
      }
  }
}

template <int UP>
__global__ void __launch_bounds__(kThreads) gram_fp32_kernel(const GramParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
  const int U = p.U, B = p.B, NS = p.n_sym;
  const int Mrows = U + NS, RS = B + 2, SU = UP + 1;
  float2* Ws = reinterpret_cast<float2*>(smem + kHeaderBytes);
  float2* slots = Ws + Mrows * RS;            // split-K partials (only when P > 1)
  const int slotSize = Mrows * SU;
  const int sc = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const float2* Hk = p.H + static_cast<size_t>(sc) * U * B;
  const float2* Yk = p.y + static_cast<size_t>(sc) * NS * B;
  if (p.bulk) {
    if (warp == 0) {
      if (lane == 0) mbar_arrive_expect_tx(bar, static_cast<uint32_t>(Mrows) * B * 8u);
      __syncwarp();
      for (int r = lane; r < Mrows; r += 32) {
        const float2* src = r < U ? Hk + static_cast<size_t>(r) * B : Yk + static_cast<size_t>(r - U) * B;
        bulk_g2s(Ws + r * RS, src, static_cast<uint32_t>(B) * 8u, bar);
      }
    }
    if (!mbar_wait_bounded(bar, 0, p.status, FFEQ_ERR_TIMEOUT)) {
      mbar_wait_bounded(bar, 0, nullptr, 0);
      return;
    }
  } else {
    for (int e = tid; e < Mrows * B; e += kThreads) {
      const int r = e / B, b = e - r * B;
      Ws[r * RS + b] = r < U ? Hk[static_cast<size_t>(r) * B + b] : Yk[static_cast<size_t>(r - U) * B + b];
    }
    __syncthreads();
  }

  const int Ceff = p.Ceff;
  const int S = B / Ceff;
  const int P = Ceff >= kWarps ? 1 : kWarps / Ceff;
  const int ncMax = Ceff >= kWarps ? kWarps : Ceff;
  const bool vec = (B & 1) == 0;
  const size_t matSize = static_cast<size_t>(Mrows) * U;
  float2* Dk = p.D + static_cast<size_t>(sc) * Ceff * matSize;

  if (P == 1) {
    // One warp per cluster, straight to the workspace.
    for (int c = warp; c < Ceff; c += kWarps) {
      float2* Dc = Dk + c * matSize;
      contract_tiles<UP>(Ws, RS, Mrows, U, c * S, (c + 1) * S, vec, lane,
                         [&](int m, int u, float2 v) { Dc[m * U + u] = v; });
    }
  } else {
    // nc = Ceff clusters, P K-parts each: partial sums in shared memory, then a
    // fixed-order reduction (deterministic) written coalesced to the workspace.
    const int nc = ncMax;
    if (warp < nc * P) {
      const int cl = warp % nc, part = warp / nc;
      const int k0 = cl * S + (part * S) / P, k1 = cl * S + ((part + 1) * S) / P;
      float2* slot = slots + warp * slotSize;
      contract_tiles<UP>(Ws, RS, Mrows, U, k0, k1, vec, lane,
                         [&](int m, int u, float2 v) { slot[m * SU + u] = v; });
    }
    __syncthreads();
    for (int e = tid; e < nc * static_cast<int>(matSize); e += kThreads) {
      const int c = e / static_cast<int>(matSize), r = e - c * static_cast<int>(matSize);
      const int m = r / U, u = r - m * U;
      float2 s = slots[c * slotSize + m * SU + u];
      for (int q = 1; q < P; ++q) s = cadd(s, slots[(q * nc + c) * slotSize + m * SU + u]);
      Dk[e] = s;
    }
  }
  // Let the dependent solve kernel start its launch while this grid drains.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <int UP>
cudaError_t launch_up(const GramParams& p, size_t smem, cudaStream_t stream) {
  static int configured[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 64 && !configured[dev]) {
    err = cudaFuncSetAttribute(gram_fp32_kernel<UP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    configured[dev] = 1;
  }
  gram_fp32_kernel<UP><<<p.n_sc, kThreads, smem, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace

int padded_users(int U) { return U <= 8 ? 8 : (U <= 16 ? 16 : 32); }

size_t gram_fp32_smem_bytes(int B, int U, int n_sym, int Ceff) {
  const size_t Mrows = static_cast<size_t>(U) + n_sym;
  const size_t SU = static_cast<size_t>(padded_users(U)) + 1;
  const bool split = Ceff < kWarps;
  return kHeaderBytes + Mrows * (static_cast<size_t>(B) + 2) * 8 + (split ? kWarps * Mrows * SU * 8 : 0);
}

cudaError_t launch_gram_fp32(const GramParams& p, cudaStream_t stream) {
  const size_t smem = gram_fp32_smem_bytes(p.B, p.U, p.n_sym, p.Ceff);
  switch (padded_users(p.U)) {
    case 8: return launch_up<8>(p, smem, stream);
    case 16: return launch_up<16>(p, smem, stream);
    default: return launch_up<32>(p, smem, stream);
  }
}

int* device_status_ptr() {
  static int* cached[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return nullptr;
  if (!cached[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_device_status) != cudaSuccess) return nullptr;
    cached[dev] = static_cast<int*>(ptr);
  }
  return cached[dev];
}

}  // namespace ffeq
