// Central / local L-MMSE solve, optimal fusion and soft outputs (FP32).
//
// Input: the workspace written by the contraction kernel, one matrix
// D = [G ; (y^MRC)^T] of (U + n_sym) x U complex per (subcarrier, cluster):
// G[u][v] = D[v][u], y^MRC_u(n) = D[U+n][u].  One group of UP lanes (UP = U
// padded to 8/16/32; lane i = user i) equalizes one matrix:
//   * Cholesky G + rho I = L L^H in registers (rho = N0/Es, Sec. III-A);
//   * column i of L^{-1} by right-looking substitution; A_ii = ||L^{-1} e_i||^2
//     is the i-th diagonal entry of A = (G + rho I)^{-1};
//   * z = A y^MRC = L^{-H} (L^{-1} y^MRC) for all n_sym right-hand sides.
// A CTA holds the C clusters of one subcarrier (FD) or several subcarriers (PD)
// and fuses per user with the optimal weights (Eq. fusionrule, Lemma 1):
//     z_u = sum_c (z_{c,u}/A_{c,uu}) / sum_c (g_{c,u}/A_{c,uu}),
//     sigma_u^2 = N0 / sum_c (g_{c,u}/A_{c,uu})             (Thm. 3)
// with g = mu = 1 - rho A_uu (unbiased pairs) or g = 1 (literal pairs); this is
// nu_c = sigma_c^-2 / sum sigma^-2 with sigma_c^2 = N0 A/g, written so that N0
// cancels from the weights (N0 = 0, zero forcing, needs no special case).  PD
// is the case C = 1.  The epilogue writes z, sigma^2 and max-log LLRs.
#include <cmath>

#include "ffeq_device.cuh"
#include "ffeq_internal.h"

namespace ffeq {
namespace {

template <int UP>
struct SolveLayout {
  // Per matrix: L / L^{-1} (UP x (UP+1)), right-hand sides (UP x kNsymMax),
  // fusion denominators (UP); padded so matrices start 64 bytes apart mod 128.
  static constexpr int kL = UP * (UP + 1);
  static constexpr int kB = UP * kNsymMax;
  static constexpr int kMat = ((kL + kB + UP / 2 + 15) / 16) * 16 + 8;   // float2 units
};

__device__ __forceinline__ float2 shfl2w(float2 v, int src, int width) {
  return make_float2(__shfl_sync(kFullMask, v.x, src, width), __shfl_sync(kFullMask, v.y, src, width));
}

// Max-log LLRs of one Gray-labelled PAM axis (labels and sign as in ffeq.h).
__device__ __forceinline__ void axis_llr(float x, float s2, float scale, int h, float* out) {
  const int L = 1 << h;
  float m0[4], m1[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) m0[t] = m1[t] = INFINITY;
  for (int l = 0; l < L; ++l) {
    const float a = scale * static_cast<float>(2 * l - (L - 1));
    const float d = (x - a) * (x - a);
    const int g = l ^ (l >> 1);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (t < h) {
        if ((g >> (h - 1 - t)) & 1) m1[t] = fminf(m1[t], d);
        else m0[t] = fminf(m0[t], d);
      }
    }
  }
  const bool s2inf = isinf(s2);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (t < h) {
      const float diff = m1[t] - m0[t];
      float v = diff / s2;
      if (s2inf || (s2 == 0.f && diff == 0.f)) v = 0.f;
      out[t] = v;
    }
  }
}

template <int UP>
__global__ void __launch_bounds__(512) solve_fuse_kernel(const SolveParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  using Lay = SolveLayout<UP>;
  const int U = p.U, NS = p.n_sym, Ceff = p.Ceff, spc = p.spc;
  const int nmat = spc * Ceff;
  const int g = threadIdx.x / UP, i = threadIdx.x % UP;
  int* fail_sc = reinterpret_cast<int*>(smem);                       // [spc]
  float2* base = reinterpret_cast<float2*>(smem + 256);
  const int sc0 = blockIdx.x * spc;

  if (threadIdx.x < spc) fail_sc[threadIdx.x] = 0;
  __syncthreads();

  const int gm = g < nmat ? g : nmat - 1;       // spare lanes shadow the last matrix
  const int scl = gm / Ceff, c = gm % Ceff;
  const int sc = sc0 + scl;
  const bool valid = g < nmat && sc < p.n_sc;
  float2* Ls = base + gm * Lay::kMat;
  float2* Bs = Ls + Lay::kL;
  float* Dn = reinterpret_cast<float*>(Bs + Lay::kB);
  const size_t matSize = static_cast<size_t>(U + NS) * U;
  const float2* Dg = p.D + (static_cast<size_t>(valid ? sc : 0) * Ceff + c) * matSize;

  // Wait for the contraction grid (programmatic dependent launch).
  asm volatile("griddepcontrol.wait;" ::: "memory");

  // ---- load row i of M = G + rho I and the right-hand sides b[i][n]
  float2 a[UP];
  float gii = 1.f;
#pragma unroll
  for (int j = 0; j < UP; ++j) {
    float2 v = make_float2(i == j ? 1.f : 0.f, 0.f);
    if (valid && i < U && j < U) {
      v = Dg[j * U + i];
      if (i == j) {
        gii = v.x;
        v = make_float2(v.x + p.rho, 0.f);
      }
    }
    a[j] = v;
  }
  if (g < nmat) {
#pragma unroll
    for (int n = 0; n < kNsymMax; ++n)
      if (n < NS) Bs[i * kNsymMax + n] = (valid && i < U) ? Dg[(U + n) * U + i] : make_float2(0.f, 0.f);
  }

  // ---- Cholesky: lane i keeps row i of L in a[0..i]
  int fail = 0;
  static_for<UP>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    const float piv = __shfl_sync(kFullMask, a[k].x, k, UP);
    const bool ok = piv > 0.f;
    if (!ok && fail == 0) fail = k + 1;
    const float d = sqrtf(ok ? piv : 1.f);
    const float inv = 1.f / d;
    if (i == k) a[k] = make_float2(d, 0.f);
    else if (i > k) a[k] = cscale(a[k], inv);
#pragma unroll
    for (int j = k + 1; j < UP; ++j) {
      const float2 ljk = shfl2w(a[k], j, UP);
      if (i >= j) a[j] = cfms_bconj(a[k], ljk, a[j]);
    }
  });
  if (g < nmat) {
#pragma unroll
    for (int j = 0; j < UP; ++j)
      if (j <= i) Ls[i * (UP + 1) + j] = a[j];
  }
  __syncwarp();

  // ---- column i of L^{-1} (right-looking forward substitution on e_i)
  float2 x[UP];
#pragma unroll
  for (int r = 0; r < UP; ++r) x[r] = make_float2(r == i ? 1.f : 0.f, 0.f);
  static_for<UP>([&](auto kc) {
    constexpr int k = decltype(kc)::value;
    const float inv = 1.f / Ls[k * (UP + 1) + k].x;
    x[k] = cscale(x[k], inv);
#pragma unroll
    for (int r = k + 1; r < UP; ++r) x[r] = cfms(Ls[r * (UP + 1) + k], x[k], x[r]);
  });
  float Aii = 0.f;
#pragma unroll
  for (int r = 0; r < UP; ++r) Aii += cabs2(x[r]);
  __syncwarp();
  // L^{-1} row-major into Ls (lane i writes column i).
  if (g < nmat) {
#pragma unroll
    for (int r = 0; r < UP; ++r) Ls[r * (UP + 1) + i] = x[r];
  }
  __syncwarp();

  // ---- w = L^{-1} b (lane i: row i), then z = L^{-H} w
  float2 acc[kNsymMax];
#pragma unroll
  for (int n = 0; n < kNsymMax; ++n) acc[n] = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < UP; ++j) {
    const float2 l = Ls[i * (UP + 1) + j];
#pragma unroll
    for (int n = 0; n < kNsymMax; n += 2) {
      if (n < NS) {
        const float4 bb = *reinterpret_cast<const float4*>(Bs + j * kNsymMax + n);
        acc[n] = cfma(l, make_float2(bb.x, bb.y), acc[n]);
        acc[n + 1] = cfma(l, make_float2(bb.z, bb.w), acc[n + 1]);
      }
    }
  }
  __syncwarp();
  if (g < nmat) {
#pragma unroll
    for (int n = 0; n < kNsymMax; ++n)
      if (n < NS) Bs[i * kNsymMax + n] = acc[n];
  }
  __syncwarp();
#pragma unroll
  for (int n = 0; n < kNsymMax; ++n) acc[n] = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < UP; ++k) {
    const float2 l = x[k];
#pragma unroll
    for (int n = 0; n < kNsymMax; n += 2) {
      if (n < NS) {
        const float4 ww = *reinterpret_cast<const float4*>(Bs + k * kNsymMax + n);
        acc[n] = cfma_conj(l, make_float2(ww.x, ww.y), acc[n]);
        acc[n + 1] = cfma_conj(l, make_float2(ww.z, ww.w), acc[n + 1]);
      }
    }
  }

  // ---- fusion terms of this matrix
  const float invA = 1.f / Aii;
  // mu = [A G]_ii = 1 - rho A_ii; a user the cluster cannot see (G_ii = 0) has
  // mu = 0 exactly, which the subtraction would only reach up to rounding.
  const float mu = gii == 0.f ? 0.f : fmaxf(1.f - p.rho * Aii, 0.f);
  __syncwarp();
  if (g < nmat) {
#pragma unroll
    for (int n = 0; n < kNsymMax; ++n)
      if (n < NS) Bs[i * kNsymMax + n] = cscale(acc[n], invA);
    Dn[i] = (p.unbiased ? mu : 1.f) * invA;
    if (i == 0 && valid) {
      if (p.info) p.info[static_cast<size_t>(sc) * Ceff + c] = fail;
      if (fail) atomicOr(&fail_sc[scl], 1);
    }
  }
  __syncthreads();

  // ---- per subcarrier: sum over clusters, outputs
  const int per = U * NS;
  const int bits = p.llr_bits, h = bits / 2;
  for (int e = threadIdx.x; e < spc * per; e += blockDim.x) {
    const int s = e / per, r = e - s * per;
    const int n = r / U, u = r - n * U;
    const int k = sc0 + s;
    if (k >= p.n_sc) break;
    float2 nm = make_float2(0.f, 0.f);
    float dn = 0.f;
    for (int cc = 0; cc < Ceff; ++cc) {
      const float2* Lm = base + (s * Ceff + cc) * Lay::kMat;
      nm = cadd(nm, (Lm + Lay::kL)[u * kNsymMax + n]);
      dn += reinterpret_cast<const float*>(Lm + Lay::kL + Lay::kB)[u];
    }
    float2 zz;
    float s2;
    if (fail_sc[s]) {
      zz = make_float2(NAN, NAN);
      s2 = NAN;
    } else if (dn > 0.f) {
      const float rr = 1.f / dn;
      zz = cscale(nm, rr);
      s2 = p.N0 * rr;
    } else {
      zz = make_float2(0.f, 0.f);
      s2 = INFINITY;
    }
    const size_t zi = (static_cast<size_t>(k) * NS + n) * U + u;
    p.z[zi] = zz;
    if (n == 0) p.sigma2[static_cast<size_t>(k) * U + u] = s2;
    if (bits) {
      float* out = p.llr + zi * bits;
      axis_llr(zz.x, s2, p.llr_scale, h, out);
      axis_llr(zz.y, s2, p.llr_scale, h, out + h);
    }
  }
}

template <int UP>
cudaError_t launch_up(const SolveParams& p, cudaStream_t stream) {
  using Lay = SolveLayout<UP>;
  const int nmat = p.spc * p.Ceff;
  const int threads = ((nmat * UP + 31) / 32) * 32;
  const size_t smem = 256 + static_cast<size_t>(nmat) * Lay::kMat * sizeof(float2);
  static int configured[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 64 && !configured[dev]) {
    err = cudaFuncSetAttribute(solve_fuse_kernel<UP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
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
  return cudaLaunchKernelEx(&cfg, solve_fuse_kernel<UP>, p);
}

}  // namespace

int solve_subcarriers_per_cta(int U, int Ceff) {
  return Ceff == 1 ? (padded_users(U) >= 32 ? 4 : 128 / padded_users(U)) : 1;
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
  switch (padded_users(p.U)) {
    case 8: return launch_up<8>(p, stream);
    case 16: return launch_up<16>(p, stream);
    default: return launch_up<32>(p, stream);
  }
}

}  // namespace ffeq
