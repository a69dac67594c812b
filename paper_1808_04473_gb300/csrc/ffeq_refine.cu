// Iterative refinement of the L-MMSE solves from the inputs (uniform problems).
//
// The mixed-precision preprocessing forms G_c = H_c^H H_c and y_c^MRC from
// operands rounded to hi + lo pairs, so the solved systems carry a relative
// perturbation u (2^-16 for BF16x3) that the solve amplifies by
// kappa(G_c + rho I).  A residual taken against the stored G_c cannot see that
// error; this kernel forms it from H and y instead (FP32, per subcarrier, all
// clusters of the subcarrier in one CTA):
//   M_c = H_c^H H_c + rho I,  b_c = H_c^H y_c                   (Sec. III-A, II-C)
//   r_c = b_c - M_c x_c = H_c^H (y_c - H_c x_c) - rho x_c,   x_c <- x_c + A~_c r_c
// with A~_c the inverse computed by the solve kernel (`steps` times).  The
// inverse itself, whose diagonal the unbiasing and the fusion weights use
// (mu = 1 - rho A_uu, sigma^2 = N0 A_uu, Eq. opt_fusion), gets a Newton-Schulz
// step from the same product V = H_c A~_c in each step:
//   A~_c <- 2 A~_c - A~_c^H M_c A~_c = 2 A~_c - V^H V - rho A~_c^H A~_c,
// which squares its relative error.  Each step shrinks the error of the
// estimates by about kappa u.  The fusion and soft outputs then follow the solve
// kernel's epilogue (Eq. fusionrule, Lemma 1, Thm. 3; PD is C = 1).  All sums
// run in a fixed order (deterministic).
#include <cmath>

#include "ffeq_device.cuh"
#include "ffeq_epilogue.cuh"
#include "ffeq_internal.h"

namespace ffeq {
namespace {

constexpr int kRefineThreads = 512;

// Shared memory: clusters are refined in chunks of CC (all of them when they
// fit); the fused numerators and denominators of every cluster persist.
struct RefineLayout {
  int B, U, NS, Ceff, S, CC, HS, W;
  size_t hs, pm, va, rb, rr, an, fz, dn, total;   // offsets in bytes
  __host__ __device__ RefineLayout(int B_, int U_, int NS_, int Ceff_, int CC_)
      : B(B_), U(U_), NS(NS_), Ceff(Ceff_), S(B_ / Ceff_), CC(CC_), HS(CC_ * (B_ / Ceff_) + 1), W(U_ + NS_) {
    size_t o = 0;
    hs = o;  o += static_cast<size_t>(U) * HS * 8;          // H rows of the chunk's antennas
    pm = o;  o += static_cast<size_t>(CC) * W * U * 8;      // per cluster: columns a_j of A~, then x_n
    va = o;  o += static_cast<size_t>(U) * HS * 8;          // V = H_c a_j per antenna
    rb = o;  o += static_cast<size_t>(NS) * HS * 8;         // y - H x per antenna
    rr = o;  o += static_cast<size_t>(CC) * NS * U * 8;     // residual
    an = o;  o += static_cast<size_t>(CC) * U * U * 8;      // next inverse
    fz = o;  o += static_cast<size_t>(Ceff) * NS * U * 8;   // fused numerators x / A_uu
    dn = o;  o += static_cast<size_t>(Ceff) * U * 4;        // fusion denominators g / A_uu
    o += 16;                                                // failure flag
    total = o;
  }
};

template <int UP>
__global__ void __launch_bounds__(kRefineThreads) refine_kernel(const RefineParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const RefineLayout L(p.B, p.U, p.n_sym, p.Ceff, p.chunk);
  const int B = L.B, U = L.U, NS = L.NS, Ceff = L.Ceff, S = L.S, HS = L.HS, W = L.W;
  float2* Hs = reinterpret_cast<float2*>(smem + L.hs);
  float2* P = reinterpret_cast<float2*>(smem + L.pm);
  float2* Va = reinterpret_cast<float2*>(smem + L.va);
  float2* Rb = reinterpret_cast<float2*>(smem + L.rb);
  float2* Rr = reinterpret_cast<float2*>(smem + L.rr);
  float2* An = reinterpret_cast<float2*>(smem + L.an);
  float2* Fz = reinterpret_cast<float2*>(smem + L.fz);
  float* Dn = reinterpret_cast<float*>(smem + L.dn);
  int* failed = reinterpret_cast<int*>(smem + L.total - 16);
  const int k = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const float rho = p.rho;
  const float2* Hk = p.H + static_cast<size_t>(k) * U * B;
  const float2* yk = p.y + static_cast<size_t>(k) * NS * B;
  const size_t sys0 = static_cast<size_t>(k) * Ceff;

  if (tid == 0) *failed = 0;
  // Wait for the solve kernel (programmatic dependent launch).
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __syncthreads();
  if (tid < Ceff && p.fails[sys0 + tid] != 0) atomicOr(failed, 1);

  for (int c0 = 0; c0 < Ceff; c0 += L.CC) {
    const int cc = Ceff - c0 < L.CC ? Ceff - c0 : L.CC;   // clusters in this chunk
    const int nb = cc * S;                                 // their antennas, from b0
    const int b0 = c0 * S;
    for (int e = tid; e < U * nb; e += nt) {
      const int u = e / nb, b = e - u * nb;
      Hs[u * HS + b] = Hk[static_cast<size_t>(u) * B + b0 + b];
    }
    for (int e = tid; e < cc * W * U; e += nt) {
      const int c = e / (W * U), r = e - c * W * U, j = r / U, i = r - j * U;
      const size_t sys = sys0 + c0 + c;
      P[e] = j < U ? p.As[(sys * U + j) * U + i] : p.Xs[(sys * NS + (j - U)) * U + i];
    }
    __syncthreads();

    for (int step = 0; step < p.steps; ++step) {
      // V = H_c [A~_c | X_c] per antenna b (cluster c = b / S); y - H_c x for the estimates.
      for (int b = tid; b < nb; b += nt) {
        const int c = b / S;
        float2 h[UP];
#pragma unroll
        for (int u = 0; u < UP; ++u) h[u] = u < U ? Hs[u * HS + b] : make_float2(0.f, 0.f);
        for (int j = 0; j < W; ++j) {
          const float2* pj = P + (c * W + j) * U;
          float2 v = make_float2(0.f, 0.f);
#pragma unroll
          for (int u = 0; u < UP; ++u)
            if (u < U) v = cfma(h[u], pj[u], v);
          if (j < U) {
            Va[j * HS + b] = v;
          } else {
            const int n = j - U;
            Rb[n * HS + b] = csub(yk[static_cast<size_t>(n) * B + b0 + b], v);
          }
        }
      }
      __syncthreads();
      // r_c = H_c^H (y_c - H_c x_c) - rho x_c;  next inverse 2 A - V^H V - rho A^H A.
      for (int e = tid; e < cc * NS * U; e += nt) {
        const int c = e / (NS * U), r = e - c * NS * U, n = r / U, u = r - n * U;
        float2 sum = make_float2(0.f, 0.f);
        for (int b = c * S; b < (c + 1) * S; ++b) sum = cfma_conj(Hs[u * HS + b], Rb[n * HS + b], sum);
        const float2 x = P[(c * W + U + n) * U + u];
        Rr[e] = make_float2(sum.x - rho * x.x, sum.y - rho * x.y);
      }
      for (int e = tid; e < cc * U * U; e += nt) {
        const int c = e / (U * U), r = e - c * U * U, j = r / U, i = r - j * U;   // entry (i, j)
        float2 vv = make_float2(0.f, 0.f);
        for (int b = c * S; b < (c + 1) * S; ++b) vv = cfma_conj(Va[i * HS + b], Va[j * HS + b], vv);
        float2 aa = make_float2(0.f, 0.f);
        const float2* ai = P + (c * W + i) * U;
        const float2* aj = P + (c * W + j) * U;
        for (int v = 0; v < U; ++v) aa = cfma_conj(ai[v], aj[v], aa);
        const float2 a = aj[i];
        An[e] = make_float2(2.f * a.x - vv.x - rho * aa.x, 2.f * a.y - vv.y - rho * aa.y);
      }
      __syncthreads();
      // x_c += A~_c r_c   (A~[u][v] = column v of A~ at row u), then A~ <- next inverse.
      for (int e = tid; e < cc * NS * U; e += nt) {
        const int c = e / (NS * U), r = e - c * NS * U, n = r / U, u = r - n * U;
        float2 d = make_float2(0.f, 0.f);
        for (int v = 0; v < U; ++v) d = cfma(P[(c * W + v) * U + u], Rr[(c * NS + n) * U + v], d);
        float2* x = P + (c * W + U + n) * U + u;
        *x = cadd(*x, d);
      }
      __syncthreads();
      for (int e = tid; e < cc * U * U; e += nt) {
        const int c = e / (U * U), r = e - c * U * U;
        P[c * W * U + r] = An[e];
      }
      __syncthreads();
    }

    // ---- fusion terms (as the solve kernel): weight g / A_uu with g = mu or 1
    for (int e = tid; e < cc * U; e += nt) {
      const int c = e / U, u = e - c * U;
      const float gii = p.D[((sys0 + c0 + c) * W + u) * U + u].x;
      const float A = P[(c * W + u) * U + u].x;
      const float invA = 1.f / A;
      const float mu = gii == 0.f ? 0.f : fmaxf(1.f - rho * A, 0.f);
      Dn[(c0 + c) * U + u] = (p.unbiased ? mu : 1.f) * invA;
      for (int n = 0; n < NS; ++n) Fz[((c0 + c) * NS + n) * U + u] = cscale(P[(c * W + U + n) * U + u], invA);
    }
    __syncthreads();
  }

  const int bits = p.llr_bits, hb = bits / 2;
  const bool fail = *failed != 0;
  for (int e = tid; e < NS * U; e += nt) {
    const int n = e / U, u = e - n * U;
    float2 nm = make_float2(0.f, 0.f);
    float dn = 0.f;
    for (int c = 0; c < Ceff; ++c) {
      nm = cadd(nm, Fz[(c * NS + n) * U + u]);
      dn += Dn[c * U + u];
    }
    float2 zz;
    float s2;
    if (fail) {
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
    if (bits) symbol_llr(zz, s2, p.llr_scale, hb, p.llr + zi * bits);
  }
}

template <int UP>
cudaError_t launch_refine_up(const RefineParams& p, cudaStream_t stream) {
  static int configured[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 64 && !configured[dev]) {
    err = cudaFuncSetAttribute(refine_kernel<UP>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    configured[dev] = 1;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.n_sc);
  cfg.blockDim = dim3(kRefineThreads);
  cfg.dynamicSmemBytes = RefineLayout(p.B, p.U, p.n_sym, p.Ceff, p.chunk).total;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, refine_kernel<UP>, p);
}

}  // namespace

int refine_chunk(int B, int U, int Ceff, int n_sym) {
  for (int cc = Ceff; cc >= 1; --cc)
    if (RefineLayout(B, U, n_sym, Ceff, cc).total <= 227 * 1024) return cc;
  return 0;
}

size_t refine_smem_bytes(int B, int U, int Ceff, int n_sym) {
  const int cc = refine_chunk(B, U, Ceff, n_sym);
  return cc ? RefineLayout(B, U, n_sym, Ceff, cc).total : 0;
}

cudaError_t launch_refine(const RefineParams& p, cudaStream_t stream) {
  switch (padded_users(p.U)) {
    case 8: return launch_refine_up<8>(p, stream);
    case 16: return launch_refine_up<16>(p, stream);
    default: return launch_refine_up<32>(p, stream);
  }
}

}  // namespace ffeq
