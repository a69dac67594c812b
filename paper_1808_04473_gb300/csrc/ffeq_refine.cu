// Iterative refinement of the L-MMSE solves from the inputs (uniform problems).
//
// The mixed-precision preprocessing forms G_c = H_c^H H_c and y_c^MRC from
// operands rounded to hi + lo pairs, so the solved systems carry a relative
// perturbation u (2^-16 for BF16x3) that the solve amplifies by
// kappa(G_c + rho I).  A residual taken against the stored G_c cannot see that
// error; these kernels form it from H and y instead (FP32, one CTA per local
// system, then one per subcarrier for the fusion):
//   M_c = H_c^H H_c + rho I,  b_c = H_c^H y_c                   (Sec. III-A, II-C)
//   r_c = b_c - M_c x_c = H_c^H (y_c - H_c x_c) - rho x_c,   x_c <- x_c + A~_c r_c
// with A~_c the inverse computed by the solve kernel (`steps` times).  The
// inverse itself, whose diagonal the unbiasing and the fusion weights use
// (mu = 1 - rho A_uu, sigma^2 = N0 A_uu, Eq. opt_fusion), gets a Newton-Schulz
// step from the same product V = H_c A~_c in each step:
//   A~_c <- 2 A~_c - A~_c^H M_c A~_c = 2 A~_c - V^H V - rho A~_c^H A~_c,
// which squares its relative error (in the last FP32 step only its diagonal,
// the part read afterwards: half of a step's products).  Each step shrinks the error of the
// estimates by about kappa u, down to the accuracy of an FP32 solve (kappa
// 2^-24, from the rounding of y_c - H_c x_c).  With the FP64 residual (always,
// or for systems whose estimate ||M_c||_1 ||A~_c||_1 of the condition number
// exceeds kCondFp64) y_c - H_c x_c and H_c^H of it accumulate in double, and the
// estimates converge to the FP32 storage of x_c instead (classical mixed-precision
// refinement).  The fusion and soft outputs then follow the solve
// kernel's epilogue (Eq. fusionrule, Lemma 1, Thm. 3; PD is C = 1).  All sums
// run in a fixed order (deterministic).
#include <cmath>

#include "ffeq_device.cuh"
#include "ffeq_epilogue.cuh"
#include "ffeq_internal.h"

namespace ffeq {
namespace {

constexpr int kRefineThreadsMax = 512;   // per system: 2 S threads, 128..512
constexpr int kFuseThreads = 256;
constexpr float kCondFp64 = 1e4f;        // condition estimate above which the residual is FP64

// Shared memory of one system (cluster c of subcarrier k; S antennas).  The two
// U x U scratch areas serve the steps before the last one (the full next
// inverse) only: with one step (full = false) they are left out, so that more
// systems share an SM.
struct RefineLayout {
  int U, NS, S, SS, W;
  size_t hs, pm, va, rb, rr, an, ae, cn, total;   // offsets in bytes
  __host__ __device__ RefineLayout(int U_, int NS_, int S_, bool full = true)
      : U(U_), NS(NS_), S(S_), SS(S_ + 1), W(U_ + NS_) {
    size_t o = 0;
    hs = o;  o += static_cast<size_t>(U) * SS * 8;      // H_c rows (stride S + 1 complex)
    pm = o;  o += static_cast<size_t>(W) * U * 8;       // columns a_j of A~, then x_n
    va = o;  o += static_cast<size_t>(U) * SS * 8;      // V = H_c a_j per antenna
    rb = o;  o += static_cast<size_t>(NS) * SS * 8;     // y_c - H_c x per antenna
    rr = o;  o += static_cast<size_t>(NS) * U * 8;      // residual
    an = o;  o += full ? static_cast<size_t>(U) * U * 8 : 0;   // next inverse (FP64 residual: E)
    ae = o;  o += full ? static_cast<size_t>(U) * U * 8 : 0;   // next inverse with the FP64 residual
    cn = o;  o += static_cast<size_t>(2) * U * 4;       // column norms for the condition estimate
    total = o;
  }
};

// acc + a b and acc + conj(a) b in double (products of FP32 values are exact).
__device__ __forceinline__ double2 dcfma(float2 a, float2 b, double2 acc) {
  const double ax = a.x, ay = a.y, bx = b.x, by = b.y;
  acc.x = fma(ax, bx, acc.x);
  acc.x = fma(-ay, by, acc.x);
  acc.y = fma(ax, by, acc.y);
  acc.y = fma(ay, bx, acc.y);
  return acc;
}
__device__ __forceinline__ double2 dcfma_conj(float2 a, float2 b, double2 acc) {
  const double ax = a.x, ay = a.y, bx = b.x, by = b.y;
  acc.x = fma(ax, bx, acc.x);
  acc.x = fma(ay, by, acc.x);
  acc.y = fma(ax, by, acc.y);
  acc.y = fma(-ay, bx, acc.y);
  return acc;
}

// C(m, n) = sum_k opA(A(m, k)) opB(B(n, k)) over an M x N output of complex FP32
// values in shared memory, in TM x TN register tiles (each operand loaded once
// per k for the whole tile, so a tile does TM TN complex FMAs per TM + TN loads
// instead of one per two); opX conjugates when CONJ_X.  A(m, k) =
// A[m am + k ak], B(n, k) = B[n bn + k bk].  Tiles go to threads tid, tid + nt, ...;
// out(m, n, c) receives every in-range element.  Out-of-range rows and columns
// of a ragged tile read the last valid row / column (in bounds) and are dropped.
template <int TM, int TN, bool CONJ_A, bool CONJ_B, typename Out>
__device__ __forceinline__ void tiled_cgemm(int M, int N, int K, const float2* A, int am, int ak, const float2* B,
                                            int bn, int bk, int tid, int nt, Out out) {
  const int tm = (M + TM - 1) / TM, tn = (N + TN - 1) / TN;
  for (int t = tid; t < tm * tn; t += nt) {
    const int m0 = (t % tm) * TM, n0 = (t / tm) * TN;
    const float2* ar[TM];
    const float2* br[TN];
#pragma unroll
    for (int i = 0; i < TM; ++i) ar[i] = A + (m0 + i < M ? m0 + i : M - 1) * am;
#pragma unroll
    for (int j = 0; j < TN; ++j) br[j] = B + (n0 + j < N ? n0 + j : N - 1) * bn;
    float2 acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int k = 0; k < K; ++k) {
      float2 a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        a[i] = ar[i][k * ak];
        if (CONJ_A) a[i].y = -a[i].y;
      }
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        b[j] = br[j][k * bk];
        if (CONJ_B) b[j].y = -b[j].y;
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = cfma(a[i], b[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j)
        if (m0 + i < M && n0 + j < N) out(m0 + i, n0 + j, acc[i][j]);
  }
}

// One CTA per local system: `steps` refinement steps, then the refined
// estimates and inverse (diagonal included) go back to the workspace.
__global__ void __launch_bounds__(kRefineThreadsMax) refine_system_kernel(const RefineParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t sys = blockIdx.x;
  const int U = p.U, NS = p.n_sym, Ceff = p.Ceff, B = p.B;
  const int k = static_cast<int>(sys / Ceff), c = static_cast<int>(sys % Ceff);
  const int S = p.cl_off[c + 1] - p.cl_off[c];   // antennas of this cluster
  const RefineLayout L(U, NS, S, p.steps > 1);
  const int SS = L.SS, W = L.W;
  float2* Hs = reinterpret_cast<float2*>(smem + L.hs);
  float2* P = reinterpret_cast<float2*>(smem + L.pm);
  float2* Va = reinterpret_cast<float2*>(smem + L.va);
  float2* Rb = reinterpret_cast<float2*>(smem + L.rb);
  float2* Rr = reinterpret_cast<float2*>(smem + L.rr);
  float2* An = reinterpret_cast<float2*>(smem + L.an);
  float2* Ae = reinterpret_cast<float2*>(smem + L.ae);
  const int tid = threadIdx.x, nt = blockDim.x;
  const float rho = p.rho;
  const float2* Hk = p.H + static_cast<size_t>(k) * U * B + p.cl_off[c];
  const float2* yk = p.y + static_cast<size_t>(k) * NS * B + p.cl_off[c];

  for (int e = tid; e < U * S; e += nt) {
    const int u = e / S, b = e - u * S;
    Hs[u * SS + b] = Hk[static_cast<size_t>(u) * B + b];
  }
  // Wait for the solve kernel (programmatic dependent launch), then its results.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  for (int e = tid; e < W * U; e += nt) {
    const int j = e / U, i = e - j * U;
    P[e] = j < U ? p.As[(sys * U + j) * U + i] : p.Xs[(sys * NS + (j - U)) * U + i];
  }
  __syncthreads();
  const bool failed = p.fails[sys] != 0;
  // Residual precision of this system (block-uniform).  Condition estimate:
  // ||G_c + rho I||_1 from the contraction output (row v of D is column v of the
  // Hermitian G_c) times ||A~_c||_1.
  bool use64 = p.res64 == 2;
  if (p.res64 == 1) {
    float* cs = reinterpret_cast<float*>(smem + L.cn);
    for (int j = tid; j < 2 * U; j += nt) {
      const float2* col = j < U ? p.D + (sys * W + j) * U : P + (j - U) * U;
      float s = j < U ? rho : 0.f;
      for (int i = 0; i < U; ++i) s += sqrtf(fmaf(col[i].x, col[i].x, col[i].y * col[i].y));
      cs[j] = s;
    }
    __syncthreads();
    float mg = 0.f, ma = 0.f;
    for (int j = 0; j < U; ++j) {
      mg = fmaxf(mg, cs[j]);
      ma = fmaxf(ma, cs[U + j]);
    }
    use64 = mg * ma > kCondFp64;
  }

  for (int step = 0; step < p.steps && !failed; ++step) {
    if (!use64) {
      // FP32 residual, register-tiled products.  V = H_c [A~ | X] per (antenna b,
      // column j): the columns a_j of A~ give V, the estimates give y_c - H_c x.
      tiled_cgemm<2, 2, false, false>(S, W, U, Hs, 1, SS, P, U, 1, tid, nt, [&](int b, int j, float2 v) {
        if (j < U) {
          Va[j * SS + b] = v;
        } else {
          const int n = j - U;
          Rb[n * SS + b] = csub(yk[static_cast<size_t>(n) * B + b], v);
        }
      });
      __syncthreads();
      // r = H_c^H (y_c - H_c x) - rho x.
      tiled_cgemm<2, 2, false, true>(NS, U, S, Rb, SS, 1, Hs, SS, 1, tid, nt, [&](int n, int u, float2 v) {
        const float2 x = P[(U + n) * U + u];
        Rr[n * U + u] = make_float2(v.x - rho * x.x, v.y - rho * x.y);
      });
      // The next inverse 2 A - V^H V - rho A^H A (entry (i, j) at j U + i); the
      // second pass gives each thread the same tiles as the first.  After the
      // last step only its diagonal is read (the unbiasing and the fusion
      // weights), which is formed below instead.
      const bool last = step + 1 == p.steps;
      if (!last) {
        tiled_cgemm<2, 2, true, false>(U, U, S, Va, SS, 1, Va, SS, 1, tid, nt, [&](int i2, int j2, float2 v) {
          const float2 a = P[j2 * U + i2];
          An[j2 * U + i2] = make_float2(2.f * a.x - v.x, 2.f * a.y - v.y);
        });
        tiled_cgemm<2, 2, true, false>(U, U, U, P, U, 1, P, U, 1, tid, nt, [&](int i2, int j2, float2 v) {
          float2& o = An[j2 * U + i2];
          o = make_float2(fmaf(-rho, v.x, o.x), fmaf(-rho, v.y, o.y));
        });
      }
      __syncthreads();
      // x += A~ r   (A~[u][v] = column v of A~ at row u).
      tiled_cgemm<2, 2, false, false>(NS, U, U, Rr, U, 1, P, 1, U, tid, nt, [&](int n, int u, float2 v) {
        float2* x = P + (U + n) * U + u;
        *x = cadd(*x, v);
      });
      __syncthreads();
      if (!last) {
        for (int e = tid; e < U * U; e += nt) P[e] = An[e];
      } else {
        // [2 A - (H_c a_j)^H (H_c a_j) - rho a_j^H a_j]_jj for column a_j of A~
        // (thread j reads and writes column j only).
        for (int j = tid; j < U; j += nt) {
          float2 d1 = make_float2(0.f, 0.f), d2 = make_float2(0.f, 0.f);
          for (int b = 0; b < S; ++b) d1 = cfma_conj(Va[j * SS + b], Va[j * SS + b], d1);
          for (int v = 0; v < U; ++v) d2 = cfma_conj(P[j * U + v], P[j * U + v], d2);
          const float2 a = P[j * U + j];
          P[j * U + j] = make_float2(fmaf(-rho, d2.x, 2.f * a.x - d1.x), fmaf(-rho, d2.y, 2.f * a.y - d1.y));
        }
      }
      __syncthreads();
      continue;
    }
    // FP64 residual.  V = H_c [A~ | X] per (antenna b, column j), accumulated in
    // double, the result rounded once (exact differences first).
    for (int e = tid; e < S * W; e += nt) {
      const int j = e / S, b = e - j * S;
      const float2* pj = P + j * U;
      double2 v = make_double2(0.0, 0.0);
      for (int u = 0; u < U; ++u) v = dcfma(Hs[u * SS + b], pj[u], v);
      if (j < U) {
        Va[j * SS + b] = make_float2(static_cast<float>(v.x), static_cast<float>(v.y));
      } else {
        const float2 yv = yk[static_cast<size_t>(j - U) * B + b];
        Rb[(j - U) * SS + b] = make_float2(static_cast<float>(static_cast<double>(yv.x) - v.x),
                                           static_cast<float>(static_cast<double>(yv.y) - v.y));
      }
    }
    __syncthreads();
    // r = H_c^H (y_c - H_c x) - rho x.
    for (int e = tid; e < NS * U; e += nt) {
      const int n = e / U, u = e - n * U;
      const float2 x = P[(U + n) * U + u];
      double2 sum = make_double2(0.0, 0.0);
      for (int b = 0; b < S; ++b) sum = dcfma_conj(Hs[u * SS + b], Rb[n * SS + b], sum);
      const double r = static_cast<double>(rho);
      Rr[e] = make_float2(static_cast<float>(fma(-r, static_cast<double>(x.x), sum.x)),
                          static_cast<float>(fma(-r, static_cast<double>(x.y), sum.y)));
    }
    const bool last = step + 1 == p.steps;
    if (!last) {
      // The residual of the inverse, E = I - M_c A~ = I - H_c^H V - rho A~ (entry
      // (i, j) at j U + i).
      for (int e = tid; e < U * U; e += nt) {
        const int j = e / U, i = e - j * U;   // entry (i, j)
        const float2* aj = P + j * U;
        double2 hv = make_double2(0.0, 0.0);
        for (int b = 0; b < S; ++b) hv = dcfma_conj(Hs[i * SS + b], Va[j * SS + b], hv);
        const double r = static_cast<double>(rho);
        const double id = i == j ? 1.0 : 0.0;
        An[e] = make_float2(static_cast<float>(fma(-r, static_cast<double>(aj[i].x), id - hv.x)),
                            static_cast<float>(fma(-r, static_cast<double>(aj[i].y), -hv.y)));
      }
    }
    __syncthreads();
    // x += A~ r   (A~[u][v] = column v of A~ at row u).
    for (int e = tid; e < NS * U; e += nt) {
      const int n = e / U, u = e - n * U;
      float2 d = make_float2(0.f, 0.f);
      for (int v = 0; v < U; ++v) d = cfma(P[v * U + u], Rr[n * U + v], d);
      float2* x = P + (U + n) * U + u;
      *x = cadd(*x, d);
    }
    if (!last) {
      // The next inverse A~ + A~ E (Newton-Schulz in residual form) into Ae.
      for (int e = tid; e < U * U; e += nt) {
        const int j = e / U, i = e - j * U;
        float2 d = make_float2(0.f, 0.f);
        for (int v = 0; v < U; ++v) d = cfma(P[v * U + i], An[j * U + v], d);
        Ae[e] = cadd(P[e], d);
      }
      __syncthreads();
      for (int e = tid; e < U * U; e += nt) P[e] = Ae[e];
      __syncthreads();
      continue;
    }
    // Last step: only the diagonal of A~ + A~ E is read afterwards,
    // [A~ + A~ E]_jj = A~_jj + sum_v A~_jv E_vj with column j of E formed on the
    // fly (E_vj rounded to FP32 as above); four lanes per column j split the v
    // sum (v = part, part + 4, ...) and add their parts in a fixed butterfly.
    // The x update above reads only the estimates' rows of P besides A~, and
    // column j's diagonal is written by its own lanes after they have read it.
    __syncthreads();
    for (int t = tid; t < ((4 * U + 31) / 32) * 32; t += nt) {
      const int j = t >> 2, part = t & 3;
      float2 d = make_float2(0.f, 0.f);
      if (j < U) {
        const double r = static_cast<double>(rho);
        for (int v = part; v < U; v += 4) {
          double2 hv = make_double2(0.0, 0.0);
          for (int b = 0; b < S; ++b) hv = dcfma_conj(Hs[v * SS + b], Va[j * SS + b], hv);
          const float2 a_vj = P[j * U + v];
          const double id = v == j ? 1.0 : 0.0;
          const float2 ev = make_float2(static_cast<float>(fma(-r, static_cast<double>(a_vj.x), id - hv.x)),
                                        static_cast<float>(fma(-r, static_cast<double>(a_vj.y), -hv.y)));
          d = cfma(P[v * U + j], ev, d);
        }
      }
      d.x += __shfl_xor_sync(kFullMask, d.x, 1);
      d.y += __shfl_xor_sync(kFullMask, d.y, 1);
      d.x += __shfl_xor_sync(kFullMask, d.x, 2);
      d.y += __shfl_xor_sync(kFullMask, d.y, 2);
      if (j < U && part == 0) P[j * U + j] = cadd(P[j * U + j], d);
    }
    __syncthreads();
  }  // Refined estimates and the diagonal of the refined inverse (all that the
  // fusion kernel reads) back to the workspace, in the same layouts.
  for (int e = tid; e < U + NS * U; e += nt) {
    if (e < U) p.As[(sys * U + e) * U + e] = P[e * U + e];
    else p.Xs[sys * NS * U + (e - U)] = P[U * U + (e - U)];
  }
  // Let the fusion kernel start its launch while this grid drains.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Per subcarrier: fusion terms from the refined systems (as the solve kernel:
// weight g / A_uu with g = mu or 1), sum over clusters, z, sigma^2 and LLRs.
__global__ void __launch_bounds__(kFuseThreads) refine_fuse_kernel(const RefineParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int U = p.U, NS = p.n_sym, Ceff = p.Ceff, W = U + NS;
  float2* Fz = reinterpret_cast<float2*>(smem);                        // [Ceff][NS][U]
  float* Dn = reinterpret_cast<float*>(Fz + static_cast<size_t>(Ceff) * NS * U);   // [Ceff][U]
  int* failed = reinterpret_cast<int*>(Dn + static_cast<size_t>(Ceff) * U);
  const int k = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const size_t sys0 = static_cast<size_t>(k) * Ceff;
  const float rho = p.rho;
  if (tid == 0) *failed = 0;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __syncthreads();
  if (tid < Ceff && p.fails[sys0 + tid] != 0) atomicOr(failed, 1);
  for (int e = tid; e < Ceff * U; e += nt) {
    const int c = e / U, u = e - c * U;
    const size_t sys = sys0 + c;
    const float gii = p.D[(sys * W + u) * U + u].x;
    const float A = p.As[(sys * U + u) * U + u].x;
    const float invA = 1.f / A;
    const float mu = gii == 0.f ? 0.f : fmaxf(1.f - rho * A, 0.f);
    Dn[e] = (p.unbiased ? mu : 1.f) * invA;
    for (int n = 0; n < NS; ++n) Fz[(c * NS + n) * U + u] = cscale(p.Xs[(sys * NS + n) * U + u], invA);
  }
  __syncthreads();
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

cudaError_t launch_pdl(const void* fn, dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       const RefineParams& p) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {const_cast<RefineParams*>(&p)};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

}  // namespace

bool refine_fits(int max_S, int U, int n_sym) { return RefineLayout(U, n_sym, max_S).total <= 227 * 1024; }

size_t refine_smem_bytes(int max_S, int U, int n_sym) { return RefineLayout(U, n_sym, max_S).total; }

cudaError_t launch_refine(const RefineParams& p, cudaStream_t stream) {
  static int configured[64] = {0};
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev < 64 && !configured[dev]) {
    err = cudaFuncSetAttribute(refine_system_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    err = cudaFuncSetAttribute(refine_fuse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (err != cudaSuccess) return err;
    configured[dev] = 1;
  }
  const size_t nsys = static_cast<size_t>(p.n_sc) * p.Ceff;
  const int S = p.max_S;   // shared memory and threads for the largest cluster
  const int threads = 2 * S < 128 ? 128 : (2 * S > kRefineThreadsMax ? kRefineThreadsMax : ((2 * S + 31) / 32) * 32);
  err = launch_pdl(reinterpret_cast<const void*>(refine_system_kernel), dim3(static_cast<unsigned>(nsys)),
                   dim3(threads), RefineLayout(p.U, p.n_sym, S, p.steps > 1).total, stream, p);
  if (err != cudaSuccess) return err;
  const size_t fsmem = static_cast<size_t>(p.Ceff) * p.n_sym * p.U * 8 + static_cast<size_t>(p.Ceff) * p.U * 4 + 16;
  return launch_pdl(reinterpret_cast<const void*>(refine_fuse_kernel), dim3(p.n_sc), dim3(kFuseThreads), fsmem,
                    stream, p);
}

}  // namespace ffeq
