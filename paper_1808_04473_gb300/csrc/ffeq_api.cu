// C ABI of the equalizer (see include/ffeq.h): plans, argument validation,
// launches and the host-buffer wrapper.  Nothing here allocates device memory.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <cuda.h>
#include <new>

#include "ffeq.h"
#include "ffeq_internal.h"

struct ffeq_plan {
  ffeq_problem p;
  int Ceff;              // clusters kept apart: C (FD) or 1 (PD: summed on chip)
  size_t workspace;      // bytes of the [n_sc][Ceff][U+n_sym][U] complex workspace
  int gram_variant = 0;  // contraction launch shape (0: default)
  int gram_stages = 0;   // staged units per CTA (0: as many as fit)
  size_t off_X = 0, off_A = 0, off_F = 0;   // refinement arrays in the workspace
  ffeq::TensorMapCache* maps = nullptr;      // streamed contraction: encoded maps of recent inputs
  bool cl_uniform = true;                    // clusters of B / C antennas
  int cl_off[ffeq::kMaxClusters + 1] = {};   // otherwise cluster c: antennas [cl_off[c], cl_off[c+1])
  int max_S = 0;                             // antennas of the largest cluster (FD; B for PD)
  ~ffeq_plan() { ffeq::tensor_map_cache_destroy(maps); }
};

namespace {

thread_local char g_last_cuda_error[256] = "no error";

ffeq_status cuda_fail(cudaError_t e) {
  std::strncpy(g_last_cuda_error, cudaGetErrorString(e), sizeof(g_last_cuda_error) - 1);
  return FFEQ_ERR_CUDA;
}

}  // namespace

namespace ffeq {
int record_cuda_error(cudaError_t e) { return static_cast<int>(cuda_fail(e)); }

unsigned long long current_context_id() {
  // cuCtxGetCurrent / cuCtxGetId from the driver, looked up once through the
  // runtime (no link-time dependency on the driver library).
  using GetCurrentFn = CUresult (*)(CUcontext*);
  using GetIdFn = CUresult (*)(CUcontext, unsigned long long*);
  static const GetCurrentFn get_current = []() -> GetCurrentFn {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<GetCurrentFn>(f);
    return nullptr;
  }();
  static const GetIdFn get_id = []() -> GetIdFn {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<GetIdFn>(f);
    return nullptr;
  }();
  CUcontext ctx = nullptr;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  unsigned long long id = 0;
  return get_id(ctx, &id) == CUDA_SUCCESS ? id : 0;
}

void* cached_symbol_address(SymbolAddressCache& cache, cudaError_t (*fetch)(void**), cudaError_t* err) {
  *err = cudaSuccess;
  unsigned long long id = current_context_id();
  std::lock_guard<std::mutex> lock(cache.m);
  for (int i = 0; i < cache.n && id != 0; ++i)
    if (cache.id[i] == id) return cache.ptr[i];
  void* p = nullptr;
  const cudaError_t e = fetch(&p);
  if (e != cudaSuccess || !p) {
    *err = e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    return nullptr;
  }
  if (id == 0) id = current_context_id();   // the lookup made the primary context current
  if (id != 0) {
    const int slot = cache.n < SymbolAddressCache::kEntries ? cache.n++ : (cache.next++ % SymbolAddressCache::kEntries);
    cache.id[slot] = id;
    cache.ptr[slot] = p;
  }
  return p;
}
}  // namespace ffeq

namespace {

constexpr size_t kSolveSmemLimit = 227 * 1024;
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

struct Sizes {
  size_t H, y, z, s2, llr, info;
};

Sizes buffer_sizes(const ffeq_problem& p) {
  Sizes s;
  const size_t nsc = static_cast<size_t>(p.n_sc);
  s.H = nsc * p.U * p.B * 8;
  s.y = nsc * p.n_sym * p.B * 8;
  s.z = nsc * p.n_sym * p.U * 8;
  s.s2 = nsc * p.U * 4 * (p.equalizer == FFEQ_LAMA ? p.n_sym : 1);   // LAMA: per received vector
  s.llr = nsc * p.n_sym * p.U * p.llr_bits * 4;
  s.info = nsc * (p.arch == FFEQ_FD ? p.C : 1) * 4;
  return s;
}

}  // namespace

extern "C" {

int ffeq_version(void) { return 100; }

const char* ffeq_status_string(ffeq_status s) {
  switch (s) {
    case FFEQ_OK: return "ok";
    case FFEQ_ERR_INVALID_ARG: return "invalid argument";
    case FFEQ_ERR_UNSUPPORTED: return "unsupported problem size for this build";
    case FFEQ_ERR_CUDA: return "CUDA runtime error";
    case FFEQ_ERR_TIMEOUT: return "bounded device wait timed out";
  }
  return "unknown status";
}

const char* ffeq_last_cuda_error(void) { return g_last_cuda_error; }

ffeq_status ffeq_plan_create(ffeq_plan** out, const ffeq_problem* p) {
  return ffeq_plan_create_clusters(out, p, nullptr);
}

ffeq_status ffeq_plan_create_clusters(ffeq_plan** out, const ffeq_problem* p, const int* cluster_sizes) {
  if (!out || !p) return FFEQ_ERR_INVALID_ARG;
  *out = nullptr;
  if (p->B <= 0 || p->U <= 0 || p->C <= 0 || p->n_sc < 0 || p->n_sym <= 0) return FFEQ_ERR_INVALID_ARG;
  if (!cluster_sizes && p->B % p->C != 0) return FFEQ_ERR_INVALID_ARG;
  // Clusters of given sizes (Sec. II-B): C sizes >= 0 summing to B.
  bool uniform = true;
  int off[ffeq::kMaxClusters + 1] = {};
  int max_S = p->B / p->C;
  if (cluster_sizes) {
    if (p->C > ffeq::kMaxClusters) return p->arch == FFEQ_FD ? FFEQ_ERR_UNSUPPORTED : FFEQ_ERR_INVALID_ARG;
    long long sum = 0;
    max_S = 0;
    for (int c = 0; c < p->C; ++c) {
      if (cluster_sizes[c] < 0) return FFEQ_ERR_INVALID_ARG;
      off[c] = static_cast<int>(sum);
      sum += cluster_sizes[c];
      if (cluster_sizes[c] > max_S) max_S = cluster_sizes[c];
      if (sum > p->B) return FFEQ_ERR_INVALID_ARG;
      if (cluster_sizes[c] != cluster_sizes[0]) uniform = false;
    }
    if (sum != p->B) return FFEQ_ERR_INVALID_ARG;
    off[p->C] = p->B;
  }
  if (p->arch != FFEQ_PD && p->arch != FFEQ_FD) return FFEQ_ERR_INVALID_ARG;
  if (p->precision != FFEQ_FP32 && p->precision != FFEQ_TF32X3 && p->precision != FFEQ_BF16X3 &&
      p->precision != FFEQ_FP16X3)
    return FFEQ_ERR_INVALID_ARG;
  if (p->estimate != FFEQ_UNBIASED && p->estimate != FFEQ_LITERAL) return FFEQ_ERR_INVALID_ARG;
  if (p->llr_bits != 0 && p->llr_bits != 2 && p->llr_bits != 4 && p->llr_bits != 6 && p->llr_bits != 8)
    return FFEQ_ERR_INVALID_ARG;
  if (p->refine < 0 || p->refine > 4) return FFEQ_ERR_INVALID_ARG;
  if (p->refine_fp64 < 0 || p->refine_fp64 > 2 || (p->refine_fp64 > 0 && p->refine == 0))
    return FFEQ_ERR_INVALID_ARG;
  if (p->equalizer != FFEQ_LMMSE && p->equalizer != FFEQ_ZF && p->equalizer != FFEQ_MRC &&
      p->equalizer != FFEQ_LAMA)
    return FFEQ_ERR_INVALID_ARG;
  if ((p->equalizer == FFEQ_MRC || p->equalizer == FFEQ_LAMA) && p->refine > 0)
    return FFEQ_ERR_INVALID_ARG;   // nothing is solved
  if (p->equalizer == FFEQ_LAMA ? (p->lama_iters < 1 || p->lama_iters > 64 || p->llr_bits == 0)
                                : p->lama_iters != 0)
    return FFEQ_ERR_INVALID_ARG;   // LAMA's prior is the LLR constellation
  if (p->U > 32 || p->n_sym > ffeq::kNsymMax) return FFEQ_ERR_UNSUPPORTED;
  const int Ceff = p->arch == FFEQ_FD ? p->C : 1;
  if (ffeq::gram_stages(p->precision, p->B, p->U, p->n_sym, Ceff, false) < 1) return FFEQ_ERR_UNSUPPORTED;
  const int spc = ffeq::solve_subcarriers_per_cta(p->U, Ceff);
  if (spc * Ceff * ffeq::padded_users(p->U) * (Ceff == 1 && ffeq::padded_users(p->U) == 16 ? 2 : 1) > 512 ||
      ffeq::solve_smem_bytes(p->U, Ceff) > kSolveSmemLimit)
    return FFEQ_ERR_UNSUPPORTED;
  if (Ceff == 1) {
    uniform = true;          // PD sums every cluster: the partition does not enter (Eq. fullMRC)
    max_S = p->B;
  }
  if (p->refine > 0 && !ffeq::refine_fits(max_S, p->U, p->n_sym)) return FFEQ_ERR_UNSUPPORTED;
  ffeq_plan* plan = new (std::nothrow) ffeq_plan;
  if (!plan) return FFEQ_ERR_INVALID_ARG;
  plan->p = *p;
  plan->Ceff = Ceff;
  plan->cl_uniform = uniform;
  plan->max_S = max_S;
  for (int c = 0; c <= Ceff && !uniform; ++c) plan->cl_off[c] = off[c];
  plan->maps = ffeq::tensor_map_cache_create();   // nullptr only on allocation failure: then encode every call
  plan->workspace = static_cast<size_t>(p->n_sc) * Ceff * (p->U + p->n_sym) * p->U * 8;
  if (p->refine > 0) {
    // Refinement keeps the local estimates, the inverses and the pivot status.
    const size_t sys = static_cast<size_t>(p->n_sc) * Ceff;
    plan->off_X = align_up(plan->workspace);
    plan->off_A = align_up(plan->off_X + sys * p->n_sym * p->U * 8);
    plan->off_F = align_up(plan->off_A + sys * p->U * p->U * 8);
    plan->workspace = plan->off_F + sys * 4;
  }
  *out = plan;
  return FFEQ_OK;
}

void ffeq_plan_destroy(ffeq_plan* plan) { delete plan; }

ffeq_status ffeq_workspace_size(const ffeq_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return FFEQ_ERR_INVALID_ARG;
  *bytes = plan->workspace;
  return FFEQ_OK;
}

namespace {

ffeq_status check_common(const ffeq_plan* plan, const void* workspace, size_t workspace_bytes) {
  if (!plan) return FFEQ_ERR_INVALID_ARG;
  if (plan->p.n_sc == 0) return FFEQ_OK;
  if (!workspace || workspace_bytes < plan->workspace || !aligned(workspace, 16)) return FFEQ_ERR_INVALID_ARG;
  return FFEQ_OK;
}

// Contraction parameters of a plan for inputs H, y (workspace D).
ffeq_status gram_params(const ffeq_plan* plan, const void* H, const void* y, void* workspace, bool host_inputs,
                        ffeq::GramParams& gp) {
  const ffeq_problem& p = plan->p;
  if (!H || !y || !aligned(H, 8) || !aligned(y, 8)) return FFEQ_ERR_INVALID_ARG;
  gp = ffeq::GramParams{};
  gp.H = static_cast<const float2*>(H);
  gp.y = static_cast<const float2*>(y);
  gp.D = static_cast<float2*>(workspace);
  gp.status = ffeq::device_status_ptr();
  gp.B = p.B;
  gp.U = p.U;
  gp.Ceff = plan->Ceff;
  gp.n_sc = p.n_sc;
  gp.n_sym = p.n_sym;
  // Inputs in host memory (read in place over the host link) take plain loads.
  gp.bulk = !host_inputs && (p.B % 2 == 0) && aligned(H, 16) && aligned(y, 16);
  gp.map_cache = plan->maps;
  gp.cl_uniform = plan->cl_uniform ? 1 : 0;
  for (int c = 0; c <= plan->Ceff && !plan->cl_uniform; ++c) gp.cl_off[c] = plan->cl_off[c];
  if (!ffeq::gram_configure(gp, p.precision, plan->gram_variant, plan->gram_stages)) return FFEQ_ERR_UNSUPPORTED;
  return FFEQ_OK;
}

ffeq_status local_preprocess(const ffeq_plan* plan, const void* H, const void* y, void* workspace,
                             cudaStream_t st, bool host_inputs = false) {
  ffeq::GramParams gp;
  const ffeq_status r = gram_params(plan, H, y, workspace, host_inputs, gp);
  if (r != FFEQ_OK) return r;
  const cudaError_t e = plan->p.precision == FFEQ_FP32 ? ffeq::launch_gram_fp32(gp, st)
                                                       : ffeq::launch_gram_tc(gp, plan->p.precision, st);
  return e == cudaSuccess ? FFEQ_OK : cuda_fail(e);
}

// Solve / fusion / soft-output parameters of a plan (outputs checked here).
ffeq_status solve_params(const ffeq_plan* plan, const void* workspace, float N0, float Es, void* z, float* sigma2,
                         float* llr, int* info, ffeq::SolveParams& sp) {
  const ffeq_problem& p = plan->p;
  if (!(N0 >= 0.f) || !std::isfinite(N0) || !(Es > 0.f) || !std::isfinite(Es)) return FFEQ_ERR_INVALID_ARG;
  if (!z || !sigma2 || !aligned(z, 8) || !aligned(sigma2, 4)) return FFEQ_ERR_INVALID_ARG;
  if (p.llr_bits && !llr) return FFEQ_ERR_INVALID_ARG;
  if (p.equalizer == FFEQ_LAMA && !(N0 > 0.f)) return FFEQ_ERR_INVALID_ARG;   // the denoiser needs tau > 0
  if ((llr && !aligned(llr, 4)) || (info && !aligned(info, 4))) return FFEQ_ERR_INVALID_ARG;
  sp = ffeq::SolveParams{};
  sp.D = static_cast<const float2*>(workspace);
  sp.z = static_cast<float2*>(z);
  sp.sigma2 = sigma2;
  sp.llr = p.llr_bits ? llr : nullptr;
  sp.info = info;
  sp.U = p.U;
  sp.Ceff = plan->Ceff;
  sp.n_sc = p.n_sc;
  sp.n_sym = p.n_sym;
  sp.spc = ffeq::solve_subcarriers_per_cta(p.U, plan->Ceff);
  // Zero forcing is the L-MMSE sweep with rho = 0 and the literal pairs (whose
  // gain is 1 there); MRC has its own kernel.
  const bool zf = p.equalizer == FFEQ_ZF;
  sp.unbiased = !zf && p.estimate == FFEQ_UNBIASED;
  sp.llr_bits = p.llr_bits;
  sp.N0 = N0;
  sp.Es = Es;
  sp.equalizer = p.equalizer;
  sp.rho = zf ? 0.f : static_cast<float>(static_cast<double>(N0) / static_cast<double>(Es));
  if (p.llr_bits) {
    const double L = static_cast<double>(1 << (p.llr_bits / 2));
    sp.llr_scale = static_cast<float>(std::sqrt(static_cast<double>(Es) / (2.0 * (L * L - 1.0) / 3.0)));
  } else {
    sp.llr_scale = 0.f;
  }
  return FFEQ_OK;
}

ffeq_status fuse_equalize(const ffeq_plan* plan, const void* workspace, float N0, float Es, void* z,
                          float* sigma2, float* llr, int* info, cudaStream_t st, const void* H = nullptr,
                          const void* y = nullptr) {
  const ffeq_problem& p = plan->p;
  ffeq::SolveParams sp;
  const ffeq_status r = solve_params(plan, workspace, N0, Es, z, sigma2, llr, info, sp);
  if (r != FFEQ_OK) return r;
  if (p.refine > 0) {
    if (!H || !y) return FFEQ_ERR_UNSUPPORTED;   // the residual needs the inputs
    unsigned char* ws = static_cast<unsigned char*>(const_cast<void*>(workspace));
    sp.Xs = reinterpret_cast<float2*>(ws + plan->off_X);
    sp.As = reinterpret_cast<float2*>(ws + plan->off_A);
    sp.fails = reinterpret_cast<int*>(ws + plan->off_F);
  }
  if (p.equalizer == FFEQ_LAMA) {
    sp.lama_iters = p.lama_iters;
    for (int c = 0; c < plan->Ceff; ++c)
      sp.cl_size[c] = plan->Ceff == 1 ? p.B
                    : (plan->cl_uniform ? p.B / plan->Ceff : plan->cl_off[c + 1] - plan->cl_off[c]);
    const cudaError_t el = ffeq::launch_lama(sp, st);
    return el == cudaSuccess ? FFEQ_OK : cuda_fail(el);
  }
  cudaError_t e = ffeq::launch_solve(sp, st);
  if (e != cudaSuccess || p.refine == 0) return e == cudaSuccess ? FFEQ_OK : cuda_fail(e);
  ffeq::RefineParams rp{};
  rp.H = static_cast<const float2*>(H);
  rp.y = static_cast<const float2*>(y);
  rp.D = static_cast<const float2*>(workspace);
  rp.As = sp.As;
  rp.Xs = sp.Xs;
  rp.fails = sp.fails;
  rp.z = sp.z;
  rp.sigma2 = sp.sigma2;
  rp.llr = sp.llr;
  rp.B = p.B;
  rp.U = p.U;
  rp.Ceff = plan->Ceff;
  rp.n_sc = p.n_sc;
  rp.n_sym = p.n_sym;
  rp.steps = p.refine;
  rp.res64 = p.refine_fp64;
  rp.max_S = plan->max_S;
  for (int c = 0; c <= plan->Ceff; ++c)
    rp.cl_off[c] = plan->cl_uniform ? c * (p.B / plan->Ceff) : plan->cl_off[c];
  rp.unbiased = sp.unbiased;
  rp.llr_bits = p.llr_bits;
  rp.N0 = sp.N0;
  rp.rho = sp.rho;
  rp.llr_scale = sp.llr_scale;
  e = ffeq::launch_refine(rp, st);
  return e == cudaSuccess ? FFEQ_OK : cuda_fail(e);
}

bool bad_scalars(float N0, float Es) {
  return !(N0 >= 0.f) || !std::isfinite(N0) || !(Es > 0.f) || !std::isfinite(Es);
}

}  // namespace

ffeq_status ffeq_local_preprocess(const ffeq_plan* plan, const void* H, const void* y, void* workspace,
                                  size_t workspace_bytes, void* stream) {
  ffeq_status r = check_common(plan, workspace, workspace_bytes);
  if (r != FFEQ_OK || plan->p.n_sc == 0) return r;
  return local_preprocess(plan, H, y, workspace, static_cast<cudaStream_t>(stream));
}

ffeq_status ffeq_fuse_equalize(const ffeq_plan* plan, const void* workspace, size_t workspace_bytes, float N0,
                               float Es, void* z, float* sigma2, float* llr, int* info, void* stream) {
  if (plan && bad_scalars(N0, Es)) return FFEQ_ERR_INVALID_ARG;
  ffeq_status r = check_common(plan, workspace, workspace_bytes);
  if (r != FFEQ_OK || plan->p.n_sc == 0) return r;
  return fuse_equalize(plan, workspace, N0, Es, z, sigma2, llr, info, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace {
ffeq_status equalize_impl(const ffeq_plan* plan, const void* H, const void* y, float N0, float Es, void* z,
                          float* sigma2, float* llr, int* info, void* workspace, size_t workspace_bytes,
                          void* stream, bool host_inputs);
}  // namespace

extern "C" {

ffeq_status ffeq_equalize(const ffeq_plan* plan, const void* H, const void* y, float N0, float Es, void* z,
                          float* sigma2, float* llr, int* info, void* workspace, size_t workspace_bytes,
                          void* stream) {
  return equalize_impl(plan, H, y, N0, Es, z, sigma2, llr, info, workspace, workspace_bytes, stream, false);
}

}  // extern "C"

namespace {

ffeq_status equalize_impl(const ffeq_plan* plan, const void* H, const void* y, float N0, float Es, void* z,
                          float* sigma2, float* llr, int* info, void* workspace, size_t workspace_bytes,
                          void* stream, bool host_inputs) {
  if (plan && bad_scalars(N0, Es)) return FFEQ_ERR_INVALID_ARG;
  ffeq_status r = check_common(plan, workspace, workspace_bytes);
  if (r != FFEQ_OK || plan->p.n_sc == 0) return r;
  const ffeq_problem& p = plan->p;
  // Validate every pointer before the first launch.
  if (!H || !y || !aligned(H, 8) || !aligned(y, 8)) return FFEQ_ERR_INVALID_ARG;
  if (!z || !sigma2 || !aligned(z, 8) || !aligned(sigma2, 4)) return FFEQ_ERR_INVALID_ARG;
  if (p.llr_bits && !llr) return FFEQ_ERR_INVALID_ARG;
  if ((llr && !aligned(llr, 4)) || (info && !aligned(info, 4))) return FFEQ_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (plan->gram_variant == ffeq::kGramFused && !host_inputs) {
    // One launch: the streamed contraction with the solve, fusion and soft
    // outputs in the same CTAs (16-byte aligned inputs; otherwise the separate
    // kernels below, which give the same results).
    ffeq::GramParams gp;
    r = gram_params(plan, H, y, workspace, false, gp);
    if (r != FFEQ_OK) return r;
    if (gp.bulk) {
      ffeq::SolveParams sp;
      r = solve_params(plan, workspace, N0, Es, z, sigma2, llr, info, sp);
      if (r != FFEQ_OK) return r;
      const cudaError_t e = ffeq::launch_gram_fused(gp, sp, p.precision, st);
      return e == cudaSuccess ? FFEQ_OK : cuda_fail(e);
    }
  }
  r = local_preprocess(plan, H, y, workspace, st, host_inputs);
  if (r != FFEQ_OK) return r;
  return fuse_equalize(plan, workspace, N0, Es, z, sigma2, llr, info, st, H, y);
}

// Device view of a host buffer the GPU can address in place (page-locked or
// registered memory), else nullptr.
void* device_view(const void* host) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

}  // namespace

extern "C" {

namespace {

struct TrainLayoutBytes {
  size_t D, X, Gb, W, P, total;
};

TrainLayoutBytes train_layout(const ffeq_plan* plan) {
  const ffeq_problem& p = plan->p;
  const size_t nsc = static_cast<size_t>(p.n_sc), C = static_cast<size_t>(p.C);
  TrainLayoutBytes t;
  t.D = align_up(plan->workspace);
  t.X = align_up(nsc * C * p.n_sym * p.U * 8);
  t.Gb = t.X;
  t.W = align_up(nsc * C * p.U * p.U * 8);
  t.P = align_up(nsc * C * (1 + p.U) * 4);
  t.total = t.D + t.X + t.Gb + t.W + t.P;
  return t;
}

ffeq_status train_params(const ffeq_plan* plan, const void* H, const void* y, const float* rho_c, const float* nu,
                         void* workspace, size_t workspace_bytes, ffeq::TrainParams& tp) {
  if (!plan) return FFEQ_ERR_INVALID_ARG;
  const ffeq_problem& p = plan->p;
  if (p.arch != FFEQ_FD) return FFEQ_ERR_INVALID_ARG;
  if (p.equalizer != FFEQ_LMMSE) return FFEQ_ERR_UNSUPPORTED;   // the differentiable form is L-MMSE
  if (ffeq::padded_users(p.U) * p.C > 512 || ffeq::train_smem_bytes(p.U, p.C) > kSolveSmemLimit)
    return FFEQ_ERR_UNSUPPORTED;
  const TrainLayoutBytes t = train_layout(plan);
  if (p.n_sc == 0) return FFEQ_OK;
  if (!H || !y || !rho_c || !nu || !workspace || workspace_bytes < t.total) return FFEQ_ERR_INVALID_ARG;
  if (!aligned(H, 8) || !aligned(y, 8) || !aligned(rho_c, 4) || !aligned(nu, 4) || !aligned(workspace, 256))
    return FFEQ_ERR_INVALID_ARG;
  char* base = static_cast<char*>(workspace);
  tp = ffeq::TrainParams{};
  tp.H = static_cast<const float2*>(H);
  tp.y = static_cast<const float2*>(y);
  tp.D = reinterpret_cast<const float2*>(base);
  tp.X = reinterpret_cast<float2*>(base + t.D);
  tp.Gb = reinterpret_cast<float2*>(base + t.D + t.X);
  tp.Wm = reinterpret_cast<float2*>(base + t.D + t.X + t.Gb);
  tp.P = reinterpret_cast<float*>(base + t.D + t.X + t.Gb + t.W);
  tp.rho_c = rho_c;
  tp.nu = nu;
  tp.B = p.B;
  tp.U = p.U;
  tp.C = p.C;
  tp.n_sc = p.n_sc;
  tp.n_sym = p.n_sym;
  tp.cl_uniform = plan->cl_uniform ? 1 : 0;   // else cluster c holds antennas [cl_off[c], cl_off[c + 1])
  for (int c = 0; c <= p.C && !plan->cl_uniform; ++c) tp.cl_off[c] = plan->cl_off[c];
  return FFEQ_OK;
}

struct OptimalLayoutBytes {
  size_t D, Gb, W, total;
};

OptimalLayoutBytes optimal_layout(const ffeq_plan* plan) {
  const ffeq_problem& p = plan->p;
  const size_t nsc = static_cast<size_t>(p.n_sc), C = static_cast<size_t>(p.C);
  OptimalLayoutBytes t;
  t.D = align_up(plan->workspace);
  t.Gb = align_up(nsc * C * p.n_sym * p.U * 8);
  t.W = align_up(nsc * C * p.U * p.U * 8);
  t.total = t.D + t.Gb + t.W;
  return t;
}

// The plan's forward must be the one differentiated: FD, L-MMSE, unbiased
// pairs, no refinement; the CTA of one subcarrier must fit.
ffeq_status optimal_plan_ok(const ffeq_plan* plan) {
  if (!plan) return FFEQ_ERR_INVALID_ARG;
  const ffeq_problem& p = plan->p;
  if (p.arch != FFEQ_FD || p.equalizer != FFEQ_LMMSE || p.estimate != FFEQ_UNBIASED || p.refine != 0)
    return FFEQ_ERR_INVALID_ARG;
  if (ffeq::padded_users(p.U) * p.C > 512 || ffeq::train_optimal_smem_bytes(p.U, p.C) > kSolveSmemLimit)
    return FFEQ_ERR_UNSUPPORTED;
  return FFEQ_OK;
}

}  // namespace

ffeq_status ffeq_fd_optimal_workspace_size(const ffeq_plan* plan, size_t* bytes) {
  if (!bytes) return FFEQ_ERR_INVALID_ARG;
  const ffeq_status r = optimal_plan_ok(plan);
  if (r != FFEQ_OK) return r;
  *bytes = optimal_layout(plan).total;
  return FFEQ_OK;
}

ffeq_status ffeq_fd_optimal_backward(const ffeq_plan* plan, const void* H, const void* y, float N0, float Es,
                                     const void* gz, void* gH, void* gy, void* workspace, size_t workspace_bytes,
                                     void* stream) {
  ffeq_status r = optimal_plan_ok(plan);
  if (r != FFEQ_OK) return r;
  if (bad_scalars(N0, Es)) return FFEQ_ERR_INVALID_ARG;
  const ffeq_problem& p = plan->p;
  if (p.n_sc == 0) return FFEQ_OK;
  const OptimalLayoutBytes t = optimal_layout(plan);
  if (!H || !y || !gz || !gH || !gy || !workspace || workspace_bytes < t.total) return FFEQ_ERR_INVALID_ARG;
  if (!aligned(H, 8) || !aligned(y, 8) || !aligned(gz, 8) || !aligned(gH, 8) || !aligned(gy, 8) ||
      !aligned(workspace, 256))
    return FFEQ_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool fused = p.precision == FFEQ_FP32 && ffeq::train_optimal_fused_fits(p.U, p.n_sym, p.B, p.C);
  if (!fused) {
    r = local_preprocess(plan, H, y, workspace, st);
    if (r != FFEQ_OK) return r;
  }
  char* base = static_cast<char*>(workspace);
  ffeq::TrainParams tp{};
  tp.H = static_cast<const float2*>(H);
  tp.y = static_cast<const float2*>(y);
  tp.D = reinterpret_cast<const float2*>(base);
  tp.Gb = reinterpret_cast<float2*>(base + t.D);
  tp.Wm = reinterpret_cast<float2*>(base + t.D + t.Gb);
  tp.gz = static_cast<const float2*>(gz);
  tp.gH = static_cast<float2*>(gH);
  tp.gy = static_cast<float2*>(gy);
  tp.B = p.B;
  tp.U = p.U;
  tp.C = p.C;
  tp.n_sc = p.n_sc;
  tp.n_sym = p.n_sym;
  tp.rho = static_cast<float>(static_cast<double>(N0) / static_cast<double>(Es));
  tp.status = ffeq::device_status_ptr();
  tp.cl_uniform = plan->cl_uniform ? 1 : 0;
  for (int c = 0; c <= p.C && !plan->cl_uniform; ++c) tp.cl_off[c] = plan->cl_off[c];
  const cudaError_t e = fused ? ffeq::launch_train_optimal_backward_fused(tp, st)
                              : ffeq::launch_train_optimal_backward(tp, st);
  return e == cudaSuccess ? FFEQ_OK : cuda_fail(e);
}

ffeq_status ffeq_fd_train_workspace_size(const ffeq_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return FFEQ_ERR_INVALID_ARG;
  *bytes = train_layout(plan).total;
  return FFEQ_OK;
}

namespace {
// The training pair runs fused (Gram matrices formed in the solving CTA) for
// FP32 plans whose subcarrier fits in one CTA's shared memory; the same choice
// for both passes, so the backward never looks for a workspace D the forward
// did not write.
bool train_fused(const ffeq_plan* plan) {
  const ffeq_problem& p = plan->p;
  return p.precision == FFEQ_FP32 && ffeq::train_fused_fits(p.U, p.n_sym, p.B, p.C);
}
}  // namespace

ffeq_status ffeq_fd_train_forward(const ffeq_plan* plan, const void* H, const void* y, const float* rho_c,
                                  const float* nu, void* z, void* workspace, size_t workspace_bytes, void* stream) {
  ffeq::TrainParams tp;
  ffeq_status r = train_params(plan, H, y, rho_c, nu, workspace, workspace_bytes, tp);
  if (r != FFEQ_OK || plan->p.n_sc == 0) return r;
  if (!z || !aligned(z, 8)) return FFEQ_ERR_INVALID_ARG;
  tp.z = static_cast<float2*>(z);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (train_fused(plan)) {
    const cudaError_t e = ffeq::launch_train_forward_fused(tp, st);
    return e == cudaSuccess ? FFEQ_OK : cuda_fail(e);
  }
  r = local_preprocess(plan, H, y, workspace, st);
  if (r != FFEQ_OK) return r;
  const cudaError_t e = ffeq::launch_train_forward(tp, st);
  return e == cudaSuccess ? FFEQ_OK : cuda_fail(e);
}

ffeq_status ffeq_fd_train_backward(const ffeq_plan* plan, const void* H, const void* y, const float* rho_c,
                                   const float* nu, const void* gz, void* gH, void* gy, float* grho, float* gnu,
                                   void* workspace, size_t workspace_bytes, void* stream) {
  ffeq::TrainParams tp;
  ffeq_status r = train_params(plan, H, y, rho_c, nu, workspace, workspace_bytes, tp);
  if (r != FFEQ_OK || plan->p.n_sc == 0) return r;
  if (!gz || !gH || !gy || !grho || !gnu) return FFEQ_ERR_INVALID_ARG;
  if (!aligned(gz, 8) || !aligned(gH, 8) || !aligned(gy, 8) || !aligned(grho, 4) || !aligned(gnu, 4))
    return FFEQ_ERR_INVALID_ARG;
  tp.gz = static_cast<const float2*>(gz);
  tp.gH = static_cast<float2*>(gH);
  tp.gy = static_cast<float2*>(gy);
  tp.grho = grho;
  tp.gnu = gnu;
  const cudaError_t e = train_fused(plan) ? ffeq::launch_train_backward_fused(tp, static_cast<cudaStream_t>(stream))
                                          : ffeq::launch_train_backward(tp, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? FFEQ_OK : cuda_fail(e);
}

ffeq_status ffeq_host_staging_size(const ffeq_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return FFEQ_ERR_INVALID_ARG;
  const Sizes s = buffer_sizes(plan->p);
  size_t ws = 0;
  ffeq_workspace_size(plan, &ws);
  *bytes = align_up(s.H) + align_up(s.y) + align_up(s.z) + align_up(s.s2) + align_up(s.llr) +
           align_up(s.info) + align_up(ws);
  return FFEQ_OK;
}

ffeq_status ffeq_plan_get_tuning(const ffeq_plan* plan, int* values, int n) {
  if (!plan || n < 0 || (n > 0 && !values)) return FFEQ_ERR_INVALID_ARG;
  const int v[2] = {plan->gram_variant, plan->gram_stages};
  for (int i = 0; i < n && i < 2; ++i) values[i] = v[i];
  return FFEQ_OK;
}

ffeq_status ffeq_plan_set_tuning(ffeq_plan* plan, const int* values, int n) {
  if (!plan || n != 2 || !values) return FFEQ_ERR_INVALID_ARG;
  if (values[0] < ffeq::kGramAuto || values[0] > ffeq::kGramVariantMax || values[1] < 0 ||
      values[1] > ((values[0] == ffeq::kGramStream || values[0] == ffeq::kGramStreamHalf) ? ffeq::kGramStreamRing : 3))
    return FFEQ_ERR_INVALID_ARG;
  // The shape must fit the problem with 16-byte aligned rows (the bulk-staged case).
  ffeq::GramParams gp{};
  gp.B = plan->p.B;
  gp.U = plan->p.U;
  gp.Ceff = plan->Ceff;
  gp.n_sc = plan->p.n_sc;
  gp.n_sym = plan->p.n_sym;
  gp.bulk = plan->p.B % 2 == 0;
  gp.cl_uniform = plan->cl_uniform ? 1 : 0;
  if (!ffeq::gram_configure(gp, plan->p.precision, values[0], values[1])) return FFEQ_ERR_UNSUPPORTED;
  // The fused shape solves in the contraction's CTAs: L-MMSE or ZF without refinement.
  if (values[0] == ffeq::kGramFused &&
      (plan->p.refine != 0 || (plan->p.equalizer != FFEQ_LMMSE && plan->p.equalizer != FFEQ_ZF)))
    return FFEQ_ERR_UNSUPPORTED;
  plan->gram_variant = values[0];
  plan->gram_stages = values[1];
  return FFEQ_OK;
}

ffeq_status ffeq_plan_autotune(ffeq_plan* plan, const void* H, const void* y, float N0, float Es, void* z,
                               float* sigma2, float* llr, int* info, void* workspace, size_t workspace_bytes,
                               void* stream, int reps) {
  return ffeq_plan_autotune_sets(plan, &H, &y, 1, N0, Es, z, sigma2, llr, info, workspace, workspace_bytes, stream,
                                 reps);
}

namespace {

// Device time of `reps` calls of ffeq_equalize on stream cs, reading the input
// sets in rotation: captured once into a CUDA graph and replayed (after one
// untimed replay), so that host launch gaps do not enter the comparison; eager
// calls if the capture is refused.  Returns a negative time on failure.
float time_equalize_calls(ffeq_plan* plan, const void* const* H, const void* const* y, int n_sets, float N0,
                          float Es, void* z, float* sigma2, float* llr, int* info, void* workspace,
                          size_t workspace_bytes, cudaStream_t cs, int reps, cudaEvent_t e0, cudaEvent_t e1,
                          ffeq_status* st_out) {
  ffeq_status s = FFEQ_OK;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    for (int r = 0; r < reps && s == FFEQ_OK; ++r)
      s = ffeq_equalize(plan, H[r % n_sets], y[r % n_sets], N0, Es, z, sigma2, llr, info, workspace,
                        workspace_bytes, cs);
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (s != FFEQ_OK || ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      graph = nullptr;
      exec = nullptr;
      cudaGetLastError();
      s = FFEQ_OK;
    }
  } else {
    cudaGetLastError();
  }
  float ms = -1.f;
  bool ok = true;
  if (exec) {
    ok = cudaGraphLaunch(exec, cs) == cudaSuccess && cudaEventRecord(e0, cs) == cudaSuccess &&
         cudaGraphLaunch(exec, cs) == cudaSuccess;
  } else {
    ok = cudaEventRecord(e0, cs) == cudaSuccess;
    for (int r = 0; r < reps && ok && s == FFEQ_OK; ++r)
      s = ffeq_equalize(plan, H[r % n_sets], y[r % n_sets], N0, Es, z, sigma2, llr, info, workspace,
                        workspace_bytes, cs);
  }
  if (ok && s == FFEQ_OK && cudaEventRecord(e1, cs) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
      cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
    // ms is set
  } else {
    ms = -1.f;
    if (s == FFEQ_OK) s = cuda_fail(cudaGetLastError());
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  *st_out = s;
  return ms;
}

}  // namespace

ffeq_status ffeq_plan_autotune_sets(ffeq_plan* plan, const void* const* H, const void* const* y, int n_sets,
                                    float N0, float Es, void* z, float* sigma2, float* llr, int* info,
                                    void* workspace, size_t workspace_bytes, void* stream, int reps) {
  if (!plan || reps < 1 || n_sets < 1 || !H || !y) return FFEQ_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return cuda_fail(e);
  if (cap != cudaStreamCaptureStatusNone) return FFEQ_ERR_INVALID_ARG;
  if (plan->p.n_sc == 0) return FFEQ_OK;
  // A private stream (capturable even when the caller's is the legacy default
  // stream), ordered after the caller's work.
  cudaStream_t cs = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr, dep = nullptr;
  if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&dep, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventRecord(dep, st)) != cudaSuccess || (e = cudaStreamWaitEvent(cs, dep, 0)) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (dep) cudaEventDestroy(dep);
    if (cs) cudaStreamDestroy(cs);
    return cuda_fail(e);
  }
  const int old[2] = {plan->gram_variant, plan->gram_stages};
  float best = -1.f;
  int best_v[2] = {old[0], old[1]};
  ffeq_status s = FFEQ_OK;
  for (int variant = ffeq::kGram16; variant <= ffeq::kGramVariantMax && s == FFEQ_OK; ++variant) {
    for (int stages = 1; stages <= 3 && s == FFEQ_OK; ++stages) {
      const int v[2] = {variant, stages};
      if (ffeq_plan_set_tuning(plan, v, 2) != FFEQ_OK) continue;
      // One eager untimed call (first-use configuration happens outside capture).
      s = ffeq_equalize(plan, H[0], y[0], N0, Es, z, sigma2, llr, info, workspace, workspace_bytes, cs);
      if (s != FFEQ_OK) break;
      const float ms = time_equalize_calls(plan, H, y, n_sets, N0, Es, z, sigma2, llr, info, workspace,
                                           workspace_bytes, cs, reps, e0, e1, &s);
      if (s != FFEQ_OK) break;
      if (ms >= 0.f && (best < 0.f || ms < best)) {
        best = ms;
        best_v[0] = variant;
        best_v[1] = stages;
      }
    }
  }
  // The caller's stream waits for everything run here.
  if (cudaEventRecord(dep, cs) == cudaSuccess) cudaStreamWaitEvent(st, dep, 0);
  cudaStreamSynchronize(cs);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(dep);
  cudaStreamDestroy(cs);
  plan->gram_variant = s == FFEQ_OK ? best_v[0] : old[0];
  plan->gram_stages = s == FFEQ_OK ? best_v[1] : old[1];
  return s;
}

ffeq_status ffeq_equalize_host(const ffeq_plan* plan, const void* H_host, const void* y_host, float N0, float Es,
                               void* z_host, float* sigma2_host, float* llr_host, int* info_host, void* staging,
                               size_t staging_bytes, void* stream) {
  if (!plan) return FFEQ_ERR_INVALID_ARG;
  const ffeq_problem& p = plan->p;
  size_t need = 0;
  ffeq_host_staging_size(plan, &need);
  if (p.n_sc == 0) return FFEQ_OK;
  if (!H_host || !y_host || !z_host || !sigma2_host || !staging) return FFEQ_ERR_INVALID_ARG;
  if (staging_bytes < need || !aligned(staging, kAlign)) return FFEQ_ERR_INVALID_ARG;
  if (p.llr_bits && !llr_host) return FFEQ_ERR_INVALID_ARG;
  // Page-locked host buffers: the kernels read H, y and write the outputs in
  // place over the host link (on Grace systems NVLink-C2C), so no staging copy
  // is made; only the workspace uses the staging buffer.
  {
    void* vH = device_view(H_host);
    void* vy = device_view(y_host);
    void* vz = device_view(z_host);
    void* vs = device_view(sigma2_host);
    void* vl = p.llr_bits ? device_view(llr_host) : nullptr;
    void* vi = info_host ? device_view(info_host) : nullptr;
    if (vH && vy && vz && vs && (!p.llr_bits || vl) && (!info_host || vi)) {
      size_t ws = 0;
      ffeq_workspace_size(plan, &ws);
      ffeq_status r = equalize_impl(plan, vH, vy, N0, Es, vz, static_cast<float*>(vs), static_cast<float*>(vl),
                                    static_cast<int*>(vi), ws ? staging : nullptr, ws, stream, true);
      if (r != FFEQ_OK) return r;
      const cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
      return e == cudaSuccess ? FFEQ_OK : cuda_fail(e);
    }
  }
  const Sizes s = buffer_sizes(p);
  char* base = static_cast<char*>(staging);
  char* dH = base;
  char* dy = dH + align_up(s.H);
  char* dz = dy + align_up(s.y);
  char* ds2 = dz + align_up(s.z);
  char* dllr = ds2 + align_up(s.s2);
  char* dinfo = dllr + align_up(s.llr);
  char* dws = dinfo + align_up(s.info);
  size_t ws = 0;
  ffeq_workspace_size(plan, &ws);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(dH, H_host, s.H, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMemcpyAsync(dy, y_host, s.y, cudaMemcpyHostToDevice, st)) != cudaSuccess) return cuda_fail(e);
  const ffeq_status r = ffeq_equalize(plan, dH, dy, N0, Es, dz, reinterpret_cast<float*>(ds2),
                                      p.llr_bits ? reinterpret_cast<float*>(dllr) : nullptr,
                                      info_host ? reinterpret_cast<int*>(dinfo) : nullptr, ws ? dws : nullptr, ws,
                                      stream);
  if (r != FFEQ_OK) return r;
  if ((e = cudaMemcpyAsync(z_host, dz, s.z, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_fail(e);
  if ((e = cudaMemcpyAsync(sigma2_host, ds2, s.s2, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_fail(e);
  if (p.llr_bits && (e = cudaMemcpyAsync(llr_host, dllr, s.llr, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e);
  if (info_host && (e = cudaMemcpyAsync(info_host, dinfo, s.info, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e);
  return FFEQ_OK;
}

ffeq_status ffeq_device_status(int* code, int clear) {
  if (!code) return FFEQ_ERR_INVALID_ARG;
  int* d = ffeq::device_status_ptr();
  if (!d) return cuda_fail(cudaGetLastError());
  cudaError_t e = cudaMemcpy(code, d, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e);
  if (clear) {
    const int zero = 0;
    e = cudaMemcpy(d, &zero, sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return FFEQ_OK;
}

}  // extern "C"
