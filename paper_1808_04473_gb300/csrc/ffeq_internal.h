// Internal interface between the C-ABI layer (ffeq_api.cu) and the kernels.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>
#include <mutex>

#include "ffeq.h"

namespace ffeq {

constexpr int kNsymMax = 16;   // OFDM symbols per subcarrier held in registers
constexpr int kMaxClusters = 64;   // FD clusters of a plan (the solve holds C * U padded <= 512 lanes)

// One unit of an uneven batch: a single subcarrier of one instance (element
// offsets into the batch's flat buffers: complex for H, y, z, D; float for
// sigma2 and llr; int for info).  Built on the host, validated on the device.
struct BatchDesc {
  long long h_off, y_off, z_off, s2_off, llr_off, info_off, d_off;
  int B, U, Ceff, n_sym;
  float N0, rho, llr_scale;
  int inst;             // index of the instance (diagnostics)
  float Es;             // symbol energy (the MRC variance scale)
};

// Element counts of the batch buffers (for the device-side bounds checks).
struct BatchLimits {
  long long h, y, z, s2, llr, info, d;
};

// [off, off + n) lies in [0, extent), written so that no sum can overflow.
__host__ __device__ inline bool span_ok(long long off, long long n, long long extent) {
  return off >= 0 && n >= 0 && off <= extent && n <= extent - off;
}

// A solve tile: descriptors [first, first + count) share one CTA; slot s of the
// tile's matrix slots holds cluster (map[s] & 0xff) of descriptor first + (map[s] >> 8).
constexpr int kTileSlots = 64;
struct SolveTile {
  int first, count;
};

// Contraction kernel: H, y -> workspace D = [n_sc][Ceff][U + n_sym][U] complex,
// D[m][u] = sum over the cluster's antennas of conj(H[u][b]) * [H; Y][m][b].
struct TensorMapCache;   // encoded tensor maps of the streamed contraction (host side)

struct GramParams {
  const float2* H;    // [n_sc][U][B]
  const float2* y;    // [n_sc][n_sym][B]
  float2* D;          // workspace
  int* status;        // device status word
  int B, U, Ceff, n_sc, n_sym;
  int bulk;           // 1: stage rows with cp.async.bulk (16-byte aligned rows)
  int stages;         // units staged ahead (1 without bulk copies)
  int stage_elems;    // capacity of one stage (float2)
  int slot_elems;     // capacity of one split-K partial slot (float2)
  int n_slots;        // partial slots in shared memory
  int n_units;        // subcarriers (uniform) or batch units
  const BatchDesc* desc;  // nullptr: uniform problem
  int* queue;         // batch: work-queue counter (zero at launch)
  int UP;             // batch: users padding of the group
  BatchLimits lim;    // batch: buffer extents
  int grid_cap;       // > 0: at most this many persistent CTAs
  int plane_bytes;    // > 0: pre-split BF16 planes of this capacity (BF16x3 pre-split contraction)
  int variant;        // contraction launch shape (kGram16 ... kGramStream)
  TensorMapCache* map_cache;   // streamed shape: maps of inputs seen before (nullptr: encode every call)
  // Uniform problems: cluster c holds antennas [cl_off[c], cl_off[c+1]) (cl_uniform:
  // every cluster B / Ceff antennas, and cl_off is not read).
  int cl_uniform;
  int cl_off[kMaxClusters + 1];
};

// Contraction launch shapes: 16 warps, one CTA per SM; 8 warps, two CTAs per SM
// (half the shared memory each, so one CTA's MMA phase overlaps the other's
// staging); BF16x3 pre-split planes (16 warps); 4 warps, three CTAs per SM;
// streamed (ffeq_gram_stream.cu: 32-antenna slices of several subcarriers per
// CTA moved by tensor-map copies, each warp owning its output tiles over the
// whole antenna range; `stages` is then the depth of each subcarrier's ring);
// fused (the streamed contraction with the solve, fusion and soft outputs in the
// same launch when a whole equalization runs; ring depth 2); streamed with
// half-size CTAs (8 MMA warps, two CTAs per SM, so that another kernel's CTA can
// share each SM).
constexpr int kGramAuto = 0, kGram16 = 1, kGram8x2 = 2, kGramPresplit = 3, kGram4x3 = 4, kGramStream = 5,
              kGramFused = 6, kGramStreamHalf = 7;
constexpr int kGramVariantMax = kGramStreamHalf;
constexpr int kGramFusedRing = 2;       // ring depth of the fused shape (its solve areas take the rest)
constexpr int kGramStreamRing = 3;      // default (and largest) ring depth of the streamed shape (least 2)

// Whether the streamed contraction takes this problem (BF16x3 or FP16x3,
// U <= 32, B even, cluster sizes whole 16-antenna steps for FD).
bool gram_stream_eligible(int precision, int B, int U, int n_sym, int Ceff);
// A plan's cache of encoded tensor maps (inputs at the addresses of a recent
// call reuse their maps instead of encoding them again on the host).
TensorMapCache* tensor_map_cache_create();
void tensor_map_cache_destroy(TensorMapCache* cache);
cudaError_t launch_gram_stream(const GramParams& p, int precision, cudaStream_t stream);
// Whether the fused shape takes this problem: the streamed shape's conditions
// with U = 8 or 16 (one lane per user, the users filling the lane group).  The
// equalizer (L-MMSE or ZF) and refine = 0 are checked by the caller.
bool gram_fused_eligible(int precision, int B, int U, int n_sym, int Ceff);
struct SolveParams;
// One launch: contraction (p, 16-byte aligned H and y, ring kGramFusedRing) and
// the solve / fusion / soft outputs of every subcarrier (s; s.D is not read).
cudaError_t launch_gram_fused(const GramParams& p, const SolveParams& s, int precision, cudaStream_t stream);

// Solve / fusion / epilogue kernel: workspace D -> z, sigma2, llr, info.
struct SolveParams {
  const float2* D;
  float2* z;          // [n_sc][n_sym][U]
  float* sigma2;      // [n_sc][U]
  float* llr;         // [n_sc][n_sym][U][llr_bits] or nullptr
  int* info;          // [n_sc][Ceff] or nullptr
  int U, Ceff, n_sc, n_sym;
  int spc;            // subcarriers per CTA
  int unbiased;       // 1: FFEQ_UNBIASED
  int llr_bits;
  float N0, rho;      // rho = N0 / Es (0 for zero forcing)
  float llr_scale;    // sqrt(Es / e_avg): amplitude of level +1
  int equalizer;      // ffeq_equalizer; FFEQ_MRC runs mrc_fuse_kernel, FFEQ_LAMA lama_kernel (uniform problems)
  float Es;
  int lama_iters;     // LAMA: iterations T
  int cl_size[kMaxClusters];   // LAMA: antennas of each cluster (B for PD)
  // Uneven batch (desc != nullptr): one CTA per tile; per-unit sizes, offsets,
  // N0, rho and llr_scale from the descriptors.
  const BatchDesc* desc;
  const SolveTile* tiles;
  const unsigned short* slot_map;   // [n_tiles][kTileSlots]
  int n_tiles, n_desc, threads;
  BatchLimits lim;
  int* status;
  // Uniform problem with refinement: write the local estimates X [n_sc][Ceff][n_sym][U],
  // the inverses transposed As [n_sc][Ceff][U][U] and the pivot status fails
  // [n_sc][Ceff] instead of the outputs.
  float2* Xs;
  float2* As;
  int* fails;
};

// Iterative refinement from the inputs (uniform problems).
struct RefineParams {
  const float2* H;      // [n_sc][U][B]
  const float2* y;      // [n_sc][n_sym][B]
  const float2* D;      // contraction output (for G_uu)
  float2* As;           // [n_sc][Ceff][U][U] inverses, transposed (the diagonal refined in place)
  float2* Xs;           // [n_sc][Ceff][n_sym][U] (refined in place)
  const int* fails;     // [n_sc][Ceff]
  float2* z;
  float* sigma2;
  float* llr;
  int B, U, Ceff, n_sc, n_sym, steps, unbiased, llr_bits;
  int res64;            // residual in FP64: 0 never, 1 above the condition threshold, 2 always
  float N0, rho, llr_scale;
  int max_S;            // antennas of the largest cluster
  int cl_off[kMaxClusters + 1];   // cluster c: antennas [cl_off[c], cl_off[c+1])
};
// Whether one local system fits the refinement kernel's shared memory.
bool refine_fits(int max_S, int U, int n_sym);
size_t refine_smem_bytes(int max_S, int U, int n_sym);
cudaError_t launch_refine(const RefineParams& p, cudaStream_t stream);

// Differentiable FD (per-cluster rho_c, free fusion weights nu) and its adjoint.
struct TrainParams {
  const float2* H;     // [n_sc][U][B]
  const float2* y;     // [n_sc][n_sym][B]
  const float2* D;     // workspace: local Gram matrices and MRC outputs (FD layout)
  float2* X;           // workspace [n_sc][C][n_sym][U]: local estimates
  float2* Gb;          // workspace [n_sc][C][n_sym][U]
  float2* Wm;          // workspace [n_sc][C][U][U]
  float* P;            // workspace [n_sc][C][1+U]: partial sums of dL/drho, dL/dnu
  const float* rho_c;  // [C]
  const float* nu;     // [C][U]
  float2* z;           // forward output [n_sc][n_sym][U]
  const float2* gz;    // backward input [n_sc][n_sym][U]
  float2* gH;          // [n_sc][U][B]
  float2* gy;          // [n_sc][n_sym][B]
  float* grho;         // [C]
  float* gnu;          // [C][U]
  int B, U, C, n_sc, n_sym;
  // Adjoint through the optimal weights (ffeq_fd_optimal_backward): rho = N0 / Es
  // shared by every cluster; clusters of cl_off (cl_uniform: B / C antennas each).
  float rho;
  int* status;
  int cl_uniform;
  int cl_off[kMaxClusters + 1];
};
size_t train_smem_bytes(int U, int C);
cudaError_t launch_train_forward(const TrainParams& p, cudaStream_t stream);
cudaError_t launch_train_backward(const TrainParams& p, cudaStream_t stream);
// Fused forms (the local Gram matrices formed in the solving CTA, from H and Y
// staged in shared memory; the gradients of H and Y in the backward CTA): for
// FP32 plans whose subcarrier fits, ffeq_fd_train_forward / _backward run these
// instead (forward: no contraction launch, no workspace D; backward: no W, G_b).
bool train_fused_fits(int U, int n_sym, int B, int C);
cudaError_t launch_train_forward_fused(const TrainParams& p, cudaStream_t stream);
cudaError_t launch_train_backward_fused(const TrainParams& p, cudaStream_t stream);
// Shared memory of the optimal-weight backward solve (one CTA per subcarrier).
size_t train_optimal_smem_bytes(int U, int C);
cudaError_t launch_train_optimal_backward(const TrainParams& p, cudaStream_t stream);
// Its fused form (FP32 plans whose subcarrier fits; no contraction launch, no D, W, G_b).
bool train_optimal_fused_fits(int U, int n_sym, int B, int C);
cudaError_t launch_train_optimal_backward_fused(const TrainParams& p, cudaStream_t stream);

// Padded user count (8, 16 or 32) used for register tiles.
int padded_users(int U);
// Subcarriers the contraction kernel of `precision` can stage ahead (0: one
// subcarrier does not fit in shared memory).
int gram_stages(int precision, int B, int U, int n_sym, int Ceff, bool bulk);
// Shared-memory capacities a contraction variant needs for one unit.
struct GramCaps {
  int stage_elems;   // one staged unit (float2)
  int slot_elems;    // one split-K partial slot (float2)
  int slots;         // partial slots
  int plane_bytes;   // pre-split planes (0: variant without them)
};
// Whether the BF16x3 pre-split variant can take a unit (B and S multiples of 4).
bool gram_presplit_eligible(int precision, int B, int Ceff);
GramCaps gram_tc_caps(int B, int U, int n_sym, int Ceff, int variant);
// Capacities of one unit under `precision` and launch shape `variant`.
GramCaps gram_instance_caps(int precision, int B, int U, int n_sym, int Ceff, int variant);
// Shared memory one CTA of `variant` may use.
size_t gram_smem_budget(int variant);
// Fill the capacities and stages of a uniform problem for `variant` (kGramAuto:
// the default shape) and `stages` (0: as many as fit, at most 3).  Returns false
// when the shape does not apply or does not fit.
bool gram_configure(GramParams& p, int precision, int variant, int stages);
int gram_stages_fit_bytes(size_t stage_elems, size_t fixed_bytes, bool bulk, size_t budget);
cudaError_t launch_gram_fp32(const GramParams& p, cudaStream_t stream);
// Tensor-core split-precision contraction (precision FFEQ_TF32X3 or FFEQ_BF16X3).
cudaError_t launch_gram_tc(const GramParams& p, int precision, cudaStream_t stream);
int solve_subcarriers_per_cta(int U, int Ceff);
size_t solve_smem_bytes(int U, int Ceff);
cudaError_t launch_solve(const SolveParams& p, cudaStream_t stream);
cudaError_t launch_lama(const SolveParams& p, cudaStream_t stream);
cudaError_t launch_lama_batch(const SolveParams& p, cudaStream_t stream);
int lama_symbols_per_cta(int U, int Ceff, int n_sym);
// Uneven batch: p.U holds the group's padded users (8/16/32), lpr its lanes per row
// (1 for MRC, p.equalizer); ZF runs the L-MMSE kernel with rho = 0 per descriptor.
cudaError_t launch_solve_batch(const SolveParams& p, int lpr, cudaStream_t stream);
size_t solve_batch_smem_bytes(int UP, int lpr, int threads, int equalizer);

// Device addresses of a __device__ symbol, one per CUDA context (a context's
// module holds its own copy; a context destroyed by cudaDeviceReset and the one
// created after it are different contexts).  Keyed by the driver's context ID,
// which is unique for the life of the process, so a stale entry can never match.
struct SymbolAddressCache {
  static constexpr int kEntries = 16;
  std::mutex m;
  unsigned long long id[kEntries] = {};
  void* ptr[kEntries] = {};
  int n = 0, next = 0;
};
// ID of the calling thread's current context, 0 when none is current.
unsigned long long current_context_id();
// The symbol's address in the current context: the cached one when this context
// looked it up before, else fetch(&ptr) (a cudaGetSymbolAddress of the symbol,
// which also makes the device's primary context current when none is), cached
// under the context's ID.  nullptr with *err set on failure.
void* cached_symbol_address(SymbolAddressCache& cache, cudaError_t (*fetch)(void**), cudaError_t* err);

// Address of the device status word in the current context (nullptr on error).
int* device_status_ptr();
// Remember the CUDA error string for ffeq_last_cuda_error(); returns FFEQ_ERR_CUDA.
int record_cuda_error(cudaError_t e);

}  // namespace ffeq
