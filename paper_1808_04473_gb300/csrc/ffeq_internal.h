// Internal interface between the C-ABI layer (ffeq_api.cu) and the kernels.
#pragma once

#include <cstddef>
#include <cuda_runtime.h>

#include "ffeq.h"

namespace ffeq {

constexpr int kNsymMax = 16;   // OFDM symbols per subcarrier held in registers

// Contraction kernel: H, y -> workspace D = [n_sc][Ceff][U + n_sym][U] complex,
// D[m][u] = sum over the cluster's antennas of conj(H[u][b]) * [H; Y][m][b].
struct GramParams {
  const float2* H;    // [n_sc][U][B]
  const float2* y;    // [n_sc][n_sym][B]
  float2* D;          // workspace
  int* status;        // device status word
  int B, U, Ceff, n_sc, n_sym;
  int bulk;           // 1: stage rows with cp.async.bulk (16-byte aligned rows)
  int stages;         // subcarriers staged ahead (1 without bulk copies)
};

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
  float N0, rho;      // rho = N0 / Es
  float llr_scale;    // sqrt(Es / e_avg): amplitude of level +1
};

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
};
size_t train_smem_bytes(int U, int C);
cudaError_t launch_train_forward(const TrainParams& p, cudaStream_t stream);
cudaError_t launch_train_backward(const TrainParams& p, cudaStream_t stream);

// Padded user count (8, 16 or 32) used for register tiles.
int padded_users(int U);
// Subcarriers the contraction kernel of `precision` can stage ahead (0: one
// subcarrier does not fit in shared memory).
int gram_stages(int precision, int B, int U, int n_sym, int Ceff, bool bulk);
int gram_tc_stages(int B, int U, int n_sym, int Ceff, bool bulk);
cudaError_t launch_gram_fp32(const GramParams& p, cudaStream_t stream);
// Tensor-core split-precision contraction (precision FFEQ_TF32X3 or FFEQ_BF16X3).
cudaError_t launch_gram_tc(const GramParams& p, int precision, cudaStream_t stream);
int solve_subcarriers_per_cta(int U, int Ceff);
size_t solve_smem_bytes(int U, int Ceff);
cudaError_t launch_solve(const SolveParams& p, cudaStream_t stream);

// Address of the device status word on the current device (nullptr on error).
int* device_status_ptr();

}  // namespace ffeq
