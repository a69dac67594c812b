/*
 * ffeq.h -- C ABI of the GB300 (sm_103a) decentralized feedforward equalizer.
 *
 * The library computes, for every subcarrier of a massive MU-MIMO uplink
 * (Sec. II-A, Eq. 1: y = H s0 + n), the partially decentralized (PD) or
 * fully decentralized (FD) L-MMSE equalizer of Jeon, Li, Cavallaro and Studer,
 * "Decentralized Equalization with Feedforward Architectures for Massive
 * MU-MIMO":
 *
 *   per cluster c (contiguous antenna block, Sec. II-B):
 *       G_c = H_c^H H_c,   y_c^MRC = H_c^H y_c                    (Sec. II-C)
 *   PD: G = sum_c G_c, y^MRC = sum_c y_c^MRC                       (Eq. fullMRC)
 *       z = (G + rho I)^{-1} y^MRC, rho = N0/Es                     (Sec. III-A)
 *   FD: z_c = (G_c + rho I)^{-1} y_c^MRC per cluster, then
 *       z_u = sum_c nu_{c,u} z_{c,u},  nu = sigma_c^-2 / sum sigma^-2 (Eq. fusionrule,
 *       Lemma 1 Eq. opt_fusion), sigma^2 = (sum_c sigma_c^-2)^-1     (Thm. 3)
 *   error variances sigma^2 and max-log LLRs of the decoupled channel (Eq. 4).
 * In place of L-MMSE, the same two architectures run the zero-forcing (ZF) or
 * maximum-ratio (MRC) equalizer of Sec. III-A or the nonlinear LAMA of
 * Sec. III-B (ffeq_problem.equalizer).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Complex numbers are interleaved float32 pairs (re, im) ("cf32", 8 bytes).
 *   H      cf32 [n_sc][U][B]       row u = the B antenna gains of user u
 *                                  (column-major layout of the paper's B x U H)
 *   y      cf32 [n_sc][n_sym][B]   receive vectors, one per OFDM symbol
 *   z      cf32 [n_sc][n_sym][U]   equalized symbols
 *   sigma2 f32  [n_sc][U]          post-equalization error variance (real);
 *                                  [n_sc][n_sym][U] for FFEQ_LAMA
 *   llr    f32  [n_sc][n_sym][U][llr_bits]   optional max-log LLRs
 *   info   i32  [n_sc] (PD) or [n_sc][C] (FD)  optional: 0, or k (1-based) when
 *                                  the k-th Cholesky pivot of G + rho I (or of
 *                                  G_c + rho I) was not positive; the outputs of
 *                                  that subcarrier are then NaN.
 * Clusters are C contiguous blocks of S = B/C antennas (B % C == 0).
 * Device pointers must be 8-byte aligned; 16-byte aligned H and y with even B
 * take the bulk-copy (TMA) staging path.
 *
 * Estimates (the paper types sigma^2 as complex; it is real here):
 *   FFEQ_LITERAL   z = (G + rho I)^{-1} y^MRC and the error variance of Sec. III-A,
 *                  diag(A G A^H N0 + (AG - I)(AG - I)^H Es) = N0 diag(A),
 *                  A = (G + rho I)^{-1}; FD fuses these pairs.
 *   FFEQ_UNBIASED  z / mu, sigma^2 / mu with mu_u = [A G]_uu = 1 - rho A_uu, the
 *                  unbiased decoupled model z_u = s_u + e_u that Lemma 1 assumes;
 *                  FD fuses the unbiased per-cluster pairs.
 *   N0 == 0 is zero forcing; fusion weights then use the N0 -> 0 limit.
 *   A user with mu <= 0 (e.g. an all-zero channel column) gets weight 0; if
 *   every cluster gives it weight 0 its z is 0 and its sigma^2 is +inf.
 *
 * LLRs (the paper names them, Sec. II-A, but gives no formula): square QAM,
 * L = 2^(llr_bits/2) odd-integer levels per axis scaled to energy Es; labels are
 * the binary-reflected Gray code of the in-phase level index (MSB first)
 * followed by that of the quadrature index; LLR_b = (min_{a: b=1}|z-a|^2 -
 * min_{a: b=0}|z-a|^2) / sigma^2 (positive favours bit 0).
 *
 * Errors: every entry point validates its arguments before launching and
 * returns a status; nothing is allocated inside the equalize calls (the caller
 * owns all device memory, including the workspace).  Kernels bound every wait;
 * a wait that runs out records FFEQ_ERR_TIMEOUT in a device status word that
 * ffeq_device_status() reads.
 */
#ifndef FFEQ_H
#define FFEQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FFEQ_OK = 0,
  FFEQ_ERR_INVALID_ARG = 1,   /* a size, pointer or enum is out of range */
  FFEQ_ERR_UNSUPPORTED = 2,   /* valid problem this build cannot run (e.g. U > 32) */
  FFEQ_ERR_CUDA = 3,          /* a CUDA runtime call failed; see ffeq_last_cuda_error() */
  FFEQ_ERR_TIMEOUT = 4        /* a bounded device wait ran out (read by ffeq_device_status) */
} ffeq_status;

typedef enum { FFEQ_PD = 0, FFEQ_FD = 1 } ffeq_arch;
/* Arithmetic of the local preprocessing (G_c, y_c^MRC); the solve and fusion
 * are FP32 in every mode.
 *   FFEQ_FP32    FP32 on the CUDA cores.
 *   FFEQ_TF32X3  tensor cores, each FP32 operand split into TF32 hi + lo, three
 *                products accumulated in FP32 (about FP32 accuracy).
 *   FFEQ_BF16X3  tensor cores, BF16 hi + lo split, three products, FP32
 *                accumulation (mixed precision: ~16 significand bits per operand).
 *   FFEQ_FP16X3  tensor cores, FP16 hi + lo split, three products, FP32
 *                accumulation: ~22 significand bits at the BF16 rate, within
 *                FP16's range (entries of H and y below 32768 in magnitude; the
 *                lo part loses bits for entries below about 2^-3, so inputs
 *                should be of order one, as with unit-variance channels). */
typedef enum { FFEQ_FP32 = 0, FFEQ_TF32X3 = 1, FFEQ_BF16X3 = 2, FFEQ_FP16X3 = 3 } ffeq_precision;
typedef enum { FFEQ_UNBIASED = 0, FFEQ_LITERAL = 1 } ffeq_estimate;
/* Equalizer of the central (PD) or local (FD) solve, Sec. III-A:
 *   FFEQ_LMMSE  z = (G + rho I)^{-1} y^MRC, rho = N0/Es (the estimate field
 *               selects the literal or unbiased pairs);
 *   FFEQ_ZF     z = G^{-1} y^MRC, sigma^2 = N0 diag(G^{-1}) (L-MMSE with rho = 0;
 *               info reports the first non-positive pivot of G or G_c);
 *   FFEQ_MRC    z = diag(G)^{-1} y^MRC, sigma^2_u = (N0 G_uu + Es sum_{v != u}
 *               |G_uv|^2) / G_uu^2 (no inversion; info is always 0).
 * ZF and MRC estimates are unbiased, so the estimate field does not apply; FD
 * fuses the per-cluster pairs with the optimal weights of Lemma 1 as for
 * L-MMSE; PD-MRC is z = diag(G)^{-1} y^MRC with no fusion step.  A user that a
 * cluster cannot see (G_c,uu = 0) gets MRC weight 0.  With N0 == 0 the weights
 * are those of the N0 -> 0 limit of Lemma 1's: for ZF proportional to
 * 1/[G_c^{-1}]_uu (every variance is 0); for MRC, per user, the clusters where
 * the user has no interference (sum_{v != u} |G_c,uv|^2 = 0: variance exactly 0)
 * share all the weight in proportion to G_c,uu and the fused variance is 0,
 * while a user with interference in every cluster keeps the ordinary weights
 * (its variance is the interference term alone).
 *   FFEQ_LAMA   Algorithm 1 (LAMA-PD) on (G, y^MRC), or per cluster on
 *               (G_c, y_c^MRC) and fused with the weights of Lemma 1 (LAMA-FD),
 *               for lama_iters iterations: z^T and sigma^2 = N0 + beta phi^T of
 *               the last one.  The system is taken in the paper's normalization
 *               (G / B, y^MRC / B, N0 / B, beta = U / B; a cluster of S_c
 *               antennas: G_c / S_c, y_c^MRC / S_c, N0 / S_c, beta_c = U / S_c),
 *               the prior is equiprobable square QAM of llr_bits bits per symbol
 *               (the LLR constellation; llr_bits > 0 is required) and the
 *               denoiser is its posterior mean and variance (Eq. F).  phi^T
 *               depends on the received vector: sigma2 is f32 [n_sc][n_sym][U]
 *               (the same value for every user of a vector), not [n_sc][U].
 *               N0 > 0 (FFEQ_ERR_INVALID_ARG otherwise); info, if given, is 0.
 *               An empty cluster gets weight 0. */
typedef enum { FFEQ_LMMSE = 0, FFEQ_ZF = 1, FFEQ_MRC = 2, FFEQ_LAMA = 3 } ffeq_equalizer;

/* Problem statement (Sec. II-A, II-B, VI): B antennas, U users, C clusters,
 * n_sc subcarriers, n_sym OFDM symbols sharing one channel per subcarrier. */
typedef struct {
  int B, U, C;
  int n_sc, n_sym;
  int arch;        /* ffeq_arch */
  int precision;   /* ffeq_precision */
  int estimate;    /* ffeq_estimate */
  int llr_bits;    /* 0 (no LLRs), 2, 4, 6 or 8 */
  int refine;      /* 0..4: steps of iterative refinement from the inputs:
                    * r_c = H_c^H (y_c - H_c x_c) - rho x_c, x_c += A_c r_c (with
                    * A_c the solve's inverse), and one Newton-Schulz step for the
                    * inverse, A_c <- 2 A_c - A_c^H (G_c + rho I) A_c, whose
                    * diagonal the unbiasing and the fusion use.  Each step
                    * multiplies the error by about the current relative error
                    * of the inverse, which the Newton-Schulz step squares:
                    * from the kappa(G_c + rho I) * 2^-16 (BF16X3) or 2^-21
                    * (FP16X3) of the preprocessing, one step suffices while
                    * that is far below 1, more steps where it nears 1
                    * (kappa ~ 1e5 for FP16X3).  Costs a second
                    * read of H and y and a larger workspace; only ffeq_equalize
                    * (and the entry points built on it) support it:
                    * ffeq_fuse_equalize returns FFEQ_ERR_UNSUPPORTED. */
  int refine_fp64; /* precision of the refinement residual r_c (needs refine > 0):
                    * 0  FP32 for every local system: the estimates converge to
                    *    the accuracy of an FP32 solve, about kappa * 2^-24;
                    * 1  FP64 (y_c - H_c x_c and H_c^H of it accumulated in
                    *    double) for the local systems whose condition estimate
                    *    ||G_c + rho I||_1 ||A_c||_1 exceeds 1e4, FP32 for the
                    *    others: the ill-conditioned ones converge to about
                    *    2^-24 (the FP32 storage of x_c) instead;
                    * 2  FP64 for every local system. */
  int equalizer;   /* ffeq_equalizer: 0 = L-MMSE.  Refinement applies to
                    * L-MMSE and ZF; MRC or LAMA with refine > 0 is
                    * FFEQ_ERR_INVALID_ARG. */
  int lama_iters;  /* LAMA: iterations T, 1..64 (T = 1 is the normalized matched
                    * filter); must be 0 for the other equalizers. */
} ffeq_problem;

typedef struct ffeq_plan ffeq_plan;

/* Validate *p and create a plan (host memory only; no device allocation).
 * Limits of this build: 1 <= U <= 32, 1 <= n_sym <= 16, B % C == 0, one
 * staged subcarrier (U + n_sym) * (B + 2) * 8 bytes (plus split-K partials
 * when fewer than 8 clusters are kept apart) must fit in 227 KiB of shared
 * memory, and the C local systems of one FD subcarrier must fit one CTA
 * (C * U padded <= 512).
 * Returns FFEQ_ERR_INVALID_ARG or FFEQ_ERR_UNSUPPORTED otherwise. */
ffeq_status ffeq_plan_create(ffeq_plan** out, const ffeq_problem* p);

/* The same with clusters of given sizes (Sec. II-B: cluster c holds B_c
 * contiguous antennas, c = 0..C-1, in order along each row of H and y):
 * cluster_sizes holds C integers >= 0 summing to B (B % C need not be 0);
 * NULL means B / C each, as ffeq_plan_create.  For PD the partition does not
 * enter the result (the local results are summed, Eq. fullMRC).  FD with
 * unequal sizes runs the contraction on shapes 1-4 (the streamed and pre-split
 * shapes need equal clusters) and at most 64 clusters; the training entry
 * points (ffeq_fd_train_*, ffeq_fd_optimal_backward) follow the plan's clusters.
 * FFEQ_ERR_INVALID_ARG for a negative size or sizes that do not sum to B. */
ffeq_status ffeq_plan_create_clusters(ffeq_plan** out, const ffeq_problem* p, const int* cluster_sizes);

/* Destroy a plan (NULL is ignored). */
void ffeq_plan_destroy(ffeq_plan* plan);

/* Device workspace bytes ffeq_equalize needs: the per-(subcarrier, cluster)
 * local Gram matrices and MRC outputs, n_sc * Ceff * (U + n_sym) * U * 8 bytes
 * with Ceff = C (FD) or 1 (PD); with refinement also the local estimates, the
 * inverses and the pivot status (n_sc * Ceff * ((n_sym + U) * U * 8 + 4) bytes
 * more, plus alignment).  Owned by the caller, 16-byte aligned. */
ffeq_status ffeq_workspace_size(const ffeq_plan* plan, size_t* bytes);

/* Equalize on the device (Sec. II-C/D, III-A, IV-A; see the header comment).
 * H, y, z, sigma2 are device pointers; llr and info are device pointers or NULL.
 * N0 >= 0 and Es > 0 (finite).  workspace is a device buffer of at least
 * ffeq_workspace_size bytes; calls that share a workspace must be ordered on
 * one stream.  stream is a cudaStream_t (NULL = legacy default stream).
 * Asynchronous: returns after the launches (a contraction kernel, then a
 * solve/fusion kernel started by programmatic dependent launch); results are
 * ready when the stream reaches them. */
ffeq_status ffeq_equalize(const ffeq_plan* plan, const void* H, const void* y, float N0, float Es,
                          void* z, float* sigma2, float* llr, int* info,
                          void* workspace, size_t workspace_bytes, void* stream);

/* The two stages of ffeq_equalize, for callers that schedule them apart.
 *
 * ffeq_local_preprocess: local preprocessing of every cluster (Sec. II-C):
 *   G_c = H_c^H H_c and y_c^MRC = H_c^H y_c, summed over clusters for PD
 *   (Eq. fullMRC), written to the workspace as [n_sc][Ceff][U + n_sym][U]
 *   complex with D[v][u] = G[u][v] (v < U) and D[U + n][u] = y^MRC_u(n).
 * ffeq_fuse_equalize: the central (PD) or per-cluster (FD) L-MMSE equalization
 *   from the workspace, optimal fusion (FD) and the soft outputs.
 * Same argument rules as ffeq_equalize; the workspace written by the first
 * must be read by the second on the same stream. */
ffeq_status ffeq_local_preprocess(const ffeq_plan* plan, const void* H, const void* y,
                                  void* workspace, size_t workspace_bytes, void* stream);
ffeq_status ffeq_fuse_equalize(const ffeq_plan* plan, const void* workspace, size_t workspace_bytes,
                               float N0, float Es, void* z, float* sigma2, float* llr, int* info,
                               void* stream);

/* Differentiable FD equalization (the paper's FD architecture, Sec. II-D /
 * IV-A, with its regularizer and fusion weights made free parameters):
 *   X_c = (G_c + rho_c I)^{-1} H_c^H Y_c     (per cluster, L-MMSE form of Sec. III-A)
 *   z_u = sum_c nu[c][u] X_c[u]              (Eq. fusionrule with free weights)
 * rho_c: f32 [C] (> 0), nu: f32 [C][U], both on the device and shared by all
 * subcarriers.  The plan must be FD.  The workspace (ffeq_fd_train_workspace_size
 * bytes, 256-byte aligned, owned by the caller) carries the local Gram matrices
 * and the local estimates from the forward call to the backward call; the
 * backward call recomputes the factorizations from them.
 * ffeq_fd_train_backward takes gz = dL/dRe z + i dL/dIm z of a real loss L
 * (cf32 [n_sc][n_sym][U]) and writes dL/dH (cf32 [n_sc][U][B]), dL/dy
 * (cf32 [n_sc][n_sym][B]) in the same convention, and dL/drho (f32 [C]) and
 * dL/dnu (f32 [C][U]) summed over all subcarriers:
 *   dL/dH_c = Y_c G_b^H - H_c (G_b X_c^H + X_c G_b^H),  dL/dY_c = H_c G_b,
 *   dL/drho_c = -sum Re tr(G_b^H X_c),  dL/dnu[c][u] = sum Re(conj(gz_u) X_c,u),
 *   G_b = (G_c + rho_c I)^{-1} diag(nu_c) gz.
 * The same H, y, rho_c, nu and workspace must be passed to both calls, in order
 * on one stream.  Outputs of a subcarrier whose system is not positive definite
 * are NaN.  Limits: C * U padded <= 512; the plan's equalizer must be
 * FFEQ_LMMSE (FFEQ_ERR_UNSUPPORTED otherwise). */
ffeq_status ffeq_fd_train_workspace_size(const ffeq_plan* plan, size_t* bytes);
ffeq_status ffeq_fd_train_forward(const ffeq_plan* plan, const void* H, const void* y, const float* rho_c,
                                  const float* nu, void* z, void* workspace, size_t workspace_bytes,
                                  void* stream);
ffeq_status ffeq_fd_train_backward(const ffeq_plan* plan, const void* H, const void* y, const float* rho_c,
                                   const float* nu, const void* gz, void* gH, void* gy, float* grho,
                                   float* gnu, void* workspace, size_t workspace_bytes, void* stream);

/* Adjoint of the FD equalizer with the paper's optimal weights (FD architecture
 * of Sec. II-D / IV-A with the unbiased L-MMSE pairs of Sec. III-A fused by
 * Lemma 1, Eq. opt_fusion: the computation ffeq_equalize performs for this plan),
 * differentiated through the weights' dependence on diag(A_c):
 *   per subcarrier and cluster, M_c = G_c + rho I, A_c = M_c^{-1}, X_c = A_c B_c,
 *   a_c = diag(A_c), w_c = 1 / a_c, D_u = sum_c (w_{c,u} - rho), rho = N0 / Es,
 *   z_u = sum_c w_{c,u} X_{c,u} / D_u;
 *   G_b = A_c diag(w_c / D) G_z,
 *   q_u = -Re(sum_n conj(g_z,u,n) (X_{c,u,n} - z_{u,n})) / (D_u a_{c,u}^2),
 *   dL/dH_c = Y_c G_b^H - H_c (X_c G_b^H + G_b X_c^H + 2 A_c diag(q) A_c),
 *   dL/dY_c = H_c G_b.
 * gz = dL/dRe z + i dL/dIm z (cf32 [n_sc][n_sym][U]) of a real loss of the
 * plan's z; gH (cf32 [n_sc][U][B]) and gy (cf32 [n_sc][n_sym][B]) in the same
 * convention.  The call recomputes the contraction and the factorizations from
 * H and y (nothing is kept from the forward call).  The plan must be FD with
 * FFEQ_LMMSE, FFEQ_UNBIASED and refine = 0 (FFEQ_ERR_INVALID_ARG otherwise);
 * clusters of given sizes are allowed; C * U padded <= 512 and one subcarrier's
 * working set in shared memory (FFEQ_ERR_UNSUPPORTED otherwise).  N0 >= 0 and
 * Es > 0 as for ffeq_equalize.  The workspace (ffeq_fd_optimal_workspace_size
 * bytes, 256-byte aligned, owned by the caller) holds the contraction output,
 * G_b and the matrices of the H term.  A user that no cluster sees contributes
 * nothing; the gradients of a subcarrier whose systems are not all positive
 * definite are NaN; users whose unbiasing gain mu is not positive lie outside
 * the region where the weights are differentiable and are not treated apart. */
ffeq_status ffeq_fd_optimal_workspace_size(const ffeq_plan* plan, size_t* bytes);
ffeq_status ffeq_fd_optimal_backward(const ffeq_plan* plan, const void* H, const void* y, float N0, float Es,
                                     const void* gz, void* gH, void* gy, void* workspace, size_t workspace_bytes,
                                     void* stream);

/* Launch shape of a plan's contraction kernel (the arithmetic is that of the
 * plan's precision in every shape; with split-K (PD) the shapes differ in how
 * the antennas are split among warps, hence in summation order only):
 *   values[0]  0 = default (5 where it applies, else 1), 1 = 16 warps, one CTA per SM,
 *              2 = 8 warps, two CTAs per SM (half the shared memory each),
 *              3 = BF16X3 only: each staged subcarrier converted once into BF16
 *                  hi/lo planes read with ldmatrix (needs B and B/C multiples of 4);
 *              4 = TF32X3 / BF16X3 only: 4 warps, three CTAs per SM;
 *              5 = BF16X3 / FP16X3 only, streamed: every warp owns output tiles
 *                  over a whole cluster (no split-K), each subcarrier streams
 *                  through a ring of 32-antenna slices moved by tensor-map
 *                  copies and split once into 16-bit planes (needs B even and,
 *                  for FD, B/C a multiple of 16; 16-byte aligned H and y, else
 *                  shape 1 runs);
 *              6 = fused: shape 5's conditions with U = 8 or 16, FFEQ_LMMSE or
 *                  FFEQ_ZF and refine = 0; ffeq_equalize then runs ONE kernel
 *                  that also solves, fuses and writes the soft outputs (each
 *                  cluster's G_c and y_c^MRC go through shared memory, not the
 *                  workspace, which is left untouched), with exactly the bits of
 *                  shape 5 with ring depth 2; ffeq_local_preprocess runs shape 5
 *                  with ring depth 2 (16-byte aligned H and y, else the separate
 *                  kernels of shape 1 run);
 *              7 = shape 5 in half-size CTAs (8 MMA warps, two CTAs per SM, half
 *                  the subcarriers in flight per CTA; the same results), so
 *                  that a kernel on another stream can share every SM;
 *   values[1]  shapes 1-4: subcarriers staged ahead per CTA, 1..3, or 0 = as
 *              many as fit; shapes 5 and 7: ring depth per subcarrier
 *              (32-antenna slices), 2 or 3, 0 = 3; shape 6: 2 or 0 (= 2).
 * FP16X3 runs on shapes 1, 5, 6 and 7 only.
 * ffeq_plan_set_tuning takes exactly 2 values and returns FFEQ_ERR_UNSUPPORTED
 * when the shape does not apply to or fit the problem (plan unchanged);
 * ffeq_plan_get_tuning writes min(n, 2) values.  ffeq_plan_autotune times every
 * shape and depth that fits with `reps` calls of ffeq_equalize on the given
 * buffers (arguments as for ffeq_equalize): the calls of each candidate are
 * captured once into a CUDA graph on a private stream (ordered after the work
 * already queued on `stream`) and the graph's replay is timed with CUDA events,
 * so that host launch gaps do not decide the choice (eager calls where capture
 * is refused).  It keeps the fastest, makes `stream` wait for its work,
 * synchronizes, and must not run during stream capture. */
ffeq_status ffeq_plan_set_tuning(ffeq_plan* plan, const int* values, int n);
ffeq_status ffeq_plan_get_tuning(const ffeq_plan* plan, int* values, int n);
ffeq_status ffeq_plan_autotune(ffeq_plan* plan, const void* H, const void* y, float N0, float Es, void* z,
                               float* sigma2, float* llr, int* info, void* workspace, size_t workspace_bytes,
                               void* stream, int reps);
/* The same with n_sets input sets (host arrays of n_sets device pointers H[i],
 * y[i], each laid out as for ffeq_equalize): timed call r reads set r % n_sets,
 * so that with sets larger than L2 in total every call reads cold inputs, as in
 * a stream of frames (with one set the inputs stay L2-resident between calls
 * and the timing favours other shapes).  FFEQ_ERR_INVALID_ARG for n_sets < 1 or
 * null arrays. */
ffeq_status ffeq_plan_autotune_sets(ffeq_plan* plan, const void* const* H, const void* const* y, int n_sets,
                                    float N0, float Es, void* z, float* sigma2, float* llr, int* info,
                                    void* workspace, size_t workspace_bytes, void* stream, int reps);

/* Device staging bytes ffeq_equalize_host needs (inputs, outputs and workspace). */
ffeq_status ffeq_host_staging_size(const ffeq_plan* plan, size_t* bytes);

/* Same computation on HOST buffers, synchronizing the stream before returning.
 * When every buffer passed is page-locked (cudaHostAlloc / cudaHostRegister, so
 * the GPU can address it in place), the kernels read H and y and write the
 * outputs directly in host memory over the host link (NVLink-C2C on Grace
 * systems) and only the workspace lives in the staging buffer.  Otherwise H and
 * y are copied to the staging buffer, ffeq_equalize runs, and z, sigma2 (and llr,
 * info when not NULL) are copied back.  Same results either way.  staging is a
 * device pointer of at least ffeq_host_staging_size bytes, 256-byte aligned. */
ffeq_status ffeq_equalize_host(const ffeq_plan* plan, const void* H_host, const void* y_host,
                               float N0, float Es, void* z_host, float* sigma2_host,
                               float* llr_host, int* info_host,
                               void* staging, size_t staging_bytes, void* stream);

/* Equalize without any device allocation (the paper has no counterpart: this
 * serves callers that cannot allocate device memory, such as a real-time
 * receive chain that must stay out of the CUDA allocator on its per-slot path,
 * or a plug-in that owns no device memory besides the buffers it is given).
 * Same computation and arguments as ffeq_equalize, minus the workspace: it
 * uses a 64 MiB array compiled into the library, one per device, which every
 * GPU that loads the library holds until the process exits.  Problems whose
 * ffeq_workspace_size exceeds 64 MiB return FFEQ_ERR_UNSUPPORTED.  The first
 * call in each CUDA context (a device's primary context, or any other context
 * made current) looks up the array's address there (cudaGetSymbolAddress) and
 * caches it under the context's unique ID, so that first call must come before
 * any stream capture in that context.  All calls share
 * the array: calls that overlap on the GPU (other streams, other threads) race
 * and must be serialized by the caller; nothing in it needs clearing between
 * calls.  It calls no cudaMalloc, cudaFree or allocating library routine. */
ffeq_status ffeq_equalize_noalloc(const ffeq_plan* plan, const void* H, const void* y, float N0, float Es,
                                  void* z, float* sigma2, float* llr, int* info, void* stream);

/* Read (and, if clear != 0, reset) the device status word written by bounded
 * waits: FFEQ_OK or FFEQ_ERR_TIMEOUT.  Synchronous with respect to the device. */
ffeq_status ffeq_device_status(int* code, int clear);

/* Human-readable status; the last CUDA error string seen by the library. */
const char* ffeq_status_string(ffeq_status s);
const char* ffeq_last_cuda_error(void);

/* ABI version: major * 10000 + minor * 100 + patch. */
int ffeq_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FFEQ_H */
