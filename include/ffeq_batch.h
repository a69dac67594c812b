/* Uneven batches: many independent equalization problems of different sizes
 * (B, U, C, n_sym, N0, Es) in one call.
 *
 * Each instance is the problem of ffeq.h (Sec. II-A..D, III-A, IV-A of the
 * paper: PD central L-MMSE from the summed local Gram matrices and MRC
 * outputs, or FD local L-MMSE with optimal fusion, Eq. fusionrule, Lemma 1,
 * Thm. 3; or the ZF or MRC equalizer in place of L-MMSE) with its own sizes
 * and noise level; the architecture, precision, equalizer, estimate and LLR
 * width are shared by the batch.  The paper treats one system
 * at a time; batching instances is this library's addition for receivers that
 * serve several cells or carriers with one GPU.
 *
 * Every instance's arrays live at element offsets in five flat device buffers:
 *   H      cf32  [n_sc][U][B]            at h_off       (complex elements)
 *   y      cf32  [n_sc][n_sym][B]        at y_off
 *   z      cf32  [n_sc][n_sym][U]        at z_off
 *   sigma2 f32   [n_sc][U]               at sigma2_off  (float elements; [n_sc][n_sym][U] for LAMA)
 *   llr    f32   [n_sc][n_sym][U][bits]  at llr_off     (only when llr_bits > 0)
 *   info   i32   [n_sc][Ceff]            at info_off    (only when info is passed)
 * with Ceff = C (FD) or 1 (PD), and the layouts and meanings of ffeq.h.  The
 * caller places instances freely (outputs must not overlap); the extents given
 * at creation bound every offset, on the host at creation and again on the
 * device for every unit of work.
 *
 * Work is grouped by users padded to 8, 16 or 32.  Per group one persistent
 * contraction kernel takes subcarriers from a device work queue in order of
 * decreasing cost, and one solve/fusion kernel packs the local systems of
 * several subcarriers into each CTA.  All launches of a call are stream-ordered
 * and may be captured into a CUDA graph. */
#ifndef FFEQ_BATCH_H
#define FFEQ_BATCH_H

#include "ffeq.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int B, U, C;              /* antennas, users, clusters (B % C == 0) */
  int n_sc, n_sym;          /* subcarriers (>= 0) and OFDM symbols (1..16) */
  float N0, Es;             /* N0 >= 0, Es > 0, finite */
  long long h_off, y_off;   /* element offsets of the inputs */
  long long z_off, sigma2_off, llr_off, info_off;   /* element offsets of the outputs */
} ffeq_instance;

typedef struct {
  int arch;        /* ffeq_arch, shared by the batch */
  int precision;   /* ffeq_precision */
  int estimate;    /* ffeq_estimate, read for L-MMSE only: ZF and MRC fuse their own pairs */
  int llr_bits;    /* 0, 2, 4, 6 or 8 */
  /* element counts of the flat buffers (info_elems = 0: info never passed) */
  long long h_elems, y_elems, z_elems, sigma2_elems, llr_elems, info_elems;
  /* ffeq_equalizer, shared by the batch: FFEQ_LMMSE (0, zero-initialized
   * configs), FFEQ_ZF or FFEQ_MRC with the meanings of ffeq.h (Sec. III-A; FD
   * fusion by Lemma 1 with the same readings, including the N0 -> 0 limit
   * weights of MRC), or FFEQ_LAMA (Sec. III-B, Algorithm 1, FD fused by
   * Lemma 1 as in ffeq.h: needs llr_bits > 0, the prior's constellation, and
   * N0 > 0 in every instance; sigma^2 per received vector). */
  int equalizer;
  /* LAMA iterations T (1..64) for FFEQ_LAMA, else 0 (FFEQ_ERR_INVALID_ARG). */
  int lama_iters;
} ffeq_batch_config;

typedef struct ffeq_batch ffeq_batch;

/* Validate the instances and build the schedule on the host (page-locked host
 * memory for the descriptor tables; no device allocation).  Per instance the
 * limits of ffeq_plan_create hold, and B even when the contraction stages rows
 * with bulk copies (always the case here: odd B or odd offsets are staged with
 * plain loads instead).  n_inst >= 0; inst is a host array.
 * Returns FFEQ_ERR_INVALID_ARG (bad sizes, scalars or offsets) or
 * FFEQ_ERR_UNSUPPORTED (an instance beyond the limits). */
ffeq_status ffeq_batch_create(ffeq_batch** out, const ffeq_batch_config* cfg, const ffeq_instance* inst,
                              int n_inst);

/* Destroy a batch plan (NULL is ignored). */
void ffeq_batch_destroy(ffeq_batch* batch);

/* Device workspace bytes: descriptor tables (copied in by the library), the
 * work-queue counters and the local Gram matrices and MRC outputs of every
 * (subcarrier, cluster).  Owned by the caller, 256-byte aligned. */
ffeq_status ffeq_batch_workspace_size(const ffeq_batch* batch, size_t* bytes);

/* Copy the descriptor tables into the workspace (stream-ordered, from the
 * plan's page-locked host memory).  ffeq_batch_equalize does this by itself
 * the first time it sees a workspace address; call it again only when the
 * workspace memory was written by anything else since. */
ffeq_status ffeq_batch_upload(ffeq_batch* batch, void* workspace, size_t workspace_bytes, void* stream);

/* Equalize every instance.  H, y, z, sigma2 device pointers; llr device
 * pointer (required when llr_bits > 0, else ignored); info device pointer or
 * NULL (requires info_elems > 0).  Asynchronous; launches: one memset of the
 * queue counters, then per user group a contraction kernel and a solve/fusion
 * kernel (programmatic dependent launch).  Capturable into a CUDA graph once
 * the workspace holds the tables (after a first call or ffeq_batch_upload).
 * Calls sharing a workspace must be ordered on one stream.  A descriptor that
 * fails the device checks is skipped and sets FFEQ_ERR_INVALID_ARG in the
 * device status word (ffeq_device_status). */
ffeq_status ffeq_batch_equalize(ffeq_batch* batch, const void* H, const void* y, void* z, float* sigma2,
                                float* llr, int* info, void* workspace, size_t workspace_bytes,
                                void* stream);

/* Autotune the launch shapes of every group (contraction pipeline depth,
 * solve CTA width, lanes per system row) by timing ffeq_batch_equalize on the
 * given buffers with CUDA events, reps calls per candidate, coordinate by
 * coordinate; keeps the fastest.  Synchronizes the stream; must not run during
 * stream capture.  Results are the same for every choice up to rounding order
 * of the solve (the contraction order is fixed). */
ffeq_status ffeq_batch_autotune(ffeq_batch* batch, const void* H, const void* y, void* z, float* sigma2,
                                float* llr, int* info, void* workspace, size_t workspace_bytes, void* stream,
                                int reps);

/* Number of user groups, and their tuning as 4 ints per group:
 * {users padded (8/16/32), contraction stages, solve threads per CTA, lanes
 * per row}.  ffeq_batch_get_tuning writes min(n, 4 * groups) ints;
 * ffeq_batch_set_tuning takes exactly 4 * groups ints and validates each
 * choice (FFEQ_ERR_INVALID_ARG otherwise, leaving the plan unchanged). */
int ffeq_batch_groups(const ffeq_batch* batch);
ffeq_status ffeq_batch_get_tuning(const ffeq_batch* batch, int* values, int n);
ffeq_status ffeq_batch_set_tuning(ffeq_batch* batch, const int* values, int n);

#ifdef __cplusplus
}
#endif

#endif /* FFEQ_BATCH_H */
