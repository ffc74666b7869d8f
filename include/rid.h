/*
 * rid.h -- C ABI of the GB300 single-pass online randomized interpolative
 * decomposition (Li, Becker & Doostan, arXiv 2405.16076).
 *
 * Problem (Sec. 1 and Algorithm 3): the columns a_1..a_n of an m x n matrix A
 * arrive once, in order.  After the stream ends the library returns an index
 * set J of t = k columns and a t x n coefficient matrix P with A ~ A(:,J) P
 * (the column ID of Eq. 2), together with single-pass NA-Hutch++ estimates of
 * ||A - A(:,J) P||_F for the four coefficient updates (Algorithm 8).
 *
 * Conventions shared by every entry point:
 *  - Return RID_OK (0) on success, a negative RID_E* code otherwise; the text
 *    of the last error is available from rid_last_error().  No C++ exception
 *    crosses this boundary.
 *  - All compute runs asynchronously on the handle's CUDA stream
 *    (rid_config.cuda_stream, NULL = the legacy default stream).  Entry points
 *    that return data to the host synchronize that stream.
 *  - Matrices are column-major.  A "column" of the stream is m contiguous
 *    elements of the configured data type; ld is the element distance
 *    between consecutive columns (ld >= m).
 *  - The handle owns all device state.  Output buffers are owned by the
 *    caller.  One handle must not be used by two host threads at once.
 *  - Indices are 0-based; -1 marks an empty basis slot.
 */
#ifndef RID_H
#define RID_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum rid_status {
  RID_OK = 0,
  RID_EINVAL = -1,      /* bad argument or configuration */
  RID_ENOMEM = -2,      /* device or host allocation failed */
  RID_ECUDA = -3,       /* a CUDA runtime call failed */
  RID_ESTATE = -4,      /* call not allowed in the current state (e.g. ingest after finalize) */
  RID_ENONFINITE = -5,  /* a NaN/Inf snapshot was ingested (detected from its squared norm) */
  RID_ENOLIB = -6,      /* the CUDA library is missing or no device is present */
  RID_ETIMEOUT = -7     /* a bounded wait inside a kernel gave up; that kernel returned early */
};

enum rid_lambda_mode {
  RID_LAMBDA_STREAMING = 0,  /* lambda = (||A_obs||_F^2 - ||S_k||_F^2)/k, Eq. 23 */
  RID_LAMBDA_FIXED = 1       /* lambda = lambda_fixed, e.g. ||A - A_k||_F^2/k (Eq. 17 with Eq. 16) */
};

enum rid_omega_kind {
  RID_OMEGA_GAUSSIAN = 0,    /* i.i.d. N(0,1) entries (Algorithm 3, randn) */
  RID_OMEGA_RADEMACHER = 1   /* i.i.d. +-1 entries (sub-Gaussian, Sec. 3.3) */
};

enum rid_dtype { RID_F64 = 0, RID_F32 = 1 };

/* Refill of an empty basis slot (Algorithm 3's inner loop over the buffered columns r, each
 * taken with probability p_r = min(1, tau^D_r c (k ln k + k ln(1/delta)/eps) / t)).  Both
 * readings decide whether the slot is refilled by scanning r in order with one uniform per
 * (batch, slot, r): the first r with u < p_r whose column is not already in the basis succeeds. */
enum rid_refill_mode {
  RID_REFILL_FIRST = 0,       /* the slot takes that first successful column (default) */
  RID_REFILL_PROPORTIONAL = 1 /* the slot takes a column drawn among those not in the basis with
                                 probability tau^D_r / sum tau^D (Sec. 2.3's normalized score),
                                 by one more uniform per slot; differs from FIRST chiefly when
                                 every p_r is clipped to 1 */
};

enum rid_sketch_prec {
  RID_SKETCH_NATIVE = 0,     /* sketch accumulated in the data type (FP64 or FP32) */
  RID_SKETCH_BF16 = 1,       /* data rounded to BF16, tensor cores, FP32 accumulation */
  RID_SKETCH_BF16X2 = 2,     /* data split hi+lo in BF16, tensor cores, FP32 accumulation */
  RID_SKETCH_FP8 = 3,        /* data in E4M3 with one power-of-two scale per 32 coordinates of a
                                column (the smallest with no element above 448), tensor cores
                                (block-scaled MMA), FP32 accumulation */
  RID_SKETCH_FP8X2 = 4       /* two block-scaled E4M3 terms: a ~ hi + lo, lo quantizing the
                                residual a - hi with its own block scales */
};

/* Sum `count` doubles of the device buffer `buf` over every shard of a row-sharded stream (see
 * rid_config.allreduce), in place, with the same result bits on every shard, ordered on the CUDA
 * stream `cuda_stream` (for example ncclAllReduce with ncclSum on that stream).  `user` is
 * rid_config.allreduce_user.  Return 0 on success, nonzero on failure (the calling entry point
 * then fails with RID_ECUDA). */
typedef int (*rid_allreduce_fn)(double* buf, int64_t count, void* cuda_stream, void* user);

typedef struct rid_config {
  int64_t m;             /* snapshot length */
  int32_t k;             /* target rank; basis size t = k (Sec. 2.2.2) */
  int32_t s;             /* left-sketch rows (ell of Algorithm 3) */
  int32_t h;             /* independent Hutch++ probe rows; 0 = shared rows of the left sketch */
  int32_t lambda_mode;   /* enum rid_lambda_mode */
  double c1, c2;         /* NA-Hutch++ split, c1 < c2, c3 = 1 - c1 - c2 (Algorithm 8) */
  double eps, delta;     /* accuracy and failure probability of the refill rule (Algorithm 3) */
  double c_const;        /* constant c of the refill probability (Algorithm 3) */
  double lambda_fixed;   /* used when lambda_mode == RID_LAMBDA_FIXED */
  int32_t omega_kind;    /* enum rid_omega_kind */
  int32_t data_dtype;    /* enum rid_dtype */
  int32_t sketch_prec;   /* enum rid_sketch_prec */
  int32_t grad_dims;     /* 0 = off; 2 = 2-D grid gradient in the leverage sketch (Sec. 3.4) */
  int32_t nx, ny;        /* grid of one field when grad_dims = 2 (x fastest) */
  int32_t nfields;       /* fields stacked in one snapshot when grad_dims = 2 */
  int64_t n_max;         /* initial capacity in columns (grows by doubling) */
  uint64_t seed;         /* key of the Philox4x32-10 streams */
  int32_t group_max;     /* columns sketched per launch (1..64; 0 = 64 on tensor cores, 16 otherwise) */
  int32_t defer_device_input; /* 1: device columns are read later, in groups (see rid_ingest) */
  void* cuda_stream;     /* cudaStream_t to run on; NULL = default stream */
  int32_t right_l;       /* columns l of the optional right sketch Y = sum_j a_j omega_j^T
                            (m x l, data dtype; not part of the paper's method); 0 = off */
  int32_t grad_coeff;    /* 1 = keep Omega G^p a_j (p = 1, 2) during the ingest for the
                            gradient-augmented coefficients of Sec. 3.4 (needs grad_dims = 2;
                            see rid_gradient_coefficients) */
  int32_t ingest_ctas;   /* CTAs per sketch launch; 0 = automatic (tensor cores: every SM for the
                            first batch, two thirds of them beside the batch steps afterwards;
                            native path: up to four per SM).  A positive value replaces the
                            tensor-core ingest's count after the first batch, or caps the native
                            one, and is clamped to the automatic maximum (see rid_autotune) */
  int32_t refill_mode;   /* enum rid_refill_mode: which buffered column refills an empty basis slot */
  int32_t lookahead;     /* batches the ingest may run ahead of the batch steps, 2..4 (0 = 3): the
                            select of step b chooses the buffer slots of batch b + lookahead, and
                            the handle keeps (lookahead + 2) t data columns of m in device memory.
                            The results do not depend on it */
  /* Row sharding (Sec. 5's in-situ parallel use; NULL allreduce = off).  Each shard -- one handle
   * per GPU or rank -- holds rows [row_offset, row_offset + m) of every snapshot of a stream of
   * m_global rows; Omega's entries are keyed by the global row, so the shards' partial sketches sum
   * to the whole one.  The library calls allreduce at the method's two exchange points, on the
   * handle's own streams: after each sketch group, on the (s + h) x ncols partial sketch and then
   * on the ncols partial squared norms; in each batch step, on the t x 2t block of partial basis
   * Gram entries (new elements x targets).  Everything else is replicated on every shard from the
   * summed values, so all shards return the same J and P; rid_get_basis returns the shard's rows.
   * Needs row_offset a multiple of 128, m_global >= row_offset + m, no gradient mode; every shard
   * must make the same calls in the same order with the same configuration apart from m and
   * row_offset.  Not meant for stream capture unless allreduce is capturable. */
  int64_t row_offset;
  int64_t m_global;
  rid_allreduce_fn allreduce;
  void* allreduce_user;
  /* SM partition (0 = off).  With batch_sms > 0 the batch steps' streams run in a CUDA green
   * context holding at least batch_sms SMs (rounded up to the device's partition granularity),
   * and the ingest of every batch after the first in a second green context holding the other
   * SMs, with one CTA per SM of it unless ingest_ctas asks for fewer; the first batch's ingest,
   * beside which no batch step runs, keeps the whole device.  Neither part then waits for SMs the
   * other holds.  rid_init fails with RID_ECUDA when the driver offers no green contexts, and with
   * RID_EINVAL when batch_sms is not below the SM count or the partition cannot co-schedule the
   * batch step's thread-block clusters.  The results do not depend on it. */
  int32_t batch_sms;
} rid_config;

typedef struct rid_handle rid_handle;

/* Fill *cfg with defaults: c1 = 1/6, c2 = 1/3, eps = 0.5, delta = 0.05,
 * c_const = 1, streaming lambda, Rademacher Omega, FP32 data, native sketch,
 * n_max = 1024.  m, k, s, h must still be set.  Returns RID_EINVAL on NULL. */
int rid_config_default(rid_config* cfg);

/* Check *cfg as rid_init does (the same conditions and messages), without creating a handle
 * or touching a device.  Returns RID_OK or RID_EINVAL (message in rid_last_error(NULL)). */
int rid_config_check(const rid_config* cfg);

/* Validate *cfg and allocate the device state (Algorithm 3, initialisation).
 * On success *out receives a new handle.  Errors: RID_EINVAL (sizes: m >= 1,
 * 1 <= k <= 1024, k < s <= 4096, 0 <= h <= 1024, h == 0 or h >= 3,
 * 0 < c1 < c2, c1 + c2 < 1, unknown enum values; gradient mode: grad_dims
 * must be 0 or 2, and with 2: nx, ny >= 2, nfields >= 1, m = nx ny nfields,
 * sketch_prec NATIVE; 0 <= right_l <= 4096; grad_coeff needs grad_dims = 2), RID_ENOMEM,
 * RID_ENOLIB.
 * Gradient mode (Sec. 3.4, Eqs. 38-43): the ridge scores and lambda use the
 * sketch of [a; G a], i.e. Omega a + Omega_g (G a) with an independent Omega_g
 * (s x 2m), and ||a||^2 + ||G a||^2; G is the least-squares gradient on each
 * field's nx x ny grid graph (central differences inside, one-sided at the
 * boundary, unit spacing).
 * On any failure every device allocation made so far is released and *out is NULL.  For tests
 * of these paths, RID_FAULT_INJECT=alloc:<n> in the environment when rid_init starts makes the
 * n-th device allocation from then on -- in this rid_init or in a later capacity growth of a
 * handle -- fail as if the device were out of memory (RID_ENOMEM); a growth that fails leaves
 * its handle as it was, with the recorded columns still pending. */
int rid_init(rid_handle** out, const rid_config* cfg);

/* Ingest ncols >= 0 columns (Algorithm 3, the loop body for each column):
 * column q starts at cols + q*ld elements of the configured dtype.
 * on_device != 0: cols is a device pointer, read in place; otherwise a host
 * pointer, copied to a device staging area on the handle's stream first.  The
 * library copies what it keeps.  A pageable host buffer may be reused
 * when the call returns; a page-locked (pinned) one is read asynchronously and
 * may be reused after the next synchronizing call (rid_sync, rid_finalize);
 * a device buffer once the handle's stream has passed this
 * call -- except with defer_device_input = 1, where device columns are only
 * recorded and read later, in groups of up to group_max columns (one read of
 * each column sketches the whole group); the caller must then keep them
 * valid and unchanged until the t-th buffered column of the batch, or
 * rid_finalize / rid_sync / rid_get_state / rid_get_basis / rid_reset, has
 * been called and the stream has passed it.  Host columns are always grouped
 * through the staging area.  Whenever t = k columns have been buffered the batch step
 * (ridge scores, prune/refill, Algorithms 4-8) runs on the device without a
 * host round trip.  Errors: RID_EINVAL (ld < m, NULL cols with ncols > 0),
 * RID_ESTATE (after rid_finalize), RID_ECUDA. */
int rid_ingest(rid_handle* h, const void* cols, int64_t ld, int32_t ncols, int32_t on_device);

/* Ingest into several independent streams in one call (configuration C5:
 * many small streams): for i < nh, ncols[i] columns for handle hs[i], given
 * as in rid_ingest by cols[i] (leading dimension ld[i]).  Equivalent to nh
 * rid_ingest calls, enqueued in order i = 0, 1, ...; every handle runs on its
 * own streams, so handles created with distinct cuda_stream values proceed
 * concurrently on the device.  Stops at the first failing handle and returns
 * its status (its message in rid_last_error of that handle); handles before it
 * have ingested their columns.  Errors: RID_EINVAL (NULL arrays, nh < 0, a
 * NULL handle), and those of rid_ingest. */
int rid_batch_ingest(rid_handle* const* hs, int32_t nh, const void* const* cols, const int64_t* ld,
                     const int32_t* ncols, int32_t on_device);

/* End the stream: run the batch step over the count < t buffered columns, if
 * any (tail batch).  Then, if J_out != NULL, write the t basis indices
 * (int64, -1 = empty slot) and, if P_out != NULL, the t x n coefficient matrix
 * (double, column-major, ldp >= t).  on_device: 0 = host output pointers,
 * 1 = device output pointers; both synchronize the stream and report device
 * errors.  RID_OUT_DEVICE_ASYNC = device output pointers without any host
 * synchronization: the copies are queued on the handle's stream, device errors
 * surface at the next synchronizing call (rid_sync), and the call may be
 * captured into a CUDA graph together with rid_reset and rid_ingest of device
 * columns (with n_max large enough that no capacity growth is needed).  May be
 * called again to re-read the result.  Errors: RID_EINVAL (ldp < t),
 * RID_ENONFINITE, RID_ECUDA. */
enum { RID_OUT_HOST = 0, RID_OUT_DEVICE = 1, RID_OUT_DEVICE_ASYNC = 2 };
int rid_finalize(rid_handle* h, int64_t* J_out, double* P_out, int64_t ldp, int32_t on_device);

/* Estimates from the last batch step (Algorithm 8): est_sq[0] = chosen
 * candidate, est_sq[1..4] = Algorithms 4..7, signed estimates of
 * ||A_obs - A_J P||_F^2; est_fro = sqrt(max(est_sq, 0)); *q_star in 4..7.
 * Any output pointer may be NULL.  Synchronizes.  RID_ESTATE before the first
 * batch step. */
int rid_error_estimate(rid_handle* h, double est_sq[5], double est_fro[5], int32_t* q_star);

/* Number of columns ingested so far. */
int64_t rid_n_obs(const rid_handle* h);

/* Copy the current basis columns A(:,J) (m x t, data dtype, ld >= m; empty
 * slots are written as zeros) to out (device or host).  Synchronizes. */
int rid_get_basis(rid_handle* h, void* out, int64_t ld, int32_t on_device);

/* Copy the optional right sketch Y = sum_{j < n_obs} a_j omega_j^T (m x right_l, data dtype,
 * column-major, ld >= m) to out (device or host).  omega_j holds right_l unit-variance entries
 * of the configured kind (Rademacher or Gaussian) drawn from their own Philox stream keyed by
 * the snapshot index j; Y is updated once per group of ingested columns.  Not part of the
 * paper's method (a running sketch of the stream's range).  Synchronizes.  Errors:
 * RID_EINVAL (NULL out, ld < m), RID_ESTATE (right_l = 0), RID_ECUDA. */
int rid_get_right_sketch(rid_handle* h, void* out, int64_t ld, int32_t on_device);

/* Gradient-augmented coefficients of Sec. 3.4 for the final basis (the stream is finalized
 * first if it was not): P(lambda) = argmin_X ||Omega (A_J X - A)||_F^2
 * + lambda sum_p ||Omega (G^p A_J X - G^p A)||_F^2 from the sketches, with lambda chosen by
 * golden-section search of the sketched GCV function GCV(lambda) = ||(I - C(lambda)) Omega A||^2
 * / tr(I - C(lambda))^2 over log10(lambda) in [-3, 3] (bracket narrower than 1e-3; the midpoint
 * of the last bracket).  C(lambda) = Omega A_J M^{-1} (Omega A_J + lambda sum_p (Omega G^p
 * Omega^T)^T Omega G^p A_J)^T, M = (Omega A_J)^T Omega A_J + lambda sum_p (Omega G^p A_J)^T
 * Omega G^p A_J, every sketch scaled by 1/sqrt(s).  Writes P (t x n, double, column-major,
 * ldp >= t, rows of empty slots 0; device or host per on_device), *lambda_out and *gcv_out
 * (may be NULL).  The first call forms Omega G^p Omega^T / s (s^2 m work per direction).
 * Allocates device scratch; synchronizes.  Errors: RID_ESTATE (grad_coeff = 0), RID_EINVAL
 * (ldp < t, NULL P_out), RID_ENOMEM / RID_ECUDA. */
int rid_gradient_coefficients(rid_handle* h, double* P_out, int64_t ldp, int32_t on_device, double* lambda_out,
                              double* gcv_out);

/* Internal state for tests (host output, synchronizes):
 *  RID_STATE_SKETCH   : (s+h) x n_obs doubles, Omega A_obs (unit-variance rows)
 *  RID_STATE_SKETCH_LEV: s x n_obs doubles, the sketch used by the ridge scores
 *  RID_STATE_SST      : s x s doubles
 *  RID_STATE_FRO2     : 2 doubles, ||A_obs||^2 and the leverage-sketch norm
 *  RID_STATE_JC       : t int64 basis indices
 *  RID_STATE_TAU_OLD  : t doubles
 *  RID_STATE_LAMBDA   : 1 double, lambda of the last batch step
 *  RID_STATE_CAND     : 4 x t x n_obs doubles, candidates P_4..P_7 of the last
 *                       batch step (rows of empty slots are 0)
 *  RID_STATE_BATCHES  : 1 int64, number of batch steps run
 *  RID_STATE_GRAD_SKETCH: 2 s x n_obs doubles, column j = [Omega G^1 a_j; Omega G^2 a_j]
 *                       (unit-variance rows; grad_coeff = 1 only)
 *  RID_STATE_GRAM_SHIFT: 1 double, the Tikhonov shift that the last batch step
 *                       added to the basis Gram of Algorithms 5 and 7, relative
 *                       to its largest diagonal entry; 0 when G = A_J^T A_J was
 *                       factored as is.  The shift is taken only when the
 *                       smallest Cholesky pivot falls below that same fraction
 *                       of the largest diagonal entry (1e-11 for FP64 sums,
 *                       3e-5 for the tensor-core Gram of FP32 data): the basis
 *                       is then so nearly dependent that the Gram's rounding
 *                       would dominate the solve.
 * count is the number of elements the caller's buffer holds. */
enum rid_state_item {
  RID_STATE_SKETCH = 0, RID_STATE_SKETCH_LEV = 1, RID_STATE_SST = 2, RID_STATE_FRO2 = 3,
  RID_STATE_JC = 4, RID_STATE_TAU_OLD = 5, RID_STATE_LAMBDA = 6, RID_STATE_CAND = 7,
  RID_STATE_BATCHES = 8, RID_STATE_GRAM_SHIFT = 9, RID_STATE_GRAD_SKETCH = 10
};
int rid_get_state(rid_handle* h, int32_t item, void* out, int64_t count);

/* Checkpoint / resume of a stream (not in the paper: a library service for long
 * streams).  rid_checkpoint_size gives the bytes rid_checkpoint needs;
 * rid_checkpoint sketches any pending columns, waits for the device, and writes
 * the stream state to the caller's host buffer: the configuration, the counters,
 * the sketch, SS^T, the norms, the basis and buffer slot tables, tau, P, the
 * pool Gram and the data columns still in use (the basis and the columns of
 * the current batch).  rid_restore puts such a state into a handle created
 * with the same configuration (any state it held is discarded); the stream
 * then continues exactly as the checkpointed one would have.  rid_restore
 * checks the whole buffer before it changes the handle: the magic number, the
 * configuration, the counters (0 <= count < t, n_prev = n_obs - count >= 0,
 * batch >= 0, finalized 0 or 1, 0 <= saved slots <= t + count), the size and
 * every saved pool slot; a rejected buffer leaves the handle's stream as it
 * was.  Errors: RID_EINVAL (buffer too small or truncated, another
 * configuration, inconsistent counters, not a checkpoint), RID_ECUDA (the
 * handle is then in the reset state). */
int rid_checkpoint_size(rid_handle* h, int64_t* bytes);
int rid_checkpoint(rid_handle* h, void* buf, int64_t bytes);
int rid_restore(rid_handle* h, const void* buf, int64_t bytes);

/* Measurement hooks (used by the benchmark).  While enabled, the library
 * brackets its launches with CUDA events on the handle's stream, per phase:
 * [0] the fused ingest/sketch kernel, [1] the ingest reductions (sketch
 * append, SS^T, ||A_obs||^2), [2] the batch step; and counts its kernel
 * launches.  rid_profile(h, 1) clears the counters; rid_profile_read
 * synchronizes and returns total milliseconds, kernel launches and bracketed
 * launch groups per phase since then (any pointer may be NULL). */
int rid_profile(rid_handle* h, int32_t enable);
int rid_profile_read(rid_handle* h, double ms[3], int64_t kernels[3], int64_t groups[3]);

/* Per-batch phase timeline of the launches made while profiling was on (a benchmark hook; the
 * paper has no counterpart).  Each record is four doubles: the batch index, the phase, and its
 * start and end in milliseconds from the rid_profile(h, 1) call, measured with CUDA events on
 * the stream the phase runs on.  Phases: 0 an ingest group (sketch launch and reductions, on the
 * handle's stream), 1 the lambda part of a batch step (tridiagonalization, top-k eigenvalues,
 * lambda and LDL^T of Eq. 23), 2 the ridge scores, 3 the uniforms and the prune / refill of
 * Algorithm 3, 4 the Gram side of the tail (basis Gram, its Cholesky factor, T of
 * Algorithm 7), 5 the sketch side of the tail (gathers, Householder QRs, projections), 6 the
 * coefficient candidates, NA-Hutch++ and the commit (Algorithms 4-8).  Writes min(max_records,
 * available) records to out (4 * max_records doubles) and their number to *n_out; with
 * max_records = 0 only the number available.  Synchronizes.  Errors: RID_EINVAL (bad buffer),
 * RID_ESTATE (profiling off), RID_ECUDA. */
int rid_profile_timeline(rid_handle* h, double* out, int32_t max_records, int32_t* n_out);

/* One record of the per-batch log: what a batch step decided (the quantities of the paper's
 * "update decision" rows, Algorithm 8 with Eqs. 23 and 36-37). */
typedef struct {
  int64_t batch;        /* 0-based index of the batch step */
  int64_t n_obs;        /* columns observed when it ran (its P covers them) */
  double lambda;        /* its ridge parameter (Eq. 23's streaming value, or the fixed one) */
  double fro2;          /* ||A_obs||_F^2 it used */
  double est_sq[4];     /* signed NA-Hutch++ estimates of ||A_obs - A_J P_q||_F^2, q = 4..7 */
  double est_unc[4];    /* rounding uncertainty of each estimate relative to fro2 (0 for FP64 sketches) */
  double gram_shift;    /* Tikhonov shift of the basis Gram relative to its largest diagonal entry */
  int32_t q_star;       /* the candidate committed to P (4..7) */
  int32_t n_active;     /* occupied basis slots after the step */
  int32_t n_kept;       /* of those, slots that held the same column before the step */
  int32_t n_new;        /* of those, slots filled by the step */
} rid_log_record;

/* Keep a log of the last `capacity` batch steps on the device (0 turns it off and frees it);
 * the log starts empty with the next batch step.  Each step adds four small device-to-device
 * copies on the handle's own streams (none while the log is off), so logging also works inside a
 * captured CUDA graph.  Synchronizes.  Errors: RID_EINVAL (capacity outside [0, 2^20]),
 * RID_ENOMEM, RID_ECUDA. */
int rid_log_enable(rid_handle* h, int32_t capacity);

/* Copy the most recent min(max_records, steps logged, capacity) records, oldest first, to out
 * (host) and their number to *n_out (may be NULL); with max_records = 0 nothing is copied and
 * *n_out receives the number of records available.  Synchronizes; pending columns are not
 * flushed.  rid_reset and rid_restore start the log afresh.  Errors: RID_EINVAL (max_records < 0,
 * NULL out with max_records > 0), RID_ESTATE (the log is off), RID_ECUDA. */
int rid_get_log(rid_handle* h, rid_log_record* out, int32_t max_records, int32_t* n_out);

/* Wait for the handle's stream; report deferred device errors. */
int rid_sync(rid_handle* h);

/* Forget the stream (keep allocations): the handle is as after rid_init. */
int rid_reset(rid_handle* h);

/* Text of the last error on h (or, when h is NULL, of the last failed
 * rid_init, rid_config_check, rid_autotune or rid_sketch_noalloc of the calling thread). */
const char* rid_last_error(const rid_handle* h);

/* Pick the ingest's launch shape for *cfg on the current device by measurement (no counterpart
 * in the paper: a tuning of this library's ingest): cfg->group_max, how many device columns one
 * sketch launch reads, and cfg->ingest_ctas, the CTAs per sketch launch.  cols: ncols >= 1
 * representative columns of the stream (device memory, m x ncols column-major, ld >= m), read
 * and not modified; 2k columns cover two batch steps.  Each candidate runs the columns through a
 * temporary handle of *cfg with defer_device_input = 1: one untimed pass, then three passes
 * timed on the host clock from the first rid_ingest to the end of rid_sync -- the ingest and
 * the batch steps it triggers -- of which the fastest counts.  First the group size, with the
 * automatic CTA count: the powers of two from 1 to 64 (tensor-core sketches) or 16 (native
 * precision), up to the first one >= min(ncols, k) since groups never span a batch of k columns;
 * the largest group within 2 % of the fastest time wins.  Then, for that group, the CTA count:
 * automatic (0), then 1/6 .. 6/6 of the SMs (tensor cores) or 1, 2, 3 per SM (native path); the
 * first within 2 % of the fastest wins.  No other field of *cfg changes; *us_per_col (may be
 * NULL) receives the winner's time per column in microseconds.  If the environment variable
 * RID_AUTOTUNE_CACHE names a file, a stored result for the same device and configuration (m,
 * k, s, h, data dtype, sketch precision, Omega kind, gradient mode and coefficients, right_l) is
 * returned without measuring, and a new result is appended to the file as a line
 * "<key> <group> <ctas> <microseconds>".  Needs device memory for one handle at a time besides
 * the caller's columns.  Errors: RID_EINVAL (NULL cfg or cols, an invalid configuration,
 * ncols < 1, ld < m, cols not in device memory), RID_ENOLIB (no device), and those of rid_init /
 * rid_ingest; messages in rid_last_error(NULL). */
int rid_autotune(rid_config* cfg, const void* cols, int64_t ld, int32_t ncols, double* us_per_col);

/* Sketch of a block of columns that allocates nothing.  The paper has no
 * counterpart: this is a library service for callers that cannot allocate
 * device memory per call -- typically a simulation compressing its snapshots
 * in situ, which reserves nearly all of HBM for its own fields and whose time
 * loop must not be stalled by the device-wide synchronisation of cudaMalloc /
 * cudaFree.  It calls no cudaMalloc, cudaFree or other allocating routine;
 * its split-K partial sums live in one fixed file-scope device array of
 * 8 MiB + 16 KiB per GPU, present from the library's first use on that GPU
 * until the process exits.
 *
 * Computes, on cfg->cuda_stream (asynchronous; nothing is synchronized):
 *   S_out(r, q) = (Omega a_q)_r for r < s + h   (the rows and scaling of
 *                 RID_STATE_SKETCH of a handle with the same m, s, h, seed)
 *   norms_out[q] = ||a_q||^2                      for q < ncols.
 * Reads from cfg: m, s, h, omega_kind (must be RID_OMEGA_RADEMACHER),
 * data_dtype (RID_F64 / RID_F32), seed, cuda_stream; ignores the rest.
 *   cols      : device, column q at cols + q*ld elements of data_dtype, ld >= m
 *   S_out     : device doubles, column q at S_out + q*lds, lds >= s + h
 *   norms_out : device, ncols doubles
 * The caller owns all three buffers.  Limits, fixed by the scratch size:
 * 1 <= ncols <= 16 and s + h <= 512; a call beyond them returns RID_EINVAL
 * with a message in rid_last_error(NULL) and launches nothing.
 * Set-up: the first call on a device, with that device current, looks up the
 * scratch array's address (cudaGetSymbolAddress) and keeps it; make that
 * first call before any stream capture.  The kept address belongs to that
 * device's primary context: after a cudaDeviceReset of the device it is stale,
 * and the entry point must not be called on that device again in the process.
 * The device is the current one; cfg->cuda_stream must belong to it (else
 * RID_EINVAL).  Every later call on the device
 * shares the array, which keeps the last call's contents (nothing in it has
 * to start at zero).  Calls whose kernels overlap on the GPU (streams with no
 * ordering between them) race on the scratch; calls on one stream are safe.
 * Errors: RID_EINVAL (NULL or non-device pointer, sizes, Gaussian Omega, a
 * stream of another device), RID_ENOLIB (no GPU), RID_ECUDA (set-up or launch
 * failure). */
int rid_sketch_noalloc(const rid_config* cfg, const void* cols, int64_t ld, int32_t ncols,
                       double* S_out, int64_t lds, double* norms_out);

/* Free everything.  NULL is ignored. */
void rid_destroy(rid_handle* h);

/* ---- Online column subset selection by residual-based sampling ----------------------------
 * The paper's Algorithm 1 (Sec. 2.2.1, after Bhaskara et al.), the online selector the accuracy
 * tables compare the single-pass ID against; it is not a step of the ID (Algorithm 3).  For each
 * arriving column a, numbered j = 0, 1, ... over the handle's life:
 *   p_a = k ||Pi_perp a||^2 / xi, Pi_perp the projector onto the orthogonal complement of the
 *         span of the previously selected columns C_pre (||a||^2 - ||Q^T a||^2 with Q an
 *         orthonormal basis of that span, FP64 sums);
 *   a joins C_cur if u_j < min(p_a, 1), u_j the 53-bit uniform of the Philox4x32-10 block at
 *         counter (j mod 2^32, j >> 32, 0x52435331, 0) and key (seed mod 2^32, seed >> 32),
 *         words 0 and 1, as every uniform of this library;
 *   if p_a < 1 the residual mass sigma grows by p_a; if p_a >= 1 or sigma >= 1, C_pre takes
 *         C_cur's columns (Q grows by each of them in order, orthogonalized twice against the
 *         basis so far; a column whose residual norm is at most tol times its norm adds no
 *         direction, tol = 1e-12 for FP64 data and 1e-4 for FP32) and sigma = 0.
 * The selection is C_pre followed by C_cur, by arrival.  Products are formed in the data's type
 * and summed in FP64 over runs of 128 coordinates; the basis is stored in the data's type.
 * Device memory: 2 cap + 1 columns of m (the basis, a candidate slot and the raw columns of
 * C_cur), plus 64 columns of staging for host input, allocated at the first host ingest. */
typedef struct rid_rcss rid_rcss;

/* New selector.  m >= 1 rows, k >= 1 (the target rank), xi > 0, data_dtype RID_F64 or RID_F32,
 * 1 <= cap <= 4096 the most columns it may select.  stop_at_cap != 0: once cap columns are
 * selected a later keep decision adds nothing and p, sigma and the steps go on (the treatment of
 * the experiments, Sec. 4.1, with cap = k); stop_at_cap = 0: a selection beyond cap is an error.
 * cuda_stream: the stream every call runs on (NULL: the legacy default stream).  Errors:
 * RID_EINVAL (sizes), RID_ENOMEM, RID_ENOLIB, RID_ECUDA (kernel set-up refused). */
int rid_rcss_init(rid_rcss** out, int64_t m, int32_t k, double xi, uint64_t seed, int32_t data_dtype,
                  int32_t cap, int32_t stop_at_cap, void* cuda_stream);

/* Decide ncols columns, column q at cols + q*ld elements (ld >= m), device memory if on_device
 * else host memory.  Blocks until they are decided.  Errors: RID_EINVAL (arguments; with
 * stop_at_cap = 0 a selection beyond cap, after which the handle's state is undefined),
 * RID_ENOMEM, RID_ECUDA. */
int rid_rcss_ingest(rid_rcss* h, const void* cols, int64_t ld, int32_t ncols, int32_t on_device);

/* The selection so far (C_pre then C_cur; global column numbers), at most max_out of them into
 * idx (host; NULL to skip), its length into *n_out, sigma into *sigma and the basis size (the
 * rank of span(C_pre)) into *basis_size; each output pointer may be NULL. */
int rid_rcss_selection(rid_rcss* h, int64_t* idx, int32_t max_out, int32_t* n_out, double* sigma,
                       int32_t* basis_size);

/* p_a of every column decided so far, by arrival (host doubles; at most max_out), count into
 * *n_out (may be NULL). */
int rid_rcss_probabilities(rid_rcss* h, double* p, int64_t max_out, int64_t* n_out);

/* The orthonormal basis Q of span(C_pre): basis_size columns of m, in the data's type, column i at
 * out + i*ld (ld >= m), device memory if on_device else host. */
int rid_rcss_basis(rid_rcss* h, void* out, int64_t ld, int32_t on_device);

/* Free everything.  NULL is ignored. */
int rid_rcss_destroy(rid_rcss* h);

/* Algorithm 1 as the handle's selector: the online rows of the paper's tables for the residual
 * CSS (Sec. 4.1), where the coefficients are computed with Algorithms 4-7 and Algorithm 8 picks
 * among them while Algorithm 1 selects.  From then on rid_ingest first passes each block to g
 * (rid_rcss_ingest), and every batch step puts the columns g kept from its batch into the empty
 * basis slots in order instead of Algorithm 3's prune / refill (Algorithm 1 never drops a column);
 * the ridge scores are still computed but decide nothing.  g must have the handle's m, data type
 * and stream, cap <= t and stop_at_cap != 0, and must outlive the handle's use of it; the handle
 * must have no row shards and no gradient mode.  Attach before the first rid_ingest; g = NULL
 * detaches.  rid_reset and rid_restore detach (a selector serves one stream); rid_checkpoint and
 * rid_checkpoint_size fail with RID_ESTATE while g is attached (its state is not in the
 * checkpoint).  Errors: RID_EINVAL (mismatch), RID_ESTATE (columns already ingested). */
int rid_attach_rcss(rid_handle* h, rid_rcss* g);

#ifdef __cplusplus
}
#endif
#endif /* RID_H */
