/*
 * gbs.h -- C ABI of libgbs: stage-1 tables of a Gaussian boson sampling emulator
 * (arXiv:2511.14923, Sec. "Pre-computing the cumulants" and App. "Correlators of
 * GBS with binary outcomes") on NVIDIA GB300 (sm_103a).
 *
 * Given the 2M x 2M covariance V of a zero-mean Gaussian state (hbar = 2, xxpp:
 * mode k owns rows/cols k and k+M), the library fills tables over every mode
 * subset S with 1 <= |S| <= kmax <= 5:
 *
 *   vacuum probability  P0(S)  = det[(V_S + I)/2]^{-1/2}
 *                        (Eq. vacuum_gaussian_prob with zero mean and hbar = 2;
 *                         V_S keeps rows/cols k and k+M for k in S)
 *   click moment        mu(S)  = p(every mode of S clicks)
 *                              = sum_{T subset S} (-1)^{|T|} P0(T)
 *                        (Eq. joint_moments_def / Eq. joint_moments_threshold)
 *   click cumulant      kt(S)  = sum over set partitions pi of S of
 *                                (-1)^{|pi|-1} (|pi|-1)! prod_{b in pi} mu(b)
 *                        (Eq. joint_cumulants_def)
 *
 * TABLE LAYOUT. A table has gbs_table_size(M, kmax) = sum_{d=1..kmax} C(M,d)
 * entries (FP64). Entries are grouped by order d (d = 1 first); the order-d group
 * starts at gbs_order_offset(M, d) and holds the d-subsets in colex order: the
 * sorted set c_1 < c_2 < ... < c_d (0-based modes) sits at rank
 * sum_{i=1..d} C(c_i, i). The empty set is not stored.
 *
 * MEMORY. Every pointer passed to a compute entry point (V, outputs, gradients,
 * workspace) is a CUDA device pointer owned by the caller; it must stay valid
 * until the work queued on cuda_stream completes. The library never allocates
 * device memory, never frees caller memory and never throws across the ABI.
 * Each compute call needs a caller-provided workspace of at least
 * gbs_workspace_bytes(M, kmax, precision) bytes, 256-byte aligned; one workspace
 * must not be used by two calls that may run at the same time.
 *
 * ERRORS. Argument errors are detected on the host before anything is queued
 * and return a nonzero gbs_status (gbs_last_error() gives a message). Device
 * errors (a non-positive-definite reduced covariance) are recorded in a status
 * word inside the workspace; the affected entries are NaN. gbs_stream_status()
 * synchronises the stream and returns that status.
 *
 * STREAMS. cuda_stream is a cudaStream_t (NULL = legacy default stream). Calls
 * are asynchronous with respect to the host; calls on one stream run in order.
 */
#ifndef GBS_H
#define GBS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GBS_OK = 0,
    GBS_ERR_INVALID_ARG = 1,  /* bad M, kmax, precision, null or misaligned pointer */
    GBS_ERR_NOT_POSDEF = 2,   /* some (V_T + I)/2 is not positive definite (device) */
    GBS_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    GBS_ERR_TIMEOUT = 4,      /* a bounded device wait of the sampler (gbs_sample) gave up */
    GBS_ERR_WORKSPACE = 5     /* workspace smaller than gbs_workspace_bytes() */
} gbs_status;

typedef enum {
    /* every determinant step in FP64 */
    GBS_FP64 = 0,
    /* determinant steps as FP32 Cholesky steps refined once to FP64 accuracy
       (log det += tr(L^{-1} E L^{-T}), residual E formed exactly from FP32
       products); inclusion-exclusion and partition sums stay in FP64 */
    GBS_FP32_REFINED = 1
} gbs_precision;

#define GBS_MAX_ORDER 5
#define GBS_MAX_MODES 1024
/* Tables with kmax <= 3 (and the K = 3 sampler) never use the prefix-tree
   kernels and accept up to this many modes, e.g. the 1152-mode state of a
   144-mode interferometer read out through 8 time bins (Sec. "High-brightness
   results for Jiuzhang 3.0"). */
#define GBS_MAX_MODES_K3 4096

/* ---------------------------------------------------------------- host helpers */

/* Number of table entries: sum_{d=1..kmax} C(M, d); 0 if the arguments are invalid
   (M < 1, kmax < 1, kmax > min(M, GBS_MAX_ORDER), M > GBS_MAX_MODES for kmax >= 4,
   M > GBS_MAX_MODES_K3 for kmax <= 3). */
uint64_t gbs_table_size(int M, int kmax);

/* First entry of the order-d group: sum_{e<d} C(M, e), e >= 1. 0 for invalid d. */
uint64_t gbs_order_offset(int M, int d);

/* Colex rank of a sorted mode set modes[0] < ... < modes[d-1]: sum C(modes[i], i+1).
   Returns UINT64_MAX if modes is NULL, d is out of [1, GBS_MAX_ORDER] or the
   modes are not strictly increasing in [0, GBS_MAX_MODES_K3). */
uint64_t gbs_rank(const int *modes, int d);

/* Inverse of gbs_rank: writes the d sorted modes of rank r to modes_out.
   Returns GBS_OK or GBS_ERR_INVALID_ARG. */
int gbs_unrank(uint64_t r, int d, int *modes_out);

/* Workspace bytes needed by any compute call with these (M, kmax, precision) on
   the current CUDA device; 0 if the arguments are invalid. */
size_t gbs_workspace_bytes(int M, int kmax, int precision);

/* Message for the most recent failing call on this host thread ("" if none). */
const char *gbs_last_error(void);

/* Synchronises cuda_stream, then returns the device status recorded in the
   workspace by the calls queued on it (GBS_OK, GBS_ERR_NOT_POSDEF, ...), or
   GBS_ERR_CUDA if the synchronisation itself failed. The status is cleared by
   the next compute call that uses the workspace. */
int gbs_stream_status(const void *workspace, void *cuda_stream);

/* The gbs_status that a status word (the first 4 bytes of a workspace, as a
   compute call leaves them) stands for, with its message for gbs_last_error():
   GBS_OK for 0, else GBS_ERR_TIMEOUT, GBS_ERR_NOT_POSDEF or GBS_ERR_INVALID_ARG
   (a failed device index check), in that order of precedence. Host-only, no
   CUDA call: it lets a caller copy the word to host memory asynchronously
   (stream-ordered, no synchronisation) and interpret it when the copy is done. */
int gbs_status_code(unsigned status_word);

/* Spin-correlator table: c_out[...] <- c(S) = E[prod_{k in S} (-1)^{x_k}]
   = (-1)^{|S|} sum_{R subset S} (-2)^{|R|} P0(R)  (Eq. correlator_sum_cov, hbar = 2),
   the correlators the paper's stage 1 computes. */
int gbs_spin_correlators(const double *V, int M, int kmax, double *c_out, int precision,
                         void *workspace, size_t ws_bytes, void *cuda_stream);

/* Spin-cumulant table: kappa_out[...] <- kappa(S), the cumulant of the spins
   (-1)^{x_k} over the partitions of S (Eq. cumulant_corr_main): the table the
   paper's sampler consumes. Computed through Eq. cumulant_exponential:
   kappa(S) = (-2)^{|S|} kt(S) for |S| >= 2 and 1 - 2 mu({k}) = 2 P0({k}) - 1. */
int gbs_spin_cumulants(const double *V, int M, int kmax, double *kappa_out, int precision,
                       void *workspace, size_t ws_bytes, void *cuda_stream);

/* ---------------------------------------------------------------- profiling */

/* Per-order kernel timing. While enabled (on != 0), every forward call records
   CUDA events on its stream before and after the kernels of each order.
   gbs_timing_read() waits for the events of the most recent call and writes
   durations in milliseconds: ms_out[0] = packing (V -> 2x2 blocks), ms_out[d] =
   the kernels of order d (d = 1..GBS_MAX_ORDER; 0 for orders above kmax).
   Events are created on first use; timing state is process-wide and not meant
   for concurrent calls from several host threads. Returns GBS_OK or GBS_ERR_CUDA. */
int gbs_timing(int on);
int gbs_timing_read(float *ms_out);

/* The same for gbs_cumulants_backward: while timing is enabled, its phases are
   bracketed by events, and this waits for those of the most recent backward call
   and writes ms_out[0] = recomputation of the P0 table (forward kernels),
   ms_out[1] = the inverse-moment table h, ms_out[2] = the dL/dP0 gather,
   ms_out[3] = the dL/dV scatter (block inverses, per-prefix accumulation,
   mirroring). Returns GBS_OK, GBS_ERR_INVALID_ARG (no timed backward call) or
   GBS_ERR_CUDA. */
int gbs_timing_read_backward(float *ms_out);

/* Bytes of device scratch gbs_pipe_peaks needs. */
#define GBS_PIPE_PEAKS_SCRATCH 65536

/* Sustained multiply-add throughput of the current GPU's FP64 and FP32 pipes,
   the peaks against which the kernels' arithmetic rooflines are reported (not
   part of the paper's method). Runs two probe kernels of about 40 ms each on
   cuda_stream -- every thread keeps 8 independent FMA chains busy, 32 warps per
   multiprocessor -- and synchronises it. scratch: device memory of at least
   GBS_PIPE_PEAKS_SCRATCH bytes (overwritten). out (host, 6 doubles): FP64
   FLOP/s, FP32 FLOP/s (an FMA counts 2), FP64 and FP32 FMAs per clock per
   multiprocessor, and the median SM clock in MHz seen by the FP64 and the FP32
   probe (from each block's cycle counter against the global nanosecond timer).
   Returns GBS_OK, GBS_ERR_INVALID_ARG or GBS_ERR_CUDA. */
int gbs_pipe_peaks(double *out, void *scratch, void *cuda_stream);

/* ---------------------------------------------------------------- forward tables */

/* P0 table: p0_out[gbs_table_size(M,kmax)] <- P0(S) for every 1 <= |S| <= kmax
   (Eq. vacuum_gaussian_prob, hbar = 2, zero mean). V: 2M x 2M row-major FP64,
   symmetric, xxpp. */
int gbs_vacuum_probs(const double *V, int M, int kmax, double *p0_out, int precision,
                     void *workspace, size_t ws_bytes, void *cuda_stream);

/* Click-moment table: mu_out[...] <- mu(S) (Eq. joint_moments_def with the
   threshold-detector moments of Eq. joint_moments_threshold). */
int gbs_click_moments(const double *V, int M, int kmax, double *mu_out, int precision,
                      void *workspace, size_t ws_bytes, void *cuda_stream);

/* Click-cumulant table: kappa_out[...] <- kt(S) (Eq. joint_cumulants_def). */
int gbs_cumulants(const double *V, int M, int kmax, double *kappa_out, int precision,
                  void *workspace, size_t ws_bytes, void *cuda_stream);

/* ---------------------------------------------------------------- displaced states */

/* Tables gbs_displaced_tables can fill. */
typedef enum {
    GBS_TABLE_P0 = 0,              /* P0(S), Eq. vacuum_gaussian_prob */
    GBS_TABLE_CLICK_MOMENT = 1,    /* mu(S), Eq. joint_moments_def */
    GBS_TABLE_CLICK_CUMULANT = 2,  /* kt(S), Eq. joint_cumulants_def */
    GBS_TABLE_SPIN_CORRELATOR = 3, /* c(S) = E[prod_{k in S} (-1)^{x_k}] */
    GBS_TABLE_SPIN_CUMULANT = 4    /* kappa(S), Eq. cumulant_corr_main */
} gbs_table;

/* One table of a DISPLACED Gaussian state: first moments mean[2M] (device, FP64,
   xxpp: mean[k] = <x_k>, mean[k+M] = <p_k>, hbar = 2) and covariance V as for
   the other entry points. The vacuum probabilities carry the exponential factor
   of Eq. vacuum_gaussian_prob,
     P0(S) = exp(-1/2 mean_S^T (V_S + I)^{-1} mean_S) / sqrt(det((V_S + I)/2)),
   and the other tables follow from P0 exactly as in the zero-mean case (the
   inclusion-exclusion and partition sums do not depend on the mean). With
   mean = 0 the tables equal those of the zero-mean entry points at GBS_FP64.
   Computed in FP64 (workspace: gbs_workspace_bytes(M, kmax, GBS_FP64)).
   table: a gbs_table value. mean must be non-NULL. Errors as elsewhere. */
int gbs_displaced_tables(const double *V, const double *mean, int M, int kmax, int table, double *out,
                         void *workspace, size_t ws_bytes, void *cuda_stream);

/* ---------------------------------------------------------------- sharded tables (rank ranges) */

/* Tables too large for one GPU (e.g. M = 1024, kmax = 4: 4.5e10 entries, 360 GB
   in FP64; the paper's scaling toward thousands of modes, Sec. "Cost estimation
   and scaling", and the 1152-mode state of Sec. "High-brightness results for
   Jiuzhang 3.0") are filled in slices of their top order. The order-kmax subsets
   whose largest mode c_kmax lies in [c_lo, c_hi) have the contiguous colex ranks
   [C(c_lo, kmax), C(c_hi, kmax)), so a slice is one contiguous block of the
   order-kmax group; slices over consecutive ranges, concatenated, are that group.

   gbs_table_range fills out[0 .. gbs_range_entries(M, kmax, c_lo, c_hi)) with the
   entries of `table` (a gbs_table value: P0, click moment, click cumulant, spin
   correlator, spin cumulant) for those subsets: out[r - C(c_lo, kmax)] is the
   entry of colex rank r. The lower orders, which the recursions read, are
   computed in full inside the workspace (gbs_range_workspace_bytes; it holds
   them besides what gbs_workspace_bytes covers) and not returned: take them
   from any whole-table call with kmax - 1. The values equal those of the
   whole-table call bit for bit. Requires 0 <= c_lo <= c_hi <= M; other errors as
   for the whole-table calls. */
size_t gbs_range_workspace_bytes(int M, int kmax, int precision);
uint64_t gbs_range_entries(int M, int kmax, int c_lo, int c_hi);
int gbs_table_range(const double *V, int M, int kmax, int table, int c_lo, int c_hi, double *out, int precision,
                    void *workspace, size_t ws_bytes, void *cuda_stream);

/* Cost-balanced split of the top elements into n_parts ranges: bounds_out[0] = 0,
   bounds_out[n_parts] = M, and part i = [bounds_out[i], bounds_out[i + 1]) holds
   about C(M, kmax) / n_parts entries (each boundary is the smallest c with
   C(c, kmax) >= i C(M, kmax) / n_parts; the entries of the prefix-tree kernels
   cost alike, so equal counts are equal work). Host only. bounds_out: n_parts + 1
   ints. Returns GBS_OK or GBS_ERR_INVALID_ARG (n_parts outside [1, M]). */
int gbs_range_split(int M, int kmax, int n_parts, int *bounds_out);

/* ---------------------------------------------------------------- stage 2: sampler */

/* Arithmetic of the sampler's tables and sums. */
typedef enum {
    GBS_SAMPLE_FP64 = 0,
    GBS_SAMPLE_FP32 = 1  /* cumulants converted to FP32 in the workspace, as the paper stores them */
} gbs_sample_precision;

/* Largest batch (samples per chunk) gbs_sample accepts. */
#define GBS_MAX_SAMPLE_BATCH (1 << 21)

/* Workspace bytes for gbs_sample with this (M, K, batch, precision); 0 if invalid
   (batch must be a multiple of 128 in [128, GBS_MAX_SAMPLE_BATCH]).
   Grows as batch x C(M, 3) entries for K = 4, 5 (the p2 table and, for K = 5,
   the stored products), batch x C(M, 2) for K = 3. */
size_t gbs_sampler_workspace_bytes(int M, int K, int batch, int precision);

/* Chain-rule sampler (Sec. "The sampling algorithm"): draws n_samples threshold-
   detector bitstrings of M bits from the spin-cumulant table kappa (orders 1..K,
   gbs.h layout, as gbs_spin_cumulants writes it), bit n from the bias of
   Eq. delta_bias truncated at order K with approximated marginals:
     K = 3: single elision (Eq. methprob, Eq. b, Eq. a);
     K = 5: double elision (Eq. probade, Eq. probpartialade, Eq. probelidedade,
            Eq. probdoubleelidedade), orders[] = expansion orders of p+, p1, p2
            (host array, NULL = the paper's 3, 3, 2; each 1..3, 1..3, 1..2);
     K = 4: the same without the |R| = 4 term (NULL orders = 2, 2, 1, the
            paper's rule for K = 5 -- one order below the minimum that keeps the
            O(M^K) time -- applied to K = 4).
   Bit n of a sample is 0 when u[s][n] < q0, q0 = max(p0, 0) / (max(p0, 0) +
   max(p1, 0)) with p0, p1 the expansion's values for the two outcomes (1/2 if
   both are <= 0). u: device [n_samples][M] uniforms in [0, 1). force (device,
   may be NULL): [n_samples][M] bits to score instead of drawing; u is then
   ignored. Outputs (device): bits_out [n_samples][M]; logp_out [n_samples]
   (may be NULL) = the natural log of the estimated probability of each
   bitstring (NaN if the estimate is <= 0); q0_out [n_samples][M] (may be
   NULL). Internally every table entry is kept multiplied by prod_v exp(H_v)
   over its variables, H_v the click entropy of mode v, which keeps the values
   of long bitstrings inside the FP32 / FP64 range. Samples run in chunks of batch (a multiple of
   128) sharing one workspace of gbs_sampler_workspace_bytes(M, K, batch,
   precision) bytes. Asynchronous on cuda_stream. */
int gbs_sample(const double *kappa, int M, int K, const int *orders, int n_samples, const double *u,
               const uint8_t *force, uint8_t *bits_out, double *logp_out, double *q0_out, int batch, int precision,
               void *workspace, size_t ws_bytes, void *cuda_stream);

/* ---------------------------------------------------------------- schedule autotuning */

/* Times gbs_cumulants for this (M, kmax, precision) under each candidate
   schedule of the prefix-tree kernels -- items per CTA (1, 2, 4, 8), children
   per shared-memory batch (16, 64), CTA shape (512 threads x 1 per SM, 256 x 2
   per SM when M <= 577; for GBS_FP32_REFINED also 640 x 1, 256 x 3 when
   M <= 577, 768 x 1 with a larger shared-memory batch area, 384 x 2 when
   M <= 961, 256 x 4 when M <= 385, the 256 x 4 and 256 x 3 shapes in
   thread-block clusters whose CTAs share one Schur-complement slot, and 256 x 4
   without slots when M <= 161, forming each Schur-complement block from the
   item's elimination rows where it is used) -- and records
   the fastest in a process-wide table that
   later forward calls of that shape use. If the environment variable
   GBS_AUTOTUNE_CACHE names a file, the table is read from it on first use and
   rewritten after tuning (JSON). Arguments as for gbs_cumulants; kappa_out is
   overwritten with the table. Synchronises cuda_stream (not capturable).
   best_ms_out (host pointer, may be NULL) receives the best time in ms. The
   schedule never changes the arithmetic: tuned and default calls return
   identical tables. */
int gbs_autotune(const double *V, int M, int kmax, double *kappa_out, int precision, void *workspace,
                 size_t ws_bytes, void *cuda_stream, float *best_ms_out);

/* Schedule the forward calls of (M, kmax, precision) run on the current device:
   the one gbs_autotune recorded (or read from GBS_AUTOTUNE_CACHE), else the
   default. schedule_out[3] (host) = {CTA shape (0: 512 threads x 1 per SM,
   1: 256 x 2, refined only 2: 640 x 1, 3: 256 x 3, 4: 768 x 1, 5: 384 x 2,
   6: 256 x 4, 7 and 8: 6 and 3 in thread-block clusters, 9: 6 without
   Schur-complement slots), items per CTA slot, children per shared-memory
   batch}, after the fallback to 512 x 1 for a shape that does not admit M.
   Host only; allocates nothing. Returns GBS_OK, GBS_ERR_INVALID_ARG (bad
   shape or precision, NULL schedule_out) or GBS_ERR_CUDA (no device). */
int gbs_schedule(int M, int kmax, int precision, int *schedule_out);

/* ---------------------------------------------------------------- ragged batches */

/* One instance of a batch: its covariance V (2M x 2M, device) and the output
   kappa_out (gbs_table_size(M, kmax) FP64 entries, device; outputs of different
   instances must not overlap). */
typedef struct {
    const double *V;
    double *kappa_out;
    int M;
    int kmax;
} gbs_instance;

/* Workspace bytes for a batch described by the HOST array inst[0..n). */
size_t gbs_batched_workspace_bytes(const gbs_instance *inst, int n, int precision);

/* Writes the batch plan into the workspace: instance order (largest M first),
   per-instance packing buffers and lower-order P0 tables, per-phase work prefix
   sums, and the prefix-tree item tables, for one schedule of the batched kernel
   (CTA shape, items per CTA, children per shared-memory batch). The schedule is
   the one gbs_batched_autotune recorded for a batch with the same multiset of
   (M, kmax) on this device (also read from GBS_AUTOTUNE_CACHE), else a default
   (256 threads x 3 CTAs per SM for GBS_FP32_REFINED and 256 x 2 for GBS_FP64
   when every M <= 577; 512 x 1 otherwise). inst is a HOST array; the pointers
   in it are device pointers that must stay valid while the plan is used. Copies
   the plan with a host-to-device copy and synchronises cuda_stream: call it
   outside any stream capture. Returns GBS_OK, GBS_ERR_INVALID_ARG,
   GBS_ERR_WORKSPACE or GBS_ERR_CUDA. */
int gbs_batched_plan(const gbs_instance *inst, int n, int precision, void *workspace, size_t ws_bytes,
                     void *cuda_stream);

/* Click-cumulant tables of every instance of the planned batch in ONE persistent
   cooperative kernel launch (phases: packing, orders 1-3, order 4, order 5,
   separated by grid-wide barriers; prefix-tree items of all instances share one
   queue per order). Reads V from the device pointers recorded by the plan, so it
   may be captured in a CUDA graph and replayed after V changes in place.
   precision must equal the plan's, and the workspace must hold a plan written by
   gbs_batched_plan or gbs_batched_autotune in this process (GBS_ERR_INVALID_ARG
   otherwise). Asynchronous; device errors go to the status word
   (gbs_stream_status). The grid-wide barriers are those of a cooperative launch,
   whose CTAs are all resident; they carry no time limit. */
int gbs_cumulants_batched(int precision, void *workspace, void *cuda_stream);

/* Batch autotuner (the schedule search of gbs_autotune, for a ragged batch):
   times gbs_cumulants_batched on this batch under candidate schedules -- every
   CTA shape allowed for the precision and the largest M (512 x 1, 256 x 2 when
   M <= 577; refined also 640 x 1, 256 x 3 when M <= 577, 768 x 1, 384 x 2
   when M <= 961, and 256 x 4 when M <= 385) at the default
   grain and batch size, then items per CTA slot (1, 2, 4, 8) x children per
   batch (16, 64) for the fastest shape -- records the fastest for this batch
   shape (multiset of (M, kmax), device, precision; persisted like gbs_autotune's
   table) and leaves its plan in the workspace, ready for gbs_cumulants_batched.
   Arguments as for gbs_batched_plan; the outputs are overwritten with the tables.
   Synchronises cuda_stream (not capturable). best_ms_out (host, may be NULL)
   receives the best time in ms. Schedules never change the arithmetic. */
int gbs_batched_autotune(const gbs_instance *inst, int n, int precision, void *workspace, size_t ws_bytes,
                         void *cuda_stream, float *best_ms_out);

/* Schedule of the batch plan in this workspace (written by gbs_batched_plan or
   gbs_batched_autotune in this process): schedule_out[5] (host) = {CTA shape
   (0: 512 threads x 1 per SM, 1: 256 x 2, 2: 640 x 1, 3: 256 x 3), threads per
   CTA, CTAs in the launch, items per CTA slot, children per shared-memory
   batch}, shape 4 being 768 threads x 1, 5 384 x 2 and 6 256 x 4. Returns GBS_OK or
   GBS_ERR_INVALID_ARG
   (no plan). */
int gbs_batched_schedule(const void *workspace, int *schedule_out);

/* ---------------------------------------------------------------- gradients */

/* Workspace bytes for gbs_cumulants_backward (includes the P0, inverse-moment and
   P0-gradient tables, 3 x 8 B x gbs_table_size, plus the forward workspace);
   0 if the arguments are invalid. The adjoint takes M <= GBS_MAX_MODES. */
size_t gbs_backward_workspace_bytes(int M, int kmax);

/* Adjoint of gbs_cumulants. grad_kappa[gbs_table_size(M,kmax)] = dL/dkt(S)
   in table layout; grad_V (2M x 2M, row-major, overwritten) receives the
   symmetric gradient G, dL = sum_ab G[a][b] dV[a][b] for symmetric dV.
   Chain (derived from Eq. joint_cumulants_def and Eq. vacuum_gaussian_prob):
   kt(S) = (-1)^{|S|} ky(S) with ky the cumulant of the no-click indicators,
   whose moments are P0; d ky(S)/d P0(B) = h(S - B) with h the coefficients of
   1/F(u), F(u) = sum_B P0(B) u^B; dP0(T)/dV_T = -1/2 P0(T) (V_T + I)^{-1}.
   Precision: P0 is recomputed by the refined FP32 path (relative error about
   1e-13), the sums over subsets run in FP64, and the per-subset inverses of the
   orders >= 4 in double-float (FP32 pairs, about 2^-44 relative per operation);
   against the FP64 oracle the largest error, relative to the largest entry, was
   1.9e-12 at M = 30, kmax = 5 and 5.3e-14 on an M = 100, kmax = 4 fitting
   gradient.
   Device errors (non-positive-definite blocks) go to the workspace status word. */
int gbs_cumulants_backward(const double *V, int M, int kmax, const double *grad_kappa, double *grad_V,
                           void *workspace, size_t ws_bytes, void *cuda_stream);

/* Covariance of M single-mode squeezed inputs after an interferometer U and
   per-mode transmissions eta (Eq. ground_truth_cov with hbar = 2 and the lossy
   transmission matrix diag(sqrt(eta)) U):
     V = D S Q S^T D + I - D^2,  S = [[Re U, -Im U], [Im U, Re U]],
     Q = diag(e^{-2 r_1}, .., e^{-2 r_M}, e^{2 r_1}, .., e^{2 r_M}),  D = diag(sqrt(eta), sqrt(eta)).
   U_re, U_im: M x M row-major; r, eta: length M (eta in (0, 1]); V_out: 2M x 2M.
   All device pointers. Returns GBS_OK, GBS_ERR_INVALID_ARG or GBS_ERR_CUDA. */
int gbs_covariance(const double *U_re, const double *U_im, const double *r, const double *eta, int M,
                   double *V_out, void *cuda_stream);

/* Adjoint of gbs_covariance: given V (its output) and G = dL/dV (2M x 2M),
   writes grad_r[M] = dL/dr and grad_eta[M] = dL/deta. Device pointers. */
int gbs_covariance_backward(const double *U_re, const double *U_im, const double *r, const double *eta, int M,
                            const double *V, const double *grad_V, double *grad_r, double *grad_eta,
                            void *cuda_stream);

/* ---------------------------------------------------------------- allocation-free variant */

/* Size of the fixed scratch array behind gbs_cumulants_noalloc, in MiB. */
#define GBS_NOALLOC_SCRATCH_MB 64

/* gbs_cumulants for callers that cannot allocate device memory. (The paper has
   no counterpart; this is a deployment convenience of this library.)

   Who needs it: code that cannot call cudaMalloc where it needs the table --
   inside an allocator or memory-pool callback, in a plugin whose host
   application owns every device allocation, or in a runtime that forbids
   allocation after start-up. Such a caller passes only V (2M x 2M FP64, device)
   and kappa_out (gbs_table_size(M, kmax) FP64 entries, device); the result
   equals gbs_cumulants(..., GBS_FP64, ...).

   Scratch: every buffer gbs_cumulants keeps in its workspace lives instead in
   one file-scope device array of GBS_NOALLOC_SCRATCH_MB MiB, reserved on each
   GPU that loads the library and held until the process exits. Calls whose
   workspace (gbs_workspace_bytes) exceeds it are rejected with
   GBS_ERR_WORKSPACE and a message; on a 152-SM GB300, M = 100 fits with
   kmax = 5 and M = 144 with kmax <= 4, while M = 144 with kmax = 5 does not.
   Nothing here calls cudaMalloc, cudaFree or any allocating routine.

   Set-up: the first call on each device looks up the array's device address
   (cudaGetSymbolAddress) with that device current; make that first call before
   any stream capture.

   Sharing: all calls in the process share the one array, which keeps the last
   call's contents (the status word and work counters are cleared at the start
   of every call). Calls whose work may overlap on the GPU -- on different
   streams, or from different host threads -- race on the array; serialise
   them (one stream). Device-side errors leave NaN in the affected entries and
   set the status word that gbs_noalloc_status reads.
   Returns GBS_OK, GBS_ERR_INVALID_ARG, GBS_ERR_WORKSPACE or GBS_ERR_CUDA. */
int gbs_cumulants_noalloc(const double *V, int M, int kmax, double *kappa_out, void *cuda_stream);

/* Device status of the allocation-free calls on the current device, the
   counterpart of gbs_stream_status for gbs_cumulants_noalloc, whose caller holds
   no workspace to pass: synchronises cuda_stream, then reads the status word kept
   in the library's fixed scratch array (allocating nothing) and returns GBS_OK,
   GBS_ERR_NOT_POSDEF or another device status, as gbs_stream_status does. The
   word is cleared by the next gbs_cumulants_noalloc call on that device. */
int gbs_noalloc_status(void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GBS_H */
