/*
 * mp.h -- C ABI of the GB300 matrix-profile library (libmp.so).
 *
 * The library computes the matrix profile P and its index I of a time series
 * (Akbarinia & Cloez, arXiv:1901.05708):
 *
 *   Def. 2.2  subsequence T_{i,m} = <t_i .. t_{i+m-1}>, 0 <= i < N = n-m+1
 *   Def. 2.4  P[i] = min_j d(i, j),  I[i] = argmin_j d(i, j)
 *
 * over all j with |i - j| > excl (the exclusion zone; excl = 0 is the
 * paper's rule, which only drops the self-match), for three distances:
 *
 *   mp_aamp   pure Euclidean  (Sec. 2, Eq. def-euclidean-distance; Algorithm 1)
 *   mp_pnorm  p-norm          (Sec. 3.4, Eq. PNormDist1;         Algorithm 3)
 *   mp_acamp  z-normalised    (Sec. 2, Eq. def-z-normalized;     Algorithm 2)
 *
 * The work is the diagonal sweep of Algorithms 1-3: for each diagonal
 * k = j - i the distance is carried from (i-1, j-1) to (i, j) in O(1)
 * (Lemmas 1-3) and offered to both P[i] and P[j].
 *
 * Conventions shared by every entry point
 *  - Indices are 0-based.  T holds n samples; P and I hold N = n - m + 1.
 *  - T, P, I and the workspace are DEVICE pointers owned by the caller.  The
 *    library never allocates during a call and never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Every call only enqueues work and returns; results are ready
 *    when the stream reaches that point.
 *  - Arguments are validated before anything is enqueued.  On any error the
 *    call returns a non-zero status, enqueues nothing and leaves P and I
 *    untouched; mp_last_error() gives a thread-local message.
 *  - Ties: among equal distances the smallest |i - j| wins, then the left
 *    neighbour (what the strict '<' of Algorithms 1-3 produces with k and i
 *    ascending).  With FP32 sweeps, candidates closer than the stated error
 *    may be ordered either way.
 *  - Rows with no candidate (N - 1 <= excl) get P = +inf, I = -1.  For the
 *    z-normalised distance a flat window (centred sum of squares at most
 *    2^-40 times its raw sum of squares) gets P = +inf, I = -1 and is never a
 *    neighbour (Sec. 1: its z-normalised distance is undefined).
 */
#ifndef MP_H
#define MP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MP_OK = 0,
    MP_ERR_INVALID_ARG = 1,  /* bad size, pointer, alignment or option     */
    MP_ERR_UNSUPPORTED = 2,  /* valid but outside this build's limits      */
    MP_ERR_WORKSPACE = 3,    /* ws NULL or ws_bytes < mp_workspace_size()  */
    MP_ERR_CUDA = 4,         /* a CUDA call failed (launch, copy, graph)   */
    MP_ERR_INTERNAL = 5      /* a device-side check failed                 */
} mp_status;

typedef enum { MP_F32 = 0, MP_F64 = 1 } mp_dtype;

typedef enum {
    /* FP32 recurrence re-anchored from exact block sums every `reanchor`
     * rows; FP64 window statistics; FP64 polish of P at I. */
    MP_PREC_FP32 = 0,
    /* FP64 recurrence (slow on this GPU: FP64 runs at 1/64 of FP32). */
    MP_PREC_FP64 = 1
} mp_precision;

typedef enum { MP_DIST_EUCLID = 0, MP_DIST_PNORM = 1, MP_DIST_ZNORM = 2 } mp_dist;

/* Kernel of the FP32 sweep.  Euclidean / p-norm, AUTO: for p = 3 with float32
 * input, the tall-tile kernel, whose p = 3 window sums are error-free (each
 * is the float-float sum of its FP32 terms |x - y|^3: the re-anchored FP32
 * kernels keep, until their next anchor, an error of the size of the largest
 * term met, which on series whose terms span many orders of magnitude puts
 * small distances far outside the FP32 tolerance; MP_VARIANT_FAST still runs
 * the two-stream kernel for p = 3, faster, with that caveat).  Otherwise the
 * two-stream kernel where it applies (FP32 input, m a multiple of 32 up to 416,
 * p in {1, 2, 3}, default re-anchor interval), with the block filter for p = 2 and
 * N >= 200,000, in tiles of 16,384 rows (each stream walks 8,192 rows in
 * staged sub-tiles of 768 and pays the O(m) anchor once) where that leaves at
 * least 16,384 tiles and p != 3, else of 2,048 rows (mp_options.tile_rows
 * overrides; the results differ only by FP32 rounding); else,
 * for m >= 512 and p in {1, 2, 3} with float32 input (or where the generic
 * kernel's shared memory does not fit m), the tall-tile kernel; else the
 * generic kernel.  (For p = 1 and 2 the tall kernel does not re-anchor within
 * a tile, so for short windows its FP32 rounding can grow past the tolerance
 * on near ties.)
 * The z-normalised distance has one FP32 kernel: AUTO takes its block filter
 * for N >= 200,000, FAST_FILTER / FAST force it on / off, GENERIC and TALL do
 * not apply.  The filter only skips candidates that cannot pass, so with or
 * without it the results are the same bit for bit.
 * The others force a choice (MP_ERR_UNSUPPORTED where it does not apply);
 * mp_autotune times them (not MP_VARIANT_ZRAW or MP_VARIANT_ZF).
 * MP_VARIANT_ZRAW runs Algorithm 2 as printed (Lemma 3): the dot product
 * C = sum t_{i+l} t_{j+l} carried along each diagonal and
 * rho = (C - A_i A_j / m) / sqrt(S_i S_j) with the window sums A, in the
 * precision of mp_options.precision, re-anchored like the other plain sweeps
 * (every `reanchor` rows, default 512 in FP32, 256 in FP64).  The numerator
 * cancels when a window's mean is large against its spread, which the
 * centred covariance of the other kernels avoids: it exists to measure that
 * loss and the speed of the paper's form, not for use.
 * MP_VARIANT_ZF is Sec. 4.3's comparison on the same raw sums: candidates are
 * ordered by F = (A_i A_j - m C) |A_i A_j - m C| / (S_i S_j) (= -m^2 rho |rho|,
 * increasing with DZ; no square root per cell) and the winner's value is
 * DZ^2 = 2m + 2 sign(F) sqrt(|F|); FP32 or FP64 sweep, re-anchored like
 * MP_VARIANT_ZRAW; also an ablation. */
typedef enum {
    MP_VARIANT_AUTO = 0,
    MP_VARIANT_FAST_FILTER = 1,  /* two-stream kernel with the block filter (p = 2); */
                                 /* z-normalised kernel with its block filter        */
    MP_VARIANT_FAST = 2,         /* two-stream kernel; z-normalised kernel, no filter */
    MP_VARIANT_GENERIC = 3,      /* generic kernel (any p, input type; reanchor;     */
                                 /* shared memory limits m to about 12,000)          */
    MP_VARIANT_TALL = 4,         /* tall-tile kernel: float-float sums, tiles of      */
                                 /* max(8192, 8m) rows (p in {1, 2, 3}; long windows) */
    MP_VARIANT_ZRAW = 5,         /* ablation, z-normalised only, FP32 or FP64 sweep:  */
                                 /* Algorithm 2's raw sums (see below)               */
    MP_VARIANT_ZF = 6,           /* ablation, z-normalised only, FP32 or FP64 sweep:  */
                                 /* raw sums compared through F (Sec. 4.3)           */
    MP_VARIANT_CACHED = 7,       /* the autotuner's cached choice for this problem    */
                                 /* class (kernel, reanchor, tile_rows) if present,  */
                                 /* else AUTO; in a batch plan, each z-normalised    */
                                 /* series' cached tile_rows                         */
    MP_VARIANT_FAST_FILTER_BOUND = 8 /* z-normalised kernel, block filter on a looser */
                                 /* bound (the block's largest 1/sqrt(S)): one packed */
                                 /* operation per cell pair instead of two; faster   */
                                 /* for i.i.d.-like data, slower on random walks;    */
                                 /* same results bit for bit                         */
} mp_variant;

typedef struct mp_options {
    uint32_t struct_size; /* = sizeof(mp_options); set by mp_options_default      */
    int32_t precision;    /* mp_precision (default MP_PREC_FP32)                  */
    int32_t reanchor;     /* rows between exact re-anchors; 0 = chosen from m     */
    int32_t polish;       /* 1 (default): P[i] recomputed in FP64 as d(i, I[i])   */
                          /* 0: P is the sweep's own (FP32 or FP64) value          */
    int32_t variant;      /* FP32 sweep kernel, mp_variant (default MP_VARIANT_AUTO) */
    int32_t tile_rows;    /* rows per tile of the two-stream kernel and of the     */
                          /* tall-tile kernels (the FP32 z-normalised kernel and   */
                          /* MP_VARIANT_TALL).  0 (default): for the two-stream   */
                          /* kernel the tallest of 16384, 8192 and 4096 rows that */
                          /* leaves at least 4096 tiles, else 2048; for the z-    */
                          /* normalised kernel max(65536, 8m); for the tall kernel */
                          /* max(8192, 8m).  Else a multiple of 2048 (two-stream) */
                          /* or of 1024 (tall-tile kernels).  Taller tiles pay the */
                          /* O(m) anchor less often; shorter ones give short      */
                          /* series more tiles.  The two-stream kernel re-anchors */
                          /* every m/Q rows whatever the tile height.  Must be 0  */
                          /* for the generic kernel (MP_ERR_UNSUPPORTED).          */
    int64_t k_begin;      /* sweep only diagonals k >= k_begin (default 0)        */
    int64_t k_end;        /* ... and k < k_end (<= 0 means no upper bound).       */
                          /* Disjoint ranges computed separately and merged with  */
                          /* the tie rule above give the full profile.            */
} mp_options;

/* Fill *opt with the defaults.  Passing opt = NULL to any call means the
 * same thing. */
void mp_options_default(mp_options *opt);

/* Bytes of device workspace that mp_aamp / mp_pnorm / mp_acamp need for this
 * problem (dist is an mp_dist, dtype an mp_dtype).  0 on invalid input.
 * The workspace must be 256-byte aligned. */
size_t mp_workspace_size(int dist, int dtype, int64_t n, int32_t m, const mp_options *opt);

/* Matrix profile with the pure Euclidean distance (AAMP, Algorithm 1).
 *   T      device, n samples of type dtype (4- or 8-byte aligned)
 *   n, m   1 <= m <= n, N = n - m + 1 < 2^31
 *   excl   >= 0; pairs with |i - j| <= excl are not considered
 *   P      device, N doubles: the distance to the nearest neighbour
 *   I      device, N int64: the nearest neighbour's index, or -1
 *   ws     device workspace of ws_bytes >= mp_workspace_size(MP_DIST_EUCLID, ...)
 * Errors: MP_ERR_INVALID_ARG (sizes, NULL or misaligned pointers, options),
 *         MP_ERR_UNSUPPORTED (N >= 2^31), MP_ERR_WORKSPACE, MP_ERR_CUDA. */
mp_status mp_aamp(const void *T, int dtype, int64_t n, int32_t m, int64_t excl,
                  double *P, int64_t *I, void *ws, size_t ws_bytes,
                  const mp_options *opt, void *stream);

/* Matrix profile with the p-norm distance (AAMP for p-norm, Algorithm 3,
 * Lemma 2), P[i] = (sum_l |t_{i+l} - t_{j+l}|^p)^(1/p).  p >= 1 (real);
 * p = 1, 2, 3 have specialised kernels, other p use powf.  Other arguments
 * and errors as mp_aamp. */
mp_status mp_pnorm(const void *T, int dtype, int64_t n, int32_t m, int64_t excl, double p,
                   double *P, int64_t *I, void *ws, size_t ws_bytes,
                   const mp_options *opt, void *stream);

/* Matrix profile with the z-normalised Euclidean distance (ACAMP,
 * Algorithm 2, Lemma 3).  Window means and centred sums of squares are
 * computed in FP64; the sweep carries the centred covariance.  m >= 2.
 * Other arguments and errors as mp_aamp. */
mp_status mp_acamp(const void *T, int dtype, int64_t n, int32_t m, int64_t excl,
                   double *P, int64_t *I, void *ws, size_t ws_bytes,
                   const mp_options *opt, void *stream);

/* Synchronise `stream` and report a sticky CUDA error or a device-side check
 * failure from earlier calls (MP_ERR_CUDA / MP_ERR_INTERNAL), else MP_OK. */
mp_status mp_sync_status(void *stream);

/* Thread-local text of the last error (empty string if none). */
const char *mp_last_error(void);

/* Static name of a status code. */
const char *mp_status_string(mp_status s);

/* Library version, as "major.minor.patch". */
const char *mp_version(void);

/* Number of kernels this library has launched in this process so far
 * (all threads, all devices).  For benchmarks: the difference across a
 * timed region is the number of the library's kernel launches in it. */
uint64_t mp_launch_count(void);

/* Profiling hook for the calling host thread.  When both are non-NULL,
 * every later mp_aamp / mp_pnorm / mp_acamp call on this thread records
 * `ev_start` (a cudaEvent_t passed as void*) on its stream right before the
 * diagonal-sweep kernel and `ev_end` right after it, so that the caller can
 * time the sweep alone with cudaEventElapsedTime.  NULL, NULL turns it off.
 * The events are owned by the caller.  Always returns MP_OK. */
mp_status mp_set_sweep_events(void *ev_start, void *ev_end);

/* Size of the library-owned device scratch used by mp_aamp_noalloc. */
#define MP_NOALLOC_SCRATCH_BYTES (32u << 20)

/* mp_aamp for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this is a deployment variant.  Some callers
 * cannot call cudaMalloc or obtain a workspace at all -- a host framework
 * that owns every device allocation and only hands out input and output
 * buffers (plugins), or a service that forbids allocation after start-up to
 * keep its memory budget fixed.  This entry point takes the same arguments
 * as mp_aamp minus the workspace and instead uses a scratch array of
 * MP_NOALLOC_SCRATCH_BYTES (32 MiB) that the library declares as static
 * device memory: every GPU that loads the library holds it until the process
 * exits.  It calls no cudaMalloc, cudaFree or other allocating routine.
 *
 *  - Problems whose workspace (mp_workspace_size(MP_DIST_EUCLID, ...)) is
 *    larger than the scratch are rejected with MP_ERR_UNSUPPORTED; with
 *    float32 input that is n up to about 1.6 million samples.
 *  - Every call looks up the scratch address on the current device (a
 *    host-side query, after the argument checks); the first lookup on a
 *    device may load the library's device code there, so make the first
 *    call on each device before any CUDA stream capture.
 *  - All calls on a device share the one scratch array, which keeps the
 *    contents of the last call (every call initialises what it reads).
 *    Calls that overlap on the GPU -- on different streams, or from
 *    different host threads without ordering -- race on it and give wrong
 *    results: serialise them.
 * Results, argument checks and errors are those of mp_aamp. */
mp_status mp_aamp_noalloc(const void *T, int dtype, int64_t n, int32_t m, int64_t excl,
                          double *P, int64_t *I, const mp_options *opt, void *stream);

/* ---- Batches: many independent profiles in one graph launch ---------------
 *
 * The paper treats one series at a time (Algorithms 1-3); a batch runs the
 * same computation for S independent series, each with its own m, exclusion
 * zone and distance, as one CUDA graph: FP64 window statistics for the
 * z-normalised series, then persistent sweep kernels that take the tiles of
 * every series from one queue per kernel (longest tiles first, one atomic
 * ticket per tile), then the finalize/polish of every window.
 *
 * Layout.  T is the S series concatenated (FP32): series s is
 * T[t_offsets[s] .. t_offsets[s+1]).  P and I are the S profiles
 * concatenated: series s has N_s = n_s - m_s + 1 entries starting at
 * w_s = N_0 + ... + N_{s-1}, and I holds indices within the series (or -1).
 * mp_batch_windows() gives the total length sum_s N_s.
 */
typedef struct mp_batch_desc {
    uint32_t struct_size;      /* = sizeof(mp_batch_desc)                              */
    int32_t num_series;        /* S >= 1                                               */
    const int64_t *t_offsets;  /* host, S + 1 non-decreasing sample offsets, n_s >= 1  */
    const int32_t *m;          /* host, S window lengths, 1 <= m_s <= n_s              */
    const uint8_t *dist;       /* host, S mp_dist values                               */
    const int64_t *excl;       /* host, S exclusion zones >= 0                         */
    double p;                  /* exponent of every MP_DIST_PNORM series (>= 1)        */
    int32_t dtype;             /* MP_F32 (the only batch input type)                   */
    int32_t reserved0;
} mp_batch_desc;

typedef struct mp_batch_plan mp_batch_plan;

/* Validate desc, split every series into sweep tiles, sort the tile queues
 * and upload them (with the per-series table) to device memory that the plan
 * owns; *ws_bytes receives the workspace size mp_batch_run needs.  The plan
 * belongs to the current device.  opt may be NULL; the batch runs the FP32
 * sweep with the default re-anchor interval and whole diagonal ranges, so
 * opt->precision must be MP_PREC_FP32, reanchor 0, k_begin = k_end = 0 (else
 * MP_ERR_UNSUPPORTED); opt->polish is honoured; opt->variant may be AUTO or
 * FAST (no block filter) or FAST_FILTER (the filter on the Euclidean
 * two-stream queue).  The tile queues take the series in turn (first tiles of
 * all series, then second tiles, ...), longest tiles first within a turn.
 * Each series' profile equals its single call (mp_aamp / mp_pnorm / mp_acamp
 * with the same options) bit for bit, except for p = 3: the batch runs p = 3
 * series on the re-anchored two-stream or generic kernel (as mp_pnorm with
 * MP_VARIANT_FAST, or MP_VARIANT_GENERIC where the two-stream kernel does not
 * apply), not on the error-free tall-tile kernel that mp_pnorm takes by
 * default, so the caveat of mp_variant on p = 3 applies.
 * desc is not kept.
 * Errors: MP_ERR_INVALID_ARG (desc, sizes, dist, p), MP_ERR_UNSUPPORTED
 * (dtype, options, N_s >= 2^31, more than 2^32 - 1 tiles in a queue, m_s too
 * large for shared memory), MP_ERR_CUDA (allocation or copy failed; nothing
 * is leaked).  Validation happens before any CUDA call. */
mp_status mp_batch_plan_create(const mp_batch_desc *desc, const mp_options *opt,
                               mp_batch_plan **plan, size_t *ws_bytes);

/* Enqueue the whole batch on `stream` as one graph launch.
 *   T   device, t_offsets[S] floats (4-byte aligned)
 *   P   device, mp_batch_windows(plan) doubles;  I  device, as many int64
 *   ws  device workspace, 256-byte aligned, ws_bytes >= the plan's size
 * The graph is built on the first run and rebuilt whenever T, P, I or ws
 * differ from the previous run's.  A plan is not thread-safe.  The queue
 * tickets live in ws, so two runs in flight at the same time (on different
 * streams) need different workspaces. */
mp_status mp_batch_run(mp_batch_plan *plan, const void *T, double *P, int64_t *I,
                       void *ws, size_t ws_bytes, void *stream);

/* sum_s N_s (the length of P and I), or -1 for a NULL plan. */
int64_t mp_batch_windows(const mp_batch_plan *plan);

/* Tiles in the plan's queues (all kernels), or -1 for a NULL plan. */
int64_t mp_batch_tiles(const mp_batch_plan *plan);

/* Free the plan's device memory and graph.  NULL is a no-op.  Call it after
 * the plan's last run has completed. */
mp_status mp_batch_plan_destroy(mp_batch_plan *plan);

/* ---- Streaming append: keep a profile current as samples arrive ----------
 *
 * Sec. 1 of the paper notes that the incremental formulation also serves to
 * maintain the profile of a growing series, without spelling out the method.
 * Here it is the diagonal recurrence (Lemma 1 / 2 / 3) run on the new last
 * row: appending one sample creates window j = N; each diagonal k = j - i
 * moves from its last cell (i - 1, j - 1) to (i, j) in O(1) (the new diagonal
 * k = j from the definition) and the cell is offered to rows i and j, so an
 * append costs O(N) and leaves P and I equal to the profile of the longer
 * series (the same distances, exclusion zone and tie rule as mp_aamp).
 * The per-diagonal state is FP64 and is recomputed from the definitions every
 * opt->reanchor appends (0: every 256); a row's new best is rescored from
 * the definition, so P carries no drift.  The object owns its device memory
 * (sized for n_max samples); appends are asynchronous on `stream`.
 */
typedef struct mp_stream mp_stream;

/* Profile of T (device, n samples of dtype) with distance `dist` (p for
 * MP_DIST_PNORM), room for n_max samples in all.  The initial profile runs the
 * one-shot path with opt (precision; polish is forced on) on a workspace
 * allocated and freed on `stream` for this call.  Errors: as mp_aamp, plus
 * MP_ERR_INVALID_ARG for n_max < n or a bad dist, MP_ERR_UNSUPPORTED for
 * opt->k_begin / k_end != 0 or n_max - m + 1 >= 2^31, MP_ERR_CUDA when the
 * device memory cannot be allocated (nothing is leaked). */
mp_status mp_stream_create(int dist, const void *T, int dtype, int64_t n, int64_t n_max,
                           int32_t m, int64_t excl, double p, const mp_options *opt,
                           mp_stream **out, void *stream);

/* Append `count` samples (device pointer x of dtype).  Fails with
 * MP_ERR_UNSUPPORTED, appending nothing, if the capacity would be exceeded. */
mp_status mp_stream_append(mp_stream *s, const void *x, int dtype, int64_t count, void *stream);

/* Copy the current profile (mp_stream_windows(s) entries) into device P, I. */
mp_status mp_stream_read(const mp_stream *s, double *P, int64_t *I, void *stream);

/* Current number of windows N = n - m + 1, or -1 for a NULL stream. */
int64_t mp_stream_windows(const mp_stream *s);

/* Free the stream's device memory (after its last append has completed). */
mp_status mp_stream_destroy(mp_stream *s);

/* ---- Anytime runs: a profile that improves tile by tile ---------------------
 *
 * The paper's algorithms can be stopped early (Sec. 1 mentions the anytime
 * use of the incremental formulation): every cell already evaluated is exact,
 * so the profile of any subset of diagonals is an upper bound that tightens
 * towards the final one.  An anytime run takes one float32 series, splits it
 * into the batch path's tiles, orders them by a seeded random permutation and
 * evaluates the next tiles of that order on each mp_anytime_run call; between
 * calls mp_anytime_read gives the profile of the cells done so far (rows
 * without a candidate yet: P = +inf, I = -1), and the keys with the queue
 * cursor can be saved to and restored from host memory.  When every tile has
 * run, P and I equal the batch path's result for the series exactly.
 */
typedef struct mp_anytime mp_anytime;

/* T: device, n float32 samples (copied; T may be freed after the call).
 * seed != 0 fixes the tile order (0 selects a built-in seed).  opt as for a
 * batch (FP32 sweep, polish honoured).  Errors: as mp_batch_plan_create. */
mp_status mp_anytime_create(int dist, const void *T, int64_t n, int32_t m, int64_t excl, double p,
                            uint64_t seed, const mp_options *opt, mp_anytime **out, void *stream);

/* Evaluate the next min(max_tiles, remaining) tiles (asynchronous). */
mp_status mp_anytime_run(mp_anytime *a, int64_t max_tiles, void *stream);

/* P, I (device, N entries) of every cell evaluated so far. */
mp_status mp_anytime_read(const mp_anytime *a, double *P, int64_t *I, void *stream);

/* Tiles evaluated so far / in all, or -1 for NULL. */
int64_t mp_anytime_tiles_done(const mp_anytime *a);
int64_t mp_anytime_tiles_total(const mp_anytime *a);

/* Checkpoint: a header (magic, seed, N, cursor) and the N profile keys, in
 * host memory of mp_anytime_checkpoint_size() bytes; the key copy is
 * asynchronous on `stream`.  mp_anytime_restore loads one into an anytime run
 * of the same series, seed and size (else MP_ERR_INVALID_ARG). */
size_t mp_anytime_checkpoint_size(const mp_anytime *a);
mp_status mp_anytime_checkpoint(const mp_anytime *a, void *host, size_t bytes, void *stream);
mp_status mp_anytime_restore(mp_anytime *a, const void *host, size_t bytes, void *stream);

/* Free the run (after its last call has completed). */
mp_status mp_anytime_destroy(mp_anytime *a);

/* ---- Autotuning -------------------------------------------------------------
 *
 * mp_autotune times the kernel variants that apply to a problem (the
 * two-stream kernel with and without the filter, and, with the filter for
 * p = 2 or without it for p = 1, at the tile height its default does not
 * take: 2,048 rows where the default is tall, 16,384 where the default is
 * 2,048 and the tall tiles still number at least 1,216; the generic kernel at its
 * default re-anchor interval and at intervals of 16, 32 and 64 rows that
 * divide m into at most 8 blocks, each distinct interval once; the tall-tile
 * kernel for m >= 512; for p = 3 with float32 input only the tall-tile
 * kernel, whose sums hold the FP32 tolerance (nothing to time: it is returned
 * as the choice); for the z-normalised distance its kernel with and
 * without the filter, each at the default tile height and at 16,384 and 4,096
 * rows per tile where those are shorter than the default and than N, and with
 * the looser filter bound at the default tile height)
 * on the caller's series, each candidate once to warm up and once timed (the
 * sweep kernel alone, CUDA events on `stream`; the call synchronises it).
 * slice_cells = 0 times the whole sweep; slice_cells > 0 only the first
 * diagonals, about that many cells (faster, but thresholds stay as loose as at
 * the start of a sweep, which understates the block filter).
 * *best receives the fastest options (opt's other fields kept); times_ms, if
 * not NULL, the times of the candidates in the order listed above (up to
 * max_times entries, -1 for one that does not apply), and *n_times their
 * number.  Results are cached in memory per (device name, dist, dtype, m,
 * log2 N, p); a cached problem returns at once without timing (*n_times = 0)
 * unless `force`.  MP_VARIANT_CACHED in later calls (and batch plans) applies
 * a cached entry.  P and I (N entries, device) are scratch for the timed runs;
 * their content afterwards is unspecified.  Arguments and errors as mp_aamp /
 * mp_pnorm / mp_acamp (ws sized by mp_workspace_size for opt). */
mp_status mp_autotune(int dist, const void *T, int dtype, int64_t n, int32_t m, int64_t excl, double p,
                      double *P, int64_t *I, void *ws, size_t ws_bytes, const mp_options *opt,
                      int64_t slice_cells, int force, mp_options *best, double *times_ms,
                      int32_t max_times, int32_t *n_times, void *stream);

/* Save / load the autotuning cache as text, one entry per line.  Loading
 * merges into the cache (entries of other devices are kept).  Errors:
 * MP_ERR_INVALID_ARG (NULL path, unreadable or malformed file). */
mp_status mp_autotune_cache_save(const char *path);
mp_status mp_autotune_cache_load(const char *path);

/* Entries in the cache. */
int64_t mp_autotune_cache_size(void);

#ifdef __cplusplus
}
#endif

#endif /* MP_H */
