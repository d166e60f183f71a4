/*
 * dfd.h -- C ABI of the GB300 discrete Frechet distance library (libdfd.so).
 *
 * The discrete Frechet distance (DFD) of two polygonal curves p (n points)
 * and q (m points) in R^dim is the value M_{n,m} of the recurrence of Eq. 1
 * of "Walking Your Frog Fast in 4 LoC" (Sec. 3):
 *     M_ij = max( min(M_{i-1,j}, M_{i-1,j-1}, M_{i,j-1}), d_ij ),
 * with d_ij = || p_i - q_j ||_2 and the first row / column taken as running
 * maxima (Alg. 1, Alg. 3).  The library carries SQUARED distances d_ij^2
 * through the recurrence and takes one square root at the end; because the
 * recurrence only selects among its inputs (min and max), this returns
 * exactly the square of the distance computed on d_ij (Sec. 3, Theorem 1
 * holds for any nondecreasing ground measure).
 *
 * Conventions shared by every entry point:
 *   - Curves are row-major arrays of n x dim coordinates (point i at
 *     p + i*dim), either float32 (DFD_F32) or int32 (DFD_I32).
 *   - Unless an entry point says otherwise, every pointer is a DEVICE
 *     pointer on the context's device, the work is enqueued on `stream`
 *     (a cudaStream_t passed as void*, NULL = the legacy default stream),
 *     and the call returns without waiting.  The caller owns every buffer
 *     and must keep it alive until the stream has passed the work.
 *   - Outputs: out_dist receives the distance delta (float for DFD_F32,
 *     double for DFD_I32); out_dist2 receives delta^2 as the recurrence
 *     computed it (float for DFD_F32, int64_t for DFD_I32, exact).  Either
 *     may be NULL, not both.
 *   - float32 results: delta^2 is one of the float32 squared distances
 *     d_ij^2 = fma-chain(t_k = p_k - q_k) (t_0*t_0 first, then
 *     fma(t_k, t_k, acc) for k = 1..dim-1, round-to-nearest), so it is within
 *     dim+1 float32 roundings of the exact value; delta = sqrtf(delta^2),
 *     correctly rounded.  int32 results: delta^2 is exact; delta is the
 *     correctly rounded double square root of (double)delta^2.
 *   - int32 precondition: every |coordinate| <= 2^30 - 1 and
 *     dim * (2 * max|coordinate|)^2 <= 2^63 - 1; otherwise DFD_ERR_RANGE
 *     (checked on the device when the context's check_inputs option is on).
 *   - float32 precondition: finite coordinates; otherwise DFD_ERR_NONFINITE
 *     (checked on the device when check_inputs is on).
 *   - Functions never abort the process.  Invalid host arguments return an
 *     error status immediately and enqueue nothing.  Errors found on the
 *     device (input checks, a bounded wait that ran out) are recorded in the
 *     context's sticky device error word, reported by dfd_get_error().
 *   - No CPU fallback exists: without a usable CUDA device every call that
 *     computes returns DFD_ERR_CUDA.
 */
#ifndef DFD_H_
#define DFD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dfd_status {
  DFD_OK = 0,
  DFD_ERR_INVALID_ARG = 1, /* bad pointer, size, dtype or dim */
  DFD_ERR_RANGE = 2,       /* int32 coordinates outside the exact range */
  DFD_ERR_NONFINITE = 3,   /* float32 coordinate is NaN or infinite */
  DFD_ERR_OOM = 4,         /* device or pinned host allocation failed */
  DFD_ERR_CUDA = 5,        /* a CUDA runtime call failed / no device */
  DFD_ERR_TIMEOUT = 6,     /* a bounded device wait ran out (no hang, no trap) */
  DFD_ERR_BUSY = 7,        /* resource limit reached, retry later */
  DFD_ERR_CANCELLED = 8,   /* work was cancelled before it finished */
  DFD_ERR_NOT_READY = 9,   /* result not available yet */
  DFD_ERR_UNSUPPORTED = 10, /* configuration the library does not support */
  DFD_ERR_CAPACITY = 11     /* input needs more than a fixed-size buffer holds */
} dfd_status;

typedef enum dfd_dtype { DFD_F32 = 0, DFD_I32 = 1 } dfd_dtype;

typedef struct dfd_context dfd_context;

typedef struct dfd_options {
  size_t struct_size;       /* sizeof(dfd_options), for forward compatibility */
  size_t mem_budget_bytes;  /* device scratch budget; 0 = no limit */
  int max_slots;            /* serving: concurrent requests admitted (0 = default) */
  double wait_timeout_ms;   /* limit of every device-side spin wait (default 2000) */
  int check_inputs;         /* 1 = validate coordinates on the device (default) */
} dfd_options;

/* Fill *opt with the defaults.  Returns DFD_ERR_INVALID_ARG for NULL. */
dfd_status dfd_options_default(dfd_options* opt);

/* Human-readable name of a status code (static string, never NULL). */
const char* dfd_status_string(dfd_status s);

/*
 * Create a context on CUDA device `device` (opt NULL = defaults).  The
 * context owns a grow-only device scratch area, a pinned host staging area
 * and the device error word; it is not thread-safe (use one per host thread
 * or serialise calls).  *out is set only on DFD_OK.
 */
dfd_status dfd_context_create(dfd_context** out, int device, const dfd_options* opt);

/* Synchronise the device, free everything the context owns.  NULL is OK. */
dfd_status dfd_context_destroy(dfd_context* ctx);

/*
 * Synchronise the device and return the sticky device error word
 * (DFD_OK if no device-side error happened), then clear it.
 */
dfd_status dfd_get_error(dfd_context* ctx);

/*
 * Discrete Frechet distance of one pair of curves (Eq. 1, Alg. 5 semantics)
 * on the whole GPU: a band wavefront over the (n x m) recurrence (rows of p
 * in bands across CTAs, warps inside a band as a systolic pipeline over the
 * columns), with O(n + m) device scratch owned by the context.  A pair of two
 * bands or more runs as two fronts in one launch -- forward over the first
 * half of the bands and backward over the rest (both curves reversed) --
 * whose last rows a final pass combines (min over the crossing steps of the
 * max of both sides): the same value, bit for bit.
 * int32 pairs whose bounding box (over p and q) keeps every squared distance
 * below 0x7F800000 (each coordinate's range at most 46,340, the squared
 * ranges summing to at most 0x7F7FFFFF) carry their exact squared distances
 * as uint32 bits in float registers (float min / max order them as
 * integers); the others carry exact int64 values.  The choice is made on the
 * device (the call launches a kernel for each class; the one that does not
 * apply returns at once), so the call stays asynchronous; both give the
 * exact int64 result.
 *   p: n x dim, q: m x dim (device, dtype), n >= 1, m >= 1, 1 <= dim <= 16.
 *   out_dist / out_dist2: device pointers to one element each (see top).
 */
dfd_status dfd_pair(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q,
                    int64_t m, void* out_dist, void* out_dist2, void* stream);

/*
 * The same distance by the plain per-pair reference form: one CTA computes
 * the recurrence row by row (Alg. 2 / Alg. 5 order); within each row the
 * dependence on the left neighbour is resolved by a block-wide scan of the
 * clamp functions x -> max(d_j, min(a_j, x)) (the paper's maxmin step,
 * Sec. 3, made associative by composing clamps).  Same arguments and
 * results as dfd_pair; bit-identical to it.  Scratch: O(m).
 */
dfd_status dfd_pair_reference(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n,
                              const void* q, int64_t m, void* out_dist, void* out_dist2, void* stream);

/*
 * dfd_pair with HOST buffers: copies p and q to the device (directly when
 * they are page-locked, e.g. from cudaHostAlloc or a pinned tensor; else
 * through the context's pinned staging area), runs dfd_pair on the
 * context's internal stream, copies the result back and waits for it.  p, q, out_dist and
 * out_dist2 are host pointers (outputs may be NULL, not both).  Device
 * errors are returned directly.
 */
dfd_status dfd_pair_host(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q,
                         int64_t m, void* out_dist, void* out_dist2);

/*
 * Distances of many independent pairs of curves in one persistent launch
 * (the batch evaluation of Sec. 4, without padding: pairs of any lengths).
 *   points:  all curves' coordinates, CSR packed (curve c is rows
 *            offsets[c] .. offsets[c+1]-1 of a [total, dim] array), device.
 *   offsets: int64[n_curves + 1], device, non-decreasing, offsets[0] = 0.
 *   pairs:   int32[2 * n_pairs] curve ids (a, b), device.
 *   out_dist / out_dist2: n_pairs elements each (types as for dfd_pair).
 * A pair's rows are the curve that needs fewer systolic steps (usually the
 * shorter; delta is symmetric), cut into stripes of 32*R rows (R <= Rmax =
 * 8 for dim <= 4, else 4), each a systolic array over the columns; of the
 * two orientations the one whose columns fit one warp's row buffer is taken
 * when only one does.  Pairs are sorted by cost on the device (a counting sort, no host
 * synchronisation) and taken by persistent CTAs and warps from atomic
 * counters, in two size classes (dfd_batch_set_team): pairs of several
 * stripes that are too wide for one warp's row buffer (4096 columns unless
 * dfd_batch_set_row_buffer widened it) -- and those for which a team is
 * expected to finish sooner, as when a launch has fewer long pairs than the
 * GPU has warps -- run first, each on the 8 warps of one CTA as a pipeline
 * of stripes; the others run one warp per pair, costliest first.  A team pair with more than 8 stripes keeps a
 * row of its longer curve in the CTA's eight warp buffers; one wider still
 * runs after all others, in the last CTA, with every warp buffer of the
 * launch as its row (2432 x the per-warp width on 152 SMs); a pair wider
 * than that gets NaN (float, double) / -1 (int64) outputs and
 * DFD_ERR_UNSUPPORTED in the error word.  Invalid curve ids or empty curves
 * put DFD_ERR_INVALID_ARG in the error word and leave that pair's outputs
 * unwritten.
 */
dfd_status dfd_batch(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                     int64_t n_curves, const int32_t* pairs, int64_t n_pairs, void* out_dist, void* out_dist2,
                     void* stream);

/*
 * Threshold decision for many pairs (the decision form of the problem,
 * Sec. 2: is delta(p, q) <= eps?) with early abandon.  M never decreases
 * along a monotone path's prefix bottleneck, so delta^2 >= min of M over any
 * set of cells every path must enter; once such a set of the running
 * recurrence exceeds eps^2 the pair is abandoned (the heuristics that avoid
 * full computations, Sec. 5).  Same inputs and engine as dfd_batch, one
 * warp per pair (no CTA teams): a pair of several stripes whose longer curve
 * is wider than 4096 points gets within = 0, out_dist2 NaN (float) / -1
 * (int64) and DFD_ERR_UNSUPPORTED in the error word.  Plus:
 *   eps2:       per-pair squared thresholds, device (float for DFD_F32,
 *               int64 for DFD_I32), or NULL to use eps2_all for every pair
 *               (compared as: float32 delta^2 <= the largest float <=
 *               eps2_all; int32 delta^2 <= floor(eps2_all)).
 *   out_dist2:  n_pairs, the exact delta^2 of pairs computed to the end,
 *               +inf (float) / INT64_MAX (int64) for abandoned ones; may be
 *               NULL if out_within is given.
 *   out_within: int32[n_pairs], 1 if delta^2 <= eps^2 else 0; may be NULL.
 *   abandoned:  device uint64 counter incremented per abandoned pair; may
 *               be NULL.
 * Ties (delta^2 == eps^2) are never abandoned.
 */
dfd_status dfd_batch_decide(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                            int64_t n_curves, const int32_t* pairs, int64_t n_pairs, const void* eps2,
                            double eps2_all, void* out_dist2, int32_t* out_within, unsigned long long* abandoned,
                            void* stream);

/*
 * Exact k nearest neighbours of one query curve among candidate curves
 * (float32), by discrete Frechet distance, with early abandon: candidates
 * are searched in ascending order of the endpoint bound max(d(p_1,q_1),
 * d(p_n,q_m))^2 <= delta^2 (every coupling contains both end pairs), skipped
 * when that bound exceeds the current k-th best, and otherwise stopped as
 * soon as a cut of the running recurrence exceeds it (see
 * dfd_batch_decide), so only the survivors are computed to the end.
 *   query:     n x dim float32, device.
 *   points / offsets / n_curves: candidate curves, CSR as for dfd_batch.
 *   cand:      int32[n_cand] candidate curve ids, device, or NULL to use
 *              curves 0 .. n_cand-1.
 *   k:         1 .. 1024.
 *   out_ids:   int32[k] candidate curve ids, ascending by (delta^2, position
 *              in cand), -1 past n_cand; out_dist2 / out_dist: float[k]
 *              delta^2 / delta (+inf past n_cand).  Any may be NULL, not all.
 *   abandoned: device uint64, set to the number of candidates abandoned
 *              or skipped by their endpoint bound (may be NULL).
 *   evaluated: device uint64, set to the number of recurrence cells
 *              actually evaluated (may be NULL).
 * The results equal the k smallest of the exact float32 delta^2 of every
 * candidate, ties broken by position.  Invalid ids / empty candidates set
 * DFD_ERR_INVALID_ARG in the error word and are skipped.
 */
dfd_status dfd_knn(dfd_context* ctx, int dim, const float* query, int64_t n, const float* points,
                   const int64_t* offsets, int64_t n_curves, const int32_t* cand, int64_t n_cand, int k,
                   int32_t* out_ids, float* out_dist2, float* out_dist, unsigned long long* abandoned,
                   unsigned long long* evaluated, void* stream);

/*
 * The appendix variants of the recurrence (DTW and the Levenshtein
 * distance), many pairs per launch on the batch engine (same inputs and
 * order as dfd_batch, one warp per pair: a pair of several stripes whose
 * longer curve is wider than 4096 points gets NaN / -1 and
 * DFD_ERR_UNSUPPORTED in the error word):
 *   DFD_VARIANT_DTW: dtype DFD_F32, 1 <= dim <= 16; out = float[n_pairs],
 *     D_{n,m} of D_ij = fl(min(D_{i-1,j}, D_{i-1,j-1}, D_{i,j-1}) + c_ij)
 *     with c_ij the float32 squared distance of dfd_pair and the first row /
 *     column as running sums; one rounding per cell, so the value is fixed
 *     (within (n+m+dim+2) * 2^-24 relative of the exact sum).
 *   DFD_VARIANT_LEVENSHTEIN: dtype DFD_I32, dim = 1 (one int32 symbol per
 *     position); out = int64[n_pairs], the unit-cost edit distance (the
 *     textbook table, E_{i,0} = i, E_{0,j} = j).
 * Other dtype / dim combinations return DFD_ERR_INVALID_ARG.
 */
typedef enum dfd_variant { DFD_VARIANT_DTW = 1, DFD_VARIANT_LEVENSHTEIN = 2 } dfd_variant;

dfd_status dfd_batch_variant(dfd_context* ctx, dfd_variant variant, dfd_dtype dtype, int dim, const void* points,
                             const int64_t* offsets, int64_t n_curves, const int32_t* pairs, int64_t n_pairs,
                             void* out, void* stream);

/*
 * Monte Carlo distance samples of two uncertain float32 curves (the
 * application to uncertain curves named in Sec. 5).  Sample s uses
 *   p_s[i][k] = fl(p[i][k] + sigma_p * noise_p[s][i][k]),
 *   q_s[j][k] = fl(q[j][k] + sigma_q * noise_q[s][j][k])   (one rounding, fmaf),
 * and out_dist2[s] / out_dist[s] receive delta_s^2 / delta_s exactly as
 * dfd_batch computes them (any of the two may be NULL, not both).
 *   p: n x dim, q: m x dim, noise_p: n_samples x n x dim, noise_q:
 *   n_samples x m x dim, all device float32; the noise is the caller's (a
 *   sample is reproducible bit for bit).
 * The samples are built in stream-ordered device memory (cudaMallocAsync,
 * freed in order after the launch) and computed in one batch launch.
 */
dfd_status dfd_mc_pair(dfd_context* ctx, int dim, const float* p, int64_t n, const float* q, int64_t m,
                       const float* noise_p, const float* noise_q, float sigma_p, float sigma_q, int64_t n_samples,
                       float* out_dist2, float* out_dist, void* stream);

/*
 * All-pairs distance matrix of n_curves curves (the paper's motivating use:
 * clustering and distance matrices of trajectories, Sec. 2), condensed upper
 * triangle: entry k = i*(2N - i - 1)/2 + (j - i - 1) for i < j (N =
 * n_curves), N*(N-1)/2 elements in out_condensed (distances) and/or
 * out_dist2.  Pairs are decoded from k on the device; the batch engine, one
 * warp per pair, tile shape per dfd_matrix_set_shape.  A pair of several
 * stripes whose longer curve is wider than 4096 points gets NaN (float,
 * double) / -1 (int64) and DFD_ERR_UNSUPPORTED in the error word.
 */
dfd_status dfd_matrix(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                      int64_t n_curves, void* out_condensed, void* out_dist2, void* stream);

/*
 * Packing autotuner of the ragged batch (the "sophisticated scheduling" the
 * paper leaves open, Sec. 4): which pair each warp takes next.  Order 0
 * (default) hands out pairs grouped by code variant (rows per lane, stripes)
 * and, inside a variant, by columns, largest first; order 1 hands them out by
 * estimated cost alone (stripes x rows per lane x (columns + 31)), largest
 * first.  Both compute every pair identically; only the timing differs.
 * dfd_batch_autotune runs dfd_batch on the arguments with each order x
 * team mode (1, 2) x tile shape (rows per lane cap Rmax or Rmax / 2, CTAs
 * per SM all or 1; see dfd_batch_set_shape) (one untimed and three timed
 * runs each, CUDA events on `stream`, synchronous), records the fastest
 * combination for (dtype, dim class) in the context -- later
 * dfd_batch, dfd_batch_capture, dfd_batch_host and dfd_batch_decide calls
 * of that class use it -- and writes it to *best_order (may be NULL).  The
 * outputs hold the batch's results afterwards.  dfd_batch_set_order sets
 * the order directly (0 or 1).
 */
dfd_status dfd_batch_autotune(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                              int64_t n_curves, const int32_t* pairs, int64_t n_pairs, void* out_dist,
                              void* out_dist2, int* best_order, void* stream);
dfd_status dfd_batch_set_order(dfd_context* ctx, dfd_dtype dtype, int dim, int order);

/*
 * Which pairs of a ragged batch run as CTA teams (no counterpart in the
 * paper, whose batches pad every curve to one length and give each lane one
 * curve, Sec. 4).  A team is the 8 warps of one CTA on one pair of several
 * stripes (more rows than one warp holds): warp w runs
 * stripes w, w + 8, ... as a pipeline over the columns, handing each
 * stripe's bottom row to the next through shared memory (and, from the last
 * warp back to the first, through the CTA's eight warp row buffers, 8 x the
 * per-warp width).  mode 1: only pairs too wide for one warp's row buffer;
 * mode 2: every pair of several stripes; mode 0 (default): the wide pairs,
 * and each pair of several stripes for which a latency model of the two
 * schedules (the launch's pairs in rounds of resident warps or of CTAs,
 * steps x cycles per step) expects the team to finish sooner -- on a few
 * hundred long pairs, teams; on thousands of pairs that already fill every
 * warp, one warp each.  Team pairs go first (costliest first), then the
 * one-warp pairs.  Every mode computes
 * every pair's value bit for bit as the others.  dfd_batch_autotune tunes
 * the mode with the packing order and the tile shape (below);
 * dfd_batch_tuned reads them back (NULL outputs are skipped; 0 = default).
 * DFD_ERR_INVALID_ARG for a mode outside 0..2.
 */
dfd_status dfd_batch_set_team(dfd_context* ctx, dfd_dtype dtype, int dim, int mode);
dfd_status dfd_batch_tuned(dfd_context* ctx, dfd_dtype dtype, int dim, int* order, int* team, int* rows_per_lane,
                           int* ctas_per_sm);

/*
 * Tile shape of the ragged batch's one-warp pairs and of the all-pairs
 * matrix (no counterpart in the paper), per (dtype, dim class):
 * rows_per_lane caps the rows a lane holds (1..8; the stripes of a pair
 * are at most 32 x this tall; 0 = the largest, 8 for dim <= 4, 4 above): a
 * lane's rows form one dependent chain per step, so fewer rows shorten the
 * step and more rows amortise its fixed instructions.  ctas_per_sm (1 or 2;
 * 0 = every resident CTA) sets the persistent grid.  Every shape computes
 * the same bits; pairs the cap would leave wider than the row buffer run
 * with the largest cap (matrix) or as CTA teams (batch), so the shape never
 * changes which pairs run.  dfd_batch_autotune and dfd_matrix_autotune time
 * the shapes on the caller's data and keep the fastest.
 */
dfd_status dfd_batch_set_shape(dfd_context* ctx, dfd_dtype dtype, int dim, int rows_per_lane, int ctas_per_sm);
dfd_status dfd_matrix_set_shape(dfd_context* ctx, dfd_dtype dtype, int dim, int rows_per_lane, int ctas_per_sm);
dfd_status dfd_matrix_tuned(dfd_context* ctx, dfd_dtype dtype, int dim, int* rows_per_lane, int* ctas_per_sm);
/* Times dfd_matrix on the arguments with rows per lane cap {Rmax, Rmax/2,
   Rmax/4} x CTAs per SM {all, 1} (one untimed and two timed runs each, CUDA
   events on `stream`, synchronous), records the fastest for (dtype, dim
   class) and writes it out (pointers may be NULL).  The outputs hold the
   matrix afterwards. */
dfd_status dfd_matrix_autotune(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                               int64_t n_curves, void* out_condensed, void* out_dist2, int* best_rows_per_lane,
                               int* best_ctas_per_sm, void* stream);

/*
 * Row buffer width (columns per warp) of the ragged batch on this context:
 * pairs that run several stripes may have up to `cols` points in their
 * longer curve.  cols in [4096, 2^28], rounded up to a multiple of 32,
 * else DFD_ERR_INVALID_ARG; the default is 4096.  The batch's scratch holds
 * one buffer per resident warp (2432 on 152 SMs): cols * 4 bytes each for
 * float32, cols * 8 for int32.  Applies to later dfd_batch and
 * dfd_batch_capture calls; dfd_batch_host widens its buffers by itself to
 * the widest pair it is given.  The decider, matrix, k-NN and variant
 * kernels keep 4096.
 */
dfd_status dfd_batch_set_row_buffer(dfd_context* ctx, int cols);

/*
 * dfd_batch with HOST buffers (points, offsets, pairs and the outputs are
 * host pointers; outputs may be NULL, not both): synchronous.  The points
 * are copied to the device in up to 8 slices of curves (about 64 MiB each)
 * on a copy stream, directly when they are page-locked and through the
 * context's pinned staging area otherwise (the offsets and pairs first,
 * as given); one launch per slice takes, from the whole pair list, the
 * pairs whose later curve lies in that slice (a filter in its device-side
 * plan) as soon as the slice has landed, so the copies overlap the
 * computation and results land at the pairs' own indices (launches
 * alternate between two internal streams, so one launch's start overlaps
 * the end of the one before).  The device staging holds the points, the results and two batch
 * scratch areas (grow-only, freed at destroy), whose row buffers are as wide
 * as the widest multi-stripe pair given (at least the context's width), so
 * any pair lengths run.  Results are bit-identical
 * to dfd_batch on the same data.  Offsets must be nondecreasing (checked on
 * the host: DFD_ERR_INVALID_ARG) and every id in [0, n_curves)
 * (DFD_ERR_INVALID_ARG: checked on the host when some curve is longer than
 * the context's row buffers, else by the last launch's device-side plan,
 * the other pairs' outputs then being written); the device-side checks are
 * dfd_batch's, returned directly.  Uses the context's
 * internal streams and staging: one host-buffer call per context at a time.
 */
dfd_status dfd_batch_host(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                          int64_t n_curves, const int32_t* pairs, int64_t n_pairs, void* out_dist, void* out_dist2);

/*
 * CUDA-graph capture of one dfd_batch / dfd_matrix call (input checks, plan
 * and the persistent launch) for repeated launches with the same pointers:
 * update the buffers' contents, not the graph.  The call runs once
 * normally (results written, device synchronised), then is captured with a
 * private scratch area owned by the graph.  dfd_graph_launch enqueues it on
 * `stream`; the graph must be destroyed before its context.
 */
typedef struct dfd_graph dfd_graph;
dfd_status dfd_batch_capture(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                             int64_t n_curves, const int32_t* pairs, int64_t n_pairs, void* out_dist, void* out_dist2,
                             dfd_graph** out);
dfd_status dfd_matrix_capture(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                              int64_t n_curves, void* out_condensed, void* out_dist2, dfd_graph** out);
dfd_status dfd_graph_launch(dfd_graph* graph, void* stream);
dfd_status dfd_graph_destroy(dfd_graph* graph);

/*
 * Serving: query-vs-candidates searches (Sec. 4's batch of curves against
 * one reference curve, as a request stream) with continuous batching.
 *
 * Candidate curves (float32) are uploaded once and stay resident on the
 * device.  dfd_server_submit (any host thread, non-blocking) queues a
 * request: one query curve and k candidate ids; the k distances are written
 * to host_out[0..k) before dfd_server_wait returns DFD_OK.  A scheduler
 * thread admits requests in arrival order while fewer than max_slots are
 * running and the device arena (mem_budget_bytes) holds their query and
 * candidate ids (O(n + k)); it runs ticks -- one persistent launch per point
 * dimension over pairs from every admitted request, oldest request first,
 * costliest pairs first inside a launch, up to tick_cells cells.  Pairs that
 * finish within a tick are expanded from per-request ranges on the device;
 * a pair with more than stripes_per_tick row stripes (or a multi-stripe pair
 * wider than 4096 points) advances at most stripes_per_tick stripes per
 * tick, its O(m) bottom row kept in the arena between ticks (the prefix
 * property of Sec. 3).  Requests that arrive while others run join the next
 * tick; two ticks are in flight.  Each distance is bit-identical to
 * dfd_pair's for the same two curves, whatever else is in the tick.
 * Ownership: submit copies the query and ids; host_out must stay valid
 * until wait returns OK or CANCELLED.  A ticket is released by the wait that
 * returns its final status.  Destroy the server before its context.
 * Limits: at most INT32_MAX candidates per dimension; a request whose query
 * and ids exceed 32 MiB of staging returns DFD_ERR_CAPACITY from submit.
 */
typedef struct dfd_server dfd_server;
typedef struct dfd_server_options {
  size_t struct_size;        /* sizeof(dfd_server_options) */
  size_t mem_budget_bytes;   /* device arena for queries, candidate ids and row states (default 1 GiB) */
  int max_slots;             /* requests running at once (default 256) */
  double tick_cells;         /* cells per tick (default 4e9) */
  int stripes_per_tick;      /* row stripes a long pair advances per tick (default 8) */
} dfd_server_options;
typedef struct dfd_serving_stats {
  uint64_t completed, cancelled, ticks;
  double cells;              /* cells of completed requests */
  double p50_ms, p99_ms, mean_ms;   /* latency: completion - arrival */
  double gpu_busy_ms;        /* device time of all ticks */
  double gcups_busy;         /* cells / gpu_busy_ms */
  double gcups_wall;         /* cells / (last completion - first arrival) */
  size_t arena_used_bytes;
} dfd_serving_stats;

dfd_status dfd_server_options_default(dfd_server_options* opt);
dfd_status dfd_server_create(dfd_context* ctx, const dfd_server_options* opt, dfd_server** out);
dfd_status dfd_server_destroy(dfd_server* server);
/* Append n_curves candidates of dimension dim (host CSR arrays, offsets[0] = 0);
   *first_id receives the id of the first one (ids are per dimension). */
dfd_status dfd_server_add_candidates(dfd_server* server, int dim, const float* host_points,
                                     const int64_t* host_offsets, int64_t n_curves, int64_t* first_id);
/* arrival_s: the request's arrival time on the dfd_server_now clock (latency is
   measured from it; < 0 = now). */
dfd_status dfd_server_submit(dfd_server* server, int dim, const float* host_query, int64_t n,
                             const int64_t* cand_ids, int64_t k, float* host_out, double arrival_s, uint64_t* ticket);
/* DFD_OK / DFD_ERR_CANCELLED (final), DFD_ERR_NOT_READY on timeout (timeout_ms < 0: no limit). */
dfd_status dfd_server_wait(dfd_server* server, uint64_t ticket, double timeout_ms);
dfd_status dfd_server_cancel(dfd_server* server, uint64_t ticket);
dfd_status dfd_server_stats(dfd_server* server, dfd_serving_stats* out);
dfd_status dfd_server_stats_reset(dfd_server* server);
/* Per-request record of each request completed since the last stats reset
   (at most 2^22), in completion order, times on the dfd_server_now clock:
   where a request's latency went -- waiting to be submitted (submit_s -
   arrival_s), queued for admission (admit_s - submit_s), for its first tick
   (launch_s - admit_s), and on the GPU (done_s - launch_s).  Copies up to
   cap records to out; *n receives the number recorded. */
typedef struct dfd_request_record {
  uint64_t ticket;
  double arrival_s, submit_s, admit_s, launch_s, done_s;
  double cells;
  int n, k, dim, pad;
  double locked_s;           /* submission took the server's lock */
} dfd_request_record;
dfd_status dfd_server_request_log(dfd_server* server, dfd_request_record* out, int64_t cap, int64_t* n);
/* Per-tick record of each tick retired since the last stats reset (at most
   2^20): when the scheduler began building it and returned from launching it,
   when it was retired, its device time (first to last event of the tick),
   its cells, long-pair items, short-pair slices, results and newly admitted
   requests; of the host time before the launch, the admission and tick
   building shares, and the slowest single CUDA call of the launch (which:
   1 event record, 2 stream wait, 3 query / id upload, 4 descriptor copy,
   5 counter reset, 6 kernel launch, 7 stream join, 8 result copy, 9 final
   event).  Copies up to cap records to out; *n receives the number. */
typedef struct dfd_tick_record {
  double build_s, launched_s, retired_s, gpu_ms, cells;
  int n_items, n_slices, n_outs, n_admitted;
  double admit_ms, build_ms, slow_call_ms;
  int slow_call, pad;
  double sync_s, synced_s, locked_s;   /* scheduler: began waiting for the tick, saw it done, retook the lock */
} dfd_tick_record;
dfd_status dfd_server_tick_log(dfd_server* server, dfd_tick_record* out, int64_t cap, int64_t* n);
/* The server's clock in seconds (monotonic). */
double dfd_server_now(dfd_server* server);

/*
 * Explicit launch shape for the band wavefront of dfd_pair (for tuning and
 * measurement).  rows_per_lane in {2, 4, 6, 8}, warps in 1..16 (compute
 * warps per CTA; one more communication warp is added), ctas in 1..#SMs
 * times the CTAs an SM holds (two for points of up to 4 coordinates, else
 * one; 0 = min(#bands, resident CTAs)).  Unsupported shapes return
 * DFD_ERR_UNSUPPORTED.
 */
typedef struct dfd_wave_shape {
  int rows_per_lane;
  int warps;
  int ctas;
} dfd_wave_shape;

dfd_status dfd_pair_shaped(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q,
                           int64_t m, void* out_dist, void* out_dist2, void* stream, const dfd_wave_shape* shape);

/*
 * dfd_pair for callers that cannot allocate device memory.  This entry point
 * has no counterpart in the paper; it exists for library users whose device
 * memory is not theirs to allocate -- a process whose HBM is reserved up
 * front by another allocator (a framework's caching pool, a serving engine
 * under a fixed memory budget) -- and for latency-critical loops where a
 * cudaMalloc / cudaFree, which can synchronise the whole device, is not
 * acceptable.  It needs no context and calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *
 * The band wavefront's scratch (band ticket, progress words, row buffer,
 * packed q) and the device error word live in one fixed array of
 * DFD_NOALLOC_SCRATCH_BYTES in the library's device image, present on
 * every GPU that loads the library until the process exits.  Scratch needed
 * (bytes): 2048 + B + 8*ceil(n / 64) + m * (4 for float32, 8 for int32) +
 * (m + 1024) * Q, where Q = 32 (float32, dim <= 4), 64 (float32, dim 5..8),
 * 128 (float32, dim 9..16), 48 (int32, dim <= 4), 96 (int32, dim 5..8),
 * 192 (int32, dim 9..16: int32 packs q for both of its value classes), and
 * B = 0 (float32) or 16,640 (int32: the bounding-box partials).  This is an
 * upper bound of one front's layout; inputs whose bound exceeds the array
 * return DFD_ERR_CAPACITY before anything is enqueued (e.g. float32 3-D: m
 * up to ~460,000; int32 2-D: m up to ~300,000).
 *
 * Arguments and results as dfd_pair, on CUDA device `device` (made current
 * for the call, then restored).  The input checks always run.  The first
 * call on a device looks up the array's device address (and the device's
 * SM count); make that first call before any stream capture.  Every call
 * clears what must start at zero and overwrites the rest, so the array
 * keeps only the last call's contents: calls whose work overlaps on the
 * GPU (on different streams, or from different threads) share the array
 * and race -- serialise them.  On a device-side error (invalid coordinates,
 * a bounded wait that ran out) the call still returns DFD_OK and the
 * outputs are left as NaN (float, double) / -1 (int64); there is no context
 * to read the error code from, so check the outputs.
 */
#define DFD_NOALLOC_SCRATCH_BYTES (16u << 20)
dfd_status dfd_pair_noalloc(int device, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q,
                            int64_t m, void* out_dist, void* out_dist2, void* stream);

/*
 * Autotuner of the band wavefront (no counterpart in the paper): runs
 * dfd_pair on (p, q) once per candidate launch shape (rows per lane 4, 6,
 * 8 x compute warps 2..10, at most two waves of bands), times each with CUDA
 * events on `stream`, and records the fastest for the size class of
 * (dtype, dim, n, m) in the context; later dfd_pair calls of that class use
 * it.  Synchronous; *best (may be NULL) receives the chosen shape.
 * dfd_autotune_save / _load write / read the context's table as text lines
 * "key rows_per_lane warps ctas".
 */
dfd_status dfd_pair_autotune(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q,
                             int64_t m, void* stream, dfd_wave_shape* best);
dfd_status dfd_autotune_save(dfd_context* ctx, const char* path);
dfd_status dfd_autotune_load(dfd_context* ctx, const char* path);

/* The launch shape dfd_pair would choose for (dtype, dim, n, m). */
dfd_status dfd_pair_plan(dfd_context* ctx, dfd_dtype dtype, int dim, int64_t n, int64_t m, dfd_wave_shape* shape);

/*
 * Measurement hooks (no counterpart in the paper).  With timing enabled the
 * context records a CUDA event pair around the main kernel launch of every
 * computing call, on that call's stream (for the band wavefront of dfd_pair:
 * around its prep kernel and the wavefront kernels, which start early on the
 * prep kernel's tail and would not with an event between them).
 * dfd_timing_last waits for the latest pair and returns its duration in
 * milliseconds (DFD_ERR_NOT_READY if none was recorded since enabling).
 */
dfd_status dfd_timing_enable(dfd_context* ctx, int on);
dfd_status dfd_timing_last(dfd_context* ctx, double* ms);

/*
 * Issue-rate measurement (the ALU roofline of the recurrence; the paper's
 * Sec. 4 "sum of all d_ij" baseline is op 10).  Runs one kernel of many
 * independent instruction chains on every SM and returns the measured
 * throughput in thread-operations per clock per SM (cells per clock per SM
 * for the cell mixes; clocks per dependent operation for the latency ops)
 * and the SM clock it ran at (MHz).  op:
 *   0 fma.f32   1 fma.f32x2   2 min.f32   3 min.f32 (3 inputs)   4 min.s32
 *   5 min.s64   6 mad.wide.s32   7 shfl.sync.up
 *   8 one float32 3-D cell (f32x2 distance + min3 + max)
 *   9 one int32 2-D cell (int64 squares + 3 x 64-bit min/max)
 *  10 one float32 3-D distance, summed instead of Eq. 1
 *  latency (one warp per SM, clocks per dependent op):
 *  11 min.f32   12 min3 -> max (one cell of the recurrence's chain)
 *  13 shfl.sync.up   14 fma.f32x2   15 min.s64 -> max.s64
 *  16 one float32 16-D cell (scalar: 16 sub + 16 mul/fma + min3 + max)
 *  17 one int32 2-D cell carried as uint32 bits (2 sub, mul.lo, mad.lo,
 *     3-input float min + float max), cells / clock / SM
 *  18 one float32 2-D DTW cell (2 sub, mul, fma, 3-input min, add)
 *  19 one Levenshtein cell (compare + select, min, add, add, min, the
 *     column mask's select)
 *  20 one float32 2-D cell (f32x2 distance + min3 + max)
 * Synchronous.  DFD_ERR_INVALID_ARG for an unknown op.
 */
dfd_status dfd_microbench(dfd_context* ctx, int op, double* per_clk_per_sm, double* sm_mhz);

/*
 * Diagnostics for the failure path of the device waits (no counterpart in
 * the paper): one CTA spins on a device flag that nothing ever sets, using
 * the same bounded wait as the wavefront, with a limit of timeout_ms; the
 * call synchronises and returns what the wait recorded -- DFD_ERR_TIMEOUT
 * when the limit works -- and clears the error word.  Nothing hangs or
 * traps; the context stays usable.
 */
dfd_status dfd_debug_bounded_wait(dfd_context* ctx, double timeout_ms);

#ifdef __cplusplus
}
#endif

#endif /* DFD_H_ */
