// batch_launch.cuh -- host launchers of K4 (ragged batch) and K5 (matrix),
// instantiated per (value type, dimension class) in batch_*.cu.
#pragma once
#include <algorithm>
#include <climits>
#include <cmath>
#include <type_traits>
#include "batch_kernel.cuh"
#include "dfd_internal.h"

namespace dfd {

static_assert(batch::BUF_COLS == kDefaultBatchBufCols, "the context's default row buffer is the kernels' fixed one");

// float32 input check over CSR points [begin[0], end[0]) (point indices on
// the device: offsets[first], offsets[n]); int32 batches are checked by the
// bounding-box kernel.
template <class V>
__global__ void check_points_kernel(const typename V::coord* x, const int64_t* begin, const int64_t* end, int dim,
                                    int* err) {
  static_assert(std::is_same<V, F32>::value, "float32 only");
  griddep_launch_dependents();   // the plan may start beside it
  const int64_t count = end[0] * dim;
  bool bad = false;
  for (int64_t i = begin[0] * dim + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_error(err, DFD_ERR_NONFINITE);
}

// Vector point loads need dim == DK in {2, 4, 8, 16} and aligned points
// (8 bytes for 2-D, 16 bytes otherwise; every curve then starts aligned too).
template <int DK>
int vector_loads_ok(const void* points, int dim) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(points);
  if (dim != DK) return 0;
  if (DK == 2) return a % 8 == 0;
  if (DK % 4 == 0) return a % 16 == 0;
  return 0;
}

// Largest |coordinate| of an int32 curve: |p_k - q_k| <= 2 * lim must keep
// dim squares summing below 2^63 (and every difference in int32).
inline long long int32_coord_limit(int dim) {
  const double l = std::floor(std::sqrt((double)LLONG_MAX / (double)dim) / 2.0);
  return std::min<long long>((1LL << 30) - 1, (long long)l);
}

// Per-curve bounding boxes (and, with input checks on, the coordinate
// range check) of curves [first, n_curves) of an int32 CSR batch.  Returns
// whether a kernel was launched (none when the range is empty).
template <int DK>
bool launch_curve_bbox(dfd_context* ctx, const void* points, const int64_t* offsets, int64_t n_curves, int dim,
                       int* bbox, cudaStream_t s, int64_t first = 0) {
  const int64_t warps_needed = n_curves - first;
  if (warps_needed < 1) return false;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((warps_needed + 7) / 8, 16 * (int64_t)ctx->num_sms));
  const int32_t* pts = static_cast<const int32_t*>(points);
  const int check = ctx->opt.check_inputs ? 1 : 0;
  if (vector_loads_ok<DK>(points, dim))
    batch::curve_bbox_kernel<DK, true><<<blocks, 256, 0, s>>>(pts, offsets, first, n_curves, dim, check,
                                                              int32_coord_limit(dim), bbox, ctx->d_err);
  else
    batch::curve_bbox_kernel<DK, false><<<blocks, 256, 0, s>>>(pts, offsets, first, n_curves, dim, check,
                                                               int32_coord_limit(dim), bbox, ctx->d_err);
  return true;
}

template <class K>
int resident_blocks(const dfd_context* ctx, K kernel, int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return per_sm * ctx->num_sms;
}

// Scratch, input checks (and int32 bounding boxes) and the device-built
// LPT work list shared by the batch and decider kernels; `blocks` persistent
// CTAs of 256 threads will run the work list.
// With `bbox_ext` (int32 batches) the per-curve boxes live in the caller's
// buffer and only curves [first_curve, n_curves) are boxed and checked
// (float32: only their points are checked): a batch run in slices of
// curves, each slice covering the curves no earlier slice covered.
// Scratch of one batch launch: [counter | hist | cursor | SM slots | meet
// words] (zeroed per launch) [bucket] [worklist]
// [bbox] [row buffers].
struct BatchLayout {
  size_t off_hist, off_cursor, off_smrank, off_meet, off_bucket, off_work, off_defer, off_bbox, off_buf, total;
};
template <class V, int DK>
BatchLayout batch_layout(int64_t n_curves, int64_t n_pairs, int blocks, bool bbox_ext, int buf_cols) {
  constexpr int THREADS = 256;
  constexpr bool kInt = std::is_same<V, I32>::value;
  BatchLayout l;
  l.off_hist = 256;
  l.off_cursor = l.off_hist + batch::NBUCKET * 4;
  l.off_smrank = align_up(l.off_cursor + batch::NBUCKET * 4, 256);
  l.off_meet = align_up(l.off_smrank + batch::kSmSlots * 4, 256);
  l.off_bucket = align_up(l.off_meet + batch::kMeetItems * 4 * 4, 256);
  l.off_work = align_up(l.off_bucket + (size_t)n_pairs * 2, 256);
  l.off_defer = align_up(l.off_work + (size_t)n_pairs * 4, 256);
  l.off_bbox = align_up(l.off_defer + (size_t)n_pairs * 4, 256);
  l.off_buf = align_up(l.off_bbox + (kInt && !bbox_ext ? (size_t)n_curves * DK * 2 * 4 : 0), 256);
  l.total = l.off_buf + (size_t)blocks * (THREADS / 32) * (size_t)buf_cols * sizeof(typename V::value);
  return l;
}

// With `scratch_ext` the launch uses the caller's scratch area (at least
// batch_scratch_bytes) instead of the context's, so launches on different
// streams can run side by side.  `buf_cols`: row buffer columns per warp.
// The pairs one launch of a host-buffer batch takes (PlanArgs): later
// curve id in [lo, hi), and those with an id outside [0, n_ids) when
// take_invalid is set.
struct SliceFilter {
  int64_t n_ids, lo, hi;
  bool take_invalid;
};

template <class V, int DK>
dfd_status batch_prepare(dfd_context* ctx, int dim, const void* points, const int64_t* offsets, int64_t n_curves,
                         const int32_t* pairs, int64_t n_pairs, cudaStream_t s, int blocks, batch::BatchArgs* ba,
                         int64_t first_curve = 0, int* bbox_ext = nullptr, char* scratch_ext = nullptr,
                         size_t scratch_ext_bytes = 0, int buf_cols = batch::BUF_COLS, int team = 0,
                         int rmax = batch::Rmax<DK>::value, const SliceFilter* slice = nullptr) {
  constexpr bool kInt = std::is_same<V, I32>::value;
  if (n_pairs >= (int64_t)batch::kNarrowBit) return DFD_ERR_UNSUPPORTED;
  const BatchLayout lay = batch_layout<V, DK>(n_curves, n_pairs, blocks, bbox_ext != nullptr, buf_cols);
  const size_t off_cursor = lay.off_cursor, off_bucket = lay.off_bucket, off_work = lay.off_work;
  const size_t off_bbox = lay.off_bbox, off_buf = lay.off_buf;
  char* base = scratch_ext;
  if (scratch_ext) {
    if (lay.total > scratch_ext_bytes) return DFD_ERR_OOM;
  } else {
    const dfd_status st = ensure_scratch(ctx, lay.total);
    if (st != DFD_OK) return st;
    base = static_cast<char*>(ctx->scratch);
  }
  const size_t off_hist = lay.off_hist;
  // a small launch zeroes its header in its one-block plan kernel
  const bool small_plan = n_pairs <= batch::kSmallPlanPairs;
  if (!small_plan) {
    cudaError_t e = cudaMemsetAsync(base, 0, off_bucket, s);
    if (e != cudaSuccess) return cuda_status(e);
  }
  int* bbox = kInt ? (bbox_ext ? bbox_ext : reinterpret_cast<int*>(base + off_bbox)) : nullptr;
  // The plan starts early (programmatic launch) only right after this call's
  // own check or box kernel, an ordinary launch that waited for everything
  // before it: a float32 plan writes the header before it waits, and the
  // scratch may still be in use by whatever ran before the call.
  bool lead = false;
  if constexpr (kInt) {
    lead = launch_curve_bbox<DK>(ctx, points, offsets, n_curves, dim, bbox, s, bbox_ext ? first_curve : 0);
  } else if (ctx->opt.check_inputs && n_curves > first_curve) {
    check_points_kernel<V><<<std::min(4 * ctx->num_sms, 1024), 256, 0, s>>>(
        static_cast<const typename V::coord*>(points), offsets + first_curve, offsets + n_curves, dim, ctx->d_err);
    lead = true;
  }
  batch::PlanArgs pa;
  pa.offsets = offsets;
  pa.pairs = pairs;
  pa.n_pairs = n_pairs;
  pa.n_curves = n_curves;
  pa.hist = reinterpret_cast<unsigned*>(base + off_hist);
  pa.cursor = reinterpret_cast<unsigned*>(base + off_cursor);
  pa.bucket = reinterpret_cast<unsigned short*>(base + off_bucket);
  pa.worklist = reinterpret_cast<unsigned*>(base + off_work);
  pa.bbox = bbox;
  pa.dk = DK;
  pa.err = ctx->d_err;
  pa.rmax = rmax;
  pa.order = ctx->batch_order[std::is_same<V, F32>::value ? 0 : 1][dim_class_index(DK)];
  pa.team = team;
  pa.buf_cols = buf_cols;
  pa.ctas = blocks;
  pa.n_ids = slice ? slice->n_ids : n_curves;
  pa.lo_curve = slice ? slice->lo : 0;
  pa.hi_curve = slice ? slice->hi : n_curves;
  pa.take_invalid = slice ? (int)slice->take_invalid : 1;
  const int pblocks = (int)std::min<int64_t>((n_pairs + 255) / 256, 8 * (int64_t)ctx->num_sms);
  cudaError_t le = cudaSuccess;
  if (small_plan) {
    if (lead)
      le = launch_pdl(batch::plan_small_kernel, dim3(1), dim3(1024), 0, s, pa, reinterpret_cast<unsigned*>(base),
                      (int)(off_bucket / 4));
    else
      batch::plan_small_kernel<<<1, 1024, 0, s>>>(pa, reinterpret_cast<unsigned*>(base), (int)(off_bucket / 4));
  } else {
    if (lead)
      le = launch_pdl(batch::plan_hist_kernel, dim3(pblocks), dim3(256), 0, s, pa);
    else
      batch::plan_hist_kernel<<<pblocks, 256, 0, s>>>(pa);
    if (le == cudaSuccess) le = launch_pdl(batch::plan_scan_kernel, dim3(1), dim3(batch::NBUCKET), 0, s, pa);
    if (le == cudaSuccess) le = launch_pdl(batch::plan_scatter_kernel, dim3(pblocks), dim3(256), 0, s, pa);
  }
  if (le != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(le);
  }
  ba->rowbuf = base + off_buf;
  ba->buf_cols = buf_cols;
  ba->sm_rank = reinterpret_cast<unsigned*>(base + lay.off_smrank);   // zeroed with the header
  ba->meet = reinterpret_cast<unsigned*>(base + lay.off_meet);        // zeroed with the header
  ba->n_sm = std::min(blocks, ctx->num_sms);
  ba->points = points;
  ba->offsets = offsets;
  ba->pairs = pairs;
  ba->worklist = pa.worklist;
  ba->n_items = n_pairs;
  // a filtered launch's items: the end of the last bucket after the scatter
  ba->n_items_dev = slice ? pa.cursor + (batch::NBUCKET - 1) : nullptr;
  ba->n_curves = n_curves;
  ba->dim = dim;
  ba->vec = vector_loads_ok<DK>(points, dim);
  ba->counter = reinterpret_cast<int*>(base);
  ba->err = ctx->d_err;
  ba->out_dist = nullptr;
  ba->out_dist2 = nullptr;
  // CTA teams: header words after the warp counter (zeroed above); the
  // number of team items is the end of the last team bucket after the scatter
  ba->n_team = team ? pa.cursor + (batch::NTB - 1) : nullptr;
  ba->team_counter = reinterpret_cast<int*>(base + 4);
  ba->done_ctas = reinterpret_cast<unsigned*>(base + 8);
  ba->n_deferred = reinterpret_cast<unsigned*>(base + 12);
  ba->deferred = reinterpret_cast<unsigned*>(base + lay.off_defer);
  ba->timeout_ns = timeout_ns(ctx);
  ba->rmax = rmax;
  return cuda_status(cudaGetLastError());
}

// Tile shape of a batch or matrix launch, tuned per (dtype, dim class): the
// cap on rows per lane (a lane's rows are one dependent chain per step, so
// fewer rows shorten the step; more rows amortise its fixed instructions)
// and the CTAs per SM (more CTAs hide latency; fewer leave registers and
// issue slots to each).  0 = the defaults: Rmax, every resident CTA.
struct TileShape {
  int rmax;
  int blocks;
};
template <int DK, class K>
TileShape tile_shape(const dfd_context* ctx, K kernel, const signed char (&rm)[2][5], const signed char (&cp)[2][5],
                     bool f32) {
  const int t = f32 ? 0 : 1, d = dim_class_index(DK);
  TileShape sh;
  sh.rmax = rm[t][d] > 0 ? std::min<int>(rm[t][d], batch::Rmax<DK>::value) : batch::Rmax<DK>::value;
  const int resident = resident_blocks(ctx, kernel, 256);
  sh.blocks = cp[t][d] > 0 ? std::min(resident, cp[t][d] * ctx->num_sms) : resident;
  return sh;
}

// Team mode of a ragged batch launch (see batch_kernel and team_pays): the
// context's setting for (dtype, dim class) -- 1 only the pairs too wide for
// one warp's row buffer, 2 every pair of several stripes -- or by default
// (3) those for which the plan's latency model expects a team to finish
// sooner, and the wide ones.
inline int batch_team_mode(const dfd_context* ctx, bool f32, int dk) {
  const int set = ctx->batch_team[f32 ? 0 : 1][dim_class_index(dk)];
  return set > 0 ? set : 3;
}

// Scratch bytes of one batch launch over `n_pairs` pairs of `n_curves`
// curves (bounding boxes in the caller's buffer when `bbox_ext`) with row
// buffers of `buf_cols` columns.
template <class V, int DK>
size_t batch_scratch_bytes(dfd_context* ctx, int64_t n_curves, int64_t n_pairs, bool bbox_ext, int buf_cols) {
  return batch_layout<V, DK>(n_curves, n_pairs, resident_blocks(ctx, batch::batch_kernel<V, DK>, 256), bbox_ext,
                             buf_cols)
      .total;
}

// `prepared` (optional) is recorded on s once the bounding boxes and the
// work list are built, before the batch kernel.
template <class V, int DK>
dfd_status batch_launch_range(dfd_context* ctx, int dim, const void* points, const int64_t* offsets,
                              int64_t n_curves, const int32_t* pairs, int64_t n_pairs, void* out_dist,
                              void* out_dist2, cudaStream_t s, int64_t first_curve, int* bbox_ext,
                              char* scratch_ext, size_t scratch_ext_bytes, cudaEvent_t prepared, int buf_cols,
                              const SliceFilter* slice = nullptr) {
  const TileShape ts = tile_shape<DK>(ctx, batch::batch_kernel<V, DK>, ctx->batch_rmax, ctx->batch_cpsm,
                                      std::is_same<V, F32>::value);
  const int blocks = ts.blocks;
  batch::BatchArgs ba;
  const int team = batch_team_mode(ctx, std::is_same<V, F32>::value, DK);
  dfd_status st = batch_prepare<V, DK>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, s, blocks, &ba,
                                       first_curve, bbox_ext, scratch_ext, scratch_ext_bytes, buf_cols, team,
                                       ts.rmax, slice);
  if (st != DFD_OK) return st;
  if (prepared) cudaEventRecord(prepared, s);
  ba.out_dist = out_dist;
  ba.out_dist2 = out_dist2;
  timing_begin(ctx, s);
  // programmatic launch: the CTAs become resident while the plan finishes
  // and wait for it (griddep_wait) before reading the work list
  const cudaError_t le = launch_pdl(batch::batch_kernel<V, DK>, dim3(blocks), dim3(256), 0, s, ba);
  timing_end(ctx, s);
  if (le != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(le);
  }
  return cuda_status(cudaGetLastError());
}

template <class V, int DK>
dfd_status batch_launch(dfd_context* ctx, int dim, const void* points, const int64_t* offsets, int64_t n_curves,
                        const int32_t* pairs, int64_t n_pairs, void* out_dist, void* out_dist2, cudaStream_t s) {
  return batch_launch_range<V, DK>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, out_dist, out_dist2, s, 0,
                                   nullptr, nullptr, 0, nullptr, ctx->batch_buf_cols);
}

template <class V, int DK>
dfd_status decide_launch(dfd_context* ctx, int dim, const void* points, const int64_t* offsets, int64_t n_curves,
                         const int32_t* pairs, int64_t n_pairs, const void* eps2, double eps2_all, void* out_dist2,
                         int32_t* out_within, unsigned long long* abandoned, cudaStream_t s) {
  const int blocks = resident_blocks(ctx, batch::decide_kernel<V, DK>, 256);
  batch::DecideArgs d;
  dfd_status st = batch_prepare<V, DK>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, s, blocks, &d.b);
  if (st != DFD_OK) return st;
  d.b.out_dist2 = out_dist2;
  d.eps2 = eps2;
  d.eps2_f = (float)eps2_all;
  d.eps2_i = eps2_all >= 9.2e18 ? LLONG_MAX : (long long)std::floor(eps2_all);
  d.within = out_within;
  d.abandoned = abandoned;
  timing_begin(ctx, s);
  batch::decide_kernel<V, DK><<<blocks, 256, 0, s>>>(d);
  timing_end(ctx, s);
  return cuda_status(cudaGetLastError());
}

template <class V, int DK>
dfd_status matrix_launch(dfd_context* ctx, int dim, const void* points, const int64_t* offsets, int64_t n_curves,
                         void* out_dist, void* out_dist2, cudaStream_t s, int chunk) {
  using T = typename V::value;
  constexpr int THREADS = 256;
  const TileShape ts = tile_shape<DK>(ctx, batch::matrix_kernel<V, DK>, ctx->matrix_rmax, ctx->matrix_cpsm,
                                      std::is_same<V, F32>::value);
  const int blocks = ts.blocks;
  const size_t warps = (size_t)blocks * (THREADS / 32);
  constexpr bool kInt = std::is_same<V, I32>::value;
  const size_t off_bbox = 256;
  const size_t off_buf = align_up(off_bbox + (kInt ? (size_t)n_curves * DK * 2 * 4 : 0), 256);
  const size_t total = off_buf + warps * batch::BUF_COLS * sizeof(T);
  dfd_status st = ensure_scratch(ctx, total);
  if (st != DFD_OK) return st;
  char* base = static_cast<char*>(ctx->scratch);
  cudaError_t e = cudaMemsetAsync(base, 0, 256, s);
  if (e != cudaSuccess) return cuda_status(e);
  int* bbox = kInt ? reinterpret_cast<int*>(base + off_bbox) : nullptr;
  if constexpr (kInt) {
    launch_curve_bbox<DK>(ctx, points, offsets, n_curves, dim, bbox, s);
  } else if (ctx->opt.check_inputs) {
    check_points_kernel<V><<<std::min(4 * ctx->num_sms, 1024), 256, 0, s>>>(
        static_cast<const typename V::coord*>(points), offsets, offsets + n_curves, dim, ctx->d_err);
  }
  batch::MatrixArgs ma;
  ma.rowbuf = base + off_buf;
  ma.points = points;
  ma.offsets = offsets;
  ma.n_curves = n_curves;
  ma.n_pairs = n_curves * (n_curves - 1) / 2;
  ma.dim = dim;
  ma.vec = vector_loads_ok<DK>(points, dim);
  ma.chunk = chunk > 0 ? chunk : 8;
  ma.rmax = ts.rmax;
  ma.bbox = bbox;
  ma.counter = reinterpret_cast<int*>(base);
  ma.err = ctx->d_err;
  ma.out_dist = out_dist;
  ma.out_dist2 = out_dist2;
  timing_begin(ctx, s);
  batch::matrix_kernel<V, DK><<<blocks, THREADS, 0, s>>>(ma);
  timing_end(ctx, s);
  return cuda_status(cudaGetLastError());
}

}  // namespace dfd

#define DFD_BATCH_INSTANTIATE(V, DK)                                                                              \
  template dfd_status dfd::batch_launch<dfd::V, DK>(dfd_context*, int, const void*, const int64_t*, int64_t,       \
                                                      const int32_t*, int64_t, void*, void*, cudaStream_t);        \
  template dfd_status dfd::batch_launch_range<dfd::V, DK>(dfd_context*, int, const void*, const int64_t*, int64_t, \
                                                            const int32_t*, int64_t, void*, void*, cudaStream_t,      \
                                                            int64_t, int*, char*, size_t, cudaEvent_t, int,           \
                                                            const dfd::SliceFilter*);                                 \
  template size_t dfd::batch_scratch_bytes<dfd::V, DK>(dfd_context*, int64_t, int64_t, bool, int);                  \
  template dfd_status dfd::decide_launch<dfd::V, DK>(dfd_context*, int, const void*, const int64_t*, int64_t,      \
                                                       const int32_t*, int64_t, const void*, double, void*, int32_t*, \
                                                       unsigned long long*, cudaStream_t);                            \
  template dfd_status dfd::matrix_launch<dfd::V, DK>(dfd_context*, int, const void*, const int64_t*, int64_t, void*, \
                                                       void*, cudaStream_t, int);
