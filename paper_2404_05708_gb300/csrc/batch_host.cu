// batch_host.cu -- dfd_batch with HOST buffers (the ragged batch, K4, Sec. 4's
// batches of curve pairs): copies the points to the device in slices of
// curves on a copy stream while the batch engine runs the pairs whose
// curves have arrived, then copies the distances back.
//
// The offsets and the pair list go first, as given; then the point slices.
// Slice k's launch runs over curves [0, end_k) and takes from the whole pair
// list the pairs whose later curve lies in slice k (its plan filters them:
// no grouping on the host), as soon as slice k has landed, so the copy of
// slice k+1 overlaps it, and every result lands at the caller's pair index.
// Launches alternate between two streams, each with its own scratch area,
// so a launch's bounding boxes, work list and first pairs start while the
// one before finishes its longest pairs.  Each launch boxes and checks only
// the curves no earlier launch covered (the int32 bounding boxes live in one
// buffer for the whole batch, and a launch waits until the one before has
// built its boxes), and the last launch waits for every slice and covers all
// curves, so the input checks are those of dfd_batch.  Results are
// bit-identical to dfd_batch on the same data: each pair is computed by the
// same engine.
#include <algorithm>
#include <cstring>
#include <memory>
#include <vector>

#include "batch_launch.cuh"
#include "dfd_internal.h"

namespace dfd {
#define DFD_RANGE_EXTERN(V, DK)                                                                                 \
  extern template dfd_status batch_launch_range<V, DK>(dfd_context*, int, const void*, const int64_t*, int64_t, \
                                                       const int32_t*, int64_t, void*, void*, cudaStream_t,     \
                                                       int64_t, int*, char*, size_t, cudaEvent_t, int,          \
                                                       const SliceFilter*);                                     \
  extern template size_t batch_scratch_bytes<V, DK>(dfd_context*, int64_t, int64_t, bool, int);
DFD_RANGE_EXTERN(F32, 2)
DFD_RANGE_EXTERN(F32, 3)
DFD_RANGE_EXTERN(F32, 4)
DFD_RANGE_EXTERN(F32, 8)
DFD_RANGE_EXTERN(F32, 16)
DFD_RANGE_EXTERN(I32, 2)
DFD_RANGE_EXTERN(I32, 3)
DFD_RANGE_EXTERN(I32, 4)
DFD_RANGE_EXTERN(I32, 8)
DFD_RANGE_EXTERN(I32, 16)
#undef DFD_RANGE_EXTERN

namespace {

// Points per copy slice (about).  The first slice's copy is not overlapped,
// and each launch adds its pre-pass and the tail of its longest pairs (half
// hidden by the next launch on the other stream): on the 65,536-pair int32
// batch (279 MB) slices of 64 and 36 MB ran at 2.25 and 2.13 Tcell/s end to
// end; a first and a last slice of 16 MB (8 MB) with three even ones between
// ran at 2.13 (2.08).
constexpr size_t kSliceBytes = (size_t)64 << 20;

dfd_status range_run(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                     int64_t n_curves, const int32_t* pairs, int64_t n_pairs, void* out_dist, void* out_dist2,
                     cudaStream_t s, int64_t first, int* bbox, char* scratch, size_t scratch_bytes,
                     cudaEvent_t prepared, int buf_cols, const SliceFilter* slice) {
#define DFD_R_CASE(V, DK)                                                                                       \
  case DK:                                                                                                      \
    return batch_launch_range<V, DK>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, out_dist, out_dist2, s, \
                                     first, bbox, scratch, scratch_bytes, prepared, buf_cols, slice);
#define DFD_R_DK(V)                                                                                          \
  switch (dim_class(dim)) {                                                                                  \
    DFD_R_CASE(V, 2)                                                                                         \
    DFD_R_CASE(V, 3)                                                                                         \
    DFD_R_CASE(V, 4)                                                                                         \
    DFD_R_CASE(V, 8)                                                                                         \
    DFD_R_CASE(V, 16)                                                                                        \
    default: return DFD_ERR_UNSUPPORTED;                                                                     \
  }
  if (dtype == DFD_F32) {
    DFD_R_DK(F32)
  } else {
    DFD_R_DK(I32)
  }
#undef DFD_R_DK
#undef DFD_R_CASE
}

// Scratch bytes of one slice launch (at most n_pairs pairs); 0: unsupported.
size_t range_scratch(dfd_context* ctx, dfd_dtype dtype, int dim, int64_t n_curves, int64_t n_pairs, int buf_cols) {
#define DFD_S_CASE(V, DK) \
  case DK: return batch_scratch_bytes<V, DK>(ctx, n_curves, n_pairs, true, buf_cols);
#define DFD_S_DK(V)          \
  switch (dim_class(dim)) {  \
    DFD_S_CASE(V, 2)         \
    DFD_S_CASE(V, 3)         \
    DFD_S_CASE(V, 4)         \
    DFD_S_CASE(V, 8)         \
    DFD_S_CASE(V, 16)        \
    default: return 0;       \
  }
  if (dtype == DFD_F32) {
    DFD_S_DK(F32)
  } else {
    DFD_S_DK(I32)
  }
#undef DFD_S_DK
#undef DFD_S_CASE
}

// Rows per lane of a full stripe (batch::Rmax) for a dimension class.
int rmax_of(int dk) { return dk <= 4 ? 8 : 4; }
static_assert(batch::Rmax<2>::value == 8 && batch::Rmax<4>::value == 8 && batch::Rmax<8>::value == 4 &&
                  batch::Rmax<16>::value == 4,
              "rmax_of mirrors batch::Rmax");

// Device scratch of the two launch streams (grow-only; cudaFree on growth
// synchronises the device, so no launch still uses the old area).
dfd_status ensure_host_scratch(dfd_context* ctx, size_t bytes) {
  if (bytes <= ctx->host_scr_bytes) return DFD_OK;
  if (ctx->opt.mem_budget_bytes && bytes > ctx->opt.mem_budget_bytes) return DFD_ERR_OOM;
  if (ctx->host_scr) cudaFree(ctx->host_scr);
  ctx->host_scr = nullptr;
  ctx->host_scr_bytes = 0;
  if (cudaMalloc(&ctx->host_scr, bytes) != cudaSuccess) {
    cudaGetLastError();
    ctx->host_scr = nullptr;
    return DFD_ERR_OOM;
  }
  ctx->host_scr_bytes = bytes;
  return DFD_OK;
}

bool page_locked(const void* x) {
  cudaPointerAttributes at;
  const bool yes = cudaPointerGetAttributes(&at, x) == cudaSuccess && at.type == cudaMemoryTypeHost;
  cudaGetLastError();
  return yes;
}

}  // namespace
}  // namespace dfd

using namespace dfd;

extern "C" dfd_status dfd_batch_host(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points,
                                     const int64_t* offsets, int64_t n_curves, const int32_t* pairs, int64_t n_pairs,
                                     void* out_dist, void* out_dist2) {
  dfd_status st = check_batch_args(ctx, dtype, dim, points, offsets, n_curves, out_dist, out_dist2);
  if (st != DFD_OK) return st;
  if (!pairs || n_pairs < 0 || n_pairs > INT32_MAX) return DFD_ERR_INVALID_ARG;
  if (n_pairs == 0) return DFD_OK;
  if (offsets[0] < 0 || offsets[n_curves] < 0) return DFD_ERR_INVALID_ARG;
  if ((st = set_device(ctx)) != DFD_OK) return st;

  const int64_t n_pts = offsets[n_curves];
  const size_t elem = 4;   // float32 and int32 coordinates
  const size_t pts_bytes = (size_t)n_pts * dim * elem;
  const bool f32 = dtype == DFD_F32;
  const size_t d1 = f32 ? 4 : 8, d2 = f32 ? 4 : 8;   // result element sizes (dist, dist2)

  // slices of curves with about kSliceBytes of points each
  const int K = (int)std::max<size_t>(1, std::min<size_t>(kMaxSlices, (pts_bytes + kSliceBytes - 1) / kSliceBytes));
  std::vector<int64_t> bound(K + 1, n_curves);
  bound[0] = 0;
  for (int k = 1; k < K; ++k) {
    const int64_t target = (int64_t)((double)n_pts * k / K);
    bound[k] = std::lower_bound(offsets, offsets + n_curves + 1, target) - offsets;
    bound[k] = std::min(std::max(bound[k], bound[k - 1]), n_curves);
  }
  // byte range of each slice's copy: the slice's curves when the offsets are
  // valid (checked below, while the copies run), and in any case a partition
  // of the caller's buffer, so no copy reads outside it
  std::vector<size_t> cut(K + 1, pts_bytes);
  cut[0] = 0;
  for (int k = 1; k < K; ++k) {
    const int64_t o = offsets[bound[k]];
    const size_t b = o < 0 ? 0 : (size_t)o * dim * elem;
    cut[k] = std::min(std::max(b, cut[k - 1]), pts_bytes);
  }

  // pinned staging: [offsets | pairs | dist | dist2 | error word | points if pageable]
  const bool pts_locked = page_locked(points);
  const size_t off_b = align_up((size_t)(n_curves + 1) * 8, 256);
  const size_t pair_b = align_up((size_t)n_pairs * 8, 256);
  const size_t dist_b = align_up((size_t)n_pairs * d1, 256), dist2_b = align_up((size_t)n_pairs * d2, 256);
  const size_t host_bytes = off_b + pair_b + dist_b + dist2_b + 256 + (pts_locked ? 0 : align_up(pts_bytes, 256));
  if ((st = ensure_pinned(ctx, host_bytes)) != DFD_OK) return st;
  char* h = static_cast<char*>(ctx->pinned);
  int* h_err = reinterpret_cast<int*>(h + off_b + pair_b + dist_b + dist2_b);
  char* h_pts = pts_locked ? nullptr : h + off_b + pair_b + dist_b + dist2_b + 256;
  const char* src_pts = pts_locked ? static_cast<const char*>(points) : h_pts;

  // device (the context's staging buffer): [points | offsets | pairs | bbox | dist | dist2];
  // the launches' scratch is sized once the pairs are known (their row buffers)
  const size_t bbox_b = f32 ? 0 : align_up((size_t)n_curves * dim_class(dim) * 2 * 4, 256);
  const size_t dev_bytes = align_up(pts_bytes, 256) + off_b + pair_b + bbox_b + dist_b + dist2_b;
  if ((st = ensure_io(ctx, dev_bytes)) != DFD_OK) return st;
  char* d = static_cast<char*>(ctx->io);
  char* d_pts = d;
  int64_t* d_off = reinterpret_cast<int64_t*>(d + align_up(pts_bytes, 256));
  int32_t* d_pairs = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(d_off) + off_b);
  int* d_bbox = f32 ? nullptr : reinterpret_cast<int*>(reinterpret_cast<char*>(d_pairs) + pair_b);
  char* d_dist = reinterpret_cast<char*>(d_pairs) + pair_b + bbox_b;
  char* d_dist2 = d_dist + dist_b;
  cudaStream_t s = ctx->stream;
  if (!ctx->copy_stream) {
    if (cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      ctx->copy_stream = nullptr;
      return DFD_ERR_CUDA;
    }
    for (auto& e : ctx->slice_ev) {
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return DFD_ERR_CUDA;
      }
    }
  }
  if (!ctx->launch_stream2) {
    if (cudaStreamCreateWithFlags(&ctx->launch_stream2, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      ctx->launch_stream2 = nullptr;
      return DFD_ERR_CUDA;
    }
    for (cudaEvent_t* e : {&ctx->prep_ev[0], &ctx->prep_ev[1], &ctx->join_ev}) {
      if (cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return DFD_ERR_CUDA;
      }
    }
  }
  cudaStream_t ls[2] = {s, ctx->launch_stream2};

  // 1. every host-to-device copy on the copy stream, in the order the
  // launches need it (copies in one direction are served in order): point
  // slice 0, the offsets and the pairs as given (1.5 MB for 65,536 pairs),
  // then the other slices.  Nothing is regrouped on the host: each launch's
  // plan picks its own pairs from the whole list, and results land at the
  // caller's indices.
  cudaStream_t cs = ctx->copy_stream;
  cudaEventRecord(ctx->slice_ev[kMaxSlices], s);   // after the previous work on s (the staging areas)
  cudaStreamWaitEvent(cs, ctx->slice_ev[kMaxSlices], 0);
  for (int k = 0; k < K; ++k) {
    const size_t b0 = cut[k], b1 = cut[k + 1];
    if (b1 > b0) {
      if (!pts_locked) std::memcpy(h_pts + b0, static_cast<const char*>(points) + b0, b1 - b0);
      cudaMemcpyAsync(d_pts + b0, src_pts + b0, b1 - b0, cudaMemcpyHostToDevice, cs);
    }
    if (k == 0) {   // the offsets and pairs right after the first slice (host copies while it is in flight)
      std::memcpy(h, offsets, (size_t)(n_curves + 1) * 8);
      std::memcpy(h + off_b, pairs, (size_t)n_pairs * 8);
      cudaMemcpyAsync(d_off, h, (size_t)(n_curves + 1) * 8, cudaMemcpyHostToDevice, cs);
      cudaMemcpyAsync(d_pairs, h + off_b, (size_t)n_pairs * 8, cudaMemcpyHostToDevice, cs);
    }
    cudaEventRecord(ctx->slice_ev[k], cs);
  }

  // 2. on the host meanwhile: check the offsets (nondecreasing; the longest
  // curve bounds the row buffers' width) and, when a curve is wider than the
  // buffers, the ids and the widest row a multi-stripe pair hands between its
  // stripes (the row buffers)
  int64_t len_max = 0;
  bool bad = false;
  for (int64_t c = 0; c < n_curves; ++c) {
    const int64_t len = offsets[c + 1] - offsets[c];
    bad |= len < 0;
    len_max = std::max(len_max, len);
  }
  if (bad) {
    // the copies read the caller's buffers: let them finish before returning
    cudaStreamSynchronize(cs);
    cudaGetLastError();
    return DFD_ERR_INVALID_ARG;
  }
  // Unless some curve is longer than the row buffers are wide, the pair list
  // needs no host pass at all: the launches go out at once, and an id out of
  // range is reported by the last launch's plan (DFD_ERR_INVALID_ARG, as the
  // host check would).
  bool bad_id = false;
  const int dk = dim_class(dim);
  const int64_t stripe_rows = 32 * (int64_t)rmax_of(dk);
  const bool any_wide = len_max > ctx->batch_buf_cols;   // else no pair can outgrow the buffers
  int64_t wide = 0;
  for (int64_t i = 0; any_wide && i < n_pairs; ++i) {
    const int32_t ia = pairs[2 * i], ib = pairs[2 * i + 1];
    if (ia < 0 || ib < 0 || ia >= n_curves || ib >= n_curves) {
      bad_id = true;
      break;
    }
    const int64_t na = offsets[ia + 1] - offsets[ia], nb = offsets[ib + 1] - offsets[ib];
    const bool sw = batch::plan_rows_from_b(na, nb, dk, rmax_of(dk), ctx->batch_buf_cols);   // the plan's orientation
    if ((sw ? nb : na) > stripe_rows) wide = std::max(wide, sw ? na : nb);
  }
  if (bad_id) {
    // the copies read the caller's buffers: let them finish before returning
    cudaStreamSynchronize(cs);
    cudaGetLastError();
    return DFD_ERR_INVALID_ARG;
  }
  // row buffers as wide as the widest such pair needs (at least the context's width)
  const int buf_cols =
      (int)std::min<int64_t>(1 << 28, std::max<int64_t>(ctx->batch_buf_cols, (wide + 31) / 32 * 32));
  if (wide > (1 << 28)) st = DFD_ERR_UNSUPPORTED;
  const size_t scr_b = align_up(range_scratch(ctx, dtype, dim, n_curves, n_pairs, buf_cols), 256);
  if (st == DFD_OK && scr_b == 0) st = DFD_ERR_UNSUPPORTED;
  if (st == DFD_OK) st = ensure_host_scratch(ctx, 2 * scr_b);
  if (st != DFD_OK) {
    cudaStreamSynchronize(cs);   // the copies read the caller's buffers
    cudaGetLastError();
    return st;
  }
  char* d_scr[2] = {static_cast<char*>(ctx->host_scr), static_cast<char*>(ctx->host_scr) + scr_b};

  // 3. one launch per slice, over the whole pair list: slice k's launch
  // takes the pairs whose later curve lies in slice k, as soon as the slice
  // has landed; the last launch waits for every slice, covers all curves and
  // also takes any pair with an id out of range (its plan reports it).
  int64_t covered = 0;   // curves boxed / checked so far
  for (int k = 0; k < K && st == DFD_OK; ++k) {
    const bool final_launch = k + 1 == K;
    cudaStream_t sk = ls[k & 1];
    for (int j = (final_launch ? 0 : k); j <= k; ++j) cudaStreamWaitEvent(sk, ctx->slice_ev[j], 0);
    if (k > 0) cudaStreamWaitEvent(sk, ctx->prep_ev[(k - 1) & 1], 0);   // boxes of the earlier curves
    const int64_t upto = final_launch ? n_curves : bound[k + 1];
    const SliceFilter filt{n_curves, bound[k], upto, final_launch};
    st = range_run(ctx, dtype, dim, d_pts, d_off, upto, d_pairs, n_pairs, out_dist ? d_dist : nullptr,
                   out_dist2 ? d_dist2 : nullptr, sk, covered, d_bbox, d_scr[k & 1], scr_b, ctx->prep_ev[k & 1],
                   buf_cols, &filt);
    covered = upto;
  }
  cudaEventRecord(ctx->join_ev, ls[1]);
  cudaStreamWaitEvent(s, ctx->join_ev, 0);
  if (st == DFD_OK) {
    if (out_dist) cudaMemcpyAsync(h + off_b + pair_b, d_dist, (size_t)n_pairs * d1, cudaMemcpyDeviceToHost, s);
    if (out_dist2)
      cudaMemcpyAsync(h + off_b + pair_b + dist_b, d_dist2, (size_t)n_pairs * d2, cudaMemcpyDeviceToHost, s);
  }
  // s is ordered after every slice copy, whether or not a launch ran, so
  // the synchronisation below covers the copy stream too
  for (int k = 0; k < K; ++k) cudaStreamWaitEvent(s, ctx->slice_ev[k], 0);
  *h_err = 0;
  cudaMemcpyAsync(h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_CUDA;
  }
  if (st != DFD_OK) return st;
  if (*h_err != 0) {
    cudaMemset(ctx->d_err, 0, sizeof(int));
    return (dfd_status)*h_err;
  }
  // 4. results, already in the caller's pair order
  if (out_dist) std::memcpy(out_dist, h + off_b + pair_b, (size_t)n_pairs * d1);
  if (out_dist2) std::memcpy(out_dist2, h + off_b + pair_b + dist_b, (size_t)n_pairs * d2);
  return DFD_OK;
}
