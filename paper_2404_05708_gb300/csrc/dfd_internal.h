// dfd_internal.h -- host-side internals shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <map>
#include <mutex>
#include <utility>
#include <cuda_runtime.h>

#include "dfd.h"

namespace dfd {
// Launch shape of the band wavefront (K2).
struct WaveShape {
  int R = 4;      // rows per lane
  int W = 4;      // compute warps per CTA
  int ctas = 0;   // persistent CTAs (0 = auto)
};
// Launch attributes of one wavefront kernel at W compute warps, queried
// once per context: the dynamic shared memory it needs and the CTAs per SM.
struct WaveAttr {
  size_t smem = 0;
  int per_sm = 1;
};
// Autotuning key: dtype, dimension class and the size classes of n and m
// (floor(log2)), packed in 64 bits.
inline uint64_t tune_key(int dtype, int dk, int64_t n, int64_t m) {
  auto lg = [](int64_t x) { int b = 0; while (x > 1) { x >>= 1; ++b; } return b; };
  return ((uint64_t)dtype << 48) | ((uint64_t)dk << 40) | ((uint64_t)lg(n) << 20) | (uint64_t)lg(m);
}
}  // namespace dfd

namespace dfd {
constexpr int kMaxSlices = 8;   // dfd_batch_host: copy slices of the points
constexpr int kDefaultBatchBufCols = 4096;   // batch::BUF_COLS (checked in batch_launch.cuh)
}

struct dfd_context {
  int device = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  dfd_options opt{};
  int* d_err = nullptr;               // sticky device error word (+ spare control ints)
  void* scratch = nullptr;            // grow-only device scratch
  size_t scratch_bytes = 0;
  void* pinned = nullptr;             // grow-only pinned host staging
  size_t pinned_bytes = 0;
  void* io = nullptr;                 // grow-only device staging of the host-buffer entry points
  size_t io_bytes = 0;
  cudaStream_t stream = nullptr;      // internal stream (host-buffer entry points)
  bool timing = false;                // record events around the main kernel
  bool timed = false;                 // ev0/ev1 hold a recorded pair
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::map<uint64_t, dfd::WaveShape> tuned;   // autotuned wavefront shapes
  std::map<std::pair<const void*, int>, dfd::WaveAttr> wave_attr;   // per (wavefront kernel, warps)
  bool attr_cache = true;                     // keep wave_attr (off in the no-allocation entry point)
  signed char batch_order[2][5] = {};         // batch packing order per (float32 / int32, dim class 2,3,4,8,16)
  signed char batch_team[2][5] = {};          // batch team mode per (dtype, dim class): 0 auto, 1 wide pairs, 2 all multi-stripe
  signed char batch_rmax[2][5] = {};          // batch tile shape: rows per lane cap (0 = Rmax)
  signed char batch_cpsm[2][5] = {};          //   and CTAs per SM (0 = every resident CTA)
  signed char matrix_rmax[2][5] = {};         // matrix tile shape, likewise
  signed char matrix_cpsm[2][5] = {};
  cudaStream_t copy_stream = nullptr;         // dfd_batch_host: point slices (created on first use)
  cudaEvent_t slice_ev[dfd::kMaxSlices + 1] = {};   // one per slice, and one for the allocation
  int batch_buf_cols = dfd::kDefaultBatchBufCols;   // ragged batch: row buffer columns per warp
  void* host_scr = nullptr;                   // dfd_batch_host: scratch of its two launch streams (grow-only)
  size_t host_scr_bytes = 0;
  cudaStream_t launch_stream2 = nullptr;      // dfd_batch_host: every other slice launch
  cudaEvent_t prep_ev[2] = {};                // dfd_batch_host: a launch's boxes and work list built
  cudaEvent_t join_ev = nullptr;              // dfd_batch_host: launch_stream2's work done
};

namespace dfd {

// Status from a CUDA error, never throwing.
inline dfd_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return DFD_OK;
  if (e == cudaErrorMemoryAllocation) return DFD_ERR_OOM;
  return DFD_ERR_CUDA;
}

// Grow the context scratch to at least `bytes`; 256-byte aligned.
dfd_status ensure_scratch(dfd_context* ctx, size_t bytes);
dfd_status ensure_pinned(dfd_context* ctx, size_t bytes);
dfd_status ensure_io(dfd_context* ctx, size_t bytes);

// Events around the main kernel of a call (measurement hooks).
inline void timing_begin(dfd_context* ctx, cudaStream_t s) {
  if (ctx->timing) cudaEventRecord(ctx->ev0, s);
}
inline void timing_end(dfd_context* ctx, cudaStream_t s) {
  if (ctx->timing) {
    cudaEventRecord(ctx->ev1, s);
    ctx->timed = true;
  }
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Launch with programmatic stream serialisation: the kernel's CTAs may start
// while the kernel before it in the stream finishes (once every CTA of that
// one has called griddepcontrol.launch_dependents or exited); the kernel
// calls griddepcontrol.wait before it reads anything that kernel (or one
// before it) wrote.  Between two kernels this hides most of a launch gap.
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

inline unsigned long long timeout_ns(const dfd_context* ctx) {
  double ms = ctx->opt.wait_timeout_ms > 0 ? ctx->opt.wait_timeout_ms : 2000.0;
  return (unsigned long long)(ms * 1.0e6);
}

// Kernel dimension class: 2, 3, 4, 8, 16 (coordinates beyond dim are zero,
// which adds exact zeros to the squared distance).
// Index of a dim class (2, 3, 4, 8, 16) in per-class tables.
inline int dim_class_index(int dk) { return dk == 2 ? 0 : dk == 3 ? 1 : dk == 4 ? 2 : dk == 8 ? 3 : 4; }

inline int dim_class(int dim) {
  if (dim <= 2) return 2;
  if (dim == 3) return 3;
  if (dim == 4) return 4;
  if (dim <= 8) return 8;
  if (dim <= 16) return 16;
  return 0;
}

// Make the context's device current.
dfd_status set_device(dfd_context* ctx);
// Host-side argument checks shared by the batch entry points.
dfd_status check_batch_args(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                            int64_t n_curves, const void* out_dist, const void* out_dist2);

// Input validation kernels: set DFD_ERR_NONFINITE / DFD_ERR_RANGE in *err.
dfd_status launch_check_inputs(dfd_dtype dtype, int dim, const void* x, int64_t count, int* err,
                               cudaStream_t s);
// Both curves of a pair in one launch.
dfd_status launch_check_inputs2(dfd_dtype dtype, int dim, const void* x, int64_t nx, const void* y, int64_t ny,
                                int* err, cudaStream_t s);

// Band wavefront (K2).
dfd_status wave_plan(const dfd_context* ctx, dfd_dtype dtype, int dim, int64_t n, int64_t m, WaveShape* shape);
// check: the launch's prep kernel also runs the input checks (dfd_pair's
// check_inputs); callers that checked already pass false.
dfd_status wave_run(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q,
                    int64_t m, void* out_dist, void* out_dist2, cudaStream_t s, const WaveShape& shape,
                    bool check);

// Ragged batch (K4) and all-pairs matrix (K5).
dfd_status batch_run(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                     int64_t n_curves, const int32_t* pairs, int64_t n_pairs, void* out_dist, void* out_dist2,
                     cudaStream_t s);
dfd_status matrix_run(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                      int64_t n_curves, void* out_dist, void* out_dist2, cudaStream_t s, int chunk);

// Per-pair reference (K1): one CTA, row-by-row clamp scan.
dfd_status rowscan_run(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q,
                       int64_t m, void* out_dist, void* out_dist2, cudaStream_t s);

}  // namespace dfd
