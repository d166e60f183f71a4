// dfd_api.cu -- the C ABI (dfd.h): contexts, argument checks, dispatch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "dfd_device.cuh"
#include "dfd_internal.h"
#include "wave_shape.h"

namespace dfd {

// ------------------------------------------------------------ declarations
template <class V, int DK, int R>
dfd_status wave_launch(dfd_context* ctx, int dim, const void* p, int64_t n, const void* q, int64_t m,
                       void* out_dist, void* out_dist2, cudaStream_t s, int W, int ctas, bool check);

#define DFD_WAVE_EXTERN(V, DK, R)                                                                              \
  extern template dfd_status wave_launch<V, DK, R>(dfd_context*, int, const void*, int64_t, const void*, int64_t, \
                                                   void*, void*, cudaStream_t, int, int, bool);
#define DFD_WAVE_EXTERN_R(V, DK) \
  DFD_WAVE_EXTERN(V, DK, 2) DFD_WAVE_EXTERN(V, DK, 4) DFD_WAVE_EXTERN(V, DK, 6) DFD_WAVE_EXTERN(V, DK, 8)
DFD_WAVE_EXTERN_R(F32, 2)
DFD_WAVE_EXTERN_R(F32, 3)
DFD_WAVE_EXTERN_R(F32, 4)
DFD_WAVE_EXTERN_R(F32, 8)
DFD_WAVE_EXTERN_R(F32, 16)
DFD_WAVE_EXTERN_R(I32, 2)
DFD_WAVE_EXTERN_R(I32, 3)
DFD_WAVE_EXTERN_R(I32, 4)
DFD_WAVE_EXTERN_R(I32, 8)
DFD_WAVE_EXTERN_R(I32, 16)

template <class V, int DK>
dfd_status batch_launch(dfd_context* ctx, int dim, const void* points, const int64_t* offsets, int64_t n_curves,
                        const int32_t* pairs, int64_t n_pairs, void* out_dist, void* out_dist2, cudaStream_t s);
template <class V, int DK>
dfd_status matrix_launch(dfd_context* ctx, int dim, const void* points, const int64_t* offsets, int64_t n_curves,
                         void* out_dist, void* out_dist2, cudaStream_t s, int chunk);
template <class V, int DK>
dfd_status decide_launch(dfd_context* ctx, int dim, const void* points, const int64_t* offsets, int64_t n_curves,
                         const int32_t* pairs, int64_t n_pairs, const void* eps2, double eps2_all, void* out_dist2,
                         int32_t* out_within, unsigned long long* abandoned, cudaStream_t s);
#define DFD_BATCH_EXTERN(V, DK)                                                                              \
  extern template dfd_status batch_launch<V, DK>(dfd_context*, int, const void*, const int64_t*, int64_t,     \
                                                 const int32_t*, int64_t, void*, void*, cudaStream_t);        \
  extern template dfd_status decide_launch<V, DK>(dfd_context*, int, const void*, const int64_t*, int64_t,    \
                                                  const int32_t*, int64_t, const void*, double, void*,        \
                                                  int32_t*, unsigned long long*, cudaStream_t);               \
  extern template dfd_status matrix_launch<V, DK>(dfd_context*, int, const void*, const int64_t*, int64_t,    \
                                                  void*, void*, cudaStream_t, int);
DFD_BATCH_EXTERN(F32, 2)
DFD_BATCH_EXTERN(F32, 3)
DFD_BATCH_EXTERN(F32, 4)
DFD_BATCH_EXTERN(F32, 8)
DFD_BATCH_EXTERN(F32, 16)
DFD_BATCH_EXTERN(I32, 2)
DFD_BATCH_EXTERN(I32, 3)
DFD_BATCH_EXTERN(I32, 4)
DFD_BATCH_EXTERN(I32, 8)
DFD_BATCH_EXTERN(I32, 16)

// ---------------------------------------------------------- scratch memory
dfd_status ensure_scratch(dfd_context* ctx, size_t bytes) {
  if (bytes <= ctx->scratch_bytes) return DFD_OK;
  if (ctx->opt.mem_budget_bytes && bytes > ctx->opt.mem_budget_bytes) return DFD_ERR_OOM;
  size_t want = std::max(bytes, ctx->scratch_bytes + ctx->scratch_bytes / 2);
  if (ctx->opt.mem_budget_bytes) want = std::min(want, ctx->opt.mem_budget_bytes);
  void* p = nullptr;
  // cudaFree synchronises the device, so no in-flight kernel still uses the old area.
  if (ctx->scratch) cudaFree(ctx->scratch);
  ctx->scratch = nullptr;
  ctx->scratch_bytes = 0;
  cudaError_t e = cudaMalloc(&p, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_OOM;
  }
  ctx->scratch = p;
  ctx->scratch_bytes = want;
  return DFD_OK;
}

// Device buffer of the host-buffer entry points (inputs and results staged
// on the device); grow-only, so repeated calls map no new memory.  Those
// calls are synchronous, so nothing still uses the old buffer on growth.
dfd_status ensure_io(dfd_context* ctx, size_t bytes) {
  if (bytes <= ctx->io_bytes) return DFD_OK;
  if (ctx->io) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->io);
  }
  ctx->io = nullptr;
  ctx->io_bytes = 0;
  const size_t want = std::max(bytes, ctx->io_bytes + ctx->io_bytes / 2);
  void* p = nullptr;
  if (cudaMalloc(&p, want) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_OOM;
  }
  ctx->io = p;
  ctx->io_bytes = want;
  return DFD_OK;
}

dfd_status ensure_pinned(dfd_context* ctx, size_t bytes) {
  if (bytes <= ctx->pinned_bytes) return DFD_OK;
  if (ctx->pinned) {
    cudaStreamSynchronize(ctx->stream);
    cudaFreeHost(ctx->pinned);
  }
  ctx->pinned = nullptr;
  ctx->pinned_bytes = 0;
  size_t want = std::max(bytes, (size_t)1 << 20);
  void* p = nullptr;
  if (cudaMallocHost(&p, want) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_OOM;
  }
  ctx->pinned = p;
  ctx->pinned_bytes = want;
  return DFD_OK;
}

// ------------------------------------------------------ input check kernels
// Both arrays in one launch: indices below nx read x, the rest y.
__global__ void check_f32_kernel(const float* x, int64_t nx, const float* y, int64_t ny, int* err) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nx + ny; i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(i < nx ? x[i] : y[i - nx]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_error(err, DFD_ERR_NONFINITE);
}

__global__ void check_i32_kernel(const int32_t* x, int64_t nx, const int32_t* y, int64_t ny, long long lim, int* err) {
  // |c| <= lim = min(2^30 - 1, sqrt((2^63 - 1) / dim) / 2), computed on the host
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nx + ny; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = i < nx ? x[i] : y[i - nx];
    const long long v = c < 0 ? -(long long)c : (long long)c;
    bad |= v > lim;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_error(err, DFD_ERR_RANGE);
}

dfd_status launch_check_inputs2(dfd_dtype dtype, int dim, const void* x, int64_t nx, const void* y, int64_t ny,
                                int* err, cudaStream_t s) {
  if (nx + ny <= 0) return DFD_OK;
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>((nx + ny + threads - 1) / threads, 1024);
  if (dtype == DFD_F32)
    check_f32_kernel<<<blocks, threads, 0, s>>>(static_cast<const float*>(x), nx, static_cast<const float*>(y), ny,
                                                err);
  else
    check_i32_kernel<<<blocks, threads, 0, s>>>(
        static_cast<const int32_t*>(x), nx, static_cast<const int32_t*>(y), ny,
        std::min<long long>((1LL << 30) - 1, (long long)std::floor(std::sqrt((double)LLONG_MAX / (double)dim) / 2.0)),
        err);
  return cuda_status(cudaGetLastError());
}

dfd_status launch_check_inputs(dfd_dtype dtype, int dim, const void* x, int64_t count, int* err, cudaStream_t s) {
  return launch_check_inputs2(dtype, dim, x, count, x, 0, err, s);
}

// ------------------------------------------------------------- wave plans
static bool shape_ok(const dfd_context* ctx, dfd_dtype dtype, int dim, int R, int W) {
  // The q ring bounds how far the last warp may trail warp 0, the register
  // file how many warps of R rows a CTA can hold (wave_shape.h); an int32
  // pair's shape must suit both of its kernels.
  (void)ctx;
  const int dk = dim_class(dim);
  return dk > 0 && (dtype == DFD_F32 ? wave::shape_supported(true, dk, R, W) : wave::int_shape_supported(dk, R, W));
}

dfd_status wave_plan(const dfd_context* ctx, dfd_dtype dtype, int dim, int64_t n, int64_t m, WaveShape* shape) {
  // Cost model: every CTA runs one band at a time; a band of H = 32*W*R rows
  // sweeps m columns plus its internal skew; bands start one inter-band lag
  // apart (W warps, each trailing the one above by 32*K + G columns), and a
  // pair of two bands or more runs as two fronts, each its own chain of
  // bands.  A step costs the cycles measured for one float32 band of each R
  // alone (in place, one compute warp per SM sub-partition: 73, 69, 74, 117
  // for R = 2, 4, 6, 8), times the compute warps sharing a sub-partition.
  // int32 pairs are planned the same way: the shape serves both of their
  // kernels, and the narrow class (the float32 stripe) is the common one.
  // Minimise the modelled completion time.
  auto hit = ctx->tuned.find(tune_key(dtype, dim_class(dim), n, m));
  if (hit != ctx->tuned.end()) {
    *shape = hit->second;
    return DFD_OK;
  }
  // one CTA per SM: bands of one chain sharing an SM slow each other down
  // more than a second CTA hides (the 200,000^2 3-D pair: 2.63 Tcell/s with
  // 152 CTAs, 1.87 with all 261 bands resident two to an SM)
  const int P = std::max(ctx->num_sms, 1);
  double best = 1e300;
  WaveShape bs;
  const int Rs[4] = {8, 6, 4, 2};
  for (int R : Rs) {
    for (int W = 1; W <= 16; ++W) {
      if (!shape_ok(ctx, dtype, dim, R, W)) continue;
      const double H = 32.0 * W * R;
      const double B = std::ceil((double)n / H);
      const double waves = std::ceil(B / P);
      const double K = R / 2;
      const double wlag = 32.0 * K + 32.0;
      const double lag = wlag * W + 96.0;
      const double conc = std::min(B, (double)P);
      const double chain = B >= 2 ? std::ceil(conc / 2.0) - 1.0 : 0.0;   // bands of one front started in turn
      const double cols = waves * ((double)m + wlag * W) + chain * lag;
      const double step = R == 2 ? 73.0 : R == 4 ? 69.0 : R == 6 ? 74.0 : 117.0;
      const double t = cols * step * std::ceil(W / 4.0);
      if (t < best * 0.999) {
        best = t;
        bs.R = R;
        bs.W = W;
        bs.ctas = (int)conc;
      }
    }
  }
  *shape = bs;
  return DFD_OK;
}

dfd_status wave_run(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q, int64_t m,
                    void* out_dist, void* out_dist2, cudaStream_t s, const WaveShape& sh, bool check) {
  if (!shape_ok(ctx, dtype, dim, sh.R, sh.W)) return DFD_ERR_UNSUPPORTED;
  const int dk = dim_class(dim);
#define DFD_W_R(V, DK)                                                                       \
  switch (sh.R) {                                                                            \
    case 2: return wave_launch<V, DK, 2>(ctx, dim, p, n, q, m, out_dist, out_dist2, s, sh.W, sh.ctas, check); \
    case 4: return wave_launch<V, DK, 4>(ctx, dim, p, n, q, m, out_dist, out_dist2, s, sh.W, sh.ctas, check); \
    case 6: return wave_launch<V, DK, 6>(ctx, dim, p, n, q, m, out_dist, out_dist2, s, sh.W, sh.ctas, check); \
    case 8: return wave_launch<V, DK, 8>(ctx, dim, p, n, q, m, out_dist, out_dist2, s, sh.W, sh.ctas, check); \
    default: return DFD_ERR_UNSUPPORTED;                                                     \
  }
#define DFD_W_DK(V)              \
  switch (dk) {                  \
    case 2: DFD_W_R(V, 2)        \
    case 3: DFD_W_R(V, 3)        \
    case 4: DFD_W_R(V, 4)        \
    case 8: DFD_W_R(V, 8)        \
    case 16: DFD_W_R(V, 16)      \
    default: return DFD_ERR_UNSUPPORTED; \
  }
  if (dtype == DFD_F32) {
    DFD_W_DK(F32)
  } else {
    DFD_W_DK(I32)
  }
#undef DFD_W_DK
#undef DFD_W_R
}

dfd_status batch_run(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                     int64_t n_curves, const int32_t* pairs, int64_t n_pairs, void* out_dist, void* out_dist2,
                     cudaStream_t s) {
#define DFD_B_DK(V)                                                                                           \
  switch (dim_class(dim)) {                                                                                   \
    case 2: return batch_launch<V, 2>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, out_dist, out_dist2, s); \
    case 3: return batch_launch<V, 3>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, out_dist, out_dist2, s); \
    case 4: return batch_launch<V, 4>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, out_dist, out_dist2, s); \
    case 8: return batch_launch<V, 8>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, out_dist, out_dist2, s); \
    case 16: return batch_launch<V, 16>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, out_dist, out_dist2, s); \
    default: return DFD_ERR_UNSUPPORTED;                                                                      \
  }
  if (dtype == DFD_F32) {
    DFD_B_DK(F32)
  } else {
    DFD_B_DK(I32)
  }
#undef DFD_B_DK
}

static dfd_status decide_run(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                             int64_t n_curves, const int32_t* pairs, int64_t n_pairs, const void* eps2,
                             double eps2_all, void* out_dist2, int32_t* within, unsigned long long* abandoned,
                             cudaStream_t s) {
#define DFD_D_CALL(V, DK) \
  return decide_launch<V, DK>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, eps2, eps2_all, out_dist2, within, \
                              abandoned, s)
#define DFD_D_DK(V)                \
  switch (dim_class(dim)) {        \
    case 2: DFD_D_CALL(V, 2);      \
    case 3: DFD_D_CALL(V, 3);      \
    case 4: DFD_D_CALL(V, 4);      \
    case 8: DFD_D_CALL(V, 8);      \
    case 16: DFD_D_CALL(V, 16);    \
    default: return DFD_ERR_UNSUPPORTED; \
  }
  if (dtype == DFD_F32) {
    DFD_D_DK(F32)
  } else {
    DFD_D_DK(I32)
  }
#undef DFD_D_DK
#undef DFD_D_CALL
}

dfd_status matrix_run(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                      int64_t n_curves, void* out_dist, void* out_dist2, cudaStream_t s, int chunk) {
#define DFD_M_DK(V)                                                                                      \
  switch (dim_class(dim)) {                                                                              \
    case 2: return matrix_launch<V, 2>(ctx, dim, points, offsets, n_curves, out_dist, out_dist2, s, chunk);   \
    case 3: return matrix_launch<V, 3>(ctx, dim, points, offsets, n_curves, out_dist, out_dist2, s, chunk);   \
    case 4: return matrix_launch<V, 4>(ctx, dim, points, offsets, n_curves, out_dist, out_dist2, s, chunk);   \
    case 8: return matrix_launch<V, 8>(ctx, dim, points, offsets, n_curves, out_dist, out_dist2, s, chunk);   \
    case 16: return matrix_launch<V, 16>(ctx, dim, points, offsets, n_curves, out_dist, out_dist2, s, chunk); \
    default: return DFD_ERR_UNSUPPORTED;                                                                 \
  }
  if (dtype == DFD_F32) {
    DFD_M_DK(F32)
  } else {
    DFD_M_DK(I32)
  }
#undef DFD_M_DK
}

__global__ void bounded_wait_kernel(const unsigned long long* flag, int* err, unsigned long long timeout_ns) {
  if (threadIdx.x == 0) wait_geq(flag, 1ull, err, timeout_ns);
}

}  // namespace dfd

dfd_status dfd::set_device(dfd_context* ctx) { return cuda_status(cudaSetDevice(ctx->device)); }

dfd_status dfd::check_batch_args(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                            int64_t n_curves, const void* out_dist, const void* out_dist2) {
  if (!ctx) return DFD_ERR_INVALID_ARG;
  if (dtype != DFD_F32 && dtype != DFD_I32) return DFD_ERR_INVALID_ARG;
  if (dim < 1 || !points || !offsets || n_curves < 1) return DFD_ERR_INVALID_ARG;
  if (!out_dist && !out_dist2) return DFD_ERR_INVALID_ARG;
  if (dim > 16) return DFD_ERR_UNSUPPORTED;
  if (n_curves > INT32_MAX) return DFD_ERR_UNSUPPORTED;
  return DFD_OK;
}

using namespace dfd;

// ======================================================================= C ABI
namespace {

dfd_status check_pair_args(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q,
                           int64_t m, const void* out_dist, const void* out_dist2) {
  if (!ctx) return DFD_ERR_INVALID_ARG;
  if (dtype != DFD_F32 && dtype != DFD_I32) return DFD_ERR_INVALID_ARG;
  if (dim < 1 || !p || !q || n < 1 || m < 1) return DFD_ERR_INVALID_ARG;
  if (!out_dist && !out_dist2) return DFD_ERR_INVALID_ARG;
  if (dim > 16) return DFD_ERR_UNSUPPORTED;
  if (m > (int64_t)1 << 29 || n > ((int64_t)1 << 40)) return DFD_ERR_UNSUPPORTED;
  return DFD_OK;
}


dfd_status pre_checks(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q, int64_t m,
                      cudaStream_t s) {
  if (!ctx->opt.check_inputs) return DFD_OK;
  return launch_check_inputs2(dtype, dim, p, n * dim, q, m * dim, ctx->d_err, s);
}

}  // namespace

extern "C" {

dfd_status dfd_options_default(dfd_options* opt) {
  if (!opt) return DFD_ERR_INVALID_ARG;
  std::memset(opt, 0, sizeof(*opt));
  opt->struct_size = sizeof(dfd_options);
  opt->mem_budget_bytes = 0;
  opt->max_slots = 0;
  opt->wait_timeout_ms = 2000.0;
  opt->check_inputs = 1;
  return DFD_OK;
}

const char* dfd_status_string(dfd_status s) {
  switch (s) {
    case DFD_OK: return "DFD_OK";
    case DFD_ERR_INVALID_ARG: return "DFD_ERR_INVALID_ARG";
    case DFD_ERR_RANGE: return "DFD_ERR_RANGE";
    case DFD_ERR_NONFINITE: return "DFD_ERR_NONFINITE";
    case DFD_ERR_OOM: return "DFD_ERR_OOM";
    case DFD_ERR_CUDA: return "DFD_ERR_CUDA";
    case DFD_ERR_TIMEOUT: return "DFD_ERR_TIMEOUT";
    case DFD_ERR_BUSY: return "DFD_ERR_BUSY";
    case DFD_ERR_CANCELLED: return "DFD_ERR_CANCELLED";
    case DFD_ERR_NOT_READY: return "DFD_ERR_NOT_READY";
    case DFD_ERR_UNSUPPORTED: return "DFD_ERR_UNSUPPORTED";
    case DFD_ERR_CAPACITY: return "DFD_ERR_CAPACITY";
  }
  return "DFD_ERR_UNKNOWN";
}

dfd_status dfd_context_create(dfd_context** out, int device, const dfd_options* opt) {
  if (!out) return DFD_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) {
    cudaGetLastError();
    return DFD_ERR_CUDA;
  }
  if (device < 0 || device >= count) return DFD_ERR_INVALID_ARG;
  dfd_context* ctx = new (std::nothrow) dfd_context();
  if (!ctx) return DFD_ERR_OOM;
  dfd_options_default(&ctx->opt);
  if (opt) {
    if (opt->struct_size != sizeof(dfd_options)) {
      delete ctx;
      return DFD_ERR_INVALID_ARG;
    }
    ctx->opt = *opt;
    if (ctx->opt.wait_timeout_ms <= 0) ctx->opt.wait_timeout_ms = 2000.0;
  }
  ctx->device = device;
  dfd_status st = set_device(ctx);
  if (st == DFD_OK) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) st = DFD_ERR_CUDA;
    else {
      ctx->num_sms = prop.multiProcessorCount;
      ctx->smem_optin = prop.sharedMemPerBlockOptin;
    }
  }
  if (st == DFD_OK && cudaMalloc(&ctx->d_err, 256) != cudaSuccess) st = DFD_ERR_OOM;
  if (st == DFD_OK && cudaMemset(ctx->d_err, 0, 256) != cudaSuccess) st = DFD_ERR_CUDA;
  if (st == DFD_OK && cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) st = DFD_ERR_CUDA;
  if (st != DFD_OK) {
    cudaGetLastError();
    if (ctx->d_err) cudaFree(ctx->d_err);
    delete ctx;
    return st;
  }
  *out = ctx;
  return DFD_OK;
}

dfd_status dfd_context_destroy(dfd_context* ctx) {
  if (!ctx) return DFD_OK;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  for (cudaEvent_t e : ctx->slice_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->launch_stream2) cudaStreamDestroy(ctx->launch_stream2);
  for (cudaEvent_t e : ctx->prep_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  if (ctx->scratch) cudaFree(ctx->scratch);
  if (ctx->io) cudaFree(ctx->io);
  if (ctx->host_scr) cudaFree(ctx->host_scr);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->d_err) cudaFree(ctx->d_err);
  cudaGetLastError();
  delete ctx;
  return DFD_OK;
}

dfd_status dfd_get_error(dfd_context* ctx) {
  if (!ctx) return DFD_ERR_INVALID_ARG;
  dfd_status st = set_device(ctx);
  if (st != DFD_OK) return st;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_CUDA;
  }
  int v = 0;
  if (cudaMemcpy(&v, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DFD_ERR_CUDA;
  if (v != 0 && cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) return DFD_ERR_CUDA;
  return (dfd_status)v;
}

dfd_status dfd_timing_enable(dfd_context* ctx, int on) {
  if (!ctx) return DFD_ERR_INVALID_ARG;
  dfd_status st = set_device(ctx);
  if (st != DFD_OK) return st;
  if (on && !ctx->ev0) {
    if (cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess) {
      cudaGetLastError();
      return DFD_ERR_CUDA;
    }
  }
  ctx->timing = on != 0;
  ctx->timed = false;
  return DFD_OK;
}

dfd_status dfd_timing_last(dfd_context* ctx, double* ms) {
  if (!ctx || !ms) return DFD_ERR_INVALID_ARG;
  if (!ctx->timing || !ctx->timed) return DFD_ERR_NOT_READY;
  if (cudaEventSynchronize(ctx->ev1) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_CUDA;
  }
  float f = 0.f;
  if (cudaEventElapsedTime(&f, ctx->ev0, ctx->ev1) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_CUDA;
  }
  *ms = f;
  return DFD_OK;
}

dfd_status dfd_pair_autotune(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q,
                             int64_t m, void* stream, dfd_wave_shape* best_out) {
  dfd_status st = check_pair_args(ctx, dtype, dim, p, n, q, m, p, nullptr);
  if (st != DFD_OK) return st;
  if ((st = set_device(ctx)) != DFD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Candidates: rows per lane {4, 6, 8} x compute warps 2..10, keeping those
  // whose band count is at most two waves of the SMs.
  void* res = nullptr;
  if (cudaMallocAsync(&res, 16, s) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_OOM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    cudaFreeAsync(res, s);
    return DFD_ERR_CUDA;
  }
  WaveShape best;
  wave_plan(ctx, dtype, dim, n, m, &best);
  float best_ms = 1e30f;
  const int Rs[3] = {4, 6, 8};
  for (int R : Rs) {
    for (int W = 2; W <= 10; ++W) {
      if (!shape_ok(ctx, dtype, dim, R, W)) continue;
      const int64_t H = (int64_t)32 * W * R;
      const int64_t B = (n + H - 1) / H;
      if (B > 2 * (int64_t)ctx->num_sms * wave::blocks_per_sm(dim_class(dim)) || (B < ctx->num_sms / 2 && W > 2))
        continue;
      // one CTA per SM, and (bands permitting) every CTA that can be resident
      const int grids[2] = {(int)std::min<int64_t>(B, ctx->num_sms), 0};
      for (int g = 0; g < (B > ctx->num_sms ? 2 : 1); ++g) {
        WaveShape sh;
        sh.R = R;
        sh.W = W;
        sh.ctas = grids[g];
        cudaEventRecord(e0, s);
        st = wave_run(ctx, dtype, dim, p, n, q, m, res, nullptr, s, sh, false);
        cudaEventRecord(e1, s);
        if (st != DFD_OK) continue;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          cudaGetLastError();
          continue;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
          best_ms = ms;
          best = sh;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(res, s);
  cudaStreamSynchronize(s);
  ctx->tuned[tune_key(dtype, dim_class(dim), n, m)] = best;
  if (best_out) {
    best_out->rows_per_lane = best.R;
    best_out->warps = best.W;
    best_out->ctas = best.ctas;
  }
  return DFD_OK;
}

dfd_status dfd_autotune_save(dfd_context* ctx, const char* path) {
  if (!ctx || !path) return DFD_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "w");
  if (!f) return DFD_ERR_INVALID_ARG;
  std::fprintf(f, "# dfd wavefront tuning: key rows_per_lane warps ctas\n");
  for (const auto& kv : ctx->tuned)
    std::fprintf(f, "%llu %d %d %d\n", (unsigned long long)kv.first, kv.second.R, kv.second.W, kv.second.ctas);
  std::fclose(f);
  return DFD_OK;
}

dfd_status dfd_autotune_load(dfd_context* ctx, const char* path) {
  if (!ctx || !path) return DFD_ERR_INVALID_ARG;
  FILE* f = std::fopen(path, "r");
  if (!f) return DFD_ERR_INVALID_ARG;
  char line[256];
  while (std::fgets(line, sizeof line, f)) {
    if (line[0] == '#') continue;
    unsigned long long key = 0;
    WaveShape sh;
    if (std::sscanf(line, "%llu %d %d %d", &key, &sh.R, &sh.W, &sh.ctas) == 4) ctx->tuned[(uint64_t)key] = sh;
  }
  std::fclose(f);
  return DFD_OK;
}

dfd_status dfd_debug_bounded_wait(dfd_context* ctx, double timeout_ms) {
  if (!ctx || !(timeout_ms > 0) || timeout_ms > 60000.0) return DFD_ERR_INVALID_ARG;
  dfd_status st = set_device(ctx);
  if (st != DFD_OK) return st;
  // ctx->d_err[0] is the error word; d_err[2..3] (8-byte aligned) is a flag
  // that stays zero.
  unsigned long long* flag = reinterpret_cast<unsigned long long*>(ctx->d_err + 2);
  if (cudaMemsetAsync(flag, 0, sizeof(*flag), ctx->stream) != cudaSuccess) return DFD_ERR_CUDA;
  bounded_wait_kernel<<<1, 32, 0, ctx->stream>>>(flag, ctx->d_err, (unsigned long long)(timeout_ms * 1.0e6));
  if (cudaGetLastError() != cudaSuccess) return DFD_ERR_CUDA;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_CUDA;
  }
  int v = 0;
  if (cudaMemcpy(&v, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DFD_ERR_CUDA;
  cudaMemset(ctx->d_err, 0, sizeof(int));
  return (dfd_status)v;
}

dfd_status dfd_pair_plan(dfd_context* ctx, dfd_dtype dtype, int dim, int64_t n, int64_t m, dfd_wave_shape* shape) {
  if (!ctx || !shape || n < 1 || m < 1 || dim < 1) return DFD_ERR_INVALID_ARG;
  WaveShape sh;
  dfd_status st = wave_plan(ctx, dtype, dim, n, m, &sh);
  if (st != DFD_OK) return st;
  shape->rows_per_lane = sh.R;
  shape->warps = sh.W;
  shape->ctas = sh.ctas;
  return DFD_OK;
}

dfd_status dfd_pair_shaped(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q,
                           int64_t m, void* out_dist, void* out_dist2, void* stream, const dfd_wave_shape* shape) {
  dfd_status st = check_pair_args(ctx, dtype, dim, p, n, q, m, out_dist, out_dist2);
  if (st != DFD_OK) return st;
  WaveShape sh;
  if (shape) {
    sh.R = shape->rows_per_lane;
    sh.W = shape->warps;
    sh.ctas = shape->ctas;
    if (sh.ctas < 0 || sh.ctas > ctx->num_sms * wave::blocks_per_sm(dim_class(dim))) return DFD_ERR_UNSUPPORTED;
  } else {
    wave_plan(ctx, dtype, dim, n, m, &sh);
  }
  if ((st = set_device(ctx)) != DFD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the input checks run in the wavefront's prep kernel
  return wave_run(ctx, dtype, dim, p, n, q, m, out_dist, out_dist2, s, sh, ctx->opt.check_inputs != 0);
}

dfd_status dfd_pair(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q, int64_t m,
                    void* out_dist, void* out_dist2, void* stream) {
  return dfd_pair_shaped(ctx, dtype, dim, p, n, q, m, out_dist, out_dist2, stream, nullptr);
}

dfd_status dfd_pair_reference(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q,
                              int64_t m, void* out_dist, void* out_dist2, void* stream) {
  dfd_status st = check_pair_args(ctx, dtype, dim, p, n, q, m, out_dist, out_dist2);
  if (st != DFD_OK) return st;
  if ((st = set_device(ctx)) != DFD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = pre_checks(ctx, dtype, dim, p, n, q, m, s)) != DFD_OK) return st;
  return rowscan_run(ctx, dtype, dim, p, n, q, m, out_dist, out_dist2, s);
}

dfd_status dfd_pair_host(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q, int64_t m,
                         void* out_dist, void* out_dist2) {
  dfd_status st = check_pair_args(ctx, dtype, dim, p, n, q, m, out_dist, out_dist2);
  if (st != DFD_OK) return st;
  if ((st = set_device(ctx)) != DFD_OK) return st;
  // Device layout of the staged inputs and results: [p | q | dist | dist2],
  // carved from the pinned host area and from a second device buffer that
  // sits after the wavefront's scratch (which it grows first).  Inputs the
  // caller already holds in page-locked memory are copied to the device
  // directly; pageable ones go through the pinned area first.
  const size_t pb = align_up((size_t)n * dim * 4, 256), qb = align_up((size_t)m * dim * 4, 256);
  const size_t host_bytes = pb + qb + 256;
  if ((st = ensure_pinned(ctx, host_bytes)) != DFD_OK) return st;
  char* h = static_cast<char*>(ctx->pinned);
  auto page_locked = [](const void* x) {
    cudaPointerAttributes at;
    const bool yes = cudaPointerGetAttributes(&at, x) == cudaSuccess && at.type == cudaMemoryTypeHost;
    cudaGetLastError();
    return yes;
  };
  const bool p_locked = page_locked(p), q_locked = page_locked(q);
  if (!p_locked) std::memcpy(h, p, (size_t)n * dim * 4);
  if (!q_locked) std::memcpy(h + pb, q, (size_t)m * dim * 4);
  if ((st = ensure_io(ctx, host_bytes)) != DFD_OK) return st;
  char* d = static_cast<char*>(ctx->io);
  cudaStream_t s = ctx->stream;
  cudaMemcpyAsync(d, p_locked ? p : h, (size_t)n * dim * 4, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d + pb, q_locked ? q : h + pb, (size_t)m * dim * 4, cudaMemcpyHostToDevice, s);
  WaveShape sh;
  wave_plan(ctx, dtype, dim, n, m, &sh);
  {
    char* dres = d + pb + qb;
    st = wave_run(ctx, dtype, dim, d, n, d + pb, m, dres, dres + 8, s, sh, ctx->opt.check_inputs != 0);
    if (st == DFD_OK) {
      cudaMemcpyAsync(h + pb + qb, dres, 16, cudaMemcpyDeviceToHost, s);
    }
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_CUDA;
  }
  if (st != DFD_OK) return st;
  int err = 0;
  cudaMemcpy(&err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (err != 0) {
    cudaMemset(ctx->d_err, 0, sizeof(int));
    return (dfd_status)err;
  }
  const char* r = h + pb + qb;
  if (dtype == DFD_F32) {
    if (out_dist) std::memcpy(out_dist, r, 4);
    if (out_dist2) std::memcpy(out_dist2, r + 8, 4);
  } else {
    if (out_dist) std::memcpy(out_dist, r, 8);
    if (out_dist2) std::memcpy(out_dist2, r + 8, 8);
  }
  return DFD_OK;
}

}  // extern "C"

// ============================================================ batch / matrix
struct dfd_graph {
  dfd_context* ctx = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* scratch = nullptr;   // owned: the captured launches point into it
};

namespace {


// Run `fn` once normally (sizes the context scratch), then capture it into a
// graph that owns a private copy of the scratch, so later calls that grow or
// reuse the context scratch cannot disturb the graph's buffers.
template <class F>
dfd_status capture_graph(dfd_context* ctx, F fn, dfd_graph** out) {
  dfd_status st = fn(ctx->stream);
  if (st != DFD_OK) return st;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_CUDA;
  }
  dfd_graph* g = new (std::nothrow) dfd_graph();
  if (!g) return DFD_ERR_OOM;
  g->ctx = ctx;
  if (cudaMalloc(&g->scratch, ctx->scratch_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete g;
    return DFD_ERR_OOM;
  }
  void* saved = ctx->scratch;
  ctx->scratch = g->scratch;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    st = fn(ctx->stream);
    cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &graph);
    if (st == DFD_OK && e2 != cudaSuccess) st = DFD_ERR_CUDA;
  } else {
    st = DFD_ERR_CUDA;
  }
  ctx->scratch = saved;
  if (st == DFD_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) st = DFD_ERR_CUDA;
  if (graph) cudaGraphDestroy(graph);
  if (st != DFD_OK) {
    cudaGetLastError();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    cudaFree(g->scratch);
    delete g;
    return st;
  }
  *out = g;
  return DFD_OK;
}

}  // namespace

extern "C" {

dfd_status dfd_batch(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                     int64_t n_curves, const int32_t* pairs, int64_t n_pairs, void* out_dist, void* out_dist2,
                     void* stream) {
  dfd_status st = check_batch_args(ctx, dtype, dim, points, offsets, n_curves, out_dist, out_dist2);
  if (st != DFD_OK) return st;
  if (!pairs || n_pairs < 0 || n_pairs > INT32_MAX) return DFD_ERR_INVALID_ARG;
  if (n_pairs == 0) return DFD_OK;
  if ((st = set_device(ctx)) != DFD_OK) return st;
  return batch_run(ctx, dtype, dim, points, offsets, n_curves, pairs, n_pairs, out_dist, out_dist2,
                   static_cast<cudaStream_t>(stream));
}

dfd_status dfd_batch_set_order(dfd_context* ctx, dfd_dtype dtype, int dim, int order) {
  if (!ctx || (dtype != DFD_F32 && dtype != DFD_I32) || dim < 1 || (order != 0 && order != 1))
    return DFD_ERR_INVALID_ARG;
  if (dim > 16) return DFD_ERR_UNSUPPORTED;
  ctx->batch_order[dtype == DFD_F32 ? 0 : 1][dim_class_index(dim_class(dim))] = (signed char)order;
  return DFD_OK;
}

dfd_status dfd_batch_set_team(dfd_context* ctx, dfd_dtype dtype, int dim, int mode) {
  if (!ctx || (dtype != DFD_F32 && dtype != DFD_I32) || dim < 1 || mode < 0 || mode > 2) return DFD_ERR_INVALID_ARG;
  if (dim > 16) return DFD_ERR_UNSUPPORTED;
  ctx->batch_team[dtype == DFD_F32 ? 0 : 1][dim_class_index(dim_class(dim))] = (signed char)mode;
  return DFD_OK;
}

dfd_status dfd_batch_set_row_buffer(dfd_context* ctx, int cols) {
  // whole 32-column blocks; the widest a warp's row index reaches is INT32_MAX
  if (!ctx || cols < kDefaultBatchBufCols || cols > (1 << 28)) return DFD_ERR_INVALID_ARG;
  ctx->batch_buf_cols = (cols + 31) / 32 * 32;
  return DFD_OK;
}

dfd_status dfd_batch_autotune(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                              int64_t n_curves, const int32_t* pairs, int64_t n_pairs, void* out_dist,
                              void* out_dist2, int* best_order, void* stream) {
  dfd_status st = check_batch_args(ctx, dtype, dim, points, offsets, n_curves, out_dist, out_dist2);
  if (st != DFD_OK) return st;
  if (!pairs || n_pairs < 0 || n_pairs > INT32_MAX) return DFD_ERR_INVALID_ARG;
  if ((st = set_device(ctx)) != DFD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int ti = dtype == DFD_F32 ? 0 : 1, di = dim_class_index(dim_class(dim));
  signed char& slot = ctx->batch_order[ti][di];
  signed char& tslot = ctx->batch_team[ti][di];
  signed char& rslot = ctx->batch_rmax[ti][di];
  signed char& cslot = ctx->batch_cpsm[ti][di];
  const signed char keep = slot, tkeep = tslot, rkeep = rslot, ckeep = cslot;
  const int rm_full = dim_class(dim) <= 4 ? 8 : 4;   // batch::Rmax of the dim class
  const int cp_full = dim_class(dim) >= 16 ? 1 : 2;  // CTAs per SM of its launch bounds
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_CUDA;
  }
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(e0);
    return DFD_ERR_CUDA;
  }
  float best_ms = 0.f;
  int best = keep, best_team = tkeep, best_rm = rkeep, best_cp = ckeep;
  // packing order x team mode (1: only pairs too wide for a warp's buffer
  // run as CTA teams, 2: every pair of several stripes does) x tile shape
  // (rows per lane cap Rmax or Rmax / 2, CTAs per SM 1 or all)
  for (int c = 0; c < 16 && st == DFD_OK && n_pairs > 0; ++c) {
    const int order = c & 1, team = 1 + ((c >> 1) & 1);
    const int rm = (c >> 2) & 1 ? rm_full / 2 : rm_full, cp = (c >> 3) & 1 ? 1 : cp_full;
    if (cp_full == 1 && cp == 1 && (c >> 3) & 1) continue;   // one CTA per SM is the only shape
    slot = (signed char)order;
    tslot = (signed char)team;
    rslot = (signed char)rm;
    cslot = (signed char)cp;
    // one untimed run (sizes the scratch), then three timed
    st = batch_run(ctx, dtype, dim, points, offsets, n_curves, pairs, n_pairs, out_dist, out_dist2, s);
    if (st != DFD_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3 && st == DFD_OK; ++r)
      st = batch_run(ctx, dtype, dim, points, offsets, n_curves, pairs, n_pairs, out_dist, out_dist2, s);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (st == DFD_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      st = DFD_ERR_CUDA;
    if (st == DFD_OK && (c == 0 || ms < best_ms)) {
      best_ms = ms;
      best = order;
      best_team = team;
      best_rm = rm;
      best_cp = cp;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  const bool ok = st == DFD_OK;
  slot = (signed char)(ok ? best : keep);
  tslot = (signed char)(ok ? best_team : tkeep);
  rslot = (signed char)(ok ? best_rm : rkeep);
  cslot = (signed char)(ok ? best_cp : ckeep);
  if (best_order) *best_order = slot;
  return st;
}

dfd_status dfd_batch_tuned(dfd_context* ctx, dfd_dtype dtype, int dim, int* order, int* team, int* rows_per_lane,
                           int* ctas_per_sm) {
  if (!ctx || (dtype != DFD_F32 && dtype != DFD_I32) || dim < 1) return DFD_ERR_INVALID_ARG;
  if (dim > 16) return DFD_ERR_UNSUPPORTED;
  const int t = dtype == DFD_F32 ? 0 : 1, d = dim_class_index(dim_class(dim));
  if (order) *order = ctx->batch_order[t][d];
  if (team) *team = ctx->batch_team[t][d];
  if (rows_per_lane) *rows_per_lane = ctx->batch_rmax[t][d];
  if (ctas_per_sm) *ctas_per_sm = ctx->batch_cpsm[t][d];
  return DFD_OK;
}

dfd_status dfd_batch_set_shape(dfd_context* ctx, dfd_dtype dtype, int dim, int rows_per_lane, int ctas_per_sm) {
  if (!ctx || (dtype != DFD_F32 && dtype != DFD_I32) || dim < 1 || rows_per_lane < 0 || rows_per_lane > 8 ||
      ctas_per_sm < 0 || ctas_per_sm > 2)
    return DFD_ERR_INVALID_ARG;
  if (dim > 16) return DFD_ERR_UNSUPPORTED;
  const int t = dtype == DFD_F32 ? 0 : 1, d = dim_class_index(dim_class(dim));
  ctx->batch_rmax[t][d] = (signed char)rows_per_lane;
  ctx->batch_cpsm[t][d] = (signed char)ctas_per_sm;
  return DFD_OK;
}

dfd_status dfd_matrix_set_shape(dfd_context* ctx, dfd_dtype dtype, int dim, int rows_per_lane, int ctas_per_sm) {
  if (!ctx || (dtype != DFD_F32 && dtype != DFD_I32) || dim < 1 || rows_per_lane < 0 || rows_per_lane > 8 ||
      ctas_per_sm < 0 || ctas_per_sm > 2)
    return DFD_ERR_INVALID_ARG;
  if (dim > 16) return DFD_ERR_UNSUPPORTED;
  const int t = dtype == DFD_F32 ? 0 : 1, d = dim_class_index(dim_class(dim));
  ctx->matrix_rmax[t][d] = (signed char)rows_per_lane;
  ctx->matrix_cpsm[t][d] = (signed char)ctas_per_sm;
  return DFD_OK;
}

dfd_status dfd_matrix_tuned(dfd_context* ctx, dfd_dtype dtype, int dim, int* rows_per_lane, int* ctas_per_sm) {
  if (!ctx || (dtype != DFD_F32 && dtype != DFD_I32) || dim < 1) return DFD_ERR_INVALID_ARG;
  if (dim > 16) return DFD_ERR_UNSUPPORTED;
  const int t = dtype == DFD_F32 ? 0 : 1, d = dim_class_index(dim_class(dim));
  if (rows_per_lane) *rows_per_lane = ctx->matrix_rmax[t][d];
  if (ctas_per_sm) *ctas_per_sm = ctx->matrix_cpsm[t][d];
  return DFD_OK;
}

dfd_status dfd_batch_decide(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                            int64_t n_curves, const int32_t* pairs, int64_t n_pairs, const void* eps2,
                            double eps2_all, void* out_dist2, int32_t* out_within, unsigned long long* abandoned,
                            void* stream) {
  dfd_status st = check_batch_args(ctx, dtype, dim, points, offsets, n_curves, out_within ? (void*)out_within : out_dist2,
                                   out_dist2);
  if (st != DFD_OK) return st;
  if (!pairs || n_pairs < 0 || n_pairs > INT32_MAX) return DFD_ERR_INVALID_ARG;
  if (!eps2 && std::isnan(eps2_all)) return DFD_ERR_INVALID_ARG;
  if (n_pairs == 0) return DFD_OK;
  if ((st = set_device(ctx)) != DFD_OK) return st;
  double e = eps2_all;
  if (dtype == DFD_F32 && !eps2 && std::isfinite(e)) {
    // largest float <= eps2_all, so that (float) delta^2 <= it  <=>  delta^2 <= eps2_all
    float f = (float)e;
    if ((double)f > e) f = std::nextafter(f, -INFINITY);
    e = (double)f;
  }
  return decide_run(ctx, dtype, dim, points, offsets, n_curves, pairs, n_pairs, eps2, e, out_dist2, out_within,
                    abandoned, static_cast<cudaStream_t>(stream));
}

dfd_status dfd_matrix(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                      int64_t n_curves, void* out_condensed, void* out_dist2, void* stream) {
  dfd_status st = check_batch_args(ctx, dtype, dim, points, offsets, n_curves, out_condensed, out_dist2);
  if (st != DFD_OK) return st;
  if (n_curves < 2) return DFD_OK;
  if ((st = set_device(ctx)) != DFD_OK) return st;
  return matrix_run(ctx, dtype, dim, points, offsets, n_curves, out_condensed, out_dist2,
                    static_cast<cudaStream_t>(stream), 0);
}

dfd_status dfd_matrix_autotune(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                               int64_t n_curves, void* out_condensed, void* out_dist2, int* best_rows_per_lane,
                               int* best_ctas_per_sm, void* stream) {
  dfd_status st = check_batch_args(ctx, dtype, dim, points, offsets, n_curves, out_condensed, out_dist2);
  if (st != DFD_OK) return st;
  if ((st = set_device(ctx)) != DFD_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int ti = dtype == DFD_F32 ? 0 : 1, di = dim_class_index(dim_class(dim));
  signed char& rslot = ctx->matrix_rmax[ti][di];
  signed char& cslot = ctx->matrix_cpsm[ti][di];
  const signed char rkeep = rslot, ckeep = cslot;
  const int rm_full = dim_class(dim) <= 4 ? 8 : 4;
  const int cp_full = dim_class(dim) >= 16 ? 1 : 2;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return DFD_ERR_CUDA;
  }
  float best_ms = 0.f;
  int best_rm = rkeep, best_cp = ckeep;
  bool any = false;
  // rows per lane cap Rmax, Rmax / 2, Rmax / 4 x CTAs per SM (all, 1)
  for (int c = 0; c < 6 && st == DFD_OK && n_curves >= 2; ++c) {
    const int rm = rm_full >> (c % 3), cp = c < 3 ? cp_full : 1;
    if (rm < 1 || (c >= 3 && cp_full == 1)) continue;
    rslot = (signed char)rm;
    cslot = (signed char)cp;
    st = matrix_run(ctx, dtype, dim, points, offsets, n_curves, out_condensed, out_dist2, s, 0);
    if (st != DFD_OK) break;
    cudaEventRecord(e0, s);
    for (int r = 0; r < 2 && st == DFD_OK; ++r)
      st = matrix_run(ctx, dtype, dim, points, offsets, n_curves, out_condensed, out_dist2, s, 0);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (st == DFD_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      st = DFD_ERR_CUDA;
    if (st == DFD_OK && (!any || ms < best_ms)) {
      best_ms = ms;
      best_rm = rm;
      best_cp = cp;
      any = true;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  rslot = (signed char)(st == DFD_OK ? best_rm : rkeep);
  cslot = (signed char)(st == DFD_OK ? best_cp : ckeep);
  if (best_rows_per_lane) *best_rows_per_lane = rslot;
  if (best_ctas_per_sm) *best_ctas_per_sm = cslot;
  return st;
}

dfd_status dfd_batch_capture(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                             int64_t n_curves, const int32_t* pairs, int64_t n_pairs, void* out_dist, void* out_dist2,
                             dfd_graph** out) {
  if (!out) return DFD_ERR_INVALID_ARG;
  *out = nullptr;
  dfd_status st = check_batch_args(ctx, dtype, dim, points, offsets, n_curves, out_dist, out_dist2);
  if (st != DFD_OK) return st;
  if (!pairs || n_pairs < 1 || n_pairs > INT32_MAX) return DFD_ERR_INVALID_ARG;
  if ((st = set_device(ctx)) != DFD_OK) return st;
  return capture_graph(
      ctx,
      [&](cudaStream_t s) {
        return batch_run(ctx, dtype, dim, points, offsets, n_curves, pairs, n_pairs, out_dist, out_dist2, s);
      },
      out);
}

dfd_status dfd_matrix_capture(dfd_context* ctx, dfd_dtype dtype, int dim, const void* points, const int64_t* offsets,
                              int64_t n_curves, void* out_condensed, void* out_dist2, dfd_graph** out) {
  if (!out) return DFD_ERR_INVALID_ARG;
  *out = nullptr;
  dfd_status st = check_batch_args(ctx, dtype, dim, points, offsets, n_curves, out_condensed, out_dist2);
  if (st != DFD_OK) return st;
  if (n_curves < 2) return DFD_ERR_INVALID_ARG;
  if ((st = set_device(ctx)) != DFD_OK) return st;
  return capture_graph(
      ctx,
      [&](cudaStream_t s) {
        return matrix_run(ctx, dtype, dim, points, offsets, n_curves, out_condensed, out_dist2, s, 0);
      },
      out);
}

dfd_status dfd_graph_launch(dfd_graph* g, void* stream) {
  if (!g || !g->exec) return DFD_ERR_INVALID_ARG;
  if (cudaSetDevice(g->ctx->device) != cudaSuccess) return DFD_ERR_CUDA;
  return cuda_status(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
}

dfd_status dfd_graph_destroy(dfd_graph* g) {
  if (!g) return DFD_OK;
  cudaSetDevice(g->ctx->device);
  cudaDeviceSynchronize();
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->scratch) cudaFree(g->scratch);
  cudaGetLastError();
  delete g;
  return DFD_OK;
}

}  // extern "C"
