// mc.cu -- Monte Carlo distance samples of a pair of uncertain curves (the
// application to uncertain curves named in Sec. 5): every sample perturbs
// both curves point-wise with the caller's noise, x' = fl(x + sigma * z)
// (one rounding, fmaf), and the batch engine computes all samples' discrete
// Frechet distances in one persistent launch (LPT order, one warp per
// sample).  The noise is an input, so a sample is reproducible bit for bit.
#include <algorithm>
#include "batch_launch.cuh"
#include "dfd_internal.h"

namespace dfd {
// instantiated in batch_f32_d*.cu
extern template dfd_status batch_launch<F32, 2>(dfd_context*, int, const void*, const int64_t*, int64_t, const int32_t*,
                                                int64_t, void*, void*, cudaStream_t);
extern template dfd_status batch_launch<F32, 3>(dfd_context*, int, const void*, const int64_t*, int64_t, const int32_t*,
                                                int64_t, void*, void*, cudaStream_t);
extern template dfd_status batch_launch<F32, 4>(dfd_context*, int, const void*, const int64_t*, int64_t, const int32_t*,
                                                int64_t, void*, void*, cudaStream_t);
extern template dfd_status batch_launch<F32, 8>(dfd_context*, int, const void*, const int64_t*, int64_t, const int32_t*,
                                                int64_t, void*, void*, cudaStream_t);
extern template dfd_status batch_launch<F32, 16>(dfd_context*, int, const void*, const int64_t*, int64_t,
                                                 const int32_t*, int64_t, void*, void*, cudaStream_t);

namespace mc {

// Sample s occupies curves 2s (p perturbed) and 2s+1 (q perturbed) of a CSR
// batch: points [s*(n+m), s*(n+m)+n) and [s*(n+m)+n, (s+1)*(n+m)).
__global__ void mc_build_kernel(const float* __restrict__ p, int64_t n, const float* __restrict__ q, int64_t m,
                                int dim, const float* __restrict__ zp, const float* __restrict__ zq, float sp,
                                float sq, int64_t S, float* pts, int64_t* offsets, int32_t* pairs) {
  const int64_t per = (n + m) * dim;
  const int64_t total = S * per;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / per, r = i % per;
    if (r < n * dim)
      pts[i] = __fmaf_rn(sp, zp[s * n * dim + r], p[r]);
    else
      pts[i] = __fmaf_rn(sq, zq[s * m * dim + (r - n * dim)], q[r - n * dim]);
  }
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s <= S; s += (int64_t)gridDim.x * blockDim.x) {
    offsets[2 * s] = s * (n + m);
    if (s < S) {
      offsets[2 * s + 1] = s * (n + m) + n;
      pairs[2 * s] = (int32_t)(2 * s);
      pairs[2 * s + 1] = (int32_t)(2 * s + 1);
    }
  }
}

template <int DK>
dfd_status mc_launch(dfd_context* ctx, int dim, const float* p, int64_t n, const float* q, int64_t m,
                     const float* zp, const float* zq, float sp, float sq, int64_t S, float* out_dist2,
                     float* out_dist, cudaStream_t s) {
  // stream-ordered buffers for the samples (freed after the launch, in order)
  const size_t pts_bytes = align_up((size_t)S * (n + m) * dim * sizeof(float), 256);
  const size_t off_bytes = align_up((size_t)(2 * S + 1) * sizeof(int64_t), 256);
  const size_t pair_bytes = align_up((size_t)S * 2 * sizeof(int32_t), 256);
  char* buf = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf), pts_bytes + off_bytes + pair_bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_OOM;
  }
  float* pts = reinterpret_cast<float*>(buf);
  int64_t* offsets = reinterpret_cast<int64_t*>(buf + pts_bytes);
  int32_t* pairs = reinterpret_cast<int32_t*>(buf + pts_bytes + off_bytes);
  const int64_t total = S * (n + m) * dim;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 8 * (int64_t)ctx->num_sms));
  mc_build_kernel<<<blocks, 256, 0, s>>>(p, n, q, m, dim, zp, zq, sp, sq, S, pts, offsets, pairs);
  dfd_status st = cuda_status(cudaGetLastError());
  if (st == DFD_OK) st = batch_launch<F32, DK>(ctx, dim, pts, offsets, 2 * S, pairs, S, out_dist, out_dist2, s);
  cudaFreeAsync(buf, s);
  return st;
}

}  // namespace mc
}  // namespace dfd

using namespace dfd;

extern "C" dfd_status dfd_mc_pair(dfd_context* ctx, int dim, const float* p, int64_t n, const float* q, int64_t m,
                                  const float* noise_p, const float* noise_q, float sigma_p, float sigma_q,
                                  int64_t n_samples, float* out_dist2, float* out_dist, void* stream) {
  if (!ctx || !p || !q || !noise_p || !noise_q || n < 1 || m < 1 || dim < 1 || n_samples < 0)
    return DFD_ERR_INVALID_ARG;
  if (!out_dist2 && !out_dist) return DFD_ERR_INVALID_ARG;
  if (dim > 16) return DFD_ERR_UNSUPPORTED;
  if (2 * n_samples >= INT32_MAX || (n + m) * n_samples > INT32_MAX) return DFD_ERR_UNSUPPORTED;
  if (n_samples == 0) return DFD_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (dim_class(dim)) {
    case 2: return mc::mc_launch<2>(ctx, dim, p, n, q, m, noise_p, noise_q, sigma_p, sigma_q, n_samples, out_dist2, out_dist, s);
    case 3: return mc::mc_launch<3>(ctx, dim, p, n, q, m, noise_p, noise_q, sigma_p, sigma_q, n_samples, out_dist2, out_dist, s);
    case 4: return mc::mc_launch<4>(ctx, dim, p, n, q, m, noise_p, noise_q, sigma_p, sigma_q, n_samples, out_dist2, out_dist, s);
    case 8: return mc::mc_launch<8>(ctx, dim, p, n, q, m, noise_p, noise_q, sigma_p, sigma_q, n_samples, out_dist2, out_dist, s);
    case 16: return mc::mc_launch<16>(ctx, dim, p, n, q, m, noise_p, noise_q, sigma_p, sigma_q, n_samples, out_dist2, out_dist, s);
    default: return DFD_ERR_UNSUPPORTED;
  }
}
