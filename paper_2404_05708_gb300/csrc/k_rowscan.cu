// k_rowscan.cu -- K1: the plain per-pair reference form.
//
// One CTA computes the recurrence of Eq. 1 row by row, in the order of
// Alg. 5 / Alg. 2: for row i, the vertical step a_j = min(M_{i-1,j-1},
// M_{i-1,j}) is elementwise; the horizontal step M_ij = max(d_ij, min(a_j,
// M_{i,j-1})) is a left-to-right scan of the clamp functions
// f_j(x) = max(d_j, min(a_j, x)).  The paper notes its maxmin operator is not
// associative (Sec. 4); the clamp functions it induces are, under
// composition, so the row scan runs in parallel: each thread composes the
// clamps of its column segment, a block-wide exclusive scan of those
// compositions gives every thread its incoming left value, and the thread
// then applies its clamps in order.  Rows alternate between two global
// buffers of m values (O(m) scratch).  Only min and max touch the values, so
// the result is bit-identical to the band wavefront and to a serial loop.
#include "dfd_device.cuh"
#include "dfd_internal.h"

namespace dfd {
namespace {

constexpr int RS_THREADS = 256;

template <class V, int DK>
__device__ __forceinline__ typename V::value cell_d2(const typename V::coord* p, const typename V::coord* q,
                                                     int dim) {
  typename V::coord a[DK], b[DK];
#pragma unroll
  for (int k = 0; k < DK; ++k) {
    a[k] = k < dim ? p[k] : (typename V::coord)0;
    b[k] = k < dim ? q[k] : (typename V::coord)0;
  }
  return dist2<DK>(a, b);
}

template <class V, int DK>
__global__ void __launch_bounds__(RS_THREADS) rowscan_kernel(const typename V::coord* __restrict__ P, int64_t n,
                                                             const typename V::coord* __restrict__ Q, int64_t m,
                                                             int dim, typename V::value* buf0,
                                                             typename V::value* buf1, int* err, void* out_dist,
                                                             void* out_dist2) {
  using T = typename V::value;
  using Cl = Clamp<V>;
  __shared__ Cl warp_tot[RS_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t seg = (m + RS_THREADS - 1) / RS_THREADS;
  const int64_t lo = min((int64_t)tid * seg, m), hi = min(lo + seg, m);
  if (ld_relaxed_i32(err) != 0) return;

  T* prev = buf0;
  T* cur = buf1;
  for (int64_t i = 0; i < n; ++i) {
    const typename V::coord* pi = P + i * dim;
    const T corner = (i == 0) ? V::zero() : V::inf();
    // Phase A: compose this thread's clamps.
    Cl F = clamp_identity<V>();
    for (int64_t j = lo; j < hi; ++j) {
      const T up = (i == 0) ? V::inf() : prev[j];
      const T dg = (j == 0) ? corner : ((i == 0) ? V::inf() : prev[j - 1]);
      const Cl f{V::vmin(up, dg), cell_d2<V, DK>(pi, Q + j * dim, dim)};
      F = compose<V>(f, F);
    }
    // Phase B: block-wide exclusive scan of the segment compositions.
    const Cl incl = warp_clamp_scan_inclusive<V>(F, lane);
    Cl excl;
    excl.a = __shfl_up_sync(0xffffffffu, incl.a, 1);
    excl.d = __shfl_up_sync(0xffffffffu, incl.d, 1);
    if (lane == 0) excl = clamp_identity<V>();
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      Cl t = lane < RS_THREADS / 32 ? warp_tot[lane] : clamp_identity<V>();
      t = warp_clamp_scan_inclusive<V>(t, lane);
      if (lane < RS_THREADS / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    const Cl before = wid == 0 ? clamp_identity<V>() : warp_tot[wid - 1];
    const Cl Gt = compose<V>(excl, before);
    // Left boundary M_{i,0} = +inf enters the scan.
    T x = apply<V>(Gt, V::inf());
    // Phase C: apply the clamps in order.
    for (int64_t j = lo; j < hi; ++j) {
      const T up = (i == 0) ? V::inf() : prev[j];
      const T dg = (j == 0) ? corner : ((i == 0) ? V::inf() : prev[j - 1]);
      const Cl f{V::vmin(up, dg), cell_d2<V, DK>(pi, Q + j * dim, dim)};
      x = apply<V>(f, x);
      cur[j] = x;
    }
    __syncthreads();
    T* t = prev;
    prev = cur;
    cur = t;
  }
  if (tid == 0) {
    const T r = prev[m - 1];
    if constexpr (sizeof(T) == 4) {
      if (out_dist2) static_cast<float*>(out_dist2)[0] = (float)r;
      if (out_dist) static_cast<float*>(out_dist)[0] = sqrtf((float)r);
    } else {
      if (out_dist2) static_cast<long long*>(out_dist2)[0] = (long long)r;
      if (out_dist) static_cast<double*>(out_dist)[0] = sqrt((double)r);
    }
  }
}

template <class V, int DK>
dfd_status launch(dfd_context* ctx, int dim, const void* p, int64_t n, const void* q, int64_t m,
                  void* out_dist, void* out_dist2, cudaStream_t s) {
  using T = typename V::value;
  const size_t row = align_up((size_t)m * sizeof(T), 256);
  dfd_status st = ensure_scratch(ctx, 2 * row);
  if (st != DFD_OK) return st;
  T* b0 = static_cast<T*>(ctx->scratch);
  T* b1 = reinterpret_cast<T*>(static_cast<char*>(ctx->scratch) + row);
  timing_begin(ctx, s);
  rowscan_kernel<V, DK><<<1, RS_THREADS, 0, s>>>(static_cast<const typename V::coord*>(p), n,
                                                 static_cast<const typename V::coord*>(q), m, dim, b0, b1,
                                                 ctx->d_err, out_dist, out_dist2);
  timing_end(ctx, s);
  return cuda_status(cudaGetLastError());
}

}  // namespace

dfd_status rowscan_run(dfd_context* ctx, dfd_dtype dtype, int dim, const void* p, int64_t n, const void* q,
                       int64_t m, void* out_dist, void* out_dist2, cudaStream_t s) {
  const int dk = dim_class(dim);
#define DFD_RS_CASE(K)                                                                      \
  case K:                                                                                   \
    return dtype == DFD_F32 ? launch<F32, K>(ctx, dim, p, n, q, m, out_dist, out_dist2, s) \
                            : launch<I32, K>(ctx, dim, p, n, q, m, out_dist, out_dist2, s);
  switch (dk) {
    DFD_RS_CASE(2)
    DFD_RS_CASE(3)
    DFD_RS_CASE(4)
    DFD_RS_CASE(8)
    DFD_RS_CASE(16)
    default:
      return DFD_ERR_UNSUPPORTED;
  }
#undef DFD_RS_CASE
}

}  // namespace dfd
