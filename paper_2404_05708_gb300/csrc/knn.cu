// knn.cu -- exact k nearest candidate curves of one query curve under the
// discrete Frechet distance, with early abandon.
//
// Persistent warps take candidates from an atomic counter and run the batch
// engine's per-pair recurrence (one warp per pair, rows = the shorter
// curve).  A candidate is abandoned as soon as a cut of its running
// recurrence exceeds the current limit (see AbandonAbove): every monotone
// path enters the cut, and a path's prefix bottleneck is at least M of the
// cell it ends in, so delta^2 >= the cut's minimum.  Finished candidates
// enter a k-slot array of keys (delta^2 bits << 32 | candidate index) by
// replacing the array's largest key (compare-and-swap, retried on
// conflict); slots only ever decrease, so the array max is an upper bound of
// the final k-th smallest key, and the limit (atomicMin of the maxima seen
// after insertions) never prunes a true neighbour.  A one-block bitonic sort
// orders the k keys at the end.  The decision form of the problem (Sec. 2)
// and the heuristics that avoid full computations (Sec. 5) motivate the
// pruning; the distance itself is Eq. 1 exactly.
#include <algorithm>
#include "batch_launch.cuh"
#include "dfd_internal.h"

namespace dfd {
namespace knn {

constexpr int KMAX = 1024;
constexpr unsigned long long kEmpty = ~0ull;

struct KnnArgs {
  const float* query;
  int n;
  int dim;
  int vec;                     // vector point loads allowed
  const float* points;
  const int64_t* offsets;
  int64_t n_curves;
  const int32_t* cand;         // candidate curve ids, or null: all curves in order
  int64_t n_cand;
  int k;
  unsigned long long* topk;    // [k]
  unsigned* limit;             // float bits of the current upper bound of the k-th best delta^2
  int* counter;
  int* err;
  float* rowbuf;               // per-warp BUF_COLS floats
  unsigned long long* abandoned;
  unsigned long long* computed;
  unsigned long long* evaluated;   // cells of the recurrence actually evaluated (may be null)
  unsigned* lb;                // [n_cand] endpoint lower bound (float bits) per position
  unsigned* order;             // [n_cand] positions, ascending lower bound
  unsigned* hist;              // [NB] counting-sort buckets
};

// Counting sort of the candidates by their endpoint lower bound: every
// coupling path contains (0,0) and (n-1,m-1), so delta^2 >= the larger of
// those two squared distances (computed in the kernels' float32 order, so
// the bound holds bit for bit).  Searching near candidates first lowers the
// limit early, and a candidate whose bound already exceeds the limit is
// skipped without running the recurrence.
constexpr int NB = 8192;   // buckets on the top bits of the bound's float bits
__device__ __forceinline__ unsigned lb_bucket(unsigned bits) { return min(bits >> 18, (unsigned)NB - 1); }

// Warp-wide largest key of the k slots and its index.
__device__ __forceinline__ void topk_max(const KnnArgs& a, int L, unsigned long long* mx, int* mi) {
  unsigned long long v = 0;
  int idx = -1;
  for (int j = L; j < a.k; j += 32) {
    const unsigned long long t = ld_relaxed_u64(a.topk + j);
    if (idx < 0 || t > v) {
      v = t;
      idx = j;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long ov = __shfl_xor_sync(0xffffffffu, v, off);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, off);
    if (oi >= 0 && (idx < 0 || ov > v || (ov == v && oi < idx))) {
      v = ov;
      idx = oi;
    }
  }
  *mx = v;
  *mi = idx;
}

__device__ __forceinline__ void topk_insert(const KnnArgs& a, unsigned long long key, int L) {
  for (int tries = 0; tries < (1 << 20); ++tries) {
    unsigned long long mx;
    int mi;
    topk_max(a, L, &mx, &mi);
    if (key >= mx) return;   // not among the k smallest seen so far
    int ok = 0;
    if (L == 0) ok = atomicCAS(a.topk + mi, mx, key) == mx;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) {
      topk_max(a, L, &mx, &mi);
      if (L == 0 && mx != kEmpty) atomicMin(a.limit, (unsigned)(mx >> 32));
      return;
    }
  }
  if (L == 0) raise_error(a.err, DFD_ERR_TIMEOUT);   // unreachable in practice: every failed CAS is another's success
}

template <int DK>
__global__ void knn_lb_kernel(KnnArgs a) {
  const int64_t total = a.offsets[a.n_curves];
  float q0[DK], q1[DK];
#pragma unroll
  for (int k = 0; k < DK; ++k) {
    q0[k] = k < a.dim ? a.query[k] : 0.f;
    q1[k] = k < a.dim ? a.query[(int64_t)(a.n - 1) * a.dim + k] : 0.f;
  }
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < a.n_cand;
       it += (int64_t)gridDim.x * blockDim.x) {
    const int64_t id = a.cand ? a.cand[it] : it;
    unsigned bits = 0;   // invalid candidates: bound 0 (the search reports them)
    if (id >= 0 && id < a.n_curves) {
      const int64_t o = a.offsets[id], e = a.offsets[id + 1];
      if (o >= 0 && e <= total && e > o) {
        float c0[DK], c1[DK];
#pragma unroll
        for (int k = 0; k < DK; ++k) {
          c0[k] = k < a.dim ? a.points[o * a.dim + k] : 0.f;
          c1[k] = k < a.dim ? a.points[(e - 1) * a.dim + k] : 0.f;
        }
        bits = __float_as_uint(fmaxf(dist2<DK>(q0, c0), dist2<DK>(q1, c1)));
      }
    }
    a.lb[it] = bits;
    atomicAdd(a.hist + lb_bucket(bits), 1u);
  }
}

// Exclusive scan of the NB bucket counts (one block of 1024 threads).
__global__ void __launch_bounds__(1024) knn_scan_kernel(unsigned* hist) {
  __shared__ unsigned part[1024];
  constexpr int PER = NB / 1024;
  unsigned loc[PER], sum = 0;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    loc[i] = hist[threadIdx.x * PER + i];
    sum += loc[i];
  }
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const unsigned v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  unsigned run = part[threadIdx.x] - sum;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    hist[threadIdx.x * PER + i] = run;
    run += loc[i];
  }
}

__global__ void knn_scatter_kernel(KnnArgs a) {
  for (int64_t it = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; it < a.n_cand;
       it += (int64_t)gridDim.x * blockDim.x)
    a.order[atomicAdd(a.hist + lb_bucket(a.lb[it]), 1u)] = (unsigned)it;
}

template <int DK>
__global__ void __launch_bounds__(256, batch::kBlocksPerSM<DK>::value) knn_kernel(KnnArgs a) {
  __shared__ uint4 stage_sm[8][batch::QStage<DK>::RECS];
  uint4* stage = stage_sm[threadIdx.x >> 5];
  const int L = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  float* buf = a.rowbuf + gw * batch::BUF_COLS;
  const int64_t total = a.offsets[a.n_curves];
  if (ld_relaxed_i32(a.err) != 0) return;
  for (;;) {
    int item = 0;
    if (L == 0) item = atomicAdd(a.counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= a.n_cand) break;
    item = (int)a.order[item];   // nearest endpoint bound first
    {
      // Positions come in ascending bucket order: once a bucket's lower edge
      // exceeds the limit, no later candidate can enter the k best.
      unsigned lim = 0;
      if (L == 0) lim = (unsigned)ld_relaxed_i32(reinterpret_cast<const int*>(a.limit));
      lim = __shfl_sync(0xffffffffu, lim, 0);
      if ((lb_bucket(a.lb[item]) << 18) > lim) break;
    }
    const int64_t id = a.cand ? a.cand[item] : item;
    if (id < 0 || id >= a.n_curves) {
      if (L == 0) raise_error(a.err, DFD_ERR_INVALID_ARG);
      continue;
    }
    const int64_t o = a.offsets[id], e = a.offsets[id + 1];
    if (o < 0 || e > total || e - o < 1 || e - o > INT32_MAX) {
      if (L == 0) raise_error(a.err, DFD_ERR_INVALID_ARG);
      continue;
    }
    const int m = (int)(e - o);
    {
      unsigned lim = 0;
      if (L == 0) lim = (unsigned)ld_relaxed_i32(reinterpret_cast<const int*>(a.limit));
      lim = __shfl_sync(0xffffffffu, lim, 0);
      if (a.lb[item] > lim) continue;   // delta^2 >= bound > k-th best: no recurrence needed
    }
    const float* C = a.points + o * a.dim;
    const bool query_rows = a.n <= m;
    const int rows = query_rows ? a.n : m, cols = query_rows ? m : a.n;
    if (!batch::fits_buffer<DK>(rows, cols)) {
      if (L == 0) raise_error(a.err, DFD_ERR_UNSUPPORTED);
      continue;
    }
    batch::AbandonAbove<F32> ab;
    ab.fixed = __int_as_float(0x7f800000);
    ab.live_bits = a.limit;
    const float r = query_rows ? batch::warp_dfd_any<F32, DK, batch::AbandonAbove<F32>>(
                                     a.query, a.n, C, m, a.dim, a.vec != 0, buf, L, 0, 1 << 30, &ab, stage)
                               : batch::warp_dfd_any<F32, DK, batch::AbandonAbove<F32>>(
                                     C, m, a.query, a.n, a.dim, a.vec != 0, buf, L, 0, 1 << 30, &ab, stage);
    if (L == 0 && a.evaluated)
      atomicAdd(a.evaluated, (unsigned long long)rows * (unsigned long long)(ab.hit ? min(ab.cols_done, cols) : cols));
    if (ab.hit) continue;
    if (L == 0 && a.computed) atomicAdd(a.computed, 1ull);
    const unsigned bits = __float_as_uint(r);
    unsigned lim = 0;
    if (L == 0) lim = (unsigned)ld_relaxed_i32(reinterpret_cast<const int*>(a.limit));
    lim = __shfl_sync(0xffffffffu, lim, 0);
    if (bits > lim) continue;   // above the k-th best seen: cannot enter
    topk_insert(a, ((unsigned long long)bits << 32) | (unsigned)item, L);
  }
}

__global__ void knn_init_kernel(unsigned long long* topk, int k, unsigned* limit, int* counter,
                                unsigned long long* abandoned, unsigned long long* computed,
                                unsigned long long* evaluated) {
  for (int j = threadIdx.x; j < k; j += blockDim.x) topk[j] = kEmpty;
  if (threadIdx.x == 0) {
    *limit = 0x7f800000u;
    *counter = 0;
    *computed = 0;
    if (abandoned) *abandoned = 0;
    if (evaluated) *evaluated = 0;
  }
}

// Sort the k keys ascending (bitonic, one block) and write ids / distances.
__global__ void __launch_bounds__(KMAX) knn_finish_kernel(const unsigned long long* topk, int k,
                                                          const int32_t* cand, int32_t* out_ids, float* out_dist2,
                                                          float* out_dist, const unsigned long long* computed,
                                                          int64_t n_cand, unsigned long long* abandoned) {
  if (threadIdx.x == 0 && abandoned) *abandoned = (unsigned long long)n_cand - *computed;
  __shared__ unsigned long long s[KMAX];
  int size = 1;
  while (size < k) size <<= 1;
  for (int j = threadIdx.x; j < size; j += blockDim.x) s[j] = j < k ? topk[j] : kEmpty;
  __syncthreads();
  for (int len = 2; len <= size; len <<= 1) {
    for (int stride = len >> 1; stride > 0; stride >>= 1) {
      for (int j = threadIdx.x; j < size; j += blockDim.x) {
        const int p = j ^ stride;
        if (p > j) {
          const bool up = (j & len) == 0;
          const unsigned long long x = s[j], y = s[p];
          if ((x > y) == up) {
            s[j] = y;
            s[p] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const unsigned long long key = s[j];
    const bool empty = key == kEmpty;
    const unsigned idx = (unsigned)(key & 0xffffffffu);
    const float d2 = __uint_as_float((unsigned)(key >> 32));
    if (out_ids) out_ids[j] = empty ? -1 : (cand ? cand[idx] : (int32_t)idx);
    if (out_dist2) out_dist2[j] = empty ? __int_as_float(0x7f800000) : d2;
    if (out_dist) out_dist[j] = empty ? __int_as_float(0x7f800000) : sqrtf(d2);
  }
}

template <int DK>
dfd_status knn_launch(dfd_context* ctx, int dim, const float* query, int n, const float* points,
                      const int64_t* offsets, int64_t n_curves, const int32_t* cand, int64_t n_cand, int k,
                      int32_t* out_ids, float* out_dist2, float* out_dist, unsigned long long* abandoned,
                      unsigned long long* evaluated, cudaStream_t s) {
  const int blocks = resident_blocks(ctx, knn_kernel<DK>, 256);
  const size_t warps = (size_t)blocks * 8;
  const size_t off_topk = 256, off_hist = align_up(off_topk + (size_t)k * 8, 256);
  const size_t off_lb = align_up(off_hist + (size_t)NB * 4, 256);
  const size_t off_order = align_up(off_lb + (size_t)n_cand * 4, 256);
  const size_t off_buf = align_up(off_order + (size_t)n_cand * 4, 256);
  const size_t total = off_buf + warps * batch::BUF_COLS * sizeof(float);
  dfd_status st = ensure_scratch(ctx, total);
  if (st != DFD_OK) return st;
  char* base = static_cast<char*>(ctx->scratch);
  if (ctx->opt.check_inputs) {
    st = launch_check_inputs(DFD_F32, dim, query, (int64_t)n * dim, ctx->d_err, s);
    if (st != DFD_OK) return st;
    check_points_kernel<F32><<<std::min(4 * ctx->num_sms, 1024), 256, 0, s>>>(points, offsets, offsets + n_curves, dim,
                                                                             ctx->d_err);
  }
  KnnArgs a;
  a.query = query;
  a.n = n;
  a.dim = dim;
  a.vec = vector_loads_ok<DK>(points, dim) && vector_loads_ok<DK>(query, dim);
  a.points = points;
  a.offsets = offsets;
  a.n_curves = n_curves;
  a.cand = cand;
  a.n_cand = n_cand;
  a.k = k;
  a.topk = reinterpret_cast<unsigned long long*>(base + off_topk);
  a.limit = reinterpret_cast<unsigned*>(base);
  a.counter = reinterpret_cast<int*>(base + 8);
  a.computed = reinterpret_cast<unsigned long long*>(base + 16);
  a.err = ctx->d_err;
  a.rowbuf = reinterpret_cast<float*>(base + off_buf);
  a.abandoned = abandoned;
  a.evaluated = evaluated;
  a.hist = reinterpret_cast<unsigned*>(base + off_hist);
  a.lb = reinterpret_cast<unsigned*>(base + off_lb);
  a.order = reinterpret_cast<unsigned*>(base + off_order);
  knn_init_kernel<<<1, 256, 0, s>>>(a.topk, k, a.limit, a.counter, abandoned, a.computed, evaluated);
  cudaError_t e = cudaMemsetAsync(a.hist, 0, (size_t)NB * 4, s);
  if (e != cudaSuccess) return cuda_status(e);
  const int lblocks = (int)std::max<int64_t>(1, std::min<int64_t>((n_cand + 255) / 256, 4 * (int64_t)ctx->num_sms));
  knn_lb_kernel<DK><<<lblocks, 256, 0, s>>>(a);
  knn_scan_kernel<<<1, 1024, 0, s>>>(a.hist);
  knn_scatter_kernel<<<lblocks, 256, 0, s>>>(a);
  timing_begin(ctx, s);
  knn_kernel<DK><<<blocks, 256, 0, s>>>(a);
  timing_end(ctx, s);
  knn_finish_kernel<<<1, KMAX, 0, s>>>(a.topk, k, cand, out_ids, out_dist2, out_dist, a.computed, n_cand, abandoned);
  return cuda_status(cudaGetLastError());
}

}  // namespace knn
}  // namespace dfd

using namespace dfd;

extern "C" dfd_status dfd_knn(dfd_context* ctx, int dim, const float* query, int64_t n, const float* points,
                              const int64_t* offsets, int64_t n_curves, const int32_t* cand, int64_t n_cand, int k,
                              int32_t* out_ids, float* out_dist2, float* out_dist, unsigned long long* abandoned,
                              unsigned long long* evaluated, void* stream) {
  if (!ctx || !query || !points || !offsets || n < 1 || n > INT32_MAX || n_curves < 1 || n_curves > INT32_MAX)
    return DFD_ERR_INVALID_ARG;
  if (dim < 1 || k < 1 || n_cand < 0 || n_cand > INT32_MAX || (!cand && n_cand > n_curves))
    return DFD_ERR_INVALID_ARG;
  if (!out_ids && !out_dist2 && !out_dist) return DFD_ERR_INVALID_ARG;
  if (dim > 16 || k > knn::KMAX) return DFD_ERR_UNSUPPORTED;
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (dim_class(dim)) {
    case 2: return knn::knn_launch<2>(ctx, dim, query, (int)n, points, offsets, n_curves, cand, n_cand, k, out_ids, out_dist2, out_dist, abandoned, evaluated, s);
    case 3: return knn::knn_launch<3>(ctx, dim, query, (int)n, points, offsets, n_curves, cand, n_cand, k, out_ids, out_dist2, out_dist, abandoned, evaluated, s);
    case 4: return knn::knn_launch<4>(ctx, dim, query, (int)n, points, offsets, n_curves, cand, n_cand, k, out_ids, out_dist2, out_dist, abandoned, evaluated, s);
    case 8: return knn::knn_launch<8>(ctx, dim, query, (int)n, points, offsets, n_curves, cand, n_cand, k, out_ids, out_dist2, out_dist, abandoned, evaluated, s);
    case 16: return knn::knn_launch<16>(ctx, dim, query, (int)n, points, offsets, n_curves, cand, n_cand, k, out_ids, out_dist2, out_dist, abandoned, evaluated, s);
    default: return DFD_ERR_UNSUPPORTED;
  }
}
