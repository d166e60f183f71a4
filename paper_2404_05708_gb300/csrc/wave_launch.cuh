// wave_launch.cuh -- host launcher of the band wavefront (K2), instantiated
// per (value type, dimension class, rows per lane) in wave_*.cu.
#pragma once
#include <algorithm>
#include <climits>
#include <cmath>
#include <mutex>
#include <type_traits>
#include "dfd_internal.h"
#include "wave_kernel.cuh"

namespace dfd {

// Rows of at most this many columns meet the two fronts inside the
// wavefront launch (its last CTA); longer ones launch combine_kernel, whose
// many CTAs read the rows in parallel.
constexpr int64_t kFusedCombineCols = 65536;

namespace wave {

// Launch attributes of wave_kernel<KV, DK, R>.  The kernel's dynamic shared
// memory allowance is a property of the function on the device (not of a
// context), so it is kept process-wide and only ever raised: the largest
// size set so far, per device.  The CTAs per SM are kept per context and
// (kernel, warps).
template <class KV, int DK, int R>
dfd_status kernel_attrs(dfd_context* ctx, int W, size_t smem, int* per_sm_out) {
  const void* kfn = reinterpret_cast<const void*>(wave_kernel<KV, DK, R>);
  static std::mutex smem_mu;
  static size_t smem_set[64] = {};
  const int dev = ctx->device >= 0 && ctx->device < 64 ? ctx->device : 0;
  {
    std::lock_guard<std::mutex> lock(smem_mu);
    if (smem_set[dev] < smem || ctx->device != dev) {
      cudaError_t e = cudaFuncSetAttribute(wave_kernel<KV, DK, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) {
        cudaGetLastError();   // leave no error behind for later calls
        return cuda_status(e);
      }
      if (ctx->device == dev) smem_set[dev] = smem;
    }
  }
  int per_sm = 0;
  auto it = ctx->attr_cache ? ctx->wave_attr.find({kfn, W}) : ctx->wave_attr.end();
  if (it != ctx->wave_attr.end()) {
    per_sm = it->second.per_sm;
  } else {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wave_kernel<KV, DK, R>, (W + 1) * 32, smem) !=
            cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    if (ctx->attr_cache) ctx->wave_attr[{kfn, W}] = WaveAttr{smem, per_sm};
  }
  *per_sm_out = per_sm;
  return DFD_OK;
}

// q stream geometry of one value class: lane 31's bottom row reaches column
// m - 1 at step m - 1 + 32*K - 1, and the look-ahead of the last steps reads
// columns up to nblk*G + 1.
template <class KV, int DK, int R>
struct Geometry {
  int nblk = 0, nch = 0;
  size_t q_bytes = 0;
  bool ok = false;
  explicit Geometry(int64_t m) {
    using Lay = Layout<KV, DK, R>;
    constexpr int K = Skew<KV, R>::value;
    const int64_t nblk64 = (m + 32 * K - 1 + G - 1) / G;
    if (nblk64 * G > (int64_t)INT32_MAX / 2) return;
    nblk = (int)nblk64;
    nch = (nblk * G + 2 + Lay::C - 1) / Lay::C;
    q_bytes = (size_t)nch * Lay::NPL * Lay::C * sizeof(typename Lay::Rec);
    ok = true;
  }
};

}  // namespace wave

// float32 pairs run one wavefront kernel.  int32 pairs launch two with the
// same shape, back to back: the narrow class (I32B: exact uint32 squared
// distances carried as float bits, the float32 stripe) and the exact int64
// class; the prep kernel reduces the pair's bounding box and each CTA of
// either kernel leaves at once unless the box makes the pair its class, so
// the choice is made on the device and the call stays asynchronous.
template <class V, int DK, int R>
dfd_status wave_launch(dfd_context* ctx, int dim, const void* p, int64_t n, const void* q, int64_t m,
                       void* out_dist, void* out_dist2, cudaStream_t s, int W, int ctas, bool check) {
  constexpr bool kInt = std::is_same<V, I32>::value;
  using VN = typename std::conditional<kInt, I32B, V>::type;   // the first kernel's class
  if constexpr (wave::kMaxWarps<V, DK, R>::value < 1 || wave::kMaxWarps<VN, DK, R>::value < 1) {
    return DFD_ERR_UNSUPPORTED;   // R rows of DK coordinates do not fit one lane's registers
  } else {
  using LayN = wave::Layout<VN, DK, R>;
  using LayW = wave::Layout<V, DK, R>;
  constexpr int C = LayN::C;
  const bool shape_ok = kInt ? wave::int_shape_supported(DK, R, W) : wave::shape_supported(true, DK, R, W);
  if (!shape_ok) return DFD_ERR_UNSUPPORTED;
  const int64_t H = (int64_t)W * 32 * R;
  const int64_t nbands_all = (n + H - 1) / H;
  const wave::Geometry<VN, DK, R> gn(m);
  const wave::Geometry<V, DK, R> gw(m);
  if (!gn.ok || !gw.ok) return DFD_ERR_UNSUPPORTED;
  const size_t vbytes = sizeof(typename V::value);   // row buffers hold the exact class's values

  // Prep grid; int32: its first nbox blocks also reduce the bounding box.
  const int threads = 256;
  int64_t prep_work = (int64_t)gn.nch * C * LayN::NPL;
  if (kInt) prep_work += (int64_t)gw.nch * C * LayW::NPL;
  const int64_t elems = kInt ? n + m : check ? (n + m) * (int64_t)dim : 0;
  const int blocks = (int)std::max<int64_t>(
      1, std::min<int64_t>((std::max(prep_work, elems) + threads - 1) / threads, 4 * (int64_t)ctx->num_sms));
  const int nbox = kInt ? std::min(blocks, 128) : 0;

  // Two wavefronts when the pair has two bands or more: the first
  // ceil(#bands / 2) bands forward from (0, 0), the remaining rows backward
  // from (n-1, m-1) on both curves reversed, met by combine_kernel.  Each
  // front starts its own chain of bands, so the launch waits for half as
  // many band start-up lags.  The scratch doubles (two row buffers, two
  // packed q streams per class); where it cannot grow (a fixed scratch
  // array), one forward wavefront runs.
  // Layout: header (256 B) | progress | progress_b | row | row_b | box |
  // q of the first class (front, back) | q of the exact int32 class.
  struct Off {
    size_t prog_b, row, row_b, box, qn, qn_b, qw, qw_b, end;
  };
  auto layout = [&](bool two, int64_t nb0, int64_t nb1) {
    Off o;
    const size_t off_prog = 256;
    o.prog_b = align_up(off_prog + (size_t)nb0 * sizeof(unsigned long long), 256);
    o.row = align_up(o.prog_b + (two ? (size_t)nb1 * sizeof(unsigned long long) : 0), 256);
    o.row_b = align_up(o.row + (size_t)m * vbytes, 256);
    o.box = align_up(o.row_b + (two ? (size_t)m * vbytes : 0), 256);
    o.qn = align_up(o.box + (size_t)nbox * 2 * DK * sizeof(int), 256);
    o.qn_b = align_up(o.qn + gn.q_bytes, 256);
    o.qw = align_up(o.qn_b + (two ? gn.q_bytes : 0), 256);
    o.qw_b = align_up(o.qw + (kInt ? gw.q_bytes : 0), 256);
    o.end = o.qw_b + (kInt && two ? gw.q_bytes : 0);
    return o;
  };
  bool two = nbands_all >= 2;
  const int64_t n1_split = ((nbands_all + 1) / 2) * H;   // forward rows when split (< n for two bands or more)
  Off off;
  dfd_status st = DFD_OK;
  if (two) {
    off = layout(true, (nbands_all + 1) / 2, (n - n1_split + H - 1) / H);
    st = ensure_scratch(ctx, off.end);
    if (st != DFD_OK) two = false;
  }
  if (!two) {
    off = layout(false, nbands_all, 0);
    st = ensure_scratch(ctx, off.end);
  }
  if (st != DFD_OK) return st;
  const int64_t n1 = two ? n1_split : n;   // rows of the forward problem
  const int64_t n2 = n - n1;               // rows of the backward problem (0: one front)
  const int64_t nb0 = (n1 + H - 1) / H;
  const int64_t nb1 = (n2 + H - 1) / H;
  char* base = static_cast<char*>(ctx->scratch);

  const size_t smem_n = LayN::bytes(W), smem_w = LayW::bytes(W);
  if (smem_n > ctx->smem_optin || (kInt && smem_w > ctx->smem_optin)) return DFD_ERR_UNSUPPORTED;
  // one launch before the wavefront: the header zeroed, the inputs checked
  // (check), q packed for each front (int32: also the bounding box).  The
  // measurement events bracket it too: an event between it and the
  // wavefront would keep the wavefront from starting early (below).
  timing_begin(ctx, s);
  const long long lim =
      std::min<long long>((1LL << 30) - 1, (long long)std::floor(std::sqrt((double)LLONG_MAX / (double)dim) / 2.0));
  if constexpr (kInt) {
    wave::wave_prep_int_kernel<DK><<<dim3(blocks, two ? 2 : 1), threads, 0, s>>>(
        static_cast<const int32_t*>(q), m, dim, static_cast<const int32_t*>(p), n, reinterpret_cast<unsigned*>(base),
        (int)(off.row / 4), check ? 1 : 0, lim, ctx->d_err, reinterpret_cast<int*>(base + off.box), nbox, gn.nch,
        wave::QTrans<VN, R>::value, base + off.qn, base + off.qn_b, gw.nch, base + off.qw, base + off.qw_b);
  } else {
    wave::wave_prep_kernel<V, DK><<<dim3(blocks, two ? 2 : 1), threads, 0, s>>>(
        static_cast<const typename V::coord*>(q), m, dim, gn.nch, wave::QTrans<V, R>::value, base + off.qn,
        base + off.qn_b, reinterpret_cast<unsigned*>(base), (int)(off.row / 4),
        static_cast<const typename V::coord*>(p), n * (int64_t)dim, check ? 1 : 0, lim, ctx->d_err);
  }
  int per_sm_n = 1, per_sm_w = 1;
  if ((st = wave::kernel_attrs<VN, DK, R>(ctx, W, smem_n, &per_sm_n)) != DFD_OK) return st;
  if (kInt && (st = wave::kernel_attrs<V, DK, R>(ctx, W, smem_w, &per_sm_w)) != DFD_OK) return st;

  const bool fused = two && m <= kFusedCombineCols;
  auto args = [&](int nblk, int nch, size_t off_q, size_t off_q_b, int want) {
    wave::Args a;
    a.p = p;
    a.n = two ? n1 : n;
    a.dim = dim;
    a.qpk = base + off_q;
    a.m = m;
    a.nch = nch;
    a.nblk = nblk;
    a.H = H;
    a.nbands = nb0;
    a.rowbuf = base + off.row;
    a.progress = reinterpret_cast<unsigned long long*>(base + 256);
    a.ticket = reinterpret_cast<int*>(base);
    a.err = ctx->d_err;
    a.out_dist = two ? nullptr : out_dist;     // two fronts: the combine writes the result
    a.out_dist2 = two ? nullptr : out_dist2;
    a.combine = fused ? 1 : 0;
    a.done = reinterpret_cast<unsigned*>(base + 24);   // zeroed header word after the merge words
    a.res_dist = out_dist;
    a.res_dist2 = out_dist2;
    a.timeout_ns = timeout_ns(ctx);
    a.pstep = dim;
    a.nprob = two ? 2 : 1;
    a.p_b = two ? static_cast<const void*>(static_cast<const typename V::coord*>(p) + (n - 1) * (int64_t)dim)
                : nullptr;
    a.n_b = n2;
    a.nbands_b = nb1;
    a.qpk_b = two ? base + off_q_b : nullptr;
    a.rowbuf_b = two ? base + off.row_b : nullptr;
    a.progress_b = reinterpret_cast<unsigned long long*>(base + off.prog_b);
    a.box = kInt ? reinterpret_cast<const int*>(base + off.box) : nullptr;
    a.nbox = nbox;
    a.want = want;
    return a;
  };
  // persistent grid: every CTA that can be resident (a band is only ever
  // awaited by a later ticket, so CTAs that are not resident wait harmlessly)
  const int64_t nbands = nb0 + nb1;
  auto grid_of = [&](int per_sm) {
    const int g = ctas > 0 ? ctas : per_sm * ctx->num_sms;
    return (int)std::min<int64_t>(g, nbands);
  };
  // The wavefronts are launched with programmatic stream serialisation: their
  // CTAs may become resident and run their prologue (q ring zeroed, barriers
  // initialised) while the kernel before them finishes, then wait for it in
  // griddep_wait, which hides most of a launch gap per kernel.
  auto launch = [&](auto kernel, int per_sm, size_t smem, const wave::Args& a) {
    return launch_pdl(kernel, dim3((unsigned)grid_of(per_sm)), dim3((unsigned)((W + 1) * 32)), smem, s, a);
  };
  cudaError_t le = launch(wave::wave_kernel<VN, DK, R>, per_sm_n, smem_n, args(gn.nblk, gn.nch, off.qn, off.qn_b, 1));
  if (le == cudaSuccess && kInt)
    le = launch(wave::wave_kernel<V, DK, R>, per_sm_w, smem_w, args(gw.nblk, gw.nch, off.qw, off.qw_b, 0));
  if (le != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(le);
  }
  if (two && !fused) {
    // the merge words sit after the ticket in the zeroed scratch header
    const int cblocks = (int)std::max<int64_t>(1, std::min<int64_t>((m + 1023) / 1024, ctx->num_sms));
    const int* box = kInt ? reinterpret_cast<const int*>(base + off.box) : nullptr;
    auto word = reinterpret_cast<unsigned long long*>(base + 16);
    auto count = reinterpret_cast<unsigned*>(base + 8);
    wave::combine_kernel<VN, DK><<<cblocks, 256, 0, s>>>(base + off.row, base + off.row_b, m, word, count, ctx->d_err,
                                                         out_dist, out_dist2, box, nbox, 1);
    if constexpr (kInt)
      wave::combine_kernel<V, DK><<<cblocks, 256, 0, s>>>(base + off.row, base + off.row_b, m, word, count,
                                                          ctx->d_err, out_dist, out_dist2, box, nbox, 0);
  }
  timing_end(ctx, s);
  return cuda_status(cudaGetLastError());
  }
}

}  // namespace dfd

#define DFD_WAVE_INSTANTIATE(V, DK, R)                                                                     \
  template dfd_status dfd::wave_launch<dfd::V, DK, R>(dfd_context*, int, const void*, int64_t, const void*, \
                                                        int64_t, void*, void*, cudaStream_t, int, int, bool);
