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

template <class V, int DK, int R>
dfd_status wave_launch(dfd_context* ctx, int dim, const void* p, int64_t n, const void* q, int64_t m,
                       void* out_dist, void* out_dist2, cudaStream_t s, int W, int ctas, bool check) {
  using Lay = wave::Layout<V, DK, R>;
  using T = typename V::value;
  using Rec = typename Lay::Rec;
  constexpr int C = Lay::C;
  constexpr int K = wave::Skew<V, R>::value;
  if constexpr (wave::kMaxWarps<V, DK, R>::value < 1) {
    return DFD_ERR_UNSUPPORTED;   // R rows of DK coordinates do not fit one lane's registers
  } else {
  if (!wave::shape_supported(std::is_same<V, F32>::value, DK, R, W)) return DFD_ERR_UNSUPPORTED;
  const int64_t H = (int64_t)W * 32 * R;
  const int64_t nbands_all = (n + H - 1) / H;
  // Lane 31's bottom row reaches column m - 1 at step m - 1 + 32*K - 1.
  const int64_t nblk64 = (m + 32 * K - 1 + wave::G - 1) / wave::G;
  if (nblk64 * wave::G > (int64_t)INT32_MAX / 2) return DFD_ERR_UNSUPPORTED;
  const int nblk = (int)nblk64;
  // The look-ahead of the last steps reads columns up to nblk*G + 1.
  const int nch = (nblk * wave::G + 2 + C - 1) / C;
  const size_t q_bytes = (size_t)nch * Lay::NPL * C * sizeof(Rec);

  // Two wavefronts when the pair has two bands or more: the first
  // ceil(#bands / 2) bands forward from (0, 0), the remaining rows backward
  // from (n-1, m-1) on both curves reversed, met by combine_kernel.  Each
  // front starts its own chain of bands, so the launch waits for half as
  // many band start-up lags.  The scratch doubles (two row buffers, two
  // packed q streams); where it cannot grow (a fixed scratch array), one
  // forward wavefront runs.
  auto layout = [&](bool two, size_t* off_prog_b, size_t* off_row, size_t* off_row_b, size_t* off_q,
                    size_t* off_q_b, int64_t nb0, int64_t nb1) {
    const size_t off_prog = 256;
    *off_prog_b = align_up(off_prog + (size_t)nb0 * sizeof(unsigned long long), 256);
    *off_row = align_up(*off_prog_b + (two ? (size_t)nb1 * sizeof(unsigned long long) : 0), 256);
    *off_row_b = align_up(*off_row + (size_t)m * sizeof(T), 256);
    *off_q = align_up(*off_row_b + (two ? (size_t)m * sizeof(T) : 0), 256);
    *off_q_b = align_up(*off_q + q_bytes, 256);
    return *off_q_b + (two ? q_bytes : 0);
  };
  bool two = nbands_all >= 2;
  const int64_t n1_split = ((nbands_all + 1) / 2) * H;   // forward rows when split (< n for two bands or more)
  size_t off_prog_b, off_row, off_row_b, off_q, off_q_b;
  dfd_status st = DFD_OK;
  if (two) {
    st = ensure_scratch(ctx, layout(true, &off_prog_b, &off_row, &off_row_b, &off_q, &off_q_b,
                                    (nbands_all + 1) / 2, (n - n1_split + H - 1) / H));
    if (st != DFD_OK) two = false;
  }
  if (!two) st = ensure_scratch(ctx, layout(false, &off_prog_b, &off_row, &off_row_b, &off_q, &off_q_b, nbands_all, 0));
  if (st != DFD_OK) return st;
  const int64_t n1 = two ? n1_split : n;   // rows of the forward problem
  const int64_t n2 = n - n1;               // rows of the backward problem (0: one front)
  const int64_t nb0 = (n1 + H - 1) / H;
  const int64_t nb1 = (n2 + H - 1) / H;
  char* base = static_cast<char*>(ctx->scratch);

  const size_t smem = Lay::bytes(W);
  if (smem > ctx->smem_optin) return DFD_ERR_UNSUPPORTED;
  // one launch before the wavefront: the header zeroed, the inputs checked
  // (check), q packed for each front
  {
    const int64_t recs = (int64_t)nch * C * Lay::NPL;
    const int64_t elems = check ? (n + m) * (int64_t)dim : 0;
    const int threads = 256;
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((std::max(recs, elems) + threads - 1) / threads, 4 * (int64_t)ctx->num_sms));
    const long long lim =
        std::min<long long>((1LL << 30) - 1, (long long)std::floor(std::sqrt((double)LLONG_MAX / (double)dim) / 2.0));
    wave::wave_prep_kernel<V, DK><<<dim3(blocks, two ? 2 : 1), threads, 0, s>>>(
        static_cast<const typename V::coord*>(q), m, dim, nch, wave::QTrans<V, R>::value, base + off_q,
        base + off_q_b, reinterpret_cast<unsigned*>(base), (int)(off_row / 4),
        static_cast<const typename V::coord*>(p), n * (int64_t)dim, check ? 1 : 0, lim, ctx->d_err);
  }
  // Launch attributes.  The kernel's dynamic shared memory allowance is a
  // property of the function on the device (not of a context), so it is kept
  // process-wide and only ever raised: the largest size set so far, per
  // device.  The CTAs per SM are kept per context and (kernel, warps).
  const void* kfn = reinterpret_cast<const void*>(wave::wave_kernel<V, DK, R>);
  int per_sm = 0;
  {
    static std::mutex smem_mu;
    static size_t smem_set[64] = {};
    const int dev = ctx->device >= 0 && ctx->device < 64 ? ctx->device : 0;
    {
      std::lock_guard<std::mutex> lock(smem_mu);
      if (smem_set[dev] < smem || ctx->device != dev) {
        cudaError_t e =
            cudaFuncSetAttribute(wave::wave_kernel<V, DK, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
          cudaGetLastError();   // leave no error behind for later calls
          return cuda_status(e);
        }
        if (ctx->device == dev) smem_set[dev] = smem;
      }
    }
    auto it = ctx->attr_cache ? ctx->wave_attr.find({kfn, W}) : ctx->wave_attr.end();
    if (it != ctx->wave_attr.end()) {
      per_sm = it->second.per_sm;
    } else {
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wave::wave_kernel<V, DK, R>, (W + 1) * 32, smem) !=
              cudaSuccess ||
          per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
      }
      if (ctx->attr_cache) ctx->wave_attr[{kfn, W}] = WaveAttr{smem, per_sm};
    }
  }

  using Coord = typename V::coord;
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
  a.rowbuf = base + off_row;
  a.progress = reinterpret_cast<unsigned long long*>(base + 256);
  a.ticket = reinterpret_cast<int*>(base);
  a.err = ctx->d_err;
  a.out_dist = two ? nullptr : out_dist;     // two fronts: the combine writes the result
  a.out_dist2 = two ? nullptr : out_dist2;
  const bool fused = two && m <= kFusedCombineCols;
  a.combine = fused ? 1 : 0;
  a.done = reinterpret_cast<unsigned*>(base + 24);   // zeroed header word after the merge words
  a.res_dist = out_dist;
  a.res_dist2 = out_dist2;
  a.timeout_ns = timeout_ns(ctx);
  a.pstep = dim;
  a.nprob = two ? 2 : 1;
  a.p_b = two ? static_cast<const void*>(static_cast<const Coord*>(p) + (n - 1) * (int64_t)dim) : nullptr;
  a.n_b = n2;
  a.nbands_b = nb1;
  a.qpk_b = two ? base + off_q_b : nullptr;
  a.rowbuf_b = two ? base + off_row_b : nullptr;
  a.progress_b = reinterpret_cast<unsigned long long*>(base + off_prog_b);
  const int64_t nbands = nb0 + nb1;
  // persistent grid: every CTA that can be resident (a band is only ever
  // awaited by a later ticket, so CTAs that are not resident wait harmlessly)
  int grid = ctas > 0 ? ctas : per_sm * ctx->num_sms;
  grid = (int)std::min<int64_t>(grid, nbands);
  timing_begin(ctx, s);
  wave::wave_kernel<V, DK, R><<<grid, (W + 1) * 32, smem, s>>>(a);
  if (two && !fused) {
    // the merge words sit after the ticket in the zeroed scratch header
    const int cblocks = (int)std::max<int64_t>(1, std::min<int64_t>((m + 1023) / 1024, ctx->num_sms));
    wave::combine_kernel<V><<<cblocks, 256, 0, s>>>(a.rowbuf, a.rowbuf_b, m,
                                                    reinterpret_cast<unsigned long long*>(base + 16),
                                                    reinterpret_cast<unsigned*>(base + 8), a.err, out_dist,
                                                    out_dist2);
  }
  timing_end(ctx, s);
  return cuda_status(cudaGetLastError());
  }
}

}  // namespace dfd

#define DFD_WAVE_INSTANTIATE(V, DK, R)                                                                     \
  template dfd_status dfd::wave_launch<dfd::V, DK, R>(dfd_context*, int, const void*, int64_t, const void*, \
                                                        int64_t, void*, void*, cudaStream_t, int, int, bool);
