// wave_launch.cuh -- host launcher of the band wavefront (K2), instantiated
// per (value type, dimension class, rows per lane) in wave_*.cu.
#pragma once
#include <algorithm>
#include <type_traits>
#include "dfd_internal.h"
#include "wave_kernel.cuh"

namespace dfd {

template <class V, int DK, int R>
dfd_status wave_launch(dfd_context* ctx, int dim, const void* p, int64_t n, const void* q, int64_t m,
                       void* out_dist, void* out_dist2, cudaStream_t s, int W, int ctas) {
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
  const int64_t nbands = (n + H - 1) / H;
  // Lane 31's bottom row reaches column m - 1 at step m - 1 + 32*K - 1.
  const int64_t nblk64 = (m + 32 * K - 1 + wave::G - 1) / wave::G;
  if (nblk64 * wave::G > (int64_t)INT32_MAX / 2) return DFD_ERR_UNSUPPORTED;
  const int nblk = (int)nblk64;
  // The look-ahead of the last steps reads columns up to nblk*G + 1.
  const int nch = (nblk * wave::G + 2 + C - 1) / C;

  const size_t off_prog = 256;
  const size_t off_row = align_up(off_prog + (size_t)nbands * sizeof(unsigned long long), 256);
  const size_t off_q = align_up(off_row + (size_t)m * sizeof(T), 256);
  const size_t total = off_q + (size_t)nch * Lay::NPL * C * sizeof(Rec);
  dfd_status st = ensure_scratch(ctx, total);
  if (st != DFD_OK) return st;
  char* base = static_cast<char*>(ctx->scratch);

  cudaError_t e = cudaMemsetAsync(base, 0, off_row, s);
  if (e != cudaSuccess) return cuda_status(e);
  {
    const int64_t recs = (int64_t)nch * C * Lay::NPL;
    const int threads = 256;
    const int blocks = (int)std::min<int64_t>((recs + threads - 1) / threads, 4 * (int64_t)ctx->num_sms);
    wave::pack_q_kernel<V, DK><<<blocks, threads, 0, s>>>(static_cast<const typename V::coord*>(q), m, dim, nch,
                                                         wave::QTrans<V, R>::value, base + off_q);
  }
  const size_t smem = Lay::bytes(W);
  if (smem > ctx->smem_optin) return DFD_ERR_UNSUPPORTED;
  e = cudaFuncSetAttribute(wave::wave_kernel<V, DK, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_status(e);

  wave::Args a;
  a.p = p;
  a.n = n;
  a.dim = dim;
  a.qpk = base + off_q;
  a.m = m;
  a.nch = nch;
  a.nblk = nblk;
  a.H = H;
  a.nbands = nbands;
  a.rowbuf = base + off_row;
  a.progress = reinterpret_cast<unsigned long long*>(base + off_prog);
  a.ticket = reinterpret_cast<int*>(base);
  a.err = ctx->d_err;
  a.out_dist = out_dist;
  a.out_dist2 = out_dist2;
  a.timeout_ns = timeout_ns(ctx);
  int grid = ctas > 0 ? ctas : ctx->num_sms;
  grid = (int)std::min<int64_t>(grid, nbands);
  timing_begin(ctx, s);
  wave::wave_kernel<V, DK, R><<<grid, (W + 1) * 32, smem, s>>>(a);
  timing_end(ctx, s);
  return cuda_status(cudaGetLastError());
  }
}

}  // namespace dfd

#define DFD_WAVE_INSTANTIATE(V, DK, R)                                                                     \
  template dfd_status dfd::wave_launch<dfd::V, DK, R>(dfd_context*, int, const void*, int64_t, const void*, \
                                                        int64_t, void*, void*, cudaStream_t, int, int);
