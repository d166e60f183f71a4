// variants.cu -- the appendix variants of the recurrence on the batch engine:
// DTW (the Frechet recurrence with the outer max replaced by a sum) and the
// Levenshtein distance (unit-cost edit distance), many pairs per launch.
//
// Same lane layout as the Frechet batch kernel (one warp per pair, rows =
// the plan's orientation, usually the shorter sequence, in stripes of 32*R,
// lane L at step s on column
// s - L, stripes handing their bottom row through a per-warp buffer) and
// the same device-built LPT work list; only the cell rule and the
// boundaries differ:
//   DTW:          D_ij = fl(min(D_{i-1,j}, D_{i-1,j-1}, D_{i,j-1}) + c_ij),
//                 c_ij the float32 squared distance, boundaries +inf,
//                 corner 0 (the running sums of the first row / column);
//   Levenshtein:  E_ij = min(min(E_{i-1,j}, E_{i,j-1}) + 1,
//                            E_{i-1,j-1} + [a_i != b_j]),
//                 boundaries E_{i,-1} = i + 1, E_{-1,j} = j + 1, corner 0
//                 (the textbook table; the appendix listing's start
//                 differs by one and is read as this); the columns left of
//                 the table (the systolic ramp) see a symbol that differs
//                 from every real one, which keeps them at E_{i,-1}.
// Unlike the Frechet distance neither is invariant under repeating a point,
// so the result is read at row n - 1 (the padding rows of the last stripe
// are computed and ignored).
#include <algorithm>
#include "batch_launch.cuh"
#include "dfd_internal.h"

namespace dfd {
namespace variant {

struct DtwOp {
  using V = F32;
  using coord = float;
  using value = float;
  static constexpr bool lev = false;
};
struct LevOp {
  using V = I32;
  using coord = int32_t;
  using value = int;
  static constexpr bool lev = true;
};

template <class Op, int DK, int R>
__device__ __forceinline__ typename Op::value warp_var(const typename Op::coord* __restrict__ P, int n,
                                                       const typename Op::coord* __restrict__ Q, int m, int dim,
                                                       bool vec, typename Op::value* buf, int L, uint4* stage) {
  using T = typename Op::value;
  using Cd = typename Op::coord;
  using V = typename Op::V;
  using QR = batch::QRec<V, DK>;
  constexpr int NPL = QR::NPL;
  const T INF = Op::lev ? (T)0x3fffffff : (T)__int_as_float(0x7f800000);
  const int nstripes = (n + 32 * R - 1) / (32 * R);
  T res = 0;
  for (int st = 0; st < nstripes; ++st) {
    Cd pr[R][DK];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = min(st * 32 * R + L * R + r, n - 1);
#pragma unroll
      for (int k = 0; k < DK; ++k) pr[r][k] = k < dim ? __ldg(P + (int64_t)i * dim + k) : (Cd)0;
    }
    // DTW: rows packed in pairs, two distances per f32x2 instruction (the
    // per-element rounding of the scalar order)
    constexpr bool kPack = !Op::lev && R >= 2;
    unsigned long long pp[kPack ? R / 2 : 1][DK];
    if constexpr (kPack) {
#pragma unroll
      for (int h = 0; h < R / 2; ++h) {
#pragma unroll
        for (int k = 0; k < DK; ++k) pp[h][k] = pack2(pr[2 * h][k], pr[2 * h + 1][k]);
      }
    }
    const bool has_top = st > 0, has_bottom = st + 1 < nstripes, last = !has_bottom;
    const int row0 = st * 32 * R + L * R;   // global row of the lane's first row
    T v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = Op::lev ? (T)(row0 + r + 1) : INF;
    T bout = v[R - 1];
    T upp = Op::lev ? (T)row0 : ((st == 0 && L == 0) ? (T)0 : INF);
    // lane and register of row n - 1 (last stripe)
    const int li = n - 1 - st * 32 * R;
    const int lres = li / R, rres = li % R;
    const int nsteps = m + 31;
    // q through the per-warp window of the batch engine (columns c0-32 ..
    // c0+31 in slots 0..63 during the block of c0, one record load per step)
    Cd qpre[DK];
    batch::load_point<Cd, DK>(Q, min(L, m - 1), dim, vec, qpre);
    const uint4* sb = stage + (32 - L);
    T* outb = reinterpret_cast<T*>(stage + NPL * 64);
    for (int c0 = 0; c0 < nsteps; c0 += 32) {
      T top_blk;
      if (has_top)
        top_blk = buf[min(c0 + L, m - 1)];
      else
        top_blk = Op::lev ? (T)(c0 + L + 1) : INF;
      __syncwarp();
#pragma unroll
      for (int c = 0; c < NPL; ++c) {
        uint4 lower = c0 > 0 ? stage[c * 64 + 32 + L] : batch::make_qrec<V, DK>(qpre, c);
        // Levenshtein: columns left of the table (the first block's lower
        // window) read a symbol with second coordinate 1, which differs from
        // every real symbol (dim 1: second coordinate 0).  With d = 1 there the
        // cell rule reproduces the boundary E_{i,-1} = i + 1 exactly
        // (min(min(i+1, i) + 1, i + 1)), so no per-cell mask is needed.
        if constexpr (Op::lev) {
          if (c0 == 0 && c == 0) lower.y = 1u;
        }
        stage[c * 64 + L] = lower;
        stage[c * 64 + 32 + L] = batch::make_qrec<V, DK>(qpre, c);
      }
      __syncwarp();
      batch::load_point<Cd, DK>(Q, min(c0 + 32 + L, m - 1), dim, vec, qpre);
      uint4 qr[NPL];
#pragma unroll
      for (int c = 0; c < NPL; ++c) qr[c] = sb[c * 64];
#pragma unroll 4
      for (int s = 0; s < 32; ++s) {
        const int j = c0 + s - L;
        uint4 qn[NPL];
        if (s + 1 < 32) {
#pragma unroll
          for (int c = 0; c < NPL; ++c) qn[c] = sb[c * 64 + s + 1];
        }
        T d[R];
        if constexpr (Op::lev) {
          Cd qk[DK];
#pragma unroll
          for (int c = 0; c < NPL; ++c) {
            qk[4 * c] = *reinterpret_cast<const Cd*>(&qr[c].x);
            if (4 * c + 1 < DK) qk[4 * c + 1] = *reinterpret_cast<const Cd*>(&qr[c].y);
            if (4 * c + 2 < DK) qk[4 * c + 2] = *reinterpret_cast<const Cd*>(&qr[c].z);
            if (4 * c + 3 < DK) qk[4 * c + 3] = *reinterpret_cast<const Cd*>(&qr[c].w);
          }
#pragma unroll
          for (int r = 0; r < R; ++r) {
            bool diff = false;
#pragma unroll
            for (int k = 0; k < DK; ++k) diff |= pr[r][k] != qk[k];   // coordinates past dim are 0 on both sides
            d[r] = diff ? 1 : 0;
          }
        } else if constexpr (QR::kind == batch::kDup) {
          unsigned long long qd[2];
          qd[0] = ((unsigned long long)qr[0].y << 32) | qr[0].x;
          qd[1] = ((unsigned long long)qr[0].w << 32) | qr[0].z;
#pragma unroll
          for (int h = 0; h < R / 2; ++h) {
            const unsigned long long t0 = sub2(pp[h][0], qd[0]);
            const unsigned long long t1 = sub2(pp[h][1], qd[1]);
            const unsigned long long acc = fma2(t1, t1, mul2(t0, t0));
            d[2 * h] = lo2(acc);
            d[2 * h + 1] = hi2(acc);
          }
          if constexpr ((R & 1) != 0) {
            const Cd qk[DK] = {__uint_as_float(qr[0].x), __uint_as_float(qr[0].z)};
            d[R - 1] = dist2<DK>(pr[R - 1], qk);
          }
        } else {
          Cd qk[DK];
#pragma unroll
          for (int c = 0; c < NPL; ++c) {
            qk[4 * c] = *reinterpret_cast<const Cd*>(&qr[c].x);
            if (4 * c + 1 < DK) qk[4 * c + 1] = *reinterpret_cast<const Cd*>(&qr[c].y);
            if (4 * c + 2 < DK) qk[4 * c + 2] = *reinterpret_cast<const Cd*>(&qr[c].z);
            if (4 * c + 3 < DK) qk[4 * c + 3] = *reinterpret_cast<const Cd*>(&qr[c].w);
          }
          if constexpr (kPack) {
            unsigned long long qd[DK];
#pragma unroll
            for (int k = 0; k < DK; ++k) qd[k] = pack2(qk[k], qk[k]);
#pragma unroll
            for (int h = 0; h < R / 2; ++h) {
              const unsigned long long t0 = sub2(pp[h][0], qd[0]);
              unsigned long long acc = mul2(t0, t0);
#pragma unroll
              for (int k = 1; k < DK; ++k) {
                const unsigned long long t = sub2(pp[h][k], qd[k]);
                acc = fma2(t, t, acc);
              }
              d[2 * h] = lo2(acc);
              d[2 * h + 1] = hi2(acc);
            }
            if constexpr ((R & 1) != 0) d[R - 1] = dist2<DK>(pr[R - 1], qk);
          } else {
#pragma unroll
            for (int r = 0; r < R; ++r) d[r] = dist2<DK>(pr[r], qk);
          }
        }
        const T tin = __shfl_sync(0xffffffffu, top_blk, s);
        T u = __shfl_up_sync(0xffffffffu, bout, 1);
        u = (L == 0) ? tin : u;
        T up = u, dg = upp;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const T l = v[r];
          T nv;
          if constexpr (Op::lev) {
            nv = min(min(l, up) + 1, dg + d[r]);   // columns left of the table keep E_{i,-1} (sentinel symbol)
          } else {
            nv = __fadd_rn(F32::vmin3(l, dg, up), d[r]);
          }
          dg = l;
          v[r] = nv;
          up = nv;
        }
        upp = u;
        bout = up;
        if (has_bottom && L == 31) outb[s] = bout;   // column c0 + s - 31 of the stripe's bottom row
        if (last && L == lres && j == m - 1) {
#pragma unroll
          for (int r = 0; r < R; ++r)
            if (r == rres) res = v[r];
        }
#pragma unroll
        for (int c = 0; c < NPL; ++c) qr[c] = qn[c];
      }
      __syncwarp();
      if (has_bottom) {
        const int oc = c0 + L - 31;
        if (oc >= 0 && oc < m) buf[oc] = outb[L];
      }
    }
    if (last) res = __shfl_sync(0xffffffffu, res, lres);
  }
  return res;
}

template <class Op, int DK>
__device__ __forceinline__ typename Op::value warp_var_any(const typename Op::coord* P, int n,
                                                           const typename Op::coord* Q, int m, int dim, bool vec,
                                                           typename Op::value* buf, int L, uint4* stage) {
  constexpr int RM = batch::Rmax<DK>::value;
  switch (batch::rows_per_lane<DK>(n)) {
#define DFD_V_CASE(RR) \
  case RR:             \
    if constexpr (RR < RM) return warp_var<Op, DK, RR>(P, n, Q, m, dim, vec, buf, L, stage); \
    break;
    DFD_V_CASE(1)
    DFD_V_CASE(2)
    DFD_V_CASE(3)
    DFD_V_CASE(4)
    DFD_V_CASE(5)
    DFD_V_CASE(6)
    DFD_V_CASE(7)
    default:
      break;
#undef DFD_V_CASE
  }
  return warp_var<Op, DK, RM>(P, n, Q, m, dim, vec, buf, L, stage);
}

template <class Op, int DK>
__global__ void __launch_bounds__(256, batch::kBlocksPerSM<DK>::value) variant_kernel(batch::BatchArgs a) {
  using T = typename Op::value;
  using Cd = typename Op::coord;
  __shared__ uint4 stage_sm[8][batch::QStage<DK>::RECS];
  uint4* stage = stage_sm[threadIdx.x >> 5];
  const int L = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  T* buf = static_cast<T*>(a.rowbuf) + gw * batch::BUF_COLS;
  const Cd* pts = static_cast<const Cd*>(a.points);
  const int64_t total = a.offsets[a.n_curves];
  if (ld_relaxed_i32(a.err) != 0) return;
  for (bool first = true;; first = false) {
    int item = 0;
    if (L == 0) item = first ? batch::pop_first(a.counter, a.sm_rank, a.n_sm, a.n_items) : atomicAdd(a.counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= a.n_items) break;
    const unsigned w = a.worklist[item];
    const int64_t k = w & (batch::kNarrowBit - 1);
    int32_t ia = a.pairs[2 * k], ib = a.pairs[2 * k + 1];
    if (w >> 31) {
      const int32_t t = ia;
      ia = ib;
      ib = t;
    }
    if (ia < 0 || ib < 0 || ia >= a.n_curves || ib >= a.n_curves) continue;  // reported by the plan
    const int64_t oa = a.offsets[ia], ob = a.offsets[ib];
    const int64_t ea = a.offsets[ia + 1], eb = a.offsets[ib + 1];
    if (oa < 0 || ob < 0 || ea > total || eb > total) continue;
    const int n = (int)(ea - oa), m = (int)(eb - ob);
    if (n < 1 || m < 1) continue;
    if (!batch::fits_buffer<DK>(n, m)) {
      // longer curve wider than a warp's row buffer: no value; NaN / -1 and the error word say so
      if (L == 0) {
        raise_error(a.err, DFD_ERR_UNSUPPORTED);
        if constexpr (Op::lev)
          static_cast<long long*>(a.out_dist2)[k] = -1;
        else
          static_cast<float*>(a.out_dist2)[k] = __int_as_float(0x7fffffff);
      }
      continue;
    }
    const T r = warp_var_any<Op, DK>(pts + oa * a.dim, n, pts + ob * a.dim, m, a.dim, a.vec != 0, buf, L, stage);
    if (L == 0) {
      if constexpr (Op::lev)
        static_cast<long long*>(a.out_dist2)[k] = (long long)r;
      else
        static_cast<float*>(a.out_dist2)[k] = r;
    }
  }
}

template <class Op, int DK>
dfd_status variant_launch(dfd_context* ctx, int dim, const void* points, const int64_t* offsets, int64_t n_curves,
                          const int32_t* pairs, int64_t n_pairs, void* out, cudaStream_t s) {
  const int blocks = resident_blocks(ctx, variant_kernel<Op, DK>, 256);
  batch::BatchArgs ba;
  dfd_status st = batch_prepare<typename Op::V, DK>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, s, blocks, &ba);
  if (st != DFD_OK) return st;
  ba.out_dist2 = out;
  timing_begin(ctx, s);
  variant_kernel<Op, DK><<<blocks, 256, 0, s>>>(ba);
  timing_end(ctx, s);
  return cuda_status(cudaGetLastError());
}

}  // namespace variant
}  // namespace dfd

using namespace dfd;

extern "C" dfd_status dfd_batch_variant(dfd_context* ctx, dfd_variant var, dfd_dtype dtype, int dim,
                                        const void* points, const int64_t* offsets, int64_t n_curves,
                                        const int32_t* pairs, int64_t n_pairs, void* out, void* stream) {
  if (!ctx || !points || !offsets || !pairs || !out || n_curves < 1 || n_pairs < 0) return DFD_ERR_INVALID_ARG;
  if (n_curves > INT32_MAX || n_pairs > INT32_MAX) return DFD_ERR_UNSUPPORTED;
  if (var == DFD_VARIANT_DTW) {
    if (dtype != DFD_F32 || dim < 1) return DFD_ERR_INVALID_ARG;
    if (dim > 16) return DFD_ERR_UNSUPPORTED;
  } else if (var == DFD_VARIANT_LEVENSHTEIN) {
    if (dtype != DFD_I32 || dim != 1) return DFD_ERR_INVALID_ARG;
  } else {
    return DFD_ERR_INVALID_ARG;
  }
  if (n_pairs == 0) return DFD_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (var == DFD_VARIANT_LEVENSHTEIN)
    return variant::variant_launch<variant::LevOp, 2>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, out, s);
  switch (dim_class(dim)) {
    case 2: return variant::variant_launch<variant::DtwOp, 2>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, out, s);
    case 3: return variant::variant_launch<variant::DtwOp, 3>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, out, s);
    case 4: return variant::variant_launch<variant::DtwOp, 4>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, out, s);
    case 8: return variant::variant_launch<variant::DtwOp, 8>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, out, s);
    case 16: return variant::variant_launch<variant::DtwOp, 16>(ctx, dim, points, offsets, n_curves, pairs, n_pairs, out, s);
    default: return DFD_ERR_UNSUPPORTED;
  }
}
