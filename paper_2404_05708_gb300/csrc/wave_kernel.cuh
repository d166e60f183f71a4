// wave_kernel.cuh -- K2: band wavefront for one (long) pair of curves.
//
// The (n x m) recurrence of Eq. 1 is cut into horizontal bands of
// H = W * 32 * R rows.  A persistent CTA takes bands in order from an atomic
// ticket, so the band it waits on is always owned by a CTA that is already
// running.  Inside a CTA:
//   * W compute warps each own a stripe of 32 * R rows; lane L holds R
//     consecutive rows (their points in registers) and the stripe is a
//     systolic array over the columns: at step s lane L updates column
//     s - L, taking its "up" input from lane L-1 (warp shuffle) and its own
//     left / diagonal values from registers (Alg. 5's row state, split by
//     rows).  Lane 0 reads the stripe above from a shared-memory ring
//     written by the previous warp's lane 31; the handoff is ordered by
//     release / acquire counters, checked every G = 32 steps.
//   * one communication warp stages the q points into a shared-memory ring
//     with 1-D TMA bulk copies (full / empty mbarriers), fills the top ring
//     of the band from the global row buffer once the band above has
//     published those columns (acquire), and copies the band's bottom row
//     back to the global row buffer and publishes it (release).
// Only the row buffer (m values) and one progress word per band live in
// HBM, so the memory is O(n + m) (the prefix property of Sec. 3: row i of M
// summarises rows 1..i).  Every wait is bounded and ends the kernel with
// DFD_ERR_TIMEOUT in the context error word instead of hanging.
#pragma once
#include <type_traits>
#include "dfd_device.cuh"
#include "wave_shape.h"

namespace dfd {
namespace wave {

template <int DK>
struct ChunkCols {
  static constexpr int value = chunk_cols(DK);
};

// Column skew between neighbouring lanes.  float32 lanes (and the narrow
// int32 class, whose values are floats) hold K = R/2 row pairs and pair h
// runs h columns behind pair 0, so the K pairs of one step are independent
// (the "up" of pair h is pair h-1's value from the step before); lane L+1
// runs K columns behind lane L.  Exact int64 lanes keep all R rows in one
// column (K = 1).
template <class V>
struct Skewed {
  static constexpr bool value = !std::is_same<V, I32>::value;
};
template <class V, int R>
struct Skew {
  static constexpr int value = skew(Skewed<V>::value, R);
};

// Compute warps per CTA the register file allows (the kernel's launch bound).
template <class V, int DK, int R>
struct kMaxWarps {
  static constexpr int value = max_warps_regs(Skewed<V>::value, DK, R, std::is_same<V, I32B>::value);
};

// Position of column cc (0 <= cc < C) inside a packed q chunk plane: lanes
// K columns apart read records K * 16 bytes apart, which for even K maps
// several lanes to one bank group, so chunks are stored by column residue
// mod TR = K ([cc mod TR][cc / TR]) for K in {2, 4} (TR = 1 otherwise).
__host__ __device__ __forceinline__ int qpos(int cc, int TR, int C) {
  return TR > 1 ? (cc & (TR - 1)) * (C / TR) + cc / TR : cc;
}

struct Args {
  const void* p;
  int64_t n;
  int dim;
  const void* qpk;        // packed q: [nch][NPL][C] 16-byte records
  int64_t m;
  int nch;                // q chunks per band
  int nblk;               // G-step blocks per band
  int64_t H;              // rows per band
  int64_t nbands;
  void* rowbuf;           // value[m]: bottom row of the latest band, in place
  unsigned long long* progress;  // [nbands] columns of rowbuf published by band b
  int* ticket;
  int* err;
  void* out_dist;
  void* out_dist2;
  unsigned long long timeout_ns;
  int64_t pstep;          // elements from one row of p to the next
  // Optional second problem in the same launch (nprob == 2): the last n_b
  // rows of the pair taken backwards (p_b points at the last row, row
  // stride -pstep) against q reversed (its own packed stream qpk_b), with
  // its own row buffer and progress words.  Tickets alternate between the
  // two problems.
  int nprob;
  const void* p_b;
  int64_t n_b;
  int64_t nbands_b;
  const void* qpk_b;
  void* rowbuf_b;
  unsigned long long* progress_b;
  // Two fronts on a row short enough (combine != 0): the last CTA to leave
  // meets them itself (combine_block) and writes res_dist / res_dist2;
  // `done` counts the CTAs that have left (zero before the launch).
  int combine;
  unsigned* done;
  void* res_dist;
  void* res_dist2;
  // int32 pairs launch a narrow-class and an exact-class kernel back to
  // back; each CTA reduces the prep kernel's bounding-box partials (box:
  // nbox blocks of DK (min, max) pairs) and leaves at once unless the pair's
  // class is its own (want: 1 narrow, 0 exact).  box == nullptr: no choice.
  const int* box;
  int nbox;
  int want;
};

// The fields of Args that differ between the two problems of a launch.
struct Prob {
  const void* p;
  int64_t n;
  int64_t pstep;
  const void* qpk;
  void* rowbuf;
  unsigned long long* progress;
  int64_t nbands;
};

// ------------------------------------------------ rows held by one lane
template <class V, int DK, int R>
struct Rows;

// float32: rows packed in pairs, two cells per f32x2 instruction.  The packed
// q record holds every coordinate twice: plane c = (q_2c, q_2c, q_2c+1, q_2c+1).
template <int DK, int R>
struct Rows<F32, DK, R> {
  static_assert(R % 2 == 0, "float32 rows are processed in pairs");
  static constexpr int NPL = (DK + 1) / 2;
  using Rec = float4;
  unsigned long long pp[R / 2][DK];

  __device__ __forceinline__ void load(const float* P, int64_t r0, int64_t rlast, int dim, int64_t pstep) {
#pragma unroll
    for (int h = 0; h < R / 2; ++h) {
      const int64_t i0 = min(r0 + 2 * h, rlast), i1 = min(r0 + 2 * h + 1, rlast);
#pragma unroll
      for (int k = 0; k < DK; ++k) {
        const float a = k < dim ? P[i0 * pstep + k] : 0.f;
        const float b = k < dim ? P[i1 * pstep + k] : 0.f;
        pp[h][k] = pack2(a, b);
      }
    }
  }

  // Rows 2h, 2h+1 against one q point given as its NPL packed planes.
  // (h must be a compile-time constant after unrolling.)
  __device__ __forceinline__ void dist_pair(int h, const float4 (&t)[NPL], float& d0, float& d1) const {
    unsigned long long qk[DK];
#pragma unroll
    for (int c = 0; c < NPL; ++c) {
      qk[2 * c] = pack2(t[c].x, t[c].y);
      if (2 * c + 1 < DK) qk[2 * c + 1] = pack2(t[c].z, t[c].w);
    }
    const unsigned long long u0 = sub2(pp[h][0], qk[0]);
    unsigned long long acc = mul2(u0, u0);
#pragma unroll
    for (int k = 1; k < DK; ++k) {
      const unsigned long long u = sub2(pp[h][k], qk[k]);
      acc = fma2(u, u, acc);
    }
    d0 = lo2(acc);
    d1 = hi2(acc);
  }

  __device__ __forceinline__ void dist(const Rec* qp, int plane_stride, float d[R]) const {
    unsigned long long qk[DK];
#pragma unroll
    for (int c = 0; c < NPL; ++c) {
      const float4 t = qp[c * plane_stride];
      qk[2 * c] = pack2(t.x, t.y);
      if (2 * c + 1 < DK) qk[2 * c + 1] = pack2(t.z, t.w);
    }
#pragma unroll
    for (int h = 0; h < R / 2; ++h) {
      const unsigned long long t = sub2(pp[h][0], qk[0]);
      unsigned long long acc = mul2(t, t);
#pragma unroll
      for (int k = 1; k < DK; ++k) {
        const unsigned long long u = sub2(pp[h][k], qk[k]);
        acc = fma2(u, u, acc);
      }
      d[2 * h] = lo2(acc);
      d[2 * h + 1] = hi2(acc);
    }
  }
};

// int32: plane c = (q_4c, q_4c+1, q_4c+2, q_4c+3), exact int64 squares.
template <int DK, int R>
struct Rows<I32, DK, R> {
  static constexpr int NPL = (DK + 3) / 4;
  using Rec = int4;
  int pr[R][DK];

  __device__ __forceinline__ void load(const int32_t* P, int64_t r0, int64_t rlast, int dim, int64_t pstep) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = min(r0 + r, rlast);
#pragma unroll
      for (int k = 0; k < DK; ++k) pr[r][k] = k < dim ? P[i * pstep + k] : 0;
    }
  }

  __device__ __forceinline__ void dist(const Rec* qp, int plane_stride, long long d[R]) const {
    int qk[NPL * 4];
#pragma unroll
    for (int c = 0; c < NPL; ++c) {
      const int4 t = qp[c * plane_stride];
      qk[4 * c] = t.x;
      qk[4 * c + 1] = t.y;
      qk[4 * c + 2] = t.z;
      qk[4 * c + 3] = t.w;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int t = pr[r][0] - qk[0];
      long long acc = (long long)t * t;
#pragma unroll
      for (int k = 1; k < DK; ++k) {
        const int u = pr[r][k] - qk[k];
        acc += (long long)u * u;
      }
      d[r] = acc;
    }
  }
};

// Narrow int32 class (values are the exact uint32 squared distances carried
// as float bits, see I32B): the float32 stripe's row pairs and q ring
// geometry (NPL 16-byte planes a column), with the q record holding the
// words (-2 q_0, ..., -2 q_{DK-1}, |q|^2, 0...) and each row its int32
// coordinates and |p|^2.  d^2 = |p|^2 + |q|^2 + sum_k p_k (-2 q_k) in uint32
// arithmetic: every term wraps mod 2^32 and the true value lies below
// 0x7F800000, so the wrapped sum is that value exactly.
template <int DK, int R>
struct Rows<I32B, DK, R> {
  static_assert(R % 2 == 0, "rows are processed in pairs");
  static constexpr int NPL = (DK + 1) / 2;
  using Rec = float4;
  int pr[R][DK];
  unsigned pn[R];

  __device__ __forceinline__ void load(const int32_t* P, int64_t r0, int64_t rlast, int dim, int64_t pstep) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = min(r0 + r, rlast);
      unsigned n2 = 0;
#pragma unroll
      for (int k = 0; k < DK; ++k) {
        pr[r][k] = k < dim ? P[i * pstep + k] : 0;
        n2 += (unsigned)pr[r][k] * (unsigned)pr[r][k];
      }
      pn[r] = n2;
    }
  }

  // word w of a record given as its NPL planes (w a compile-time constant
  // after unrolling)
  static __device__ __forceinline__ unsigned word(const float4 (&t)[NPL], int w) {
    const float4 v = t[w >> 2];
    const float x = (w & 3) == 0 ? v.x : (w & 3) == 1 ? v.y : (w & 3) == 2 ? v.z : v.w;
    return __float_as_uint(x);
  }

  __device__ __forceinline__ void dist_pair(int h, const float4 (&t)[NPL], float& d0, float& d1) const {
    const unsigned qn = word(t, DK);
    unsigned a0 = pn[2 * h] + qn, a1 = pn[2 * h + 1] + qn;
#pragma unroll
    for (int k = 0; k < DK; ++k) {
      const unsigned w = word(t, k);
      a0 += (unsigned)pr[2 * h][k] * w;
      a1 += (unsigned)pr[2 * h + 1][k] * w;
    }
    d0 = __uint_as_float(a0);
    d1 = __uint_as_float(a1);
  }
};

// One pair's result from its squared distance in the value type: float32
// as is; int32 as int64 delta^2 and double delta (the narrow class's float
// bits are the uint32 value).
template <class V>
__device__ __forceinline__ void write_pair_result(void* out_dist, void* out_dist2, typename V::value x) {
  if constexpr (std::is_same<V, F32>::value) {
    if (out_dist2) static_cast<float*>(out_dist2)[0] = x;
    if (out_dist) static_cast<float*>(out_dist)[0] = sqrtf(x);
  } else {
    long long v;
    if constexpr (std::is_same<V, I32B>::value)
      v = (long long)__float_as_uint(x);
    else
      v = (long long)x;
    if (out_dist2) static_cast<long long*>(out_dist2)[0] = v;
    if (out_dist) static_cast<double*>(out_dist)[0] = sqrt((double)v);
  }
}

// Whether an int32 pair is narrow: every coordinate's range over p and q at
// most 46340 and the sum of the squared ranges at most 0x7F7FFFFF, so that
// every squared distance is exact in uint32 below the first float NaN
// pattern.  box holds nbox partial boxes of DK (min, max) pairs (the prep
// kernel's blocks; coordinates past dim are zero).  Called by every thread
// of the block; sh: 2 * DK + 1 ints of shared memory, free on return.
template <int DK>
__device__ __forceinline__ bool box_narrow_block(const int* box, int nbox, int* sh) {
  if (threadIdx.x < 2 * DK) sh[threadIdx.x] = (threadIdx.x & 1) ? INT_MIN : INT_MAX;
  __syncthreads();
  // one coordinate at a time: two values live, whatever DK
#pragma unroll 1
  for (int k = 0; k < DK; ++k) {
    int lo = INT_MAX, hi = INT_MIN;
    for (int b = threadIdx.x; b < nbox; b += blockDim.x) {
      lo = min(lo, __ldcg(box + (b * DK + k) * 2));
      hi = max(hi, __ldcg(box + (b * DK + k) * 2 + 1));
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&sh[2 * k], lo);
      atomicMax(&sh[2 * k + 1], hi);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    bool narrow = true;
    unsigned long long s2 = 0;
    for (int k = 0; k < DK; ++k) {
      const long long r = (long long)sh[2 * k + 1] - (long long)sh[2 * k];
      if (r < 0 || r > (long long)kI32BMaxRange)
        narrow = false;
      else
        s2 += (unsigned long long)(r * r);
    }
    sh[2 * DK] = narrow && s2 <= kI32BMaxD2 ? 1 : 0;
  }
  __syncthreads();
  const bool narrow = sh[2 * DK] != 0;
  __syncthreads();
  return narrow;
}

// --------------------------------------------------- shared-memory counters
__device__ __forceinline__ int ld_acquire_cta(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared::cta.s32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_cta(const int* p) {
  int v;
  asm volatile("ld.relaxed.cta.shared::cta.s32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_cta(int* p, int v) {
  asm volatile("st.release.cta.shared::cta.s32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_smem(const int* p) {
  return *reinterpret_cast<const volatile int*>(p);
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// A block's publication: one fence for the whole warp, then each counter
// store under a predicate.  The fence followed by a relaxed store is a
// release; __syncwarp before it has made the other lanes' ring stores
// visible to the storing lane.  (One fence and no divergent branch, where
// a release store per lane took two of each.)
__device__ __forceinline__ void fence_acq_rel_cta() { asm volatile("fence.acq_rel.cta;" ::: "memory"); }
__device__ __forceinline__ void st_relaxed_cta_if(int* p, int v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred P;\n\tsetp.ne.u32 P, %2, 0;\n\t@P st.relaxed.cta.shared::cta.s32 [%0], %1;\n\t}" ::"r"(
          smem_addr(p)),
      "r"(v), "r"((unsigned)pred)
      : "memory");
}
__device__ __forceinline__ void mbar_arrive_if(uint64_t* bar, bool pred) {
  asm volatile(
      "{\n\t.reg .pred P;\n\tsetp.ne.u32 P, %1, 0;\n\t@P mbarrier.arrive.shared::cta.b64 _, [%0];\n\t}" ::"r"(
          smem_addr(bar)),
      "r"((unsigned)pred)
      : "memory");
}

// Predicated shared-memory store without a branch (keeps the unrolled
// systolic block one basic block, so loads and distances of later steps can
// be scheduled under the min/max chain of earlier ones).
__device__ __forceinline__ void st_shared_if(float* p, float v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred P;\n\tsetp.ne.u32 P, %2, 0;\n\t@P st.shared.f32 [%0], %1;\n\t}" ::"r"(smem_addr(p)), "f"(v),
      "r"((unsigned)pred)
      : "memory");
}
__device__ __forceinline__ void st_shared_if(long long* p, long long v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred P;\n\tsetp.ne.u32 P, %2, 0;\n\t@P st.shared.s64 [%0], %1;\n\t}" ::"r"(smem_addr(p)), "l"(v),
      "r"((unsigned)pred)
      : "memory");
}

// Four-float variant (16-byte aligned address).  No "memory" clobber: the
// ring it writes is published by a later st.release (asm volatile, kept in
// order), and q / ring loads of later steps may be scheduled across it.
__device__ __forceinline__ void st_shared_if4(float* p, float4 v, bool pred) {
  asm volatile(
      "{\n\t.reg .pred P;\n\tsetp.ne.u32 P, %5, 0;\n\t@P st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n\t}" ::"r"(
          smem_addr(p)),
      "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"((unsigned)pred));
}

template <class T>
__device__ __forceinline__ T ld_cg(const T* p) {
  return __ldcg(p);
}
template <class T>
__device__ __forceinline__ void st_cg(T* p, T v) {
  __stcg(p, v);
}

struct Ctl {
  int band;
  int abort;
  int prod[17];   // columns written into ring k (k = 0..W)
  int cons[17];   // columns read from ring k
};

// Spin on a shared-memory counter; bounded by time and by the abort flag.
__device__ __forceinline__ bool spin_smem_geq(const int* cnt, int need, Ctl* ctl, int* err,
                                              unsigned long long timeout_ns) {
  if (ld_acquire_cta(cnt) >= need) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    if (ld_acquire_cta(cnt) >= need) return true;
    if (ld_volatile_smem(&ctl->abort)) return false;
    if (globaltimer_ns() - t0 > timeout_ns) {
      raise_error(err, DFD_ERR_TIMEOUT);
      *reinterpret_cast<volatile int*>(&ctl->abort) = 1;
      return false;
    }
  }
}

// Records mirrored past the end of each q ring row (see QRow).
constexpr int kQMirror = 64;

// q ring row geometry: a row (one plane and column residue) holds NQ*C/TR
// records followed by a mirror of its first kQMirror records, so the 34
// records a 32-step block reads from any start are contiguous and a step
// addresses its record at a fixed offset from the block's base.
template <int C, int TR>
struct QRow {
  static constexpr int NQ = nq_slots(C);
  static constexpr int RING_LEN = NQ * C / TR;      // records of the ring proper
  static constexpr int LEN = RING_LEN + kQMirror;   // records per row
  static constexpr int PLANE = TR * LEN;            // records per plane
};

template <class V, int DK, int R>
struct Layout {
  using Rows_ = Rows<V, DK, R>;
  using Rec = typename Rows_::Rec;
  using T = typename V::value;
  static constexpr int C = ChunkCols<DK>::value;
  static constexpr int NPL = Rows_::NPL;
  static constexpr int TR = (Skew<V, R>::value == 2 || Skew<V, R>::value == 4) ? Skew<V, R>::value : 1;
  using QR = QRow<C, TR>;
  static constexpr size_t q_bytes = (size_t)NPL * QR::PLANE * sizeof(Rec);
  static constexpr size_t bar_off = q_bytes;
  static constexpr int NQ = nq_slots(C);
  static constexpr size_t ring_off = bar_off + 2 * NQ * sizeof(uint64_t);
  static __host__ __device__ size_t ctl_off(int W) { return ring_off + (size_t)(W + 1) * RING * sizeof(T); }
  static __host__ __device__ size_t bytes(int W) { return ctl_off(W) + sizeof(Ctl); }
};

// ----------------------------------------------------------- ring indexing
// Inter-warp rings hold column c at index (c + 3) mod RING: lane 31 emits
// column c0 + s - (32K - 1) at step s and 32K - 1 = 3 (mod 4), so the four
// outputs of steps 4t..4t+3 land in one aligned 16-byte slot.
__device__ __forceinline__ int ridx(int c) { return (c + 3) & (RING - 1); }

// q ring: NQ chunks of C columns, plane-major ([plane][NQ*C] records); for
// lane skew K in {2, 4} each plane is further split by column residue mod
// TR = K ([plane][residue][NQ*C/TR]), so the 32 lanes of a step (K columns
// apart) read 32 consecutive records.  x is the column's position in the
// band-stream (chunk sequence * C + column), taken mod the ring size.
template <class V, int R>
struct QTrans {
  static constexpr int value = (Skew<V, R>::value == 2 || Skew<V, R>::value == 4) ? Skew<V, R>::value : 1;
};

// ----------------------------------------------------------- compute warp
// float32: one G-step block of the skewed systolic stripe.  At step s pair h
// of lane L updates column c0 + s - K*L - h (rows 2h, 2h+1 of the lane):
//   row 2h:   up = pair h-1's bottom value of the previous step, diag = that
//             of the step before (lane L-1's bottom row by shuffle for h = 0,
//             the ring above for lane 0), left = its own previous value;
//   row 2h+1: up = row 2h of this step, diag / left = the previous values.
// The K pairs of a step are independent, so the only chain a step carries
// is two cells long.  Pair 0's q record is loaded two steps ahead and slides
// to pair h after h steps in registers; the shuffle for the next step is
// issued as soon as the bottom pair is done.
template <int DK, int R>
struct SkewState {
  static constexpr int K = R / 2;
  static constexpr int NPL = (DK + 1) / 2;
  float v0[K], v1[K], pv1[K];   // rows 2h, 2h+1 now; row 2h+1 one step ago
  float dcur[K][2];             // distances of the coming step
  float4 win[K][NPL];           // win[j]: pair 0's record j steps ago (j < K-1 used)
  float4 nrec1[NPL];            // pair 0's record of the coming step + 1
  float upp;                    // lane's diagonal input
  float ush;                    // lane L-1's bottom value, shuffled for the coming step
};

template <class RowsT, int DK, int R>
__device__ __forceinline__ void skew_block(const RowsT& rows, SkewState<DK, R>& st, const float* ring_in,
                                           float* ring_out, const float4* qring, unsigned xbase, int c0, int L) {
  constexpr int K = R / 2;
  constexpr int NPL = (DK + 1) / 2;
  constexpr int C = ChunkCols<DK>::value;
  constexpr int TR = (K == 2 || K == 4) ? K : 1;
  using QR = QRow<C, TR>;
  constexpr int SK = 32 * K - 1;
  // Lane 0's inputs from the ring above: columns c0..c0+31 at indices
  // c0+3..c0+34 (9 aligned float4 loads, broadcast).
  float rin[36];
#pragma unroll
  for (int k = 0; k < 36; k += 4) {
    const float4 t4 = *reinterpret_cast<const float4*>(ring_in + ((c0 + k) & (RING - 1)));
    rin[k] = t4.x;
    rin[k + 1] = t4.y;
    rin[k + 2] = t4.z;
    rin[k + 3] = t4.w;
  }
  float u = (L == 0) ? rin[3] : st.ush;
  // Stream position of pair 0's column at step 0 of this block; X = 0 mod TR.
  const unsigned X = xbase + (unsigned)(c0 - K * L);
  // the block's records start at ring position Xq mod the row length and
  // run on into the mirror: fixed offsets from one base
  const float4* qb = qring + ((X / TR) & (unsigned)(QR::RING_LEN - 1));
  float obuf[4];
#pragma unroll
  for (int s = 0; s < G; ++s) {
    // (1) pair 0's record for step s + 2
    float4 nrec2[NPL];
    {
      const float4* qp = qb + ((s + 2) % TR) * QR::LEN + (s + 2) / TR;
#pragma unroll
      for (int c = 0; c < NPL; ++c) nrec2[c] = qp[c * QR::PLANE];
    }
    // (2) the first rows of all pairs (independent), then the second rows
    // with the bottom pair first, so the shuffle for step s + 1 leaves early
    float unext;
    {
      float n0[K], n1[K];
#pragma unroll
      for (int h = K - 1; h >= 0; --h) {
        const int hp = h > 0 ? h - 1 : 0;
        const float up0 = h > 0 ? st.v1[hp] : u;   // pair 0: lane L-1 / ring above
        const float dg0 = h > 0 ? st.pv1[hp] : st.upp;
        n0[h] = F32::vmax(F32::vmin3(st.v0[h], dg0, up0), st.dcur[h][0]);
      }
#pragma unroll
      for (int h = K - 1; h >= 0; --h) n1[h] = F32::vmax(F32::vmin3(st.v1[h], st.v0[h], n0[h]), st.dcur[h][1]);
      unext = __shfl_up_sync(0xffffffffu, n1[K - 1], 1);
      obuf[s & 3] = n1[K - 1];
#pragma unroll
      for (int h = 0; h < K; ++h) {
        st.pv1[h] = st.v1[h];
        st.v0[h] = n0[h];
        st.v1[h] = n1[h];
      }
    }
    st.upp = u;
    // (4) distances of step s + 1
    rows.dist_pair(0, st.nrec1, st.dcur[0][0], st.dcur[0][1]);
#pragma unroll
    for (int h = 1; h < K; ++h) rows.dist_pair(h, st.win[h - 1], st.dcur[h][0], st.dcur[h][1]);
    // (5) lane 31's bottom values, four steps per store
    if ((s & 3) == 3) {
      const int c_last = c0 + s - SK;   // column of this step's output
      st_shared_if4(ring_out + ridx(c_last - 3), make_float4(obuf[0], obuf[1], obuf[2], obuf[3]),
                    L == 31 && c_last >= 0);
    }
    // (6) slide the records
#pragma unroll
    for (int j = K - 2; j > 0; --j) {
#pragma unroll
      for (int c = 0; c < NPL; ++c) st.win[j][c] = st.win[j - 1][c];
    }
#pragma unroll
    for (int c = 0; c < NPL; ++c) {
      st.win[0][c] = st.nrec1[c];
      st.nrec1[c] = nrec2[c];
    }
    if (s + 1 < G) {
      u = (L == 0) ? rin[s + 4] : unext;
    } else {
      st.ush = unext;
    }
  }
}

template <class V, int DK, int R>
__device__ __forceinline__ void compute_stripe(const Args& a, const Prob& pb, int w, int64_t band, unsigned gbase,
                                               unsigned char* smem) {
  using Lay = Layout<V, DK, R>;
  using T = typename V::value;
  using Rec = typename Lay::Rec;
  constexpr int C = Lay::C;
  constexpr int NPL = Lay::NPL;
  constexpr int NQ = Lay::NQ;
  constexpr int NQC = NQ * C;
  constexpr int K = Skew<V, R>::value;
  constexpr int SK = 32 * K - 1;
  constexpr bool kSkew = Skewed<V>::value;
  const int L = threadIdx.x & 31;
  const int W = (int)(blockDim.x >> 5) - 1;
  const Rec* qring = reinterpret_cast<const Rec*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Lay::bar_off);
  uint64_t* empty = full + NQ;
  T* rings = reinterpret_cast<T*>(smem + Lay::ring_off);
  Ctl* ctl = reinterpret_cast<Ctl*>(smem + Lay::ctl_off(W));
  const T* ring_in = rings + (size_t)w * RING;
  T* ring_out = rings + (size_t)(w + 1) * RING;

  using Coord = typename V::coord;
  Rows<V, DK, R> rows;
  const int64_t rb0 = band * a.H;
  const int64_t rend = min(rb0 + a.H, pb.n);
  rows.load(static_cast<const Coord*>(pb.p), rb0 + (int64_t)(w * 32 + L) * R, rend - 1, a.dim, pb.pstep);

  const bool corner = band == 0 && w == 0 && L == 0;
  const unsigned xbase = gbase * (unsigned)C;   // stream position of the band's column 0
  // int32 state: R rows in one column.
  T v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = V::inf();
  T bout = V::inf();
  T upp = corner ? V::zero() : V::inf();
  // float32 state: skewed pairs.
  using SS = SkewState<DK, (kSkew ? R : 2)>;
  SS ss;
  if constexpr (kSkew) {
#pragma unroll
    for (int h = 0; h < SS::K; ++h) ss.v0[h] = ss.v1[h] = ss.pv1[h] = V::inf();
    ss.upp = corner ? 0.f : V::inf();
    ss.ush = V::inf();
  }
  const int m = (int)a.m;
  int qdone = 0, qready = 0;

  for (int blk = 0; blk < a.nblk; ++blk) {
    const int c0 = blk * G;
    // One uniform check of both ring counters, the abort flag and the q
    // chunks through the one holding column c0 + G + 1 (the last steps'
    // look-ahead reads it); the slow path (a wait, or the first block,
    // which always waits for its first chunk) handles them one by one.
    const int need_in = min(c0 + G, m);
    const int need_out = c0 + G - SK - RING;
    const int qneed = min((c0 + G + 1) / C + 1, a.nch);
    const float4* qr = reinterpret_cast<const float4*>(qring);
    {
      // relaxed reads and one fence after the check (an acquire): cheaper
      // than two acquire loads (measured: 2 cycles a step)
      const int pv = ld_relaxed_cta(&ctl->prod[w]);
      const int cv = ld_relaxed_cta(&ctl->cons[w + 1]);
      const int ab = ld_volatile_smem(&ctl->abort);
      if (pv < need_in || cv < need_out || ab || qready < qneed) {
        if (pv < need_in || cv < need_out || ab) {
          // spin (bounded) only on the counter that is not there yet
          if (L == 0) spin_smem_geq(&ctl->prod[w], need_in, ctl, a.err, a.timeout_ns);
          if (L == 31) spin_smem_geq(&ctl->cons[w + 1], need_out, ctl, a.err, a.timeout_ns);
          __syncwarp();
          if (ld_volatile_smem(&ctl->abort)) break;
        }
        bool qok = true;
        while (qready < qneed) {
          const unsigned seq = gbase + (unsigned)qready;
          if (!mbar_wait(&full[seq & (NQ - 1)], (seq / NQ) & 1, a.err, a.timeout_ns)) {
            *reinterpret_cast<volatile int*>(&ctl->abort) = 1;
            qok = false;
            break;
          }
          ++qready;
        }
        if (!qok) break;
        if constexpr (kSkew) {
          if (blk == 0) {
            // Step 0 and step 1 records of pair 0 (columns -K*L and 1 - K*L;
            // negative columns read stale records and only ever produce +inf).
            constexpr int TRk = Lay::TR;
            using QRk = typename Lay::QR;
            auto rec_at = [&](unsigned x, float4 (&r)[NPL]) {
              const float4* qp = qr + (x % TRk) * QRk::LEN + ((x / TRk) & (unsigned)(QRk::RING_LEN - 1));
#pragma unroll
              for (int c = 0; c < NPL; ++c) r[c] = qp[c * QRk::PLANE];
            };
            float4 r0[NPL];
            rec_at(xbase - (unsigned)(K * L), r0);
            rec_at(xbase + 1u - (unsigned)(K * L), ss.nrec1);
#pragma unroll
            for (int h = 0; h < SS::K; ++h) {
#pragma unroll
              for (int c = 0; c < NPL; ++c) ss.win[h][c] = r0[c];
            }
            rows.dist_pair(0, r0, ss.dcur[0][0], ss.dcur[0][1]);
#pragma unroll
            for (int h = 1; h < SS::K; ++h) {
              ss.dcur[h][0] = ss.dcur[0][0];
              ss.dcur[h][1] = ss.dcur[0][1];
            }
          }
        }
      }
      fence_acq_rel_cta();
    }

    if constexpr (kSkew) {
      skew_block<Rows<V, DK, R>, DK, R>(rows, ss, reinterpret_cast<const float*>(ring_in),
                                        reinterpret_cast<float*>(ring_out), qr, xbase, c0, L);
    } else {
      auto qaddr = [&](int cq) { return qring + ((xbase + (unsigned)cq) & (unsigned)(NQC - 1)); };
      // The block's 32 ring inputs, one per lane (lane s holds column c0 + s);
      // at step s lane 0 takes lane s's value.  Lane 31's outputs are gathered
      // the same way (lane s keeps step s's) and stored after the block, so
      // the unrolled block has no shared-memory store and no branch.
      const T in_blk = ring_in[ridx(c0 + L)];
      T out_blk = V::inf();
#pragma unroll
      for (int s = 0; s < G; ++s) {
        const int col = c0 + s - L;
        const T rin = __shfl_sync(0xffffffffu, in_blk, s);
        T u = __shfl_up_sync(0xffffffffu, bout, 1);
        u = (L == 0) ? rin : u;
        T d[R];
        rows.dist(qaddr(max(col, 0)), Lay::QR::PLANE, d);
        T up = u, dg = upp;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const T l = v[r];
          const T nv = V::vmax(V::vmin3(l, dg, up), d[r]);
          dg = l;
          v[r] = nv;
          up = nv;
        }
        upp = u;
        bout = up;
        const T b31 = __shfl_sync(0xffffffffu, bout, 31);
        out_blk = (L == s) ? b31 : out_blk;
      }
      {
        const int oc = c0 + L - 31;   // column lane 31 produced at step L
        st_shared_if(ring_out + ridx(oc), out_blk, oc >= 0);
      }
    }
    __syncwarp();
    fence_acq_rel_cta();
    st_relaxed_cta_if(&ctl->prod[w + 1], c0 + G - SK, L == 31);
    st_relaxed_cta_if(&ctl->cons[w], c0 + G, L == 0);
    // q chunks no lane of this warp will read again: the next read is lane
    // 31's first one in the next block (float32: the look-ahead of step 2).
    // A block of G <= C columns finishes at most one chunk.
    static_assert(G <= C, "one chunk release per block");
    const int first_unread = c0 + G - 31 * K + (kSkew ? 2 : 0);
    const int consumed = min(max(0, first_unread) / C, a.nch);
    const bool release = qdone < consumed;
    mbar_arrive_if(&empty[(gbase + (unsigned)qdone) & (NQ - 1)], release && L == 0);
    qdone += release ? 1 : 0;
  }
  __syncwarp();
  while (qdone < a.nch) {
    if (L == 0) mbar_arrive(&empty[(gbase + (unsigned)qdone) & (NQ - 1)]);
    ++qdone;
  }
}

// ------------------------------------------------------- communication warp
template <class V, int DK, int R>
__device__ __forceinline__ void comm_warp(const Args& a, const Prob& pb, int64_t band, unsigned gbase,
                                          unsigned char* smem) {
  using Lay = Layout<V, DK, R>;
  using T = typename V::value;
  using Rec = typename Lay::Rec;
  constexpr int C = Lay::C;
  constexpr int NPL = Lay::NPL;
  constexpr unsigned CHUNK_BYTES = (unsigned)(NPL * C * sizeof(Rec));
  constexpr int NQ = Lay::NQ;
  constexpr int TR = Lay::TR;
  using QR = typename Lay::QR;
  static_assert(QTrans<V, R>::value == TR, "q ring residue split");
  const int L = threadIdx.x & 31;
  const int W = (int)(blockDim.x >> 5) - 1;
  Rec* qring = reinterpret_cast<Rec*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Lay::bar_off);
  uint64_t* empty = full + NQ;
  T* rings = reinterpret_cast<T*>(smem + Lay::ring_off);
  Ctl* ctl = reinterpret_cast<Ctl*>(smem + Lay::ctl_off(W));
  T* ring0 = rings;
  const T* ringW = rings + (size_t)W * RING;
  const Rec* qpk = static_cast<const Rec*>(pb.qpk);
  T* rowbuf = static_cast<T*>(pb.rowbuf);

  const int m = (int)a.m;
  const int fill_end = a.nblk * G;
  int issued = 0, filled = 0, drained = 0;
  unsigned long long pub = 0;   // columns of the band above known published
  unsigned long long t_idle = globaltimer_ns();
  bool aborted = false;

  for (;;) {
    bool progressed = false;
    // (1) next q chunk, once every compute warp has released its slot
    if (issued < a.nch) {
      const unsigned seq = gbase + (unsigned)issued;
      const unsigned slot = seq & (NQ - 1);
      const bool slot_free = seq < (unsigned)NQ || mbar_test_wait(&empty[slot], ((seq / NQ) - 1) & 1);
      if (slot_free) {
        if (L == 0) {
          // The first slots' leading records also go to the rows' mirrors.
          const int mir0 = (int)slot * (C / TR);
          const int nmir = mir0 < kQMirror ? min(C / TR, kQMirror - mir0) : 0;
          mbar_arrive_expect_tx(&full[slot], CHUNK_BYTES + (unsigned)(NPL * TR * nmir * sizeof(Rec)));
          // One copy per plane and column residue (the ring layout of QTrans).
#pragma unroll
          for (int pl = 0; pl < NPL; ++pl) {
#pragma unroll
            for (int r = 0; r < TR; ++r) {
              Rec* row = qring + (size_t)pl * QR::PLANE + (size_t)r * QR::LEN;
              const Rec* src = qpk + ((size_t)issued * NPL + pl) * C + (size_t)r * (C / TR);
              tma_load_1d(row + (size_t)slot * (C / TR), src, (unsigned)((C / TR) * sizeof(Rec)), &full[slot]);
              if (nmir > 0) tma_load_1d(row + QR::RING_LEN + mir0, src, (unsigned)(nmir * sizeof(Rec)), &full[slot]);
            }
          }
        }
        ++issued;
        progressed = true;
      }
    }
    // (2) top ring of the band: every 32-column unit that the band above
    // has published (acquire; re-polled only when the cached value falls
    // short) and the ring has room for, up to 4 units per L2 round trip.
    if (filled < fill_end) {
      const int room = ld_acquire_cta(&ctl->cons[0]) + RING - filled;
      int ready = fill_end - filled;
      if (band > 0) {
        if (pub < (unsigned long long)min(filled + 32, m)) {
          unsigned long long pv = 0;
          if (L == 0) pv = ld_acquire_u64(&pb.progress[band - 1]);
          pub = __shfl_sync(0xffffffffu, pv, 0);
        }
        // Columns past m are +inf padding, ready once column m - 1 is.
        ready = pub >= (unsigned long long)m ? fill_end - filled : (int)pub - filled;
      }
      const int units = min(min(ready, room) >> 5, 4);
      if (units > 0) {
        __syncwarp();   // order the lanes' loads after lane 0's acquire
        T val[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int col = filled + 32 * k + L;
          val[k] = V::inf();
          if (k < units && band > 0 && col < m) val[k] = ld_cg(rowbuf + col);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (k < units) ring0[ridx(filled + 32 * k + L)] = val[k];
        __syncwarp();
        filled += 32 * units;
        if (L == 0) st_release_cta(&ctl->prod[0], filled);
        progressed = true;
      }
    }
    // (3) drain the bottom ring to the global row buffer and publish it,
    // up to 4 units of 32 columns per release.
    if (drained < m) {
      const int pw = min(ld_acquire_cta(&ctl->prod[W]), m);
      const int units = min((pw - drained + (pw == m ? 31 : 0)) >> 5, 4);
      if (units > 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int col = drained + 32 * k + L;
          if (k < units && col < m) {
            const T val = ringW[ridx(col)];
            st_cg(rowbuf + col, val);
            if (band == pb.nbands - 1 && col == m - 1) write_pair_result<V>(a.out_dist, a.out_dist2, val);
          }
        }
        __syncwarp();
        drained = min(drained + 32 * units, m);
        if (L == 0) {
          st_release_cta(&ctl->cons[W], drained);
          // The release orders the warp's row-buffer stores (made visible to
          // lane 0 by __syncwarp) before the progress word at GPU scope.
          st_release_u64(&pb.progress[band], (unsigned long long)drained);
        }
        progressed = true;
      }
    }
    if (issued >= a.nch && filled >= fill_end && drained >= m) break;
    if (ld_volatile_smem(&ctl->abort) || ld_relaxed_i32(a.err) != 0) {
      aborted = true;
      break;
    }
    const unsigned long long now = globaltimer_ns();
    if (progressed) {
      t_idle = now;
    } else {
      if (now - t_idle > a.timeout_ns) {
        raise_error(a.err, DFD_ERR_TIMEOUT);
        aborted = true;
        break;
      }
      __nanosleep(64);
    }
  }
  if (aborted) {
    *reinterpret_cast<volatile int*>(&ctl->abort) = 1;
    // Let every bulk copy this warp started land before the CTA can leave.
    const int first = issued > NQ ? issued - NQ : 0;
    for (int c = first; c < issued; ++c) {
      const unsigned seq = gbase + (unsigned)c;
      mbar_wait(&full[seq & (NQ - 1)], (seq / NQ) & 1, a.err, a.timeout_ns);
    }
  }
}

// The meeting of the two fronts (see combine_kernel) by one CTA, at the end
// of the wavefront launch when the row is short: every other CTA has left,
// so both row buffers are final.  Loads bypass L1 (the rows were written by
// other SMs).  Nothing is written when the error word is set.
template <class V>
__device__ __forceinline__ void combine_block(const void* rowbuf_f, const void* rowbuf_b, int64_t m, const int* err,
                                              void* out_dist, void* out_dist2, typename V::value* part) {
  using T = typename V::value;
  const T* F = static_cast<const T*>(rowbuf_f);
  const T* B = static_cast<const T*>(rowbuf_b);
  T best = V::inf();
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x) {
    const T bj = __ldcg(B + (m - 1 - j));
    const T bj1 = j + 1 < m ? __ldcg(B + (m - 2 - j)) : V::inf();
    best = V::vmin(best, V::vmax(__ldcg(F + j), V::vmin(bj, bj1)));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) best = V::vmin(best, __shfl_xor_sync(0xffffffffu, best, off));
  const int warp = threadIdx.x >> 5, L = threadIdx.x & 31;
  if (L == 0) part[warp] = best;   // part: one value per warp (shared memory the caller no longer uses)
  __syncthreads();
  if (warp == 0) {
    T x = L < (int)(blockDim.x >> 5) ? part[L] : V::inf();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = V::vmin(x, __shfl_xor_sync(0xffffffffu, x, off));
    if (L == 0 && *(volatile const int*)err == 0) write_pair_result<V>(out_dist, out_dist2, x);
  }
}

// ------------------------------------------------------------------ kernel
template <class V, int DK, int R>
__global__ void __launch_bounds__((kMaxWarps<V, DK, R>::value + 1) * 32, 1) wave_kernel(Args a) {
  using Lay = Layout<V, DK, R>;
  using T = typename V::value;
  constexpr int NQ = Lay::NQ;
  extern __shared__ __align__(128) unsigned char smem[];
  const int W = (int)(blockDim.x >> 5) - 1;
  const int warp = threadIdx.x >> 5;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Lay::bar_off);
  uint64_t* empty = full + NQ;
  T* rings = reinterpret_cast<T*>(smem + Lay::ring_off);
  Ctl* ctl = reinterpret_cast<Ctl*>(smem + Lay::ctl_off(W));

  // The kernel that follows in the stream (an int32 pair's other class) may
  // start its prologue now; it waits for this one to finish.
  griddep_launch_dependents();
  // zero the q ring once (never-read slots stay finite); this needs nothing
  // from the kernel before, so it overlaps that kernel's tail
  {
    uint4* q4 = reinterpret_cast<uint4*>(smem);
    for (size_t i = threadIdx.x; i < Lay::q_bytes / 16; i += blockDim.x) q4[i] = make_uint4(0, 0, 0, 0);
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < NQ; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], (unsigned)W);
    }
    fence_mbar_init();
    ctl->abort = 0;
  }
  // the prep kernel's header, box and packed q from here on
  griddep_wait();
  // an int32 pair's other class: leave before touching the header (the
  // rings serve as the reduction's scratch; no bulk copy has been issued)
  if (a.box && box_narrow_block<DK>(a.box, a.nbox, reinterpret_cast<int*>(rings)) != (a.want != 0)) return;
  for (size_t i = threadIdx.x; i < (size_t)(W + 1) * RING; i += blockDim.x) rings[i] = V::inf();
  __syncthreads();

  unsigned gbase = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      int b = (ld_relaxed_i32(a.err) != 0) ? INT_MAX : atomicAdd(a.ticket, 1);
      ctl->band = b;
      for (int k = 0; k <= W; ++k) {
        ctl->prod[k] = 0;
        ctl->cons[k] = 0;
      }
    }
    __syncthreads();
    const int t = ctl->band;
    const int prob = a.nprob == 2 ? (t & 1) : 0;
    const int64_t band = a.nprob == 2 ? (int64_t)(t >> 1) : (int64_t)t;
    if (band >= max(a.nbands, a.nprob == 2 ? a.nbands_b : (int64_t)0)) break;
    Prob pb;
    if (prob == 0) {
      pb = Prob{a.p, a.n, a.pstep, a.qpk, a.rowbuf, a.progress, a.nbands};
    } else {
      pb = Prob{a.p_b, a.n_b, -a.pstep, a.qpk_b, a.rowbuf_b, a.progress_b, a.nbands_b};
    }
    if (band >= pb.nbands) {   // this problem has one band fewer than the other
      __syncthreads();
      continue;
    }
    if (warp == W)
      comm_warp<V, DK, R>(a, pb, band, gbase, smem);
    else
      compute_stripe<V, DK, R>(a, pb, warp, band, gbase, smem);
    gbase += (unsigned)a.nch;
    __syncthreads();
    if (ctl->abort) break;
  }
  if (a.combine) {
    // (no static shared memory: the control block and the rings are free now)
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();   // this CTA's row-buffer stores before its count
      ctl->band = atomicAdd(a.done, 1u) == gridDim.x - 1 ? 1 : 0;
    }
    __syncthreads();
    if (ctl->band) {
      __threadfence();
      combine_block<V>(a.rowbuf, a.rowbuf_b, a.m, a.err, a.res_dist, a.res_dist2, rings);
    }
  }
}

// --------------------------------------------------------- prep kernel
// Everything the wavefront needs before its first band, in one launch:
//   * the scratch header (ticket, merge words, progress words) zeroed by
//     block (0, 0);
//   * the input check, when `check` is set (blockIdx.y == 0): every
//     coordinate of p and q finite (DFD_ERR_NONFINITE), raised in the error
//     word, which makes the wavefront skip its bands;
//   * the per-band q stream: nch chunks of C columns, NPL 16-byte planes per
//     column, each plane in the column order qpos(., TR, C); columns past m
//     repeat q_{m-1} (a repeated point does not change the distance, Sec. 4
//     footnote; they are never read into the result).  blockIdx.y == 1 writes
//     the stream of q reversed (column j is q_{m-1-j}) for the backward front.
// (Was a memset, a check kernel and a packing kernel: on the 2000 x 1500
// pair, three launches whose gaps cost more than their work.)
// (float32; int32 pairs use wave_prep_int_kernel)
template <class V, int DK>
__global__ void wave_prep_kernel(const typename V::coord* q, int64_t m, int dim, int nch, int TR, void* out0,
                                 void* out1, unsigned* header, int header_words, const typename V::coord* p,
                                 int64_t p_elems, int check, long long lim, int* err) {
  static_assert(std::is_same<V, F32>::value, "float32 prep");
  (void)lim;
  griddep_launch_dependents();   // the wavefront may start its prologue
  const int rev = (int)blockIdx.y;
  if (blockIdx.x == 0 && rev == 0)
    for (int i = threadIdx.x; i < header_words; i += blockDim.x) header[i] = 0u;
  if (check && rev == 0) {
    const int64_t q_elems = m * dim;
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < p_elems + q_elems;
         i += (int64_t)gridDim.x * blockDim.x) {
      const float c = i < p_elems ? p[i] : q[i - p_elems];
      bad |= !isfinite(c);
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_error(err, DFD_ERR_NONFINITE);
  }
  void* out = rev ? out1 : out0;
  constexpr int C = ChunkCols<DK>::value;
  using Rows_ = Rows<V, DK, 2>;
  constexpr int NPL = Rows_::NPL;
  using Rec = typename Rows_::Rec;
  Rec* o = static_cast<Rec*>(out);
  const int64_t total = (int64_t)nch * C * NPL;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t chunk = idx / (C * NPL);
    const int rem = (int)(idx % (C * NPL));
    const int plane = rem / C;
    const int jj = rem % C;
    const int64_t jc = min(chunk * C + jj, m - 1);
    const int64_t j = rev ? m - 1 - jc : jc;   // the reversed problem's column jc is q's column m-1-jc
    const float* qj = q + j * dim;
    const int k0 = 2 * plane, k1 = 2 * plane + 1;
    const float x0 = k0 < dim ? qj[k0] : 0.f;
    const float x1 = k1 < dim ? qj[k1] : 0.f;
    o[chunk * (C * NPL) + plane * C + qpos(jj, TR, C)] = make_float4(x0, x0, x1, x1);
  }
}

// The int32 form of the prep kernel.  Besides the header and the range
// check it reduces the bounding box of p and q: blocks blockIdx.x < nbox of
// blockIdx.y == 0 take points in a grid stride of nbox blocks and write their
// (min, max) per coordinate (zero past dim) to box[blockIdx.x], which every
// CTA of the launches that follow reduces to choose the value class.  It
// packs q for both classes, each front its own streams: the narrow class's
// (out_n0 / out_n1: nch_n chunks of NPL = (DK+1)/2 planes, words
// (-2 q_0, ..., -2 q_{DK-1}, |q|^2, 0...), order qpos(., TR_n, C)) and the
// exact class's (out_w0 / out_w1: nch_w chunks of (DK+3)/4 int4 planes).
template <int DK>
__global__ void wave_prep_int_kernel(const int32_t* q, int64_t m, int dim, const int32_t* p, int64_t n,
                                     unsigned* header, int header_words, int check, long long lim, int* err,
                                     int* box, int nbox, int nch_n, int TR_n, void* out_n0, void* out_n1, int nch_w,
                                     void* out_w0, void* out_w1) {
  griddep_launch_dependents();   // the wavefronts may start their prologue
  const int rev = (int)blockIdx.y;
  if (blockIdx.x == 0 && rev == 0)
    for (int i = threadIdx.x; i < header_words; i += blockDim.x) header[i] = 0u;
  if (rev == 0 && (int)blockIdx.x < nbox) {
    __shared__ int sh[2 * DK];
    if (threadIdx.x < 2 * DK) sh[threadIdx.x] = (threadIdx.x & 1) ? INT_MIN : INT_MAX;
    __syncthreads();
    int lo[DK], hi[DK];
#pragma unroll
    for (int k = 0; k < DK; ++k) {
      lo[k] = INT_MAX;
      hi[k] = INT_MIN;
    }
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n + m; i += (int64_t)nbox * blockDim.x) {
      const int32_t* x = i < n ? p + i * dim : q + (i - n) * dim;
#pragma unroll
      for (int k = 0; k < DK; ++k) {
        const int c = k < dim ? x[k] : 0;
        lo[k] = min(lo[k], c);
        hi[k] = max(hi[k], c);
        if (check && k < dim) {
          const long long v = c < 0 ? -(long long)c : (long long)c;
          bad |= v > lim;
        }
      }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) raise_error(err, DFD_ERR_RANGE);
#pragma unroll
    for (int k = 0; k < DK; ++k) {
      lo[k] = __reduce_min_sync(0xffffffffu, lo[k]);
      hi[k] = __reduce_max_sync(0xffffffffu, hi[k]);
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
      for (int k = 0; k < DK; ++k) {
        atomicMin(&sh[2 * k], lo[k]);
        atomicMax(&sh[2 * k + 1], hi[k]);
      }
    }
    __syncthreads();
    if (threadIdx.x < 2 * DK) box[blockIdx.x * 2 * DK + threadIdx.x] = sh[threadIdx.x];
  }
  constexpr int C = ChunkCols<DK>::value;
  constexpr int NPL_N = Rows<I32B, DK, 2>::NPL;
  constexpr int NPL_W = Rows<I32, DK, 2>::NPL;
  const int64_t total_n = (int64_t)nch_n * C * NPL_N;
  const int64_t total_w = (int64_t)nch_w * C * NPL_W;
  int4* on = static_cast<int4*>(rev ? out_n1 : out_n0);
  int4* ow = static_cast<int4*>(rev ? out_w1 : out_w0);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total_n + total_w;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const bool nar = idx < total_n;
    const int64_t id = nar ? idx : idx - total_n;
    const int npl = nar ? NPL_N : NPL_W;
    const int64_t chunk = id / (C * npl);
    const int rem = (int)(id % (C * npl));
    const int plane = rem / C;
    const int jj = rem % C;
    const int64_t jc = min(chunk * C + jj, m - 1);
    const int64_t j = rev ? m - 1 - jc : jc;   // the reversed problem's column jc is q's column m-1-jc
    const int32_t* qj = q + j * dim;
    int w[4];
    if (nar) {
      unsigned n2 = 0;
      if (4 * plane <= DK && DK < 4 * plane + 4) {
#pragma unroll
        for (int k = 0; k < DK; ++k) {
          const unsigned c = k < dim ? (unsigned)qj[k] : 0u;
          n2 += c * c;
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k = 4 * plane + i;
        w[i] = k < DK ? (k < dim ? (int)(0u - 2u * (unsigned)qj[k]) : 0) : k == DK ? (int)n2 : 0;
      }
      on[chunk * (C * NPL_N) + plane * C + qpos(jj, TR_n, C)] = make_int4(w[0], w[1], w[2], w[3]);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k = 4 * plane + i;
        w[i] = k < dim ? qj[k] : 0;
      }
      ow[chunk * (C * NPL_W) + plane * C + jj] = make_int4(w[0], w[1], w[2], w[3]);
    }
  }
}

// ------------------------------------------------------------ combine
// Two wavefronts meet between rows n1-1 and n1: F[j] = M[n1-1][j] of the
// forward problem, and B[j], the bottleneck of the best path from (n1, j)
// to (n-1, m-1), is the backward problem's bottom row read in reverse
// (rowbuf_b[m-1-j]).  Every monotone path crosses from row n1-1 to row n1
// once, by a vertical step (to column j) or a diagonal one (to j+1), so
// delta^2 = min_j max(F[j], min(B[j], B[j+1])): a selection among the same
// squared distances, bit-identical to the single wavefront's result.
// Each CTA reduces a stretch of columns; the values are non-negative, so
// their bit patterns order like the values and the CTAs merge by an atomic
// max of the complemented bits in `word` (zero before the launch); the last
// CTA to finish (`count`, zero before the launch) writes the result, unless
// the error word is set: an input check that failed or a wait that ran out
// made the wavefront skip its bands, so the row buffers hold no result and
// the outputs keep whatever the caller put there.
template <class V, int DK>
__global__ void combine_kernel(const void* rowbuf_f, const void* rowbuf_b, int64_t m, unsigned long long* word,
                               unsigned* count, const int* err, void* out_dist, void* out_dist2, const int* box,
                               int nbox, int want) {
  using T = typename V::value;
  __shared__ int sel[2 * DK + 1];
  if (box && box_narrow_block<DK>(box, nbox, sel) != (want != 0)) return;   // the other class's launch
  const T* F = static_cast<const T*>(rowbuf_f);
  const T* B = static_cast<const T*>(rowbuf_b);
  T best = V::inf();
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const T bj = B[m - 1 - j];
    const T bj1 = j + 1 < m ? B[m - 2 - j] : V::inf();
    best = V::vmin(best, V::vmax(F[j], V::vmin(bj, bj1)));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) best = V::vmin(best, __shfl_xor_sync(0xffffffffu, best, off));
  __shared__ T part[32];
  const int warp = threadIdx.x >> 5, L = threadIdx.x & 31;
  if (L == 0) part[warp] = best;
  __syncthreads();
  if (warp == 0) {
    T x = L < (int)(blockDim.x >> 5) ? part[L] : V::inf();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x = V::vmin(x, __shfl_xor_sync(0xffffffffu, x, off));
    if (L == 0) {
      unsigned long long bits;
      if constexpr (sizeof(T) == 4)
        bits = __float_as_uint((float)x);
      else
        bits = (unsigned long long)(long long)x;
      atomicMax(word, ~bits);
      __threadfence();
      if (atomicAdd(count, 1u) == gridDim.x - 1 && *(volatile const int*)err == 0) {
        const unsigned long long mb = ~atomicAdd(word, 0ull);
        if constexpr (sizeof(T) == 4)
          write_pair_result<V>(out_dist, out_dist2, __uint_as_float((unsigned)mb));
        else
          write_pair_result<V>(out_dist, out_dist2, (T)(long long)mb);
      }
    }
  }
}

}  // namespace wave
}  // namespace dfd
