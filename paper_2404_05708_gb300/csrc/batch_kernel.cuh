// batch_kernel.cuh -- K4 (ragged batch) and K5 (all-pairs matrix).
//
// Many independent pairs: one warp per pair.  The rows of the recurrence of
// Eq. 1 are the curve that costs fewer steps (delta(p,q) = delta(q,p); see
// orient_cost: usually the shorter one), split into stripes
// of 32*R rows; lane L holds R consecutive rows in registers and the stripe
// runs as a systolic array over the columns (lane L at step s updates column
// s - L).  Rows past the curve's end repeat its last point (a repeated point
// does not change the distance, Sec. 4 footnote).  A pair longer than one
// stripe hands each stripe's bottom row to the next through a per-warp
// shared-memory buffer (in place: a column is read for stripe k+1 before
// stripe k+1 overwrites it).  Persistent warps take work items from an
// atomic counter over a device-built, cost-descending (LPT) work list.
#pragma once
#include <type_traits>
#include "dfd_device.cuh"

namespace dfd {
namespace batch {

// Rows per lane of one stripe is at most Rmax: 8 for points of up to 4
// coordinates and 4 beyond (a lane's R rows form one dependent chain per
// step).  Points of dim class 16 hold their packed rows in up to 172
// registers, so those kernels run one 256-thread CTA per SM: each step's
// four q planes then serve four rows instead of two, and a pair needs half
// the stripes (16-D matrix: 0.59 Tcell/s, was 0.49 with two rows and two
// CTAs per SM).  Other classes run two CTAs per SM.  Pairs with more rows
// run several stripes.
template <int DK>
struct Rmax {
  static constexpr int value = DK <= 4 ? 8 : 4;
};
template <int DK>
struct kBlocksPerSM {
  static constexpr int value = DK >= 16 ? 1 : 2;
};

// q streams through a per-warp shared-memory window instead of per-lane
// L1/L2 loads: the warp loads the next 32 points cooperatively one block
// ahead (one point per lane, coalesced) and every step reads them from
// shared memory.  During the block of columns c0 .. c0+31 the window holds
// columns c0-32 .. c0+31 in slots 0 .. 63, so lane L reads column
// c0 + s - L from slot 32 + s - L: one load per 16-byte plane at a fixed
// offset from a per-lane base, no index arithmetic per step.  Planes are
// stored plane-major ([plane][64 slots]) so lanes one column apart read
// consecutive records.  (Per-lane loads left lane 0 waiting on L2 for every
// new point.)  After the planes, 16 records hold the stripe's bottom row of
// the current block (lane 31 stores four values at a time), and 16 more the
// stripe above's values for the block's columns (lane 0 reads eight at a
// time).
template <int DK>
struct QStage {
  static constexpr bool on = true;
  static constexpr int NPL = (DK + 3) / 4;
  static constexpr int RECS = NPL * 64 + 32;   // uint4 records per warp
};

// Form of a column's record in the window.
//   kRaw:  the coordinates, 4 per plane.
//   kDup:  float32 points of dim class 2 as (x, x, y, y): the operand of the
//          packed row pairs, read as is.
//   kNorm: uint32-bits points of dim class <= 3 as (-2x, -2y, -2z, |q|^2),
//          mod 2^32.  With |p|^2 per row, d^2 = |p|^2 + |q|^2 - 2 p.q is
//          three integer instructions a cell instead of four, and exact: the
//          arithmetic is modulo 2^32 and the true d^2 is below 2^31.
enum QRecKind { kRaw = 0, kDup = 1, kNorm = 2 };
template <class V, int DK>
struct QRec {
  static constexpr int kind = (std::is_same<V, F32>::value && DK == 2)   ? kDup
                              : (std::is_same<V, I32B>::value && DK <= 3) ? kNorm
                                                                         : kRaw;
  static constexpr int NPL = QStage<DK>::NPL;   // 1 for kDup and kNorm
};

// Plane c of the record of point q.
template <class V, int DK>
__device__ __forceinline__ uint4 make_qrec(const typename V::coord (&q)[DK], int c) {
  uint4 r;
  if constexpr (QRec<V, DK>::kind == kDup) {
    r.x = r.y = __float_as_uint(q[0]);
    r.z = r.w = __float_as_uint(q[1]);
  } else if constexpr (QRec<V, DK>::kind == kNorm) {
    unsigned n2 = 0;
#pragma unroll
    for (int k = 0; k < DK; ++k) n2 += (unsigned)q[k] * (unsigned)q[k];
    r.x = 0u - 2u * (unsigned)q[0];
    r.y = DK > 1 ? 0u - 2u * (unsigned)q[DK > 1 ? 1 : 0] : 0u;
    r.z = DK > 2 ? 0u - 2u * (unsigned)q[DK > 2 ? 2 : 0] : 0u;
    r.w = n2;
  } else {
    unsigned w[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int k = 4 * c + t;
      w[t] = 0u;
#pragma unroll
      for (int kk = 0; kk < DK; ++kk)
        if (kk == k) w[t] = *reinterpret_cast<const unsigned*>(&q[kk]);
    }
    r = make_uint4(w[0], w[1], w[2], w[3]);
  }
  return r;
}
// Per-warp row buffer (columns) of multi-stripe pairs: the default width,
// and the fixed one of the decider, matrix, k-NN and variant kernels; the
// ragged batch takes a wider one per launch (BatchArgs::buf_cols).
constexpr int BUF_COLS = 4096;

// First pops of a small launch spread over the SMs' sub-partitions.
// Persistent warps race for the work counter, and all warps of a CTA start
// together, so a launch with fewer pairs than resident warps would give its
// pairs to the first CTAs' warps, two or more to a sub-partition, while
// other sub-partitions idle; such a warp is latency-bound (its lane's rows
// form one dependent chain per step), and one warp alone on a
// sub-partition runs its pair about twice as fast (512 pairs of 1,024-point
// curves: 0.33 ms instead of 0.63).  So when every pair fits one round of
// 4 * n_sm sub-partitions, a warp's first pop waits until every item is
// taken unless it is the first warp of its sub-partition (warp slot mod 4)
// to arrive.  The wait is bounded (kSpreadWaitNs): it orders placement
// only, never correctness.  Larger launches pop plainly: ordering their
// first pops this way made the 65,536-pair batch 9-14% slower.
// `sm_rank`: kSmSlots counters, zeroed per launch.
constexpr int kSmSlots = 1024;
constexpr unsigned long long kSpreadWaitNs = 20000;
constexpr int kSpreadPolls = 64;
__device__ __forceinline__ int pop_first(int* counter, unsigned* sm_rank, int n_sm, long long total) {
  if (sm_rank && total <= 4LL * n_sm) {
    unsigned sm, slot;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    asm volatile("mov.u32 %0, %%warpid;" : "=r"(slot));
    const unsigned q = sm * 4u + (slot & 3u);
    const unsigned r = q < (unsigned)kSmSlots ? atomicAdd(&sm_rank[q], 1u) : 0u;
    if (r > 0) {
      // bounded twice: by the timer, and by a count of L2 round trips
      // (kSpreadPolls) that holds even if the timer does not advance
      const unsigned long long t0 = globaltimer_ns();
      for (int it = 0; it < kSpreadPolls && (long long)ld_relaxed_i32(counter) < total &&
                       globaltimer_ns() - t0 < kSpreadWaitNs;
           ++it) {
      }
    }
  }
  return atomicAdd(counter, 1);
}

// Progress words of a team (shared memory, CTA scope): the producer's lane
// 0 publishes after its lanes' stores (__syncwarp, then a fence and a
// relaxed store: a release), the consumer's lane 0 polls relaxed and fences
// once the value is there (an acquire) before its lanes' loads.
// Bounded wait until *p >= need: by the timer and by a count of polls that
// holds even if the timer does not advance; gives up at once when the
// error word is set.  On expiry it records DFD_ERR_TIMEOUT and returns, and
// the team goes on without waiting (its results are then not to be used:
// the error word says so).
constexpr long long kTeamPolls = 1LL << 26;
__device__ __forceinline__ unsigned long long ld_relaxed_cta_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.cta.shared::cta.u64 %0, [%1];" : "=l"(v) : "r"(smem_addr(p)) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_cta_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.cta.shared::cta.u64 [%0], %1;" ::"r"(smem_addr(p)), "l"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_cta_team() { asm volatile("fence.acq_rel.cta;" ::: "memory"); }
// Relaxed polls, then one fence: with the producer's fence before its
// relaxed store, an acquire of what it published.
__device__ __forceinline__ void team_wait(const unsigned long long* p, unsigned long long need, int* err,
                                          unsigned long long timeout_ns) {
  if (ld_relaxed_cta_u64(p) < need) {
    const unsigned long long t0 = globaltimer_ns();
    for (long long it = 1;; ++it) {
      if (ld_relaxed_cta_u64(p) >= need) break;
      if ((it & 255) == 0) {
        if (ld_relaxed_i32(err) != 0) break;
        if (it >= kTeamPolls || globaltimer_ns() - t0 > timeout_ns) {
          raise_error(err, DFD_ERR_TIMEOUT);
          break;
        }
      }
    }
  }
  fence_acq_rel_cta_team();
}

// Eight values of a warp's staging area into registers (16-byte loads), and
// four out of them (16-byte stores); the addresses are 16-byte aligned.
template <class T>
__device__ __forceinline__ void load8(const T* p, T (&v)[8]) {
  const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
  for (int i = 0; i < (int)(8 * sizeof(T) / 16); ++i) {
    const uint4 x = q[i];
    const unsigned w[4] = {x.x, x.y, x.z, x.w};
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int j = 0; j < 4; ++j) v[4 * i + j] = __uint_as_float(w[j]);
    } else {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const unsigned long long z = ((unsigned long long)w[2 * j + 1] << 32) | w[2 * j];
        v[2 * i + j] = (T)(long long)z;
      }
    }
  }
}
template <class T>
__device__ __forceinline__ void store4(T* p, const T (&v)[4]) {
  uint4* q = reinterpret_cast<uint4*>(p);
  if constexpr (sizeof(T) == 4) {
    q[0] = make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]), __float_as_uint(v[3]));
  } else {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const unsigned long long a = (unsigned long long)(long long)v[2 * i], b = (unsigned long long)(long long)v[2 * i + 1];
      q[i] = make_uint4((unsigned)a, (unsigned)(a >> 32), (unsigned)b, (unsigned)(b >> 32));
    }
  }
}

// Rows per lane chosen for a pair with `rows` rows: the fewest stripes
// (one when rows <= 32 * Rmax), with the rows spread evenly over them, so a
// pair of 300 rows runs two stripes of 160 rows rather than two of 256.
// `rmax` (at most Rmax, a launch's tuned cap) bounds the rows per lane.
template <int DK>
__host__ __device__ __forceinline__ int rows_per_lane(int rows, int rmax = Rmax<DK>::value) {
  const int RM = rmax < 1 ? 1 : (rmax > Rmax<DK>::value ? Rmax<DK>::value : rmax);
  if (rows <= 32) return 1;
  const int st = (rows + 32 * RM - 1) / (32 * RM);
  const int r = (rows + 32 * st - 1) / (32 * st);
  return r > RM ? RM : r;
}

// Point j of a curve into registers, coordinates past dim zero.  With `vec`
// (dim == DK in {2, 4, 8, 16} and 16-byte aligned curves, checked by the
// host) one 8- or 16-byte load per 2 or 4 coordinates.
template <class Cd, int DK>
__device__ __forceinline__ void load_point(const Cd* __restrict__ Q, int j, int dim, bool vec, Cd (&qk)[DK]) {
  if constexpr (DK == 2) {
    if (vec) {
      if constexpr (sizeof(Cd) == 4 && std::is_same<Cd, float>::value) {
        const float2 t = __ldg(reinterpret_cast<const float2*>(Q) + j);
        qk[0] = t.x;
        qk[1] = t.y;
      } else {
        const int2 t = __ldg(reinterpret_cast<const int2*>(Q) + j);
        qk[0] = t.x;
        qk[1] = t.y;
      }
      return;
    }
  } else if constexpr (DK % 4 == 0) {
    if (vec) {
#pragma unroll
      for (int c = 0; c < DK / 4; ++c) {
        if constexpr (std::is_same<Cd, float>::value) {
          const float4 t = __ldg(reinterpret_cast<const float4*>(Q) + (int64_t)j * (DK / 4) + c);
          qk[4 * c] = t.x;
          qk[4 * c + 1] = t.y;
          qk[4 * c + 2] = t.z;
          qk[4 * c + 3] = t.w;
        } else {
          const int4 t = __ldg(reinterpret_cast<const int4*>(Q) + (int64_t)j * (DK / 4) + c);
          qk[4 * c] = t.x;
          qk[4 * c + 1] = t.y;
          qk[4 * c + 2] = t.z;
          qk[4 * c + 3] = t.w;
        }
      }
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < DK; ++k) qk[k] = k < dim ? __ldg(Q + (int64_t)j * dim + k) : (Cd)0;
}

// Stripes [st_begin, st_end) of the pair (all of them by default).  `buf`
// holds the bottom row of stripe st_begin - 1 on entry (when st_begin > 0)
// and of stripe st_end - 1 on exit (when st_end < #stripes): this is the
// O(m) row state that lets a long pair pause between serving ticks (row i of
// the recurrence summarises rows 1..i, Sec. 3).  Returns delta^2 when the
// last stripe ran, +inf otherwise.
// Early abandon (decider and k-NN forms).  Along any monotone path the
// bottleneck of its prefix ending at a cell is at least M of that cell, so
// delta >= min over any set of cells that every path from (0,0) to
// (n-1,m-1) must enter.  After each 32-step block of a single-stripe pair
// the lanes' current cells (one column per lane, lane L at column s - L)
// together with, for each lane, the left neighbour of the upper lane's
// bottom cell (the lane's `upp`, which a diagonal step could otherwise slip
// past) form such a set while lane 0 has not passed the last column: a path
// starts left of it in row 0 and must reach column m-1 in the last row.  A
// stripe of a taller pair adds the cells through which a path can avoid its
// frontier (see bmin / sufb in warp_dfd).  A pair whose minimum there
// exceeds the limit has delta^2 above it and is abandoned; ties never
// abandon.
template <class V>
struct NoAbandon {
  static constexpr bool on = false;
  bool hit = false;
  __device__ __forceinline__ typename V::value limit() const { return V::inf(); }
};

// A fixed limit, or one read (lane 0, relaxed, broadcast) from device memory
// each time it is checked: the k-NN search lowers it while warps run.
template <class V>
struct AbandonAbove {
  static constexpr bool on = true;
  typename V::value fixed;
  const unsigned* live_bits;   // k-NN: current limit as float bits (float values only), else null
  bool hit = false;
  int cols_done = 0;           // columns of the (single) stripe swept when abandoned
  __device__ __forceinline__ typename V::value limit() const {
    if constexpr (sizeof(typename V::value) == 4) {
      if (live_bits) {
        unsigned b = 0;
        if ((threadIdx.x & 31) == 0) b = (unsigned)ld_relaxed_i32(reinterpret_cast<const int*>(live_bits));
        b = __shfl_sync(0xffffffffu, b, 0);
        return __uint_as_float(b);
      }
    }
    return fixed;
  }
};

// Where a stripe reads its top row (the bottom row of the stripe above) and
// writes its bottom row, per 32-column block.
// SoloIO: one warp runs all stripes of the pair in order, through its own
// row buffer in global memory (in place: a column is read for stripe k+1
// before stripe k+1 overwrites it).
struct SoloIO {
  static constexpr bool kTeam = false;
  template <class T>
  __device__ __forceinline__ static T top(SoloIO*, const T* buf, int, int c0, int L, int m) {
    return buf[min(c0 + L, m - 1)];
  }
  template <class T>
  __device__ __forceinline__ static void bottom(SoloIO*, T* buf, int, int c0, int L, int m, const T* outb) {
    const int oc = c0 + L - 31;
    if (oc >= 0 && oc < m) buf[oc] = outb[L];
  }
  __device__ __forceinline__ static void end_block(SoloIO*, int, int, int, int, bool, bool) {}
  __device__ __forceinline__ static bool final_row(const SoloIO*) { return false; }
};

// Team of the CTA's warps on one pair: warp w runs stripes w, w + nw,
// w + 2 nw, ... as a pipeline over the columns.  Stripe s hands its bottom
// row to stripe s + 1 through warp w's shared-memory ring of RING slots,
// or, from the last warp to warp 0 of the next cycle, through the CTA's row
// buffer in global memory (m columns, in place).  Positions count over a
// warp's stripes: column c of its stripe in cycle k is position k * m + c,
// kept in ring slot (k * m + c) mod RING, so the ring is one FIFO across
// cycles.  prog[w] counts the positions of warp w's bottom rows published,
// cons[w] the positions of its top rows read (both in shared memory).  A
// consumer waits for the producer before each block; a producer waits
// before overwriting slots the consumer has not read (position - RING).
// The global buffer needs no such wait: the last warp writes column c of a
// later cycle only after that column has passed down through every stripe
// in between, each of which read it after warp 0 did.  Every wait is
// bounded.
template <int RING>
struct TeamIO {
  static constexpr bool kTeam = true;
  static_assert((RING & (RING - 1)) == 0 && RING >= 128, "ring: a power of two of at least 128 columns");
  void* gbuf;                  // the CTA's row buffer (global), >= m values when the pair has more stripes than warps
  void* ring;                  // shared: nw rings of RING values of up to 8 bytes
  unsigned long long* prog;    // shared [nw]
  unsigned long long* cons;    // shared [nw]
  int w, nw;
  int* err;
  unsigned long long timeout_ns;
  void* final_out;             // global, m values: stripe last_st's bottom row (a half-pair), or null
  int last_st;
  __device__ __forceinline__ static bool final_row(const TeamIO* io) { return io->final_out != nullptr; }

  template <class T>
  __device__ __forceinline__ static T top(TeamIO* io, const T*, int st, int c0, int L, int m) {
    const int wp = io->w == 0 ? io->nw - 1 : io->w - 1;   // the warp of stripe st - 1
    const unsigned long long kp = (unsigned long long)((st - 1) / io->nw);
    const int need = min(c0 + 32, m);
    if (L == 0) team_wait(&io->prog[wp], kp * (unsigned long long)m + need, io->err, io->timeout_ns);
    __syncwarp();
    const int c = min(c0 + L, m - 1);
    const T v = wp == io->nw - 1
                    ? static_cast<const T*>(io->gbuf)[c]
                    : reinterpret_cast<const T*>(static_cast<const unsigned long long*>(io->ring) +
                                                 wp * RING)[(kp * (unsigned long long)m + c) & (RING - 1)];
    return v;   // the read is published (cons) with the block's output, in end_block
  }
  template <class T>
  __device__ __forceinline__ static void bottom(TeamIO* io, T*, int st, int c0, int L, int m, const T* outb) {
    const int oc = c0 + L - 31;
    if (io->final_out && st == io->last_st) {   // the half-pair's last row: no consumer but the meeting
      if (oc >= 0 && oc < m) static_cast<T*>(io->final_out)[oc] = outb[L];
      return;
    }
    const unsigned long long k = (unsigned long long)(st / io->nw);
    if (io->w == io->nw - 1) {
      if (oc >= 0 && oc < m) static_cast<T*>(io->gbuf)[oc] = outb[L];
    } else {
      // the slots of positions k*m + c0-31 .. k*m + c0 last held positions up
      // to k*m + c0 - RING: the consumer (stripe st + 1, same cycle) must have read them
      const long long need = (long long)(k * (unsigned long long)m) + c0 + 1 - RING;
      if (need > 0 && L == 0) team_wait(&io->cons[io->w + 1], (unsigned long long)need, io->err, io->timeout_ns);
      __syncwarp();
      if (oc >= 0 && oc < m)
        reinterpret_cast<T*>(static_cast<unsigned long long*>(io->ring) +
                             io->w * RING)[(k * (unsigned long long)m + oc) & (RING - 1)] = outb[L];
    }
  }
  // After each block: one release for both progress words -- the block's
  // bottom row (columns 0 .. c0 of stripe st) and the top row it read
  // (columns up to c0 + 31).  A fence, then relaxed stores, where a release
  // store per word took two fences; holding the read back to here delays the
  // producer's flow control by one block, well within the ring (the producer
  // waits for positions RING behind its own, the consumer trails it by about
  // two blocks).
  __device__ __forceinline__ static void end_block(TeamIO* io, int st, int c0, int L, int m, bool has_top,
                                                   bool has_bottom) {
    __syncwarp();
    if (L == 0) {
      fence_acq_rel_cta_team();
      const unsigned long long k = (unsigned long long)(st / io->nw);
      if (has_bottom) st_relaxed_cta_u64(&io->prog[io->w], k * m + min(c0 + 1, m));
      if (has_top) st_relaxed_cta_u64(&io->cons[io->w], k * m + min(c0 + 32, m));
    }
  }
};

template <class V, int DK, int R, class AB = NoAbandon<V>, class IO = SoloIO>
__device__ __forceinline__ typename V::value warp_dfd(const typename V::coord* __restrict__ P, int n,
                                                      const typename V::coord* __restrict__ Q, int m, int dim,
                                                      bool vec, typename V::value* buf, int L, int st_begin = 0,
                                                      int st_end = 1 << 30, AB* ab = nullptr,
                                                      uint4* stage = nullptr, IO* io = nullptr,
                                                      int st_step = 1, int pstep = 0, int qsign = 1) {
  // pstep: elements from one row of P to the next (0: dim; -dim runs the rows
  // backwards from P); qsign = -1 runs the columns backwards from Q.
  const int64_t prow = pstep ? pstep : dim;
  using T = typename V::value;
  using Cd = typename V::coord;
  const int nstripes = (n + 32 * R - 1) / (32 * R);
  T res = V::inf();
  for (int st = st_begin; st < min(st_end, nstripes); st += st_step) {
    Cd pr[R][DK];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = min(st * 32 * R + L * R + r, n - 1);
#pragma unroll
      for (int k = 0; k < DK; ++k) pr[r][k] = k < dim ? __ldg(P + (int64_t)i * prow + k) : (Cd)0;
    }
    // float32: rows packed in pairs, two cells per f32x2 instruction (the
    // same per-element rounding as the scalar order; odd R: last row scalar)
    constexpr bool kPack = std::is_same<V, F32>::value && R >= 2;
    unsigned long long pp[kPack ? R / 2 : 1][DK];
    if constexpr (kPack) {
#pragma unroll
      for (int h = 0; h < R / 2; ++h) {
#pragma unroll
        for (int k = 0; k < DK; ++k) pp[h][k] = pack2(pr[2 * h][k], pr[2 * h + 1][k]);
      }
    }
    // (a team half-pair also hands its last stripe's bottom row out: IO::final_row)
    const bool has_top = st > 0, has_bottom = st + 1 < nstripes || IO::final_row(io), last = st + 1 >= nstripes;
    T v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = V::inf();
    T bout = V::inf();
    T upp = (st == 0 && L == 0) ? V::zero() : V::inf();
    // Early abandon of a multi-stripe pair: the stripe's frontier cut is
    // completed by (a) the cells of the stripe's bottom row already swept
    // (`bmin`, lane 31: a path passing left of the frontier leaves through
    // them) and (b) the previous stripe's bottom row from lane 0's column on
    // (a path entering right of the frontier comes through it), kept as
    // suffix minima per 32-column block (`sufb`, block L + 32t on lane L).
    T bmin = V::inf();
    T sufb[AB::on ? BUF_COLS / 1024 : 1];
    if constexpr (AB::on) {
#pragma unroll
      for (int t = 0; t < BUF_COLS / 1024; ++t) sufb[t] = V::inf();
      if (has_top) {
        const int nb = (m + 31) / 32;
        for (int b = 0; b < nb; ++b) {
          const int c = 32 * b + L;
          T x = c < m ? buf[c] : V::inf();
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) x = V::vmin(x, __shfl_xor_sync(0xffffffffu, x, off));
#pragma unroll
          for (int t = 0; t < BUF_COLS / 1024; ++t)
            if (L == (b & 31) && t == (b >> 5)) sufb[t] = x;
        }
        T carry = V::inf();   // minimum over the blocks of higher t
#pragma unroll
        for (int t = BUF_COLS / 1024 - 1; t >= 0; --t) {
          T x = sufb[t];
#pragma unroll
          for (int off = 1; off < 32; off <<= 1) {
            const T y = __shfl_down_sync(0xffffffffu, x, off);
            if (L + off < 32) x = V::vmin(x, y);
          }
          x = V::vmin(x, carry);
          carry = __shfl_sync(0xffffffffu, x, 0);
          sufb[t] = x;
        }
      }
    }
    const int nsteps = m + 31;
    using QR = QRec<V, DK>;
    constexpr int NPL = QR::NPL;
    // |p|^2 per row (kNorm)
    unsigned pn[QR::kind == kNorm ? R : 1];
    if constexpr (QR::kind == kNorm) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        unsigned acc = 0;
#pragma unroll
        for (int k = 0; k < DK; ++k) acc += (unsigned)pr[r][k] * (unsigned)pr[r][k];
        pn[r] = acc;
      }
    }
    // this lane's point of the coming block (in flight during the block before)
    Cd qpre[DK];
    load_point<Cd, DK>(Q, min(L, m - 1) * qsign, dim, vec, qpre);
    const uint4* sb = stage + (32 - L);   // column c0 + s - L of the window is sb[s]
    T* outb = reinterpret_cast<T*>(stage + NPL * 64);
    T* topb = reinterpret_cast<T*>(stage + NPL * 64 + 16);
    for (int c0 = 0; c0 < nsteps; c0 += 32) {
      const T top_blk = has_top ? IO::top(io, buf, st, c0, L, m) : V::inf();
      // slide the window: the block before's columns (slot 32 + L, written
      // by this lane) move to slot L, this block's column to slot 32 + L
      __syncwarp();
#pragma unroll
      for (int c = 0; c < NPL; ++c) {
        stage[c * 64 + L] = c0 > 0 ? stage[c * 64 + 32 + L] : make_qrec<V, DK>(qpre, c);
        stage[c * 64 + 32 + L] = make_qrec<V, DK>(qpre, c);
      }
      topb[L] = top_blk;   // the stripe above's columns c0 .. c0 + 31, read by lane 0 eight at a time
      __syncwarp();
      load_point<Cd, DK>(Q, min(c0 + 32 + L, m - 1) * qsign, dim, vec, qpre);   // next block, in flight
      uint4 qr[NPL];
#pragma unroll
      for (int c = 0; c < NPL; ++c) qr[c] = sb[c * 64];
      // Groups of 8 steps unrolled (not 32): a kernel holds every R variant,
      // and warps running different variants side by side must not thrash
      // the instruction cache (the ragged int32 batch: 2.86 Tcell/s unrolled
      // by 4, 3.04 by 8, 2.78 fully).  Per group, lane 0's inputs from the
      // stripe above come from the staging area in two or four 16-byte loads
      // (was a shuffle per step) and lane 31's bottom values leave in
      // 16-byte stores of four (was a store per step): 3.04 -> 3.26.  The
      // next step's record is read unconditionally: at the block's last step
      // that read lands on the next plane's (or the bottom row's) first
      // slots of this warp's window, inside the array, and is never used.
#pragma unroll 1
      for (int s8 = 0; s8 < 32; s8 += 8) {
        T tv[8];
        load8<T>(topb + s8, tv);
        T ob[4];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int s = s8 + t;
          uint4 qn[NPL];   // the next step's record, read one step ahead
  #pragma unroll
          for (int c = 0; c < NPL; ++c) qn[c] = sb[c * 64 + s + 1];
          T d[R];
          if constexpr (QR::kind == kNorm) {
  #pragma unroll
            for (int r = 0; r < R; ++r) {
              unsigned acc = pn[r] + qr[0].w;
              acc += (unsigned)pr[r][0] * qr[0].x;
              if (DK > 1) acc += (unsigned)pr[r][1] * qr[0].y;
              if (DK > 2) acc += (unsigned)pr[r][2 < DK ? 2 : 0] * qr[0].z;
              d[r] = __uint_as_float(acc);
            }
          } else if constexpr (QR::kind == kDup) {
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
              d[R - 1] = vdist2<V, DK>(pr[R - 1], qk);
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
              if constexpr ((R & 1) != 0) d[R - 1] = vdist2<V, DK>(pr[R - 1], qk);
            } else {
  #pragma unroll
              for (int r = 0; r < R; ++r) d[r] = vdist2<V, DK>(pr[r], qk);
            }
          }
          T u = __shfl_up_sync(0xffffffffu, bout, 1);
          u = (L == 0) ? tv[t] : u;
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
          if constexpr (AB::on) bmin = V::vmin(bmin, bout);
          ob[t & 3] = bout;   // column c0 + s - 31 of the stripe's bottom row
          if ((t & 3) == 3 && has_bottom && L == 31) store4<T>(outb + (s - 3), ob);
  #pragma unroll
          for (int c = 0; c < NPL; ++c) qr[c] = qn[c];

        }
      }
      __syncwarp();
      if (has_bottom) IO::bottom(io, buf, st, c0, L, m, outb);
      IO::end_block(io, st, c0, L, m, has_top, has_bottom);
      if constexpr (AB::on) {
        if (c0 + 31 <= m - 1) {
          T cut = upp;
#pragma unroll
          for (int r = 0; r < R; ++r) cut = V::vmin(cut, v[r]);
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) cut = V::vmin(cut, __shfl_xor_sync(0xffffffffu, cut, off));
          if (has_bottom) cut = V::vmin(cut, __shfl_sync(0xffffffffu, bmin, 31));
          if (has_top) {
            // previous stripe's bottom row from column c0 + 31 on: that column
            // (lane 31's top value of this block) and the blocks after it
            const int nb = c0 / 32 + 1;
            T sv = V::inf();
#pragma unroll
            for (int t = 0; t < BUF_COLS / 1024; ++t)
              if (t == (nb >> 5)) sv = sufb[t];
            sv = __shfl_sync(0xffffffffu, sv, nb & 31);
            if (nb >= (m + 31) / 32) sv = V::inf();
            cut = V::vmin(cut, V::vmin(sv, __shfl_sync(0xffffffffu, top_blk, 31)));
          }
          if (cut > ab->limit()) {
            ab->hit = true;
            ab->cols_done = c0 + 32;
            return V::inf();
          }
        }
      }
    }
    // Lane 31's bottom row has swept past column m - 1 over q padded by
    // repeating its last point, which leaves the value unchanged (Sec. 4
    // footnote): its last value is delta^2.
    if (last) res = bout;
  }
  return __shfl_sync(0xffffffffu, res, 31);
}

template <class V, int DK, class AB = NoAbandon<V>>
__device__ __forceinline__ typename V::value warp_dfd_any(const typename V::coord* P, int n,
                                                          const typename V::coord* Q, int m, int dim, bool vec,
                                                          typename V::value* buf, int L, int st_begin = 0,
                                                          int st_end = 1 << 30, AB* ab = nullptr,
                                                          uint4* stage = nullptr, int rmax = Rmax<DK>::value) {
  constexpr int RM = Rmax<DK>::value;
  switch (rows_per_lane<DK>(n, rmax)) {
#define DFD_B_CASE(RR)                                                                                       \
  case RR:                                                                                                   \
    if constexpr (RR < RM) return warp_dfd<V, DK, RR, AB>(P, n, Q, m, dim, vec, buf, L, st_begin, st_end, ab, stage); \
    break;
    DFD_B_CASE(1)
    DFD_B_CASE(2)
    DFD_B_CASE(3)
    DFD_B_CASE(4)
    DFD_B_CASE(5)
    DFD_B_CASE(6)
    DFD_B_CASE(7)
    default:
      break;
#undef DFD_B_CASE
  }
  return warp_dfd<V, DK, RM, AB>(P, n, Q, m, dim, vec, buf, L, st_begin, st_end, ab, stage);
}

// Number of stripes warp_dfd_any uses for a pair with `rows` rows.
template <int DK>
__host__ __device__ __forceinline__ int num_stripes(int rows, int rmax = Rmax<DK>::value) {
  const int r = rows_per_lane<DK>(rows, rmax);
  return (rows + 32 * r - 1) / (32 * r);
}

// A pair needs the row buffer when its rows span several stripes.
template <int DK>
__device__ __forceinline__ bool fits_buffer(int rows, int cols, int buf_cols = BUF_COLS,
                                            int rmax = Rmax<DK>::value) {
  return num_stripes<DK>(rows, rmax) <= 1 || cols <= buf_cols;
}

template <class V>
__device__ __forceinline__ void write_result(void* out_dist, void* out_dist2, int64_t k, typename V::value r) {
  if constexpr (std::is_same<V, F32>::value) {
    if (out_dist2) static_cast<float*>(out_dist2)[k] = r;
    if (out_dist) static_cast<float*>(out_dist)[k] = sqrtf(r);
  } else {
    long long v;
    if constexpr (std::is_same<V, I32B>::value)
      v = (long long)__float_as_uint(r);
    else
      v = (long long)r;
    if (out_dist2) static_cast<long long*>(out_dist2)[k] = v;
    if (out_dist) static_cast<double*>(out_dist)[k] = sqrt((double)v);
  }
}

// Outputs of a pair the kernel cannot run (a row wider than its buffer):
// NaN (float, double) / -1 (int64), beside DFD_ERR_UNSUPPORTED in the error word.
template <class V>
__device__ __forceinline__ void write_unsupported(void* out_dist, void* out_dist2, int64_t k) {
  if constexpr (std::is_same<V, F32>::value) {
    if (out_dist2) static_cast<float*>(out_dist2)[k] = __int_as_float(0x7fffffff);
    if (out_dist) static_cast<float*>(out_dist)[k] = __int_as_float(0x7fffffff);
  } else {
    if (out_dist2) static_cast<long long*>(out_dist2)[k] = -1;
    if (out_dist) static_cast<double*>(out_dist)[k] = __longlong_as_double(0x7fffffffffffffffLL);
  }
}

// int32 pairs whose bounding boxes keep every squared distance exact in
// uint32 (below the first float NaN pattern) run as I32B.  bbox holds per
// curve and coordinate (min, max).
__device__ __forceinline__ bool narrow_pair(const int* __restrict__ bbox, int dk, int64_t ia, int64_t ib) {
  unsigned long long s = 0;
  for (int k = 0; k < dk; ++k) {
    const long long lo = min(bbox[(ia * dk + k) * 2], bbox[(ib * dk + k) * 2]);
    const long long hi = max(bbox[(ia * dk + k) * 2 + 1], bbox[(ib * dk + k) * 2 + 1]);
    const unsigned long long r = (unsigned long long)(hi - lo);
    if (r > kI32BMaxRange) return false;
    s += r * r;
  }
  return s <= kI32BMaxD2;
}

// Per-curve bounding boxes (one warp per curve) of int32 points, and the
// coordinate range check (|c| <= lim) when `check` is set, for curves
// [first, n_curves).  Every lane issues BoxLoads<DK> point loads per round
// before it reduces any, so a round of 32 * BoxLoads points costs one memory
// round trip (indices past the curve's end read its last point again, which
// changes neither the box nor the check), and the next curve's offsets are
// read while the current curve is reduced.  (A loop of one load per
// iteration left each warp waiting on DRAM for every 32 points: 2 TB/s.)
// The range check reads the box, not every point: all |c| <= lim exactly
// when the box lies within [-lim, lim] (a check per coordinate against the
// 64-bit limit kept the kernel issue-bound, at a third of DRAM bandwidth).
template <int DK>
struct BoxLoads {
  static constexpr int value = DK <= 2 ? 8 : DK <= 4 ? 4 : DK <= 8 ? 2 : 1;
};

template <int DK, bool VEC>
__global__ void curve_bbox_kernel(const int32_t* __restrict__ pts, const int64_t* __restrict__ offsets,
                                  int64_t first, int64_t n_curves, int dim, int check, long long lim, int* bbox,
                                  int* err) {
  griddep_launch_dependents();   // the plan may start (it waits for the boxes)
  constexpr int NL = BoxLoads<DK>::value;
  const int L = threadIdx.x & 31;
  const int64_t total = offsets[n_curves];
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  bool bad = false;
  int64_t c = first + (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  int64_t o = 0, e = 0;
  if (c < n_curves) {
    o = offsets[c];
    e = offsets[c + 1];
  }
  for (; c < n_curves; c += wstride) {
    int64_t on = 0, en = 0;
    if (c + wstride < n_curves) {
      on = offsets[c + wstride];
      en = offsets[c + wstride + 1];
    }
    int lo[DK], hi[DK];
#pragma unroll
    for (int k = 0; k < DK; ++k) {
      lo[k] = INT_MAX;
      hi[k] = INT_MIN;
    }
    if (o >= 0 && e <= total && o < e) {
      const int64_t len = e - o;
      for (int64_t j0 = 0; j0 < len; j0 += 32 * NL) {
        const int32_t* Q = pts + (o + j0) * dim;
        const int last = (int)min(len - 1 - j0, (int64_t)(32 * NL - 1));
        int32_t qk[NL][DK];
#pragma unroll
        for (int u = 0; u < NL; ++u) load_point<int32_t, DK>(Q, min(32 * u + L, last), dim, VEC, qk[u]);
#pragma unroll
        for (int u = 0; u < NL; ++u) {
#pragma unroll
          for (int k = 0; k < DK; ++k) {
            lo[k] = min(lo[k], qk[u][k]);
            hi[k] = max(hi[k], qk[u][k]);
          }
        }
      }
    }
    if (check) {
#pragma unroll
      for (int k = 0; k < DK; ++k)
        if (k < dim) bad |= (long long)lo[k] < -lim || (long long)hi[k] > lim;   // empty: lo > hi, passes
    }
#pragma unroll
    for (int k = 0; k < DK; ++k) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], off));
        hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], off));
      }
    }
    if (L == 0) {
#pragma unroll
      for (int k = 0; k < DK; ++k) {
        bbox[(c * DK + k) * 2] = lo[k];
        bbox[(c * DK + k) * 2 + 1] = hi[k];
      }
    }
    o = on;
    e = en;
  }
  if (__any_sync(0xffffffffu, bad) && L == 0) raise_error(err, DFD_ERR_RANGE);
}

// ------------------------------------------------------------- planning
// Work order: by code variant first (rows per lane R, then the number of
// stripes), largest first, then by column count, largest first (LPT within
// a variant).  Warps resident together then mostly run the same variant,
// and the costliest pairs start first.  16 variant classes x 16 column
// buckets of 256 per value class; int32 pairs come in two value classes
// (exact int64 first, then exact uint32 bits, I32B).
constexpr int NBUCKET1 = 256;
// Team buckets come first: pairs of several stripes that a whole CTA runs
// together (see batch_kernel), 16 cost buckets per value class, costliest
// first.  The warp buckets follow.
constexpr int NTB1 = 16;
constexpr int NTB = 2 * NTB1;
constexpr int NBUCKET = NTB + 2 * NBUCKET1;
constexpr unsigned kNarrowBit = 1u << 30;   // worklist: pair index | narrow << 30 | swap << 31

// Orientation of a pair (delta(p, q) = delta(q, p), bit for bit: the ground
// distance is symmetric in every value class).  A warp spends about
// stripes x (cols + 31) steps on a pair -- the 31 being the systolic ramp --
// and a step costs a cell's instructions per row of a lane (5 for points of
// up to 4 coordinates, 10 for 8, 18 for 16) and about eight more (the
// shuffle from the lane above, the column record's load, lane 0's select,
// the loop), measured on uniform int32 2-D batches (47.9 per step at R = 8,
// 27.7 at R = 4).  The rows are the curve for which that estimate is lower,
// with Rmax rows per lane whatever the launch's cap, so that the host can
// repeat the choice: e.g. 100 x 500 2-D points run as two stripes of 8 rows
// a lane over 131 steps each (12.6k instructions) rather than one stripe of
// 4 rows over 531 steps (14.9k).  Ties keep rows = the shorter curve.
__host__ __device__ __forceinline__ int rmax_of_class(int dk) { return dk <= 4 ? 8 : 4; }
// (32-bit divisions: a 64-bit one is a long software routine on the GPU,
// and the one-block plan of a small launch waits on it; lengths past 2^30,
// which no curve here reaches, count as 2^30.)
__host__ __device__ __forceinline__ long long orient_cost(int64_t rows, int64_t cols, int dk) {
  const unsigned rmax = (unsigned)rmax_of_class(dk);
  const unsigned cell = dk <= 4 ? 5u : dk <= 8 ? 10u : 18u;
  const unsigned R = (unsigned)(rows < (1LL << 30) ? rows : (1LL << 30));
  const unsigned st = (R + 32u * rmax - 1u) / (32u * rmax);
  const unsigned r = R <= 32u ? 1u : (R + 32u * st - 1u) / (32u * st);
  return (long long)st * (long long)(cols + 31) * (long long)(cell * r + 8u);
}
// Whether curve b supplies the rows of pair (a, b) (a has na points, b nb;
// dk = the dimension class).
__host__ __device__ __forceinline__ bool rows_from_b(int64_t na, int64_t nb, int dk) {
  const long long ca = orient_cost(na, nb, dk), cb = orient_cost(nb, na, dk);
  return cb < ca || (cb == ca && nb < na);
}
// The plan's choice: the cheaper orientation, unless only the other one
// keeps a pair of several stripes (of 32 * rmax rows) within a warp's row
// buffer (buf_cols columns).
__host__ __device__ __forceinline__ bool plan_rows_from_b(int64_t na, int64_t nb, int dk, int rmax, int64_t buf_cols) {
  const bool sw = rows_from_b(na, nb, dk);
  const int64_t rows = sw ? nb : na, cols = sw ? na : nb;
  const bool fits = rows <= 32 * (int64_t)rmax || cols <= buf_cols;
  const bool fits_other = cols <= 32 * (int64_t)rmax || rows <= buf_cols;
  return (!fits && fits_other) ? !sw : sw;
}

// Team bucket of a pair: floor(log2(rows * (cols + 31))) from 2^16 (15) up
// to 2^31 and beyond (0), so the costliest team pairs start first.
__device__ __forceinline__ int team_bucket(int64_t rows, int64_t cols) {
  const unsigned long long cost = (unsigned long long)rows * (unsigned long long)(cols + 31);
  const int msb = 63 - __clzll((long long)cost);
  return 15 - min(15, max(0, msb - 16));
}

__device__ __forceinline__ int cost_bucket(int64_t rows, int64_t cols, int rmax) {
  const int64_t per_stripe = 32 * (int64_t)rmax;
  const int64_t stripes = (rows + per_stripe - 1) / per_stripe;
  const int cls = stripes > 1 ? rmax + (int)min(stripes - 1, (int64_t)6) : (int)((rows + 31) / 32);
  const int sub = 15 - (int)min((int64_t)15, (cols - 1) / 256);
  return (15 - min(cls, 15)) * 16 + sub;
}

// The packing order the autotuner can pick instead (order 1): pairs by
// estimated cost alone, largest first -- stripes x rows per lane x (columns +
// the 31-step ramp), on a log scale of 1/8 octave -- whatever their code
// variant.  Either order computes every pair the same way; only the
// assignment of pairs to warps over time differs.
__device__ __forceinline__ int cost_bucket_lpt(int64_t rows, int64_t cols, int rmax) {
  const int64_t per_stripe = 32 * (int64_t)rmax;
  const int64_t st = (rows + per_stripe - 1) / per_stripe;
  const int64_t r = rows <= 32 ? 1 : min((int64_t)rmax, (rows + 32 * st - 1) / (32 * st));
  const unsigned long long cost = (unsigned long long)(st * r) * (unsigned long long)(cols + 31);   // >= 32
  const int msb = 63 - __clzll((long long)cost);
  const int b = 8 * msb + (int)((cost >> (msb - 3)) & 7);
  return NBUCKET1 - 1 - min(NBUCKET1 - 1, b);
}

// Whether a pair of several stripes should run as a CTA team (mode 3), from
// a latency model of the two schedules in steps x cycles per step (a step
// of R rows per lane costs about 24 + 8 R cycles: the shuffle from the lane
// above, then R dependent cells), with the launch's pairs taking rounds of
// the resident warps (one warp per pair) or CTAs (one team per pair):
//   one warp:  ceil(N / (8 C)) * stripes * (cols + 31) * (24 + 8 Rmax)
//   team:      ceil(N / C) * (cycles * (cols + 31) + (warps used - 1) * 64) * (24 + 8 Rt)
// where a team spreads its rows over 8 warps with Rt rows per lane and the
// hand-off between consecutive stripes lags 64 steps.  On the paper's
// Experiment 1 shapes this picks teams for 32 .. 512 pairs of 1,024 points
// and for 1,024 pairs of 2,048 points and more, one warp otherwise (measured
// both ways).
// (float32 and 32-bit divisions: the decision changes no result, and FP64
// arithmetic and 64-bit division are slow paths that the one-block plan of a
// small launch would wait on; lengths and counts past 2^30 count as 2^30.)
__device__ __forceinline__ bool team_pays(int64_t rows64, int64_t cols, int rmax, int64_t n_pairs, int ctas) {
  const unsigned rows = (unsigned)min(rows64, (int64_t)1 << 30);
  const unsigned np = (unsigned)min(n_pairs, (int64_t)1 << 30);
  const unsigned rm = (unsigned)rmax, cs = (unsigned)max(ctas, 1);
  const float c = (float)cols + 31.0f;
  const unsigned sw = (rows + 32u * rm - 1u) / (32u * rm);
  const float warp_rounds = (float)((np + 8u * cs - 1u) / (8u * cs));
  const float warp_cost = warp_rounds * (float)sw * c * (24.0f + 8.0f * (float)rm);
  unsigned rt = (rows + 32u * 8u - 1u) / (32u * 8u);
  rt = rt < 1u ? 1u : (rt > rm ? rm : rt);
  const unsigned st = (rows + 32u * rt - 1u) / (32u * rt);
  const unsigned cyc = (st + 7u) / 8u;
  const unsigned used = st < 8u ? st : 8u;
  const float team_rounds = (float)((np + cs - 1u) / cs);
  const float team_cost = team_rounds * ((float)cyc * c + (float)(used - 1u) * 64.0f) * (24.0f + 8.0f * (float)rt);
  return team_cost < warp_cost;
}

struct PlanArgs {
  int order;           // 0: variant-major buckets (cost_bucket), 1: cost-descending (cost_bucket_lpt)
  int team;            // 0: no team buckets; 1: pairs of several stripes wider than buf_cols; 2: every pair of
                       // several stripes; 3: those, when team_pays says so, and the wide ones
  int buf_cols;        // row buffer columns of one warp
  int ctas;            // persistent CTAs of the batch kernel (8 warps each)
  const int64_t* offsets;
  const int32_t* pairs;
  int64_t n_pairs;
  int64_t n_curves;
  unsigned* hist;      // [NBUCKET]
  unsigned* cursor;    // [NBUCKET]
  unsigned short* bucket;  // [n_pairs]
  unsigned* worklist;  // [n_pairs]: pair index | narrow << 30 | swap << 31
  const int* bbox;     // int32 batches: per curve and coordinate (min, max); else null
  int dk;              // coordinates per bbox entry
  int* err;
  int rmax;            // rows per lane of one stripe for this dimension class
  // Pairs this launch takes (a host-buffer call runs one launch per copy
  // slice over the whole pair list): those whose later curve id lies in
  // [lo_curve, hi_curve), and the pairs with an id outside [0, n_ids) when
  // take_invalid is set (they only raise DFD_ERR_INVALID_ARG).  The others
  // get bucket kNoBucket and no work-list slot.
  int64_t n_ids;
  int64_t lo_curve, hi_curve;
  int take_invalid;
};
constexpr unsigned short kNoBucket = 0xFFFF;

// The counting sort's atomics are aggregated per warp: the lanes of a warp
// that fall in one bucket add their count with one atomic (hist) or take
// consecutive slots from one (scatter), since a batch's pairs crowd into a
// few buckets.  Each warp walks the pairs 32 at a time with all lanes
// together, so the match covers the whole warp.
// (static: this header is compiled into several translation units)
// Bucket of pair k (k < n_pairs), or -1 when the pair belongs to another
// launch; also raises the plan's input errors.
__device__ __forceinline__ int plan_bucket(const PlanArgs& a, int64_t k) {
  const int32_t ia = a.pairs[2 * k], ib = a.pairs[2 * k + 1];
  const bool valid_id = ia >= 0 && ib >= 0 && ia < a.n_ids && ib < a.n_ids;
  const int64_t c = max(ia, ib);
  if (!(valid_id ? (c >= a.lo_curve && c < a.hi_curve) : a.take_invalid != 0)) return -1;
  int b = NTB + NBUCKET1 - 1;   // invalid pairs: last of the int64 warp class (skipped by the kernel)
  if (ia < 0 || ib < 0 || ia >= a.n_curves || ib >= a.n_curves) {
    raise_error(a.err, DFD_ERR_INVALID_ARG);
  } else {
    const int64_t total = a.offsets[a.n_curves];
    const int64_t oa = a.offsets[ia], ob = a.offsets[ib], ea = a.offsets[ia + 1], eb = a.offsets[ib + 1];
    const int64_t na = ea - oa, nb = eb - ob;
    if (na < 1 || nb < 1 || oa < 0 || ob < 0 || ea > total || eb > total || na > INT32_MAX || nb > INT32_MAX)
      raise_error(a.err, DFD_ERR_INVALID_ARG);
    const bool sw = plan_rows_from_b(na, nb, a.dk, a.rmax, a.buf_cols);
    const int64_t rows = max(sw ? nb : na, (int64_t)1), cols = max(sw ? na : nb, (int64_t)1);
    const bool narrow = a.bbox && narrow_pair(a.bbox, a.dk, ia, ib);
    const bool multi = rows > 32 * (int64_t)a.rmax;
    if (a.team && multi &&
        (a.team == 2 || cols > a.buf_cols || (a.team == 3 && team_pays(rows, cols, a.rmax, a.n_pairs, a.ctas)))) {
      b = team_bucket(rows, cols) + (narrow ? NTB1 : 0);
    } else {
      b = NTB + (a.order ? cost_bucket_lpt(rows, cols, a.rmax) : cost_bucket(rows, cols, a.rmax));
      if (narrow) b += NBUCKET1;
    }
  }
  return b;
}

// Work-list entry of pair k in bucket b: index | narrow << 30 | swap << 31.
__device__ __forceinline__ unsigned plan_entry(const PlanArgs& a, int64_t k, int b) {
  const int32_t ia = a.pairs[2 * k], ib = a.pairs[2 * k + 1];
  unsigned swap = 0;
  if (ia >= 0 && ib >= 0 && ia < a.n_curves && ib < a.n_curves) {
    const int64_t na = a.offsets[ia + 1] - a.offsets[ia], nb = a.offsets[ib + 1] - a.offsets[ib];
    swap = plan_rows_from_b(na, nb, a.dk, a.rmax, a.buf_cols) ? 1u : 0u;   // as in plan_bucket
  }
  const unsigned narrow = (b < NTB ? b >= NTB1 : b - NTB >= NBUCKET1) ? kNarrowBit : 0u;
  return (unsigned)k | narrow | (swap << 31);
}

// Plan kernels run with programmatic stream serialisation (launch_pdl) right
// after the call's own check or box kernel: an int32 plan waits for the
// bounding boxes before it classifies; a float32 plan needs nothing from the
// input check, runs beside it and waits for it only before it finishes, so
// that the batch kernel, which waits for the plan, also finds the check done.
static __global__ void plan_hist_kernel(PlanArgs a) {
  griddep_launch_dependents();
  if (a.bbox) griddep_wait();
  const int L = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k0 = 32 * w0; k0 < a.n_pairs; k0 += 32 * wstride) {
    const int64_t k = k0 + L;
    int b = -1;
    if (k < a.n_pairs) {
      b = plan_bucket(a, k);
      a.bucket[k] = b >= 0 ? (unsigned short)b : kNoBucket;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    if (b >= 0 && L == __ffs(peers) - 1) atomicAdd(&a.hist[b], (unsigned)__popc(peers));
  }
  griddep_wait();
}

// One block of NBUCKET threads: exclusive scan of the bucket counts into
// the cursors (a shuffle scan per warp, then over the warp totals).
static __global__ void plan_scan_kernel(PlanArgs a) {
  static_assert(NBUCKET % 32 == 0 && NBUCKET / 32 <= 32 && NBUCKET <= 1024, "one block, one warp of warp totals");
  __shared__ unsigned wsum[NBUCKET / 32];
  griddep_launch_dependents();
  griddep_wait();   // the counts
  const int b = threadIdx.x, L = b & 31, w = b >> 5;
  const unsigned x = a.hist[b];
  unsigned inc = x;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, inc, off);
    if (L >= off) inc += y;
  }
  if (L == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    unsigned t = L < NBUCKET / 32 ? wsum[L] : 0u;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, t, off);
      if (L >= off) t += y;
    }
    if (L < NBUCKET / 32) wsum[L] = t;   // inclusive totals through warp L
  }
  __syncthreads();
  a.cursor[b] = (w > 0 ? wsum[w - 1] : 0u) + inc - x;
}

static __global__ void plan_scatter_kernel(PlanArgs a) {
  griddep_launch_dependents();
  griddep_wait();   // the cursors (and, through the scan, the buckets)
  const int L = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k0 = 32 * w0; k0 < a.n_pairs; k0 += 32 * wstride) {
    const int64_t k = k0 + L;
    const int b = k < a.n_pairs && a.bucket[k] != kNoBucket ? (int)a.bucket[k] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(peers) - 1;
    unsigned pos = 0;
    if (b >= 0 && L == leader) pos = atomicAdd(&a.cursor[b], (unsigned)__popc(peers));
    pos = __shfl_sync(0xffffffffu, pos, leader) + __popc(peers & ((1u << L) - 1u));
    if (b < 0) continue;
    a.worklist[pos] = plan_entry(a, k, b);
  }
}

// The whole plan of a launch of at most kSmallPlanPairs pairs in one block
// of 1024 threads: the scratch header (zero_words words: counters, bucket
// counts, cursors, SM slots) zeroed, the bucket counts and their scan in
// shared memory, the scatter, and the final cursors (read by the batch
// kernel) stored.  The general plan takes a memset and three kernels, whose
// launch gaps dominate a small launch (32 pairs of 1,024 points).
constexpr int64_t kSmallPlanPairs = 2048;
static __global__ void __launch_bounds__(1024) plan_small_kernel(PlanArgs a, unsigned* zero_base, int zero_words) {
  static_assert(NBUCKET <= 1024, "one bucket per thread");
  __shared__ unsigned cnt[NBUCKET];
  __shared__ unsigned wsum[32];
  griddep_launch_dependents();
  if (a.bbox) griddep_wait();   // int32: the bounding boxes (see plan_hist_kernel)
  const int t = threadIdx.x, L = t & 31, w = t >> 5;
  for (int i = t; i < zero_words; i += blockDim.x) zero_base[i] = 0u;
  for (int i = t; i < NBUCKET; i += blockDim.x) cnt[i] = 0u;
  __syncthreads();
  for (int64_t k = t; k < a.n_pairs; k += blockDim.x) {
    const int b = plan_bucket(a, k);
    a.bucket[k] = b >= 0 ? (unsigned short)b : kNoBucket;
    if (b >= 0) atomicAdd(&cnt[b], 1u);
  }
  __syncthreads();
  // exclusive scan of the counts: a shuffle scan per warp, then over the warp totals
  const unsigned x = t < NBUCKET ? cnt[t] : 0u;
  unsigned inc = x;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, inc, off);
    if (L >= off) inc += y;
  }
  if (L == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    unsigned v = wsum[L];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, v, off);
      if (L >= off) v += y;
    }
    wsum[L] = v;   // inclusive totals through warp L
  }
  __syncthreads();
  if (t < NBUCKET) cnt[t] = (w > 0 ? wsum[w - 1] : 0u) + inc - x;
  __syncthreads();
  for (int64_t k = t; k < a.n_pairs; k += blockDim.x) {
    const unsigned short bb = a.bucket[k];
    if (bb == kNoBucket) continue;
    const unsigned pos = atomicAdd(&cnt[bb], 1u);
    a.worklist[pos] = plan_entry(a, k, (int)bb);
  }
  __syncthreads();
  for (int i = t; i < NBUCKET; i += blockDim.x) a.cursor[i] = cnt[i];
  griddep_wait();
}

// ------------------------------------------------------------ batch kernel
struct BatchArgs {
  unsigned* sm_rank;   // kSmSlots counters, zeroed per launch (pop_first, team_pop_first)
  int n_sm;            // SMs the grid covers
  void* rowbuf;        // per-warp buf_cols values (multi-stripe pairs); a CTA's eight are contiguous
  int buf_cols;        // row buffer columns per warp (>= BUF_COLS; the decider uses BUF_COLS)
  const void* points;
  const int64_t* offsets;
  const int32_t* pairs;
  const unsigned* worklist;
  int64_t n_items;
  const unsigned* n_items_dev;   // batch kernel: items of the work list, written by the plan (null: n_items)
  int64_t n_curves;
  int dim;
  int vec;             // 1: vector point loads allowed (dim == DK, 16-byte aligned points)
  int* counter;
  int* err;
  void* out_dist;
  void* out_dist2;
  // CTA teams (batch kernel only; null n_team: none)
  const unsigned* n_team;   // items at the front of the worklist run by CTA teams (written by the plan)
  int* team_counter;
  unsigned* done_ctas;      // CTAs finished with the team and warp items
  unsigned* deferred;       // worklist entries of team pairs wider than one CTA's row buffers
  unsigned* n_deferred;
  unsigned long long timeout_ns;
  int rmax;                 // rows per lane cap of one-warp pairs (<= Rmax; the launch's tuned shape)
  unsigned* meet;           // kMeetItems x 4 words, zeroed per launch: team pairs split over two CTAs
};

// Team pairs run as two halves on two CTAs (see run_team_pair) when at most
// this many team items exist and their halves fit one per SM.
constexpr int kMeetItems = 128;

// Ring columns of a team's shared-memory hand-off (per warp, 8 bytes a slot).
template <int DK>
struct TeamRing {
  static constexpr int value = DK >= 16 ? 128 : 256;
};
constexpr int kTeamWarps = 8;   // a team is the CTA's 8 warps

// Rows per lane of a team pair: the rows spread over all the team's warps
// (one stripe each) when they fit, else the largest stripes, cycling.
template <int DK>
__host__ __device__ __forceinline__ int team_rows_per_lane(int rows, int nw = kTeamWarps) {
  constexpr int RM = Rmax<DK>::value;
  if (rows <= 32) return 1;
  const int r = (rows + 32 * nw - 1) / (32 * nw);
  return r > RM ? RM : r;
}

template <class V, int DK, class IO>
__device__ __forceinline__ typename V::value team_dfd_any(const typename V::coord* P, int n,
                                                          const typename V::coord* Q, int m, int dim, bool vec,
                                                          int L, int w, uint4* stage, IO* io, int nw = kTeamWarps,
                                                          int pstep = 0, int qsign = 1) {
  constexpr int RM = Rmax<DK>::value;
  using T = typename V::value;
  switch (team_rows_per_lane<DK>(n, nw)) {
#define DFD_T_CASE(RR)                                                                                         \
  case RR:                                                                                                     \
    if constexpr (RR < RM)                                                                                     \
      return warp_dfd<V, DK, RR, NoAbandon<V>, IO>(P, n, Q, m, dim, vec, static_cast<T*>(nullptr), L, w,       \
                                                   1 << 30, static_cast<NoAbandon<V>*>(nullptr), stage, io, nw, \
                                                   pstep, qsign);                                              \
    break;
    DFD_T_CASE(1)
    DFD_T_CASE(2)
    DFD_T_CASE(3)
    DFD_T_CASE(4)
    DFD_T_CASE(5)
    DFD_T_CASE(6)
    DFD_T_CASE(7)
    default:
      break;
#undef DFD_T_CASE
  }
  return warp_dfd<V, DK, RM, NoAbandon<V>, IO>(P, n, Q, m, dim, vec, static_cast<T*>(nullptr), L, w, 1 << 30,
                                               static_cast<NoAbandon<V>*>(nullptr), stage, io, nw, pstep, qsign);
}

// First team pop of a CTA: when every team item fits one round of the SMs,
// a CTA that is not the first on its SM waits (bounded, placement only)
// until every item is taken, so the teams spread one per SM.
__device__ __forceinline__ int team_pop_first(int* counter, unsigned* sm_rank, int n_sm, long long total) {
  if (sm_rank && total <= n_sm) {
    unsigned sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    const unsigned q = 640u + sm;
    const unsigned r = q < (unsigned)kSmSlots ? atomicAdd(&sm_rank[q], 1u) : 0u;
    if (r > 0) {
      const unsigned long long t0 = globaltimer_ns();
      for (int it = 0; it < kSpreadPolls && (long long)ld_relaxed_i32(counter) < total &&
                       globaltimer_ns() - t0 < kSpreadWaitNs;
           ++it) {
      }
    }
  }
  return atomicAdd(counter, 1);
}

// Meeting of a split team pair's halves (see combine_kernel): F is the
// forward half's last row (row h - 1), B the backward half's (row h, taken
// with q reversed, so B[m-1-j] is column j); every monotone path steps from
// row h - 1 to row h once, so delta^2 = min_j max(F[j], min(B at j, B at
// j + 1)) -- a selection among the same values, bit for bit the one-front
// result.  All threads of the CTA call it; thread 0 gets the result.
// `scratch`: 8 shared-memory words the CTA no longer uses (its rings).
// Rows written by another SM are read through L2 (CG).
template <class V, bool CG = false>
__device__ __forceinline__ typename V::value meet_rows(const typename V::value* F, const typename V::value* B, int m,
                                                       unsigned long long* scratch) {
  using T = typename V::value;
  auto ld = [](const T* p) { return CG ? __ldcg(p) : *p; };
  T best = V::inf();
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const T bj = ld(B + (m - 1 - j));
    const T bj1 = j + 1 < m ? ld(B + (m - 2 - j)) : V::inf();
    best = V::vmin(best, V::vmax(ld(F + j), V::vmin(bj, bj1)));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) best = V::vmin(best, __shfl_xor_sync(0xffffffffu, best, off));
  T* part = reinterpret_cast<T*>(scratch);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = best;
  __syncthreads();
  T r = V::inf();
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r = V::vmin(r, part[k]);
  return r;
}

// One team pair (all 256 threads of the CTA call it): the rows (the plan's
// orientation) in stripes over the 8 warps (TeamIO), the result written by
// the warp that runs the last stripe.  `gbuf` holds `gcols` values; a pair
// with more stripes than warps needs m of them, else it is not run here and
// false is returned (CTA-uniform).
// With only_half = 0 or 1 the CTA runs one half of a two-front pair (below)
// and another CTA the other: `meet` is the pair's 4 words (count, the two
// halves' CTAs + 1), `xw` a shared word, and *hold is set when this CTA
// finished first, so its row buffer holds its half's row until the other
// CTA has read it.  A pair that does not split runs whole in half 0's CTA.
template <class V, int DK>
__device__ __forceinline__ bool run_team_pair(const BatchArgs& a, unsigned wentry, void* gbuf, long long gcols,
                                              uint4* stage, unsigned long long* ring, unsigned long long* prog,
                                              unsigned long long* cons, int only_half = -1,
                                              unsigned* meet = nullptr, int* xw = nullptr, bool* hold = nullptr) {
  using Cd = typename V::coord;
  const int L = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t k = wentry & (kNarrowBit - 1);
  int32_t ia = a.pairs[2 * k], ib = a.pairs[2 * k + 1];
  if (wentry >> 31) {
    const int32_t t = ia;
    ia = ib;
    ib = t;
  }
  if (ia < 0 || ib < 0 || ia >= a.n_curves || ib >= a.n_curves) return true;   // reported by the plan
  const int64_t total = a.offsets[a.n_curves];
  const int64_t oa = a.offsets[ia], ob = a.offsets[ib];
  const int64_t ea = a.offsets[ia + 1], eb = a.offsets[ib + 1];
  if (oa < 0 || ob < 0 || ea > total || eb > total) return true;                // reported by the plan
  const int n = (int)(ea - oa), m = (int)(eb - ob);
  if (n < 1 || m < 1) return true;                                               // reported by the plan
  const Cd* pts = static_cast<const Cd*>(a.points);
  // Two fronts (as the band wavefront's): when each half of the rows fits
  // kHalf stripes, warps 0..3 run the first h rows forward and warps 4..7 the
  // other n - h rows backwards against q reversed, each half a pipeline of
  // its own, and their last rows meet in the CTA (meet_rows): the pipeline
  // is half as deep.  The halves' last rows sit in the CTA's row buffer.
  // With only_half set, the CTA's warps of that half run it (one warp per
  // SM sub-partition, the others wait at the barrier) and the CTA that
  // finishes second meets the two rows, the other's read through L2.
  constexpr int kHalf = kTeamWarps / 2;
  const int h = (n + 1) / 2;
  const bool split = n >= 64 && h <= kHalf * 32 * Rmax<DK>::value && 2LL * m <= gcols;
  if (only_half == 1 && !split) return true;   // half 0's CTA runs the whole pair
  if (split) {
    if (threadIdx.x < kTeamWarps) {
      prog[threadIdx.x] = 0;
      cons[threadIdx.x] = 0;
    }
    __syncthreads();
    const int half = w / kHalf;
    const int nh = half == 0 ? h : n - h;
    const int Rh = team_rows_per_lane<DK>(nh, kHalf);
    TeamIO<TeamRing<DK>::value> io;
    io.gbuf = gbuf;   // (no wrap-around: a half has at most kHalf stripes)
    io.ring = ring + (size_t)half * kHalf * TeamRing<DK>::value;
    io.prog = prog + half * kHalf;
    io.cons = cons + half * kHalf;
    io.w = w % kHalf;
    io.nw = kHalf;
    io.err = a.err;
    io.timeout_ns = a.timeout_ns;
    io.last_st = (nh + 32 * Rh - 1) / (32 * Rh) - 1;
    const Cd* P = pts + (half == 0 ? oa : oa + n - 1) * a.dim;
    const Cd* Q = pts + (half == 0 ? ob : ob + m - 1) * a.dim;
    const int ps = half == 0 ? a.dim : -a.dim, qs = half == 0 ? 1 : -1;
    const bool mine = only_half < 0 || half == only_half;
    auto run = [&](auto cls) {
      using VV = decltype(cls);
      using TT = typename VV::value;
      TT* rows = static_cast<TT*>(gbuf);
      io.final_out = rows + (size_t)half * m;
      if (mine) team_dfd_any<VV, DK>(P, nh, Q, m, a.dim, a.vec != 0, L, io.w, stage, &io, kHalf, ps, qs);
      __syncthreads();
      if (only_half < 0) {
        const TT r = meet_rows<VV>(rows, rows + m, m, ring);
        if (threadIdx.x == 0) write_result<VV>(a.out_dist, a.out_dist2, k, r);
        __syncthreads();
        return;
      }
      // publish this half's row (every writer's stores before the count),
      // then count; the second CTA reads the first's CTA index and meets
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        *reinterpret_cast<volatile unsigned*>(&meet[1 + only_half]) = blockIdx.x + 1u;
        __threadfence();
        const unsigned before = atomicAdd(&meet[0], 1u);
        int other = -1;
        if (before == 1) {
          other = (int)*reinterpret_cast<volatile unsigned*>(&meet[2 - only_half]) - 1;
          __threadfence();
        }
        *xw = before == 0 ? -2 : other;
      }
      __syncthreads();
      const int other = *xw;
      *hold = other == -2;
      if (other >= 0) {
        // the other CTA's row buffer, offset as gbuf is (in the launch's value type)
        const TT* orow = reinterpret_cast<const TT*>(static_cast<const typename V::value*>(a.rowbuf) +
                                                     (int64_t)other * kTeamWarps * a.buf_cols);
        const TT* F = only_half == 0 ? rows : orow;
        const TT* B = only_half == 1 ? rows + m : orow + m;
        const TT r = meet_rows<VV, true>(F, B, m, ring);
        if (threadIdx.x == 0) write_result<VV>(a.out_dist, a.out_dist2, k, r);
      }
      __syncthreads();
    };
    if constexpr (std::is_same<V, I32>::value) {
      if (wentry & kNarrowBit) {
        run(I32B{});
        return true;
      }
    }
    run(V{});
    return true;
  }
  const int R = team_rows_per_lane<DK>(n);
  const int S = (n + 32 * R - 1) / (32 * R);
  if (S > kTeamWarps && (long long)m > gcols) return false;
  if (threadIdx.x < kTeamWarps) {
    prog[threadIdx.x] = 0;
    cons[threadIdx.x] = 0;
  }
  __syncthreads();
  TeamIO<TeamRing<DK>::value> io;
  io.gbuf = gbuf;
  io.ring = ring;
  io.prog = prog;
  io.cons = cons;
  io.w = w;
  io.nw = kTeamWarps;
  io.err = a.err;
  io.timeout_ns = a.timeout_ns;
  io.final_out = nullptr;
  io.last_st = S - 1;
  const bool last_warp = w == (S - 1) % kTeamWarps;
  if constexpr (std::is_same<V, I32>::value) {
    if (wentry & kNarrowBit) {
      const float r = team_dfd_any<I32B, DK>(pts + oa * a.dim, n, pts + ob * a.dim, m, a.dim, a.vec != 0, L, w,
                                             stage, &io);
      if (last_warp && L == 0) write_result<I32B>(a.out_dist, a.out_dist2, k, r);
      __syncthreads();
      return true;
    }
  }
  const typename V::value r =
      team_dfd_any<V, DK>(pts + oa * a.dim, n, pts + ob * a.dim, m, a.dim, a.vec != 0, L, w, stage, &io);
  if (last_warp && L == 0) write_result<V>(a.out_dist, a.out_dist2, k, r);
  __syncthreads();
  return true;
}

// Persistent CTAs in three phases:
//  1. team items (the front of the worklist): the CTA's 8 warps run one
//     pair of several stripes together, as a pipeline over the columns --
//     pairs too long for one warp to finish early, or too wide for one
//     warp's row buffer; their wrap-around row lives in the CTA's eight
//     contiguous warp buffers (8 * buf_cols columns);
//  2. warp items: one warp per pair (warp_dfd), as many at a time as warps;
//  3. the last CTA to finish runs the team pairs that were wider than a
//     CTA's buffers, with every warp buffer of the launch as one row buffer
//     (all other CTAs are done with theirs); a pair wider still gets NaN /
//     -1 outputs and DFD_ERR_UNSUPPORTED in the error word.
template <class V, int DK>
__global__ void __launch_bounds__(256, kBlocksPerSM<DK>::value) batch_kernel(BatchArgs a) {
  using T = typename V::value;
  using Cd = typename V::coord;
  __shared__ uint4 stage_sm[8][QStage<DK>::RECS];
  __shared__ unsigned long long team_ring[kTeamWarps * TeamRing<DK>::value];
  __shared__ unsigned long long team_prog[kTeamWarps], team_cons[kTeamWarps];
  __shared__ int cta_word;
  uint4* stage = stage_sm[threadIdx.x >> 5];
  const int L = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  T* buf = static_cast<T*>(a.rowbuf) + gw * (int64_t)a.buf_cols;
  const Cd* pts = static_cast<const Cd*>(a.points);
  // the plan (and through it the input check) is done from here on
  griddep_wait();
  const int64_t total = a.offsets[a.n_curves];
  if (threadIdx.x == 0) cta_word = ld_relaxed_i32(a.err);
  __syncthreads();
  if (cta_word != 0) return;   // CTA-uniform
  const long long n_team = a.n_team ? (long long)*a.n_team : 0;

  // 1. team items.  When every team pair's two halves fit one per SM, the
  // items are halves (2t: pair t's first half, 2t + 1 its second), each CTA
  // runs one with one warp per SM sub-partition, and the CTA that finishes
  // a half first keeps its row buffer (hold): no more items for it.
  bool hold = false;
  if (n_team > 0) {
    void* gbuf = static_cast<T*>(a.rowbuf) + (int64_t)blockIdx.x * kTeamWarps * a.buf_cols;
    const bool halves = a.meet && n_team <= kMeetItems && 2 * n_team <= a.n_sm;
    const long long n_pop = halves ? 2 * n_team : n_team;
    for (bool first = true; !hold; first = false) {
      __syncthreads();
      if (threadIdx.x == 0)
        cta_word = first ? team_pop_first(a.team_counter, a.sm_rank, a.n_sm, n_pop) : atomicAdd(a.team_counter, 1);
      __syncthreads();
      const int item = cta_word;
      if (item >= n_pop) break;
      const int ti = halves ? item >> 1 : item;
      const unsigned we = a.worklist[ti];
      const bool ran = halves ? run_team_pair<V, DK>(a, we, gbuf, (long long)kTeamWarps * a.buf_cols, stage, team_ring,
                                                     team_prog, team_cons, item & 1, a.meet + 4 * ti, &cta_word, &hold)
                              : run_team_pair<V, DK>(a, we, gbuf, (long long)kTeamWarps * a.buf_cols, stage, team_ring,
                                                     team_prog, team_cons);
      if (!ran && threadIdx.x == 0) a.deferred[atomicAdd(a.n_deferred, 1u)] = we;
    }
  }

  // 2. warp items (none for a CTA whose row buffer holds a half's row)
  const long long n_items = a.n_items_dev ? (long long)*a.n_items_dev : a.n_items;
  const long long n_warp = hold ? 0 : n_items - n_team;
  for (bool first = true;; first = false) {
    int item = 0;
    if (L == 0) item = first ? pop_first(a.counter, a.sm_rank, a.n_sm, n_warp) : atomicAdd(a.counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= n_warp) break;
    const unsigned w = a.worklist[n_team + item];
    const int64_t k = w & (kNarrowBit - 1);
    int32_t ia = a.pairs[2 * k], ib = a.pairs[2 * k + 1];
    if (w >> 31) {
      const int32_t t = ia;
      ia = ib;
      ib = t;
    }
    if (ia < 0 || ib < 0 || ia >= a.n_curves || ib >= a.n_curves) continue;  // reported by the plan
    const int64_t oa = a.offsets[ia], ob = a.offsets[ib];
    const int64_t ea = a.offsets[ia + 1], eb = a.offsets[ib + 1];
    if (oa < 0 || ob < 0 || ea > total || eb > total) continue;             // reported by the plan
    const int n = (int)(ea - oa), m = (int)(eb - ob);
    if (n < 1 || m < 1) continue;                                            // reported by the plan
    if (!fits_buffer<DK>(n, m, a.buf_cols, a.rmax)) {
      // only when the plan made no team items (decider-style launches)
      if (L == 0) {
        raise_error(a.err, DFD_ERR_UNSUPPORTED);
        write_unsupported<V>(a.out_dist, a.out_dist2, k);
      }
      continue;
    }
    if constexpr (std::is_same<V, I32>::value) {
      if (w & kNarrowBit) {
        const float r = warp_dfd_any<I32B, DK>(pts + oa * a.dim, n, pts + ob * a.dim, m, a.dim, a.vec != 0,
                                               reinterpret_cast<float*>(buf), L, 0, 1 << 30,
                                               static_cast<NoAbandon<I32B>*>(nullptr), stage, a.rmax);
        if (L == 0) write_result<I32B>(a.out_dist, a.out_dist2, k, r);
        continue;
      }
    }
    const T r = warp_dfd_any<V, DK>(pts + oa * a.dim, n, pts + ob * a.dim, m, a.dim, a.vec != 0, buf, L, 0, 1 << 30,
                                    static_cast<NoAbandon<V>*>(nullptr), stage, a.rmax);
    if (L == 0) write_result<V>(a.out_dist, a.out_dist2, k, r);
  }

  // 3. the last CTA: team pairs wider than one CTA's buffers
  if (n_team == 0) return;   // uniform: nothing was deferred
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    cta_word = atomicAdd(a.done_ctas, 1u) == gridDim.x - 1 ? 1 : 0;
  }
  __syncthreads();
  if (cta_word == 0) return;
  __threadfence();
  const unsigned nd = *static_cast<volatile unsigned*>(a.n_deferred);
  const long long pool = (long long)gridDim.x * kTeamWarps * a.buf_cols;
  for (unsigned d = 0; d < nd; ++d) {
    const unsigned we = static_cast<volatile unsigned*>(a.deferred)[d];
    if (!run_team_pair<V, DK>(a, we, a.rowbuf, pool, stage, team_ring, team_prog, team_cons) && threadIdx.x == 0) {
      write_unsupported<V>(a.out_dist, a.out_dist2, we & (kNarrowBit - 1));
      raise_error(a.err, DFD_ERR_UNSUPPORTED);
    }
  }
}

// ----------------------------------------------------------- decider kernel
// Threshold decision per pair: within[k] = (delta^2 <= eps2_k), with early
// abandon once a cut of the recurrence exceeds eps2_k.  dist2[k] is the
// exact delta^2 of pairs computed to the end and +inf (float) / INT64_MAX
// (int32) for abandoned ones.
struct DecideArgs {
  BatchArgs b;
  const void* eps2;        // per pair (float / int64), or null: eps2_f / eps2_i for all
  float eps2_f;
  long long eps2_i;
  int* within;             // [n_pairs] 1 / 0 (may be null)
  unsigned long long* abandoned;   // pairs abandoned (may be null)
};

// The limit in the value domain of the uint32-bits class.
__device__ __forceinline__ float bits_limit(long long e) {
  if (e < 0) return __int_as_float(0xff800000);
  if (e >= 0x7f800000LL) return __int_as_float(0x7f800000);
  return __uint_as_float((unsigned)e);
}

template <class V, int DK>
__global__ void __launch_bounds__(256, kBlocksPerSM<DK>::value) decide_kernel(DecideArgs d) {
  using T = typename V::value;
  using Cd = typename V::coord;
  __shared__ uint4 stage_sm[8][QStage<DK>::RECS];
  uint4* stage = stage_sm[threadIdx.x >> 5];
  const BatchArgs& a = d.b;
  const int L = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  T* buf = static_cast<T*>(a.rowbuf) + gw * BUF_COLS;
  const Cd* pts = static_cast<const Cd*>(a.points);
  const int64_t total = a.offsets[a.n_curves];
  if (ld_relaxed_i32(a.err) != 0) return;
  for (bool first = true;; first = false) {
    int item = 0;
    if (L == 0) item = first ? pop_first(a.counter, a.sm_rank, a.n_sm, a.n_items) : atomicAdd(a.counter, 1);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= a.n_items) break;
    const unsigned w = a.worklist[item];
    const int64_t k = w & (kNarrowBit - 1);
    int32_t ia = a.pairs[2 * k], ib = a.pairs[2 * k + 1];
    if (w >> 31) {
      const int32_t t = ia;
      ia = ib;
      ib = t;
    }
    if (ia < 0 || ib < 0 || ia >= a.n_curves || ib >= a.n_curves) continue;
    const int64_t oa = a.offsets[ia], ob = a.offsets[ib];
    const int64_t ea = a.offsets[ia + 1], eb = a.offsets[ib + 1];
    if (oa < 0 || ob < 0 || ea > total || eb > total) continue;
    const int n = (int)(ea - oa), m = (int)(eb - ob);
    if (n < 1 || m < 1) continue;
    if (!fits_buffer<DK>(n, m)) {
      // no decision: not within, delta^2 NaN / -1, and the error word says so
      if (L == 0) {
        raise_error(a.err, DFD_ERR_UNSUPPORTED);
        if (d.within) d.within[k] = 0;
        write_unsupported<V>(nullptr, a.out_dist2, k);
      }
      continue;
    }
    bool hit = false, within = false;
    long long exact = 0;
    float exact_f = 0.f;
    if constexpr (std::is_same<V, F32>::value) {
      AbandonAbove<F32> ab;
      ab.fixed = d.eps2 ? static_cast<const float*>(d.eps2)[k] : d.eps2_f;
      ab.live_bits = nullptr;
      const float r = warp_dfd_any<F32, DK, AbandonAbove<F32>>(pts + oa * a.dim, n, pts + ob * a.dim, m, a.dim,
                                                               a.vec != 0, buf, L, 0, 1 << 30, &ab, stage);
      hit = ab.hit;
      exact_f = r;
      within = !hit && r <= ab.fixed;
    } else {
      const long long e = d.eps2 ? static_cast<const long long*>(d.eps2)[k] : d.eps2_i;
      if (w & kNarrowBit) {
        AbandonAbove<I32B> ab;
        ab.fixed = bits_limit(e);
        ab.live_bits = nullptr;
        const float r = warp_dfd_any<I32B, DK, AbandonAbove<I32B>>(pts + oa * a.dim, n, pts + ob * a.dim, m, a.dim,
                                                                   a.vec != 0, reinterpret_cast<float*>(buf), L, 0,
                                                                   1 << 30, &ab, stage);
        hit = ab.hit;
        exact = (long long)__float_as_uint(r);
      } else {
        AbandonAbove<I32> ab;
        ab.fixed = e;
        ab.live_bits = nullptr;
        exact = warp_dfd_any<I32, DK, AbandonAbove<I32>>(pts + oa * a.dim, n, pts + ob * a.dim, m, a.dim,
                                                         a.vec != 0, buf, L, 0, 1 << 30, &ab, stage);
        hit = ab.hit;
      }
      within = !hit && exact <= e;
    }
    if (L == 0) {
      if (d.within) d.within[k] = within ? 1 : 0;
      if (a.out_dist2) {
        if constexpr (std::is_same<V, F32>::value)
          static_cast<float*>(a.out_dist2)[k] = hit ? __int_as_float(0x7f800000) : exact_f;
        else
          static_cast<long long*>(a.out_dist2)[k] = hit ? LLONG_MAX : exact;
      }
      if (hit && d.abandoned) atomicAdd(d.abandoned, 1ull);
    }
  }
}

// ----------------------------------------------------------- matrix kernel
// Condensed upper triangle: k = i*(2N - i - 1)/2 + (j - i - 1), i < j.
__device__ __forceinline__ void decode_pair(int64_t k, int64_t N, int64_t* pi, int64_t* pj) {
  const double b = 2.0 * (double)N - 1.0;
  int64_t i = (int64_t)floor((b - sqrt(b * b - 8.0 * (double)k)) / 2.0);
  // fix the floating-point estimate with exact integer checks
  auto start = [N](int64_t r) { return r * (2 * N - r - 1) / 2; };
  if (i < 0) i = 0;
  if (i > N - 2) i = N - 2;
  while (i > 0 && start(i) > k) --i;
  while (i + 1 <= N - 2 && start(i + 1) <= k) ++i;
  *pi = i;
  *pj = k - start(i) + i + 1;
}

struct MatrixArgs {
  void* rowbuf;        // per-warp BUF_COLS values (multi-stripe pairs)
  const void* points;
  const int64_t* offsets;
  int64_t n_curves;
  int64_t n_pairs;
  int dim;
  int vec;             // 1: vector point loads allowed (dim == DK, 16-byte aligned points)
  int chunk;        // pairs per pop
  int rmax;         // rows per lane cap (<= Rmax; the tuned shape); a pair it would leave wider than the
                    // row buffer runs with Rmax
  const int* bbox;  // int32 matrices: per curve and coordinate (min, max); else null
  int* counter;
  int* err;
  void* out_dist;
  void* out_dist2;
};

template <class V, int DK>
__global__ void __launch_bounds__(256, kBlocksPerSM<DK>::value) matrix_kernel(MatrixArgs a) {
  using T = typename V::value;
  using Cd = typename V::coord;
  __shared__ uint4 stage_sm[8][QStage<DK>::RECS];
  uint4* stage = stage_sm[threadIdx.x >> 5];
  const int L = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  T* buf = static_cast<T*>(a.rowbuf) + gw * BUF_COLS;
  const Cd* pts = static_cast<const Cd*>(a.points);
  const int64_t total = a.offsets[a.n_curves];
  if (ld_relaxed_i32(a.err) != 0) return;
  for (;;) {
    long long base = 0;
    if (L == 0) base = (long long)atomicAdd(a.counter, 1) * a.chunk;
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= a.n_pairs) break;
    const int64_t end = min((int64_t)base + a.chunk, a.n_pairs);
    int64_t i, j;
    decode_pair(base, a.n_curves, &i, &j);
    for (int64_t k = base; k < end; ++k) {
      const int64_t oi = a.offsets[i], oj = a.offsets[j], ei = a.offsets[i + 1], ej = a.offsets[j + 1];
      const bool ok = oi >= 0 && oj >= 0 && ei <= total && ej <= total && ei - oi <= INT32_MAX &&
                      ej - oj <= INT32_MAX;
      const int ni = ok ? (int)(ei - oi) : 0, nj = ok ? (int)(ej - oj) : 0;
      // the cheaper orientation, unless only the other one fits the row buffer
      bool sw = rows_from_b(ni, nj, DK);
      if (!fits_buffer<DK>(sw ? nj : ni, sw ? ni : nj) && fits_buffer<DK>(sw ? ni : nj, sw ? nj : ni)) sw = !sw;
      const int rows = sw ? nj : ni, cols = sw ? ni : nj;
      if (rows < 1 || cols < 1) {
        if (L == 0) raise_error(a.err, DFD_ERR_INVALID_ARG);
      } else if (fits_buffer<DK>(rows, cols)) {
        const int rm = fits_buffer<DK>(rows, cols, BUF_COLS, a.rmax) ? a.rmax : Rmax<DK>::value;
        const int64_t ia = sw ? j : i, ib = sw ? i : j;
        const int64_t oa = sw ? oj : oi, ob = sw ? oi : oj;
        bool narrow = false;
        if constexpr (std::is_same<V, I32>::value) narrow = a.bbox && narrow_pair(a.bbox, DK, ia, ib);
        if (narrow) {
          if constexpr (std::is_same<V, I32>::value) {
            const float r = warp_dfd_any<I32B, DK>(pts + oa * a.dim, rows, pts + ob * a.dim, cols, a.dim,
                                                   a.vec != 0, reinterpret_cast<float*>(buf), L, 0, 1 << 30,
                                                   static_cast<NoAbandon<I32B>*>(nullptr), stage, rm);
            if (L == 0) write_result<I32B>(a.out_dist, a.out_dist2, k, r);
          }
        } else {
          const T r = warp_dfd_any<V, DK>(pts + oa * a.dim, rows, pts + ob * a.dim, cols, a.dim, a.vec != 0, buf, L,
                                          0, 1 << 30, static_cast<NoAbandon<V>*>(nullptr), stage, rm);
          if (L == 0) write_result<V>(a.out_dist, a.out_dist2, k, r);
        }
      } else if (L == 0) {
        raise_error(a.err, DFD_ERR_UNSUPPORTED);
        write_unsupported<V>(a.out_dist, a.out_dist2, k);
      }
      if (++j == a.n_curves) {
        ++i;
        j = i + 1;
      }
    }
  }
}

}  // namespace batch
}  // namespace dfd
