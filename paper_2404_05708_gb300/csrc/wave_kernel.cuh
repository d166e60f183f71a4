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

namespace dfd {
namespace wave {

constexpr int G = 32;        // systolic steps between synchronisations
constexpr int RING = 256;    // columns held by each inter-warp ring (power of 2)
constexpr int NQ = 16;       // q chunk slots (power of 2)

template <int DK>
struct ChunkCols {
  static constexpr int value = DK <= 4 ? 128 : 64;  // q columns per TMA chunk
};

// With every ring saturated, warp w+1 trails warp w by two G-blocks, so the
// last of W warps trails warp 0 by 2*G*(W-1) columns plus its 31-lane skew.
// The q ring must hold that window, or warp 0 could wait for a slot that
// only the last warp can free:  (NQ - 1) * C >= 2*G*(W-1) + 31.
__host__ __device__ constexpr int max_warps(int C) {
  return ((NQ - 1) * C - 31) / (2 * G) + 1;
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

  __device__ __forceinline__ void load(const float* P, int64_t r0, int64_t rlast, int dim) {
#pragma unroll
    for (int h = 0; h < R / 2; ++h) {
      const int64_t i0 = min(r0 + 2 * h, rlast), i1 = min(r0 + 2 * h + 1, rlast);
#pragma unroll
      for (int k = 0; k < DK; ++k) {
        const float a = k < dim ? P[i0 * dim + k] : 0.f;
        const float b = k < dim ? P[i1 * dim + k] : 0.f;
        pp[h][k] = pack2(a, b);
      }
    }
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

  __device__ __forceinline__ void load(const int32_t* P, int64_t r0, int64_t rlast, int dim) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int64_t i = min(r0 + r, rlast);
#pragma unroll
      for (int k = 0; k < DK; ++k) pr[r][k] = k < dim ? P[i * dim + k] : 0;
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

// --------------------------------------------------- shared-memory counters
__device__ __forceinline__ int ld_acquire_cta(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared::cta.s32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
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

template <class V, int DK, int R>
struct Layout {
  using Rows_ = Rows<V, DK, R>;
  using Rec = typename Rows_::Rec;
  using T = typename V::value;
  static constexpr int C = ChunkCols<DK>::value;
  static constexpr int NPL = Rows_::NPL;
  static constexpr size_t q_bytes = (size_t)NQ * NPL * C * sizeof(Rec);
  static constexpr size_t bar_off = q_bytes;
  static constexpr size_t ring_off = bar_off + 2 * NQ * sizeof(uint64_t);
  static __host__ __device__ size_t ctl_off(int W) { return ring_off + (size_t)(W + 1) * RING * sizeof(T); }
  static __host__ __device__ size_t bytes(int W) { return ctl_off(W) + sizeof(Ctl); }
};

// ----------------------------------------------------------- compute warp
template <class V, int DK, int R>
__device__ __forceinline__ void compute_stripe(const Args& a, int w, int64_t band, unsigned gbase,
                                               unsigned char* smem) {
  using Lay = Layout<V, DK, R>;
  using T = typename V::value;
  using Rec = typename Lay::Rec;
  constexpr int C = Lay::C;
  constexpr int NPL = Lay::NPL;
  constexpr int LOGC = C == 128 ? 7 : 6;
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
  const int64_t rend = min(rb0 + a.H, a.n);
  rows.load(static_cast<const Coord*>(a.p), rb0 + (int64_t)(w * 32 + L) * R, rend - 1, a.dim);

  T v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = V::inf();
  T bout = V::inf();
  T upp = (band == 0 && w == 0 && L == 0) ? V::zero() : V::inf();
  const int m = (int)a.m;
  int qdone = 0;

  for (int blk = 0; blk < a.nblk; ++blk) {
    const int c0 = blk * G;
    bool ok = true;
    if (L == 0) ok = spin_smem_geq(&ctl->prod[w], min(c0 + G, m), ctl, a.err, a.timeout_ns);
    if (L == 31) ok = spin_smem_geq(&ctl->cons[w + 1], c0 + G - 31 - RING, ctl, a.err, a.timeout_ns);
    if ((c0 & (C - 1)) == 0) {
      const unsigned seq = gbase + (unsigned)(c0 >> LOGC);
      if (!mbar_wait(&full[seq & (NQ - 1)], (seq / NQ) & 1, a.err, a.timeout_ns)) {
        *reinterpret_cast<volatile int*>(&ctl->abort) = 1;
      }
    }
    (void)ok;
    __syncwarp();
    if (ld_volatile_smem(&ctl->abort)) break;

    auto qaddr = [&](int cq) {
      const unsigned slot = (gbase + (unsigned)(cq >> LOGC)) & (NQ - 1);
      return qring + (size_t)slot * NPL * C + (cq & (C - 1));
    };
    if constexpr (sizeof(T) == 4) {
      // Each warp issues in order, so whatever waits on the previous step's
      // chain blocks every later instruction.  Per step only one instruction
      // does (the shuffle of the bottom value): lane 0's 32 ring inputs are
      // loaded into registers at block start (broadcast), the next step's q
      // point and distances are computed ahead of this step's chain, and
      // lane 31's output is a predicated store that nothing waits on.
      T rv[G];
#pragma unroll
      for (int k = 0; k < G; k += 4) {
        const float4 t4 = *reinterpret_cast<const float4*>(ring_in + ((c0 + k) & (RING - 1)));
        rv[k] = t4.x;
        rv[k + 1] = t4.y;
        rv[k + 2] = t4.z;
        rv[k + 3] = t4.w;
      }
      T dcur[R];
      rows.dist(qaddr(max(c0 - L, 0)), C, dcur);
#pragma unroll
      for (int s = 0; s < G; ++s) {
        const int col = c0 + s - L;
        T dnext[R];
        if (s + 1 < G) rows.dist(qaddr(max(col + 1, 0)), C, dnext);
        T u = __shfl_up_sync(0xffffffffu, bout, 1);
        u = (L == 0) ? rv[s] : u;
        T up = u, dg = upp;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const T l = v[r];
          const T nv = V::vmax(V::vmin3(l, dg, up), dcur[r]);
          dg = l;
          v[r] = nv;
          up = nv;
        }
        upp = u;
        bout = up;
        st_shared_if(ring_out + (col & (RING - 1)), bout, L == 31 && col >= 0);
        if (s + 1 < G) {
#pragma unroll
          for (int r = 0; r < R; ++r) dcur[r] = dnext[r];
        }
      }
    } else {
    // The block's 32 ring inputs, one per lane (lane s holds column c0 + s);
    // at step s lane 0 takes lane s's value.  Lane 31's outputs are gathered
    // the same way (lane s keeps step s's) and stored after the block, so
    // the unrolled block has no shared-memory store and no branch.
    const T in_blk = ring_in[(c0 + L) & (RING - 1)];
    T out_blk = V::inf();
#pragma unroll
    for (int s = 0; s < G; ++s) {
      const int col = c0 + s - L;
      const T rin = __shfl_sync(0xffffffffu, in_blk, s);
      T u = __shfl_up_sync(0xffffffffu, bout, 1);
      u = (L == 0) ? rin : u;
      T d[R];
      rows.dist(qaddr(max(col, 0)), C, d);
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
      st_shared_if(ring_out + (oc & (RING - 1)), out_blk, oc >= 0);
    }
    }
    __syncwarp();
    if (L == 31) st_release_cta(&ctl->prod[w + 1], c0 + G - 31);
    if (L == 0) st_release_cta(&ctl->cons[w], c0 + G);
    // q chunks no lane of this warp will read again: columns < c0 + G - 31.
    const int consumed = max(0, c0 + G - 31) >> LOGC;
    while (qdone < consumed && qdone < a.nch) {
      if (L == 0) mbar_arrive(&empty[(gbase + (unsigned)qdone) & (NQ - 1)]);
      ++qdone;
    }
  }
  __syncwarp();
  while (qdone < a.nch) {
    if (L == 0) mbar_arrive(&empty[(gbase + (unsigned)qdone) & (NQ - 1)]);
    ++qdone;
  }
}

// ------------------------------------------------------- communication warp
template <class V, int DK, int R>
__device__ __forceinline__ void comm_warp(const Args& a, int64_t band, unsigned gbase, unsigned char* smem) {
  using Lay = Layout<V, DK, R>;
  using T = typename V::value;
  using Rec = typename Lay::Rec;
  constexpr int C = Lay::C;
  constexpr int NPL = Lay::NPL;
  constexpr unsigned CHUNK_BYTES = (unsigned)(NPL * C * sizeof(Rec));
  const int L = threadIdx.x & 31;
  const int W = (int)(blockDim.x >> 5) - 1;
  Rec* qring = reinterpret_cast<Rec*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Lay::bar_off);
  uint64_t* empty = full + NQ;
  T* rings = reinterpret_cast<T*>(smem + Lay::ring_off);
  Ctl* ctl = reinterpret_cast<Ctl*>(smem + Lay::ctl_off(W));
  T* ring0 = rings;
  const T* ringW = rings + (size_t)W * RING;
  const Rec* qpk = static_cast<const Rec*>(a.qpk);
  T* rowbuf = static_cast<T*>(a.rowbuf);

  const int m = (int)a.m;
  const int fill_end = a.nblk * G;
  int issued = 0, filled = 0, drained = 0;
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
          mbar_arrive_expect_tx(&full[slot], CHUNK_BYTES);
          tma_load_1d(qring + (size_t)slot * NPL * C, qpk + (size_t)issued * NPL * C, CHUNK_BYTES, &full[slot]);
        }
        ++issued;
        progressed = true;
      }
    }
    // (2) top ring of the band, 32 columns at a time
    if (filled < fill_end && ld_acquire_cta(&ctl->cons[0]) >= filled + 32 - RING) {
      bool avail = true;
      const int need = min(filled + 32, m);
      if (band > 0 && need > 0) {
        unsigned long long pv = 0;
        if (L == 0) pv = ld_acquire_u64(&a.progress[band - 1]);
        pv = __shfl_sync(0xffffffffu, pv, 0);
        __syncwarp();
        avail = pv >= (unsigned long long)need;
      }
      if (avail) {
        const int col = filled + L;
        T val = V::inf();
        if (band > 0 && col < m) val = ld_cg(rowbuf + col);
        ring0[col & (RING - 1)] = val;
        __syncwarp();
        if (L == 0) st_release_cta(&ctl->prod[0], filled + 32);
        filled += 32;
        progressed = true;
      }
    }
    // (3) drain the bottom ring to the global row buffer and publish it
    if (drained < m) {
      const int need = min(drained + 32, m);
      if (ld_acquire_cta(&ctl->prod[W]) >= need) {
        const int col = drained + L;
        if (col < m) {
          const T val = ringW[col & (RING - 1)];
          st_cg(rowbuf + col, val);
          if (band == a.nbands - 1 && col == m - 1) {
            if constexpr (sizeof(T) == 4) {
              if (a.out_dist2) static_cast<float*>(a.out_dist2)[0] = (float)val;
              if (a.out_dist) static_cast<float*>(a.out_dist)[0] = sqrtf((float)val);
            } else {
              if (a.out_dist2) static_cast<long long*>(a.out_dist2)[0] = (long long)val;
              if (a.out_dist) static_cast<double*>(a.out_dist)[0] = sqrt((double)val);
            }
          }
        }
        __syncwarp();
        if (L == 0) {
          st_release_cta(&ctl->cons[W], drained + 32);
          // The release orders the warp's row-buffer stores (made visible to
          // lane 0 by __syncwarp) before the progress word at GPU scope.
          st_release_u64(&a.progress[band], (unsigned long long)need);
        }
        drained += 32;
        if (drained > m) drained = m;
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

// ------------------------------------------------------------------ kernel
template <class V, int DK, int R>
__global__ void __launch_bounds__(17 * 32, 1) wave_kernel(Args a) {
  using Lay = Layout<V, DK, R>;
  using T = typename V::value;
  extern __shared__ __align__(128) unsigned char smem[];
  const int W = (int)(blockDim.x >> 5) - 1;
  const int warp = threadIdx.x >> 5;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Lay::bar_off);
  uint64_t* empty = full + NQ;
  T* rings = reinterpret_cast<T*>(smem + Lay::ring_off);
  Ctl* ctl = reinterpret_cast<Ctl*>(smem + Lay::ctl_off(W));

  // zero the q ring once (never-read slots stay finite), rings to +inf
  {
    uint4* q4 = reinterpret_cast<uint4*>(smem);
    for (size_t i = threadIdx.x; i < Lay::q_bytes / 16; i += blockDim.x) q4[i] = make_uint4(0, 0, 0, 0);
    for (size_t i = threadIdx.x; i < (size_t)(W + 1) * RING; i += blockDim.x) rings[i] = V::inf();
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < NQ; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], (unsigned)W);
    }
    fence_mbar_init();
    ctl->abort = 0;
  }
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
    const int64_t band = ctl->band;
    if (band >= a.nbands) break;
    if (warp == W)
      comm_warp<V, DK, R>(a, band, gbase, smem);
    else
      compute_stripe<V, DK, R>(a, warp, band, gbase, smem);
    gbase += (unsigned)a.nch;
    __syncthreads();
    if (ctl->abort) break;
  }
}

// --------------------------------------------------------- q packing kernel
// Writes the per-band q stream: nch chunks of C columns, NPL 16-byte planes
// per column, columns past m repeat q_{m-1} (a repeated point does not change
// the distance, Sec. 4 footnote; they are never read into the result).
template <class V, int DK>
__global__ void pack_q_kernel(const typename V::coord* q, int64_t m, int dim, int nch, void* out) {
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
    const int64_t j = min(chunk * C + jj, m - 1);
    const typename V::coord* qj = q + j * dim;
    Rec r;
    if constexpr (std::is_same<V, F32>::value) {
      const int k0 = 2 * plane, k1 = 2 * plane + 1;
      const float x0 = k0 < dim ? qj[k0] : 0.f;
      const float x1 = k1 < dim ? qj[k1] : 0.f;
      r = make_float4(x0, x0, x1, x1);
    } else {
      const int k = 4 * plane;
      r.x = k < dim ? qj[k] : 0;
      r.y = k + 1 < dim ? qj[k + 1] : 0;
      r.z = k + 2 < dim ? qj[k + 2] : 0;
      r.w = k + 3 < dim ? qj[k + 3] : 0;
    }
    o[idx] = r;
  }
}

}  // namespace wave
}  // namespace dfd
