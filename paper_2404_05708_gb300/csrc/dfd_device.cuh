// dfd_device.cuh -- device primitives for the discrete Frechet distance kernels.
//
// Value traits (float32 or int32 coordinates), the squared ground distance,
// clamp functions and their composition (the exact associative form of the
// paper's non-associative maxmin scan, Sec. 4), the warp clamp-scan, bounded
// spin waits, and 1-D TMA bulk copies with mbarriers.
#pragma once
#include <cstdint>
#include <climits>
#include <type_traits>
#include <cuda_runtime.h>

#include "dfd_status.h"

namespace dfd {

// ------------------------------------------------------------------ traits
// F32: coordinates float, DP values float (squared distances), +inf sentinel.
// I32: coordinates int32, DP values int64 (exact squared distances).
struct F32 {
  using coord = float;
  using value = float;
  __device__ __forceinline__ static value inf() { return __int_as_float(0x7f800000); }
  __device__ __forceinline__ static value ninf() { return __int_as_float(0xff800000); }
  __device__ __forceinline__ static value zero() { return 0.0f; }
  __device__ __forceinline__ static value vmin(value a, value b) { return fminf(a, b); }
  __device__ __forceinline__ static value vmax(value a, value b) { return fmaxf(a, b); }
  __device__ __forceinline__ static value vmin3(value a, value b, value c) {
    value r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
  }
};

struct I32 {
  using coord = int32_t;
  using value = long long;
  __device__ __forceinline__ static value inf() { return LLONG_MAX; }
  __device__ __forceinline__ static value ninf() { return LLONG_MIN; }
  __device__ __forceinline__ static value zero() { return 0; }
  __device__ __forceinline__ static value vmin(value a, value b) { return a < b ? a : b; }
  __device__ __forceinline__ static value vmax(value a, value b) { return a > b ? a : b; }
  __device__ __forceinline__ static value vmin3(value a, value b, value c) { return vmin(vmin(a, b), c); }
};

// I32B: int32 coordinates whose squared distances are known (from the
// pair's bounding boxes) to stay below 0x7F800000.  The squared distance is
// computed exactly in uint32 and carried as the float with those bits: for
// such non-negative patterns the float order is the integer order, so the
// recurrence (pure selection) runs on float min/max (full rate, 3-input
// min) and returns the exact int64 value's bit pattern.  +inf (0x7F800000)
// is above every value.
struct I32B {
  using coord = int32_t;
  using value = float;
  __device__ __forceinline__ static value inf() { return __int_as_float(0x7f800000); }
  __device__ __forceinline__ static value ninf() { return __int_as_float(0xff800000); }
  __device__ __forceinline__ static value zero() { return 0.0f; }
  __device__ __forceinline__ static value vmin(value a, value b) { return fminf(a, b); }
  __device__ __forceinline__ static value vmax(value a, value b) { return fmaxf(a, b); }
  __device__ __forceinline__ static value vmin3(value a, value b, value c) {
    value r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
  }
};

// Largest bounding-box range per coordinate (and sum of squared ranges) for
// which a pair may use I32B: every |p_k - q_k| <= 46340 keeps each square in
// int32 and the sum below the first NaN pattern.
constexpr unsigned kI32BMaxRange = 46340u;
constexpr unsigned long long kI32BMaxD2 = 0x7f7fffffull;

// ---------------------------------------------------------- ground distance
// Squared Euclidean distance.  float32: t_k = p_k - q_k rounded, then
// acc = t_0*t_0, acc = fma(t_k, t_k, acc) for k = 1..D-1, each op rounded to
// nearest (explicit intrinsics, so no contraction choice is left to the
// compiler).  int32: exact, t_k in int32 (the coordinate range precondition
// keeps |p_k - q_k| < 2^31), products and sum in int64.
template <int D>
__device__ __forceinline__ float dist2(const float* p, const float* q) {
  float t = __fsub_rn(p[0], q[0]);
  float acc = __fmul_rn(t, t);
#pragma unroll
  for (int k = 1; k < D; ++k) {
    float u = __fsub_rn(p[k], q[k]);
    acc = __fmaf_rn(u, u, acc);
  }
  return acc;
}

template <int D>
__device__ __forceinline__ long long dist2(const int32_t* p, const int32_t* q) {
  int t = p[0] - q[0];
  long long acc = (long long)t * (long long)t;
#pragma unroll
  for (int k = 1; k < D; ++k) {
    int u = p[k] - q[k];
    acc += (long long)u * (long long)u;
  }
  return acc;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the kernel before it in the stream runs, as
// soon as every CTA of that kernel has called launch_dependents (or exited);
// griddep_wait then blocks until that kernel has completed and its memory
// operations are visible.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void griddep_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Squared distance in the value type of V (F32: float, I32: exact int64,
// I32B: exact uint32 bits as a float).
template <class V, int D>
__device__ __forceinline__ typename V::value vdist2(const typename V::coord* p, const typename V::coord* q) {
  if constexpr (std::is_same<V, I32B>::value) {
    unsigned acc = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const unsigned t = (unsigned)(p[k] - q[k]);
      acc += t * t;   // |p_k - q_k| <= 46340: each square < 2^31, the sum < 0x7F800000
    }
    return __uint_as_float(acc);
  } else {
    return dist2<D>(p, q);
  }
}

// Packed float32x2 arithmetic (two independent lanes in one 64-bit register),
// per-element IEEE round-to-nearest: bit-identical to the scalar ops above.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float lo2(unsigned long long v) { return __uint_as_float((unsigned)(v & 0xffffffffu)); }
__device__ __forceinline__ float hi2(unsigned long long v) { return __uint_as_float((unsigned)(v >> 32)); }
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// ------------------------------------------------------------ clamp algebra
// One cell of a row of Eq. 1, once the row above is known, is the clamp
// function f(x) = max(d, min(a, x)) of its left neighbour x, with
// a = min(up, diag) and d the ground distance.  Clamp functions are closed
// under composition:  (a2,d2) o (a1,d1) = (min(a1,a2), max(d2, min(a2,d1))),
// and composition is associative, so a row can be scanned in parallel with
// only min and max (no rounding).  Identity: (+inf, -inf).
template <class V>
struct Clamp {
  typename V::value a, d;
};

template <class V>
__device__ __forceinline__ Clamp<V> clamp_identity() {
  return Clamp<V>{V::inf(), V::ninf()};
}

// later o earlier (apply `earlier` first)
template <class V>
__device__ __forceinline__ Clamp<V> compose(Clamp<V> later, Clamp<V> earlier) {
  Clamp<V> r;
  r.a = V::vmin(earlier.a, later.a);
  r.d = V::vmax(later.d, V::vmin(later.a, earlier.d));
  return r;
}

template <class V>
__device__ __forceinline__ typename V::value apply(Clamp<V> f, typename V::value x) {
  return V::vmax(f.d, V::vmin(f.a, x));
}

template <class T>
__device__ __forceinline__ T shfl_up_any(T v, int delta) {
  return __shfl_up_sync(0xffffffffu, v, delta);
}

// Inclusive warp scan of clamp functions over lanes (lane 0 first).
template <class V>
__device__ __forceinline__ Clamp<V> warp_clamp_scan_inclusive(Clamp<V> f, int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    Clamp<V> g;
    g.a = shfl_up_any(f.a, off);
    g.d = shfl_up_any(f.d, off);
    if (lane >= off) f = compose<V>(f, g);
  }
  return f;
}

// ---------------------------------------------------------- bounded waits
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void raise_error(int* err, int code) {
  atomicCAS(err, 0, code);
}

// Spin until *flag >= need, the context error word becomes nonzero, or
// timeout_ns elapses.  Returns true when the value was reached; on timeout
// it records DFD_ERR_TIMEOUT in *err.  Never traps.
__device__ __forceinline__ bool wait_geq(const unsigned long long* flag, unsigned long long need, int* err,
                                         unsigned long long timeout_ns) {
  if (ld_acquire_u64(flag) >= need) return true;
  const unsigned long long t0 = globaltimer_ns();
  unsigned ns = 32;
  for (;;) {
    if (ld_acquire_u64(flag) >= need) return true;
    if (ld_relaxed_i32(err) != 0) return false;
    if (globaltimer_ns() - t0 > timeout_ns) {
      raise_error(err, DFD_ERR_TIMEOUT);
      return false;
    }
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
  }
}

// ------------------------------------------------- mbarrier + 1-D TMA bulk
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred P;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, P;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking test of an mbarrier phase (never suspends the thread).  A
// polling loop must use this rather than try_wait: a try_wait that
// suspends was measured to stall the other warps of the SM by ~12,000
// cycles at a time.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred P;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, P;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for an mbarrier phase; records DFD_ERR_TIMEOUT on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err, unsigned long long timeout_ns) {
  if (mbar_test_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    if (mbar_test_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > timeout_ns) {
      raise_error(err, DFD_ERR_TIMEOUT);
      return false;
    }
  }
}

// Untiled bulk copy global -> shared; src, dst 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void tma_load_1d(void* dst_smem, const void* src_gmem, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

}  // namespace dfd
