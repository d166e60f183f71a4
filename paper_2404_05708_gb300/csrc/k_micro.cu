// k_micro.cu -- measurement kernels for the ALU roofline.
//
// The recurrence has no dense contraction and reads almost nothing from HBM
// per cell, so its ceiling is the issue / pipe rate of the instructions one
// cell needs.  These kernels measure, on the running GPU:
//   * throughput of each instruction kind (thread-instructions per clock per
//     SM, many independent chains, one full wave of resident blocks);
//   * throughput of the exact instruction mix of one DP cell without the
//     DP's serial dependence (the cell-rate roofline reported beside the
//     kernels' achieved rate), and of the distance alone summed instead of
//     running Eq. 1 (the paper's "sum of all d_ij" ceiling, Sec. 4);
//   * latency of the dependent chains the systolic step waits on (clocks per
//     dependent operation, one warp per SM).
#include <cstdint>
#include "dfd_device.cuh"
#include "dfd_internal.h"

namespace dfd {
namespace {

constexpr int MB_THREADS = 256;
constexpr int MB_ITERS = 16384;

enum MicroOp {
  MB_FFMA = 0,      // fma.rn.f32
  MB_FFMA2 = 1,     // fma.rn.f32x2
  MB_FMNMX = 2,     // min.f32
  MB_FMNMX3 = 3,    // min.f32 with three inputs
  MB_IMNMX = 4,     // min.s32
  MB_IMNMX64 = 5,   // min.s64
  MB_IMADWIDE = 6,  // mad.wide.s32
  MB_SHFL = 7,      // shfl.sync.up.b32
  MB_MIX_F32D3 = 8, // one float32 3-D cell: 3 f32x2 (per 2 cells x 2) + min3 + max
  MB_MIX_I32D2 = 9, // one int32 2-D cell: 2 sub, mul.wide, mad.wide, 3 x min/max.s64
  MB_DISTONLY_F32D3 = 10,  // sum of float32 3-D squared distances (no recurrence)
  MB_LAT_FMNMX = 11,       // latency: dependent min.f32 chain (clocks per op)
  MB_LAT_CELL = 12,        // latency: dependent min3 -> max (one cell of the chain)
  MB_LAT_SHFL = 13,        // latency: dependent shfl.up chain
  MB_LAT_FFMA2 = 14,       // latency: dependent fma.f32x2 chain
  MB_LAT_MNMX64 = 15,      // latency: dependent min.s64 -> max.s64 (int cell chain)
  MB_MIX_F32D16 = 16,      // one float32 16-D cell: 16 sub + 16 fma/mul + min3 + max (scalar)
  MB_MIX_I32B_D2 = 17,     // one int32 2-D cell in uint32 bits: 2 sub, mul.lo, mad.lo, min3.f32 + max.f32
  MB_MIX_DTW_F32D2 = 18,   // one float32 2-D DTW cell: sub, mul, sub, fma, min3.f32, add
  MB_MIX_LEV_I32 = 19,     // one Levenshtein cell: compare + select, min, add, add, min, column mask select
  MB_MIX_F32D2 = 20,       // one float32 2-D cell: 2 f32x2 (per 2 cells: 2 sub, mul, fma) + min3 + max
  MB_COUNT = 21
};

__host__ __device__ constexpr bool is_latency(int op) { return op >= MB_LAT_FMNMX && op <= MB_LAT_MNMX64; }

// operations (thread-instructions, cells, or dependent ops) per iteration
__host__ __device__ constexpr int ops_per_iter(int op) {
  return op == MB_MIX_F32D3 || op == MB_MIX_F32D2 ? 16
         : op == MB_MIX_I32D2 ? 8 : op == MB_DISTONLY_F32D3 ? 16 : op == MB_MIX_F32D16 ? 2 : 8;
}

template <int OP>
__global__ void __launch_bounds__(MB_THREADS) micro_kernel(float seed, unsigned long long* stamps, float* sink) {
  float f[8];
  unsigned long long u[8];
  int iv[8];
  long long lv[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    f[k] = seed * (k + 1) + threadIdx.x;
    u[k] = pack2(f[k], f[k] + 1.f);
    iv[k] = (int)f[k];
    lv[k] = (long long)iv[k] << 20;
  }
  const float c1 = seed + 0.5f, c2 = seed - 0.25f;
  const unsigned long long cu = pack2(c1, c2);
  __syncthreads();
  const unsigned long long t0 = clock64();
  const unsigned long long g0 = globaltimer_ns();
#pragma unroll 1
  for (int it = 0; it < MB_ITERS; ++it) {
    if constexpr (OP == MB_LAT_FMNMX) {
#pragma unroll
      for (int k = 0; k < 8; ++k) asm volatile("min.f32 %0, %0, %1;" : "+f"(f[0]) : "f"(f[k & 3 ? 1 : 2]));
    } else if constexpr (OP == MB_LAT_CELL) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        asm volatile("min.f32 %0, %1, %2, %0;" : "+f"(f[0]) : "f"(f[1]), "f"(f[2]));
        asm volatile("max.f32 %0, %0, %1;" : "+f"(f[0]) : "f"(f[3]));
      }
    } else if constexpr (OP == MB_LAT_SHFL) {
#pragma unroll
      for (int k = 0; k < 8; ++k) asm volatile("shfl.sync.up.b32 %0, %0, 1, 0, 0xffffffff;" : "+r"(iv[0]));
    } else if constexpr (OP == MB_LAT_FFMA2) {
#pragma unroll
      for (int k = 0; k < 8; ++k) asm volatile("fma.rn.f32x2 %0, %0, %1, %1;" : "+l"(u[0]) : "l"(cu));
    } else if constexpr (OP == MB_MIX_F32D16) {
      // two independent 16-D cells per iteration (coordinates loop-carried,
      // 16 distinct subtrahends so no subtraction can be merged)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        float acc, t;
        asm volatile("sub.rn.f32 %0, %1, %2;" : "=f"(t) : "f"(f[c]), "f"(c1));
        asm volatile("mul.rn.f32 %0, %1, %1;" : "=f"(acc) : "f"(t));
#pragma unroll
        for (int k = 1; k < 16; ++k) {
          asm volatile("sub.rn.f32 %0, %1, %2;" : "=f"(t) : "f"(f[c]), "f"(c2 + (float)k));
          asm volatile("fma.rn.f32 %0, %1, %1, %0;" : "+f"(acc) : "f"(t));
        }
        asm volatile("min.f32 %0, %0, %1, %2;" : "+f"(f[c + 4]) : "f"(c1), "f"(c2));
        asm volatile("max.f32 %0, %0, %1;" : "+f"(f[c + 4]) : "f"(acc));
        f[c] = acc;
      }
    } else if constexpr (OP == MB_LAT_MNMX64) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        asm volatile("min.s64 %0, %0, %1;" : "+l"(lv[0]) : "l"(lv[1]));
        asm volatile("max.s64 %0, %0, %1;" : "+l"(lv[0]) : "l"(lv[2]));
      }
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if constexpr (OP == MB_FFMA) {
          asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[k]) : "f"(c1), "f"(c2));
        } else if constexpr (OP == MB_FFMA2) {
          asm volatile("fma.rn.f32x2 %0, %0, %1, %1;" : "+l"(u[k]) : "l"(cu));
        } else if constexpr (OP == MB_FMNMX) {
          asm volatile("min.f32 %0, %0, %1;" : "+f"(f[k]) : "f"(c1));
        } else if constexpr (OP == MB_FMNMX3) {
          asm volatile("min.f32 %0, %0, %1, %2;" : "+f"(f[k]) : "f"(c1), "f"(c2));
        } else if constexpr (OP == MB_IMNMX) {
          asm volatile("min.s32 %0, %0, %1;" : "+r"(iv[k]) : "r"(it));
        } else if constexpr (OP == MB_IMNMX64) {
          asm volatile("min.s64 %0, %0, %1;" : "+l"(lv[k]) : "l"((long long)it));
        } else if constexpr (OP == MB_IMADWIDE) {
          asm volatile("mad.wide.s32 %0, %1, %1, %0;" : "+l"(lv[k]) : "r"(iv[k]));
        } else if constexpr (OP == MB_SHFL) {
          asm volatile("shfl.sync.up.b32 %0, %0, 1, 0, 0xffffffff;" : "+r"(iv[k]));
        } else if constexpr (OP == MB_MIX_F32D3) {
          // two cells (a row pair) per k: 3 sub2 + mul2 + 2 fma2, then min3 + max per cell.
          // The sub2 operands are loop-carried (u[k] is rewritten below), so
          // nothing can be hoisted out of the loop.
          unsigned long long t0_, t1_, t2_, acc;
          asm volatile("sub.rn.f32x2 %0, %1, %2;" : "=l"(t0_) : "l"(u[k]), "l"(cu));
          asm volatile("sub.rn.f32x2 %0, %1, %2;" : "=l"(t1_) : "l"(u[k]), "l"(u[(k + 1) & 7]));
          asm volatile("sub.rn.f32x2 %0, %1, %2;" : "=l"(t2_) : "l"(u[k]), "l"(u[(k + 2) & 7]));
          asm volatile("mul.rn.f32x2 %0, %1, %1;" : "=l"(acc) : "l"(t0_));
          asm volatile("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc) : "l"(t1_));
          asm volatile("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc) : "l"(t2_));
          u[k] = acc;
          const float lo = lo2(acc), hi = hi2(acc);
          asm volatile("min.f32 %0, %0, %1, %2;" : "+f"(f[k]) : "f"(c1), "f"(c2));
          asm volatile("max.f32 %0, %0, %1;" : "+f"(f[k]) : "f"(lo));
          asm volatile("min.f32 %0, %0, %1, %2;" : "+f"(f[(k + 4) & 7]) : "f"(c1), "f"(c2));
          asm volatile("max.f32 %0, %0, %1;" : "+f"(f[(k + 4) & 7]) : "f"(hi));
        } else if constexpr (OP == MB_MIX_F32D2) {
          // two cells (a row pair) per k: 2 sub2 + mul2 + fma2, then min3 + max per cell
          unsigned long long t0_, t1_, acc;
          asm volatile("sub.rn.f32x2 %0, %1, %2;" : "=l"(t0_) : "l"(u[k]), "l"(cu));
          asm volatile("sub.rn.f32x2 %0, %1, %2;" : "=l"(t1_) : "l"(u[k]), "l"(u[(k + 1) & 7]));
          asm volatile("mul.rn.f32x2 %0, %1, %1;" : "=l"(acc) : "l"(t0_));
          asm volatile("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc) : "l"(t1_));
          u[k] = acc;
          const float lo = lo2(acc), hi = hi2(acc);
          asm volatile("min.f32 %0, %0, %1, %2;" : "+f"(f[k]) : "f"(c1), "f"(c2));
          asm volatile("max.f32 %0, %0, %1;" : "+f"(f[k]) : "f"(lo));
          asm volatile("min.f32 %0, %0, %1, %2;" : "+f"(f[(k + 4) & 7]) : "f"(c1), "f"(c2));
          asm volatile("max.f32 %0, %0, %1;" : "+f"(f[(k + 4) & 7]) : "f"(hi));
        } else if constexpr (OP == MB_MIX_DTW_F32D2) {
          // the point coordinates are loop-carried (rewritten below), so no
          // distance can be hoisted out of the loop
          float t, acc;
          asm volatile("sub.rn.f32 %0, %1, %2;" : "=f"(t) : "f"(f[k]), "f"(c1));
          asm volatile("mul.rn.f32 %0, %1, %1;" : "=f"(acc) : "f"(t));
          asm volatile("sub.rn.f32 %0, %1, %2;" : "=f"(t) : "f"(f[(k + 1) & 7]), "f"(c2));
          asm volatile("fma.rn.f32 %0, %1, %1, %0;" : "+f"(acc) : "f"(t));
          float mn;
          asm volatile("min.f32 %0, %1, %2, %3;" : "=f"(mn) : "f"(f[k]), "f"(f[(k + 2) & 7]), "f"(f[(k + 3) & 7]));
          asm volatile("add.rn.f32 %0, %1, %2;" : "=f"(f[k]) : "f"(mn), "f"(acc));
        } else if constexpr (OP == MB_MIX_LEV_I32) {
          int dd, t0, t1;
          asm volatile("{\n\t.reg .pred P;\n\tsetp.ne.s32 P, %1, %2;\n\tselp.s32 %0, 1, 0, P;\n\t}"
                       : "=r"(dd) : "r"(iv[k]), "r"(it));
          asm volatile("min.s32 %0, %1, %2;" : "=r"(t0) : "r"(iv[k]), "r"(iv[(k + 1) & 7]));
          asm volatile("add.s32 %0, %0, 1;" : "+r"(t0));
          asm volatile("add.s32 %0, %1, %2;" : "=r"(t1) : "r"(iv[(k + 2) & 7]), "r"(dd));
          asm volatile("min.s32 %0, %0, %1;" : "+r"(t0) : "r"(t1));
          asm volatile("{\n\t.reg .pred Q;\n\tsetp.lt.s32 Q, %2, 0;\n\tselp.s32 %0, %1, %0, Q;\n\t}"
                       : "+r"(t0) : "r"(iv[k]), "r"(iv[(k + 3) & 7]));
          iv[k] = t0;
        } else if constexpr (OP == MB_MIX_I32B_D2) {
          int dx, dy;
          unsigned d2;
          asm volatile("sub.s32 %0, %1, %2;" : "=r"(dx) : "r"(iv[k]), "r"(it));
          asm volatile("sub.s32 %0, %1, %2;" : "=r"(dy) : "r"(iv[(k + 1) & 7]), "r"(it));
          iv[k] = dy;
          asm volatile("mul.lo.u32 %0, %1, %1;" : "=r"(d2) : "r"(dx));
          asm volatile("mad.lo.u32 %0, %1, %1, %0;" : "+r"(d2) : "r"(dy));
          asm volatile("min.f32 %0, %0, %1, %2;" : "+f"(f[k]) : "f"(f[(k + 1) & 7]), "f"(f[(k + 2) & 7]));
          asm volatile("max.f32 %0, %0, %1;" : "+f"(f[k]) : "f"(__uint_as_float(d2)));
        } else if constexpr (OP == MB_MIX_I32D2) {
          long long d2;
          int dx, dy;
          asm volatile("sub.s32 %0, %1, %2;" : "=r"(dx) : "r"(iv[k]), "r"(it));
          asm volatile("sub.s32 %0, %1, %2;" : "=r"(dy) : "r"(iv[(k + 1) & 7]), "r"(it));
          iv[k] = dy;
          asm volatile("mul.wide.s32 %0, %1, %1;" : "=l"(d2) : "r"(dx));
          asm volatile("mad.wide.s32 %0, %1, %1, %0;" : "+l"(d2) : "r"(dy));
          asm volatile("min.s64 %0, %0, %1;" : "+l"(lv[k]) : "l"(lv[(k + 1) & 7]));
          asm volatile("min.s64 %0, %0, %1;" : "+l"(lv[k]) : "l"(lv[(k + 2) & 7]));
          asm volatile("max.s64 %0, %0, %1;" : "+l"(lv[k]) : "l"(d2));
        } else if constexpr (OP == MB_DISTONLY_F32D3) {
          unsigned long long t0_, t1_, t2_, acc;
          asm volatile("sub.rn.f32x2 %0, %1, %2;" : "=l"(t0_) : "l"(u[k]), "l"(cu));
          asm volatile("sub.rn.f32x2 %0, %1, %2;" : "=l"(t1_) : "l"(u[k]), "l"(u[(k + 1) & 7]));
          asm volatile("sub.rn.f32x2 %0, %1, %2;" : "=l"(t2_) : "l"(u[k]), "l"(u[(k + 2) & 7]));
          asm volatile("mul.rn.f32x2 %0, %1, %1;" : "=l"(acc) : "l"(t0_));
          asm volatile("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc) : "l"(t1_));
          asm volatile("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc) : "l"(t2_));
          asm volatile("add.rn.f32x2 %0, %0, %1;" : "+l"(u[(k + 4) & 7]) : "l"(acc));
        }
      }
    }
  }
  // every warp of the block has finished its loop before the end stamp:
  // warps of one sub-partition are not issued evenly (the first may finish
  // well ahead of the others), so a stamp taken when thread 0 alone is done
  // would undercount the block's cycles and overstate the rate
  __syncthreads();
  const unsigned long long g1 = globaltimer_ns();
  const unsigned long long t1 = clock64();
  if (threadIdx.x == 0) {
    stamps[2 * blockIdx.x] = t1 - t0;
    stamps[2 * blockIdx.x + 1] = g1 - g0;
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += f[k] + lo2(u[k]) + (float)iv[k] + (float)lv[k];
  if (s == 1.2345f) sink[blockIdx.x] = s;
}

template <int OP>
dfd_status run_op(dfd_context* ctx, double* rate, double* mhz) {
  int per_sm = 1, threads = 32;
  if (!is_latency(OP)) {
    threads = MB_THREADS;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, micro_kernel<OP>, threads, 0) != cudaSuccess ||
        per_sm < 1)
      return DFD_ERR_CUDA;
    per_sm = per_sm > 4 ? 4 : per_sm;   // one full wave, every block resident
  }
  const int blocks = ctx->num_sms * per_sm;
  unsigned long long* st = nullptr;
  float* sink = nullptr;
  if (cudaMalloc(&st, 2 * blocks * sizeof(unsigned long long)) != cudaSuccess) return DFD_ERR_OOM;
  if (cudaMalloc(&sink, blocks * sizeof(float)) != cudaSuccess) {
    cudaFree(st);
    return DFD_ERR_OOM;
  }
  micro_kernel<OP><<<blocks, threads, 0, ctx->stream>>>(1.0f, st, sink);  // warm-up
  micro_kernel<OP><<<blocks, threads, 0, ctx->stream>>>(1.0f, st, sink);
  dfd_status s = cuda_status(cudaStreamSynchronize(ctx->stream));
  if (s == DFD_OK) {
    unsigned long long* h = new unsigned long long[2 * blocks];
    cudaMemcpy(h, st, 2 * blocks * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    double cyc = 0, ns = 0;
    for (int b = 0; b < blocks; ++b) {
      cyc += (double)h[2 * b];
      ns += (double)h[2 * b + 1];
    }
    cyc /= blocks;
    ns /= blocks;
    delete[] h;
    const double ops = (double)MB_ITERS * ops_per_iter(OP);
    if (is_latency(OP))
      *rate = cyc / ops;                               // clocks per dependent op
    else
      *rate = (double)per_sm * threads * ops / cyc;    // per clock per SM
    *mhz = ns > 0 ? cyc / ns * 1.0e3 : 0.0;
  }
  cudaFree(st);
  cudaFree(sink);
  return s;
}

}  // namespace
}  // namespace dfd

extern "C" dfd_status dfd_microbench(dfd_context* ctx, int op, double* result, double* sm_mhz) {
  using namespace dfd;
  if (!ctx || !result || !sm_mhz) return DFD_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DFD_ERR_CUDA;
  switch (op) {
    case MB_FFMA: return run_op<MB_FFMA>(ctx, result, sm_mhz);
    case MB_FFMA2: return run_op<MB_FFMA2>(ctx, result, sm_mhz);
    case MB_FMNMX: return run_op<MB_FMNMX>(ctx, result, sm_mhz);
    case MB_FMNMX3: return run_op<MB_FMNMX3>(ctx, result, sm_mhz);
    case MB_IMNMX: return run_op<MB_IMNMX>(ctx, result, sm_mhz);
    case MB_IMNMX64: return run_op<MB_IMNMX64>(ctx, result, sm_mhz);
    case MB_IMADWIDE: return run_op<MB_IMADWIDE>(ctx, result, sm_mhz);
    case MB_SHFL: return run_op<MB_SHFL>(ctx, result, sm_mhz);
    case MB_MIX_F32D3: return run_op<MB_MIX_F32D3>(ctx, result, sm_mhz);
    case MB_MIX_I32D2: return run_op<MB_MIX_I32D2>(ctx, result, sm_mhz);
    case MB_DISTONLY_F32D3: return run_op<MB_DISTONLY_F32D3>(ctx, result, sm_mhz);
    case MB_LAT_FMNMX: return run_op<MB_LAT_FMNMX>(ctx, result, sm_mhz);
    case MB_LAT_CELL: return run_op<MB_LAT_CELL>(ctx, result, sm_mhz);
    case MB_LAT_SHFL: return run_op<MB_LAT_SHFL>(ctx, result, sm_mhz);
    case MB_LAT_FFMA2: return run_op<MB_LAT_FFMA2>(ctx, result, sm_mhz);
    case MB_LAT_MNMX64: return run_op<MB_LAT_MNMX64>(ctx, result, sm_mhz);
    case MB_MIX_F32D16: return run_op<MB_MIX_F32D16>(ctx, result, sm_mhz);
    case MB_MIX_I32B_D2: return run_op<MB_MIX_I32B_D2>(ctx, result, sm_mhz);
    case MB_MIX_DTW_F32D2: return run_op<MB_MIX_DTW_F32D2>(ctx, result, sm_mhz);
    case MB_MIX_LEV_I32: return run_op<MB_MIX_LEV_I32>(ctx, result, sm_mhz);
    case MB_MIX_F32D2: return run_op<MB_MIX_F32D2>(ctx, result, sm_mhz);
    default: return DFD_ERR_INVALID_ARG;
  }
}
