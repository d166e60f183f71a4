// k_micro.cu -- K7/K8: measurement kernels for the ALU roofline.
//
// The recurrence has no dense contraction and reads almost nothing from HBM
// per cell, so its ceiling is the issue / pipe rate of the instructions one
// cell needs.  These kernels measure, on the running GPU, the throughput of
// each instruction kind (thread-instructions per clock per SM, with many
// independent chains so latency is hidden) and of the exact instruction mix
// of one DP cell without the DP's serial dependence.  The mix rate is the
// cell-rate roofline reported next to the kernels' achieved rate.
//
// The Sigma d^2 "distance only" ceiling of the paper (Sec. 4, the baseline
// that sums all d_ij instead of running Eq. 1) is the DISTONLY mix.
#include <cstdint>
#include "dfd_device.cuh"
#include "dfd_internal.h"

namespace dfd {
namespace {

constexpr int MB_THREADS = 256;
constexpr int MB_BLOCKS_PER_SM = 4;
constexpr int MB_ITERS = 2048;

enum MicroOp {
  MB_FFMA = 0,      // fma.rn.f32
  MB_FFMA2 = 1,     // fma.rn.f32x2
  MB_FMNMX = 2,     // min.f32
  MB_FMNMX3 = 3,    // min.f32 with three inputs
  MB_IMNMX = 4,     // min.s32
  MB_IMNMX64 = 5,   // min.s64
  MB_IMADWIDE = 6,  // mad.wide.s32
  MB_SHFL = 7,      // shfl.sync.up.b32
  MB_MIX_F32D3 = 8, // one float32 3-D cell: 3 f32x2 + min3 + max per cell (f32x2 covers two cells)
  MB_MIX_I32D2 = 9, // one int32 2-D cell: 2 sub, mul.wide, mad.wide, 3 x min/max.s64
  MB_DISTONLY_F32D3 = 10, // Sigma d^2: the same distance work, summed (no recurrence)
  MB_COUNT = 11
};

// ops (thread-instructions or cells) per iteration per thread
__host__ __device__ constexpr int ops_per_iter(int op) {
  return op == MB_MIX_F32D3 ? 16 : op == MB_MIX_I32D2 ? 8 : op == MB_DISTONLY_F32D3 ? 16 : 8;
}

template <int OP>
__global__ void __launch_bounds__(MB_THREADS) micro_kernel(float seed, unsigned long long* cycles, float* sink) {
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
#pragma unroll 1
  for (int it = 0; it < MB_ITERS; ++it) {
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
        // two cells (a row pair) per k: 3 sub2 + mul2 + 2 fma2, then min3 + max per cell
        unsigned long long t0_, t1_, t2_, acc;
        asm volatile("sub.rn.f32x2 %0, %1, %2;" : "=l"(t0_) : "l"(u[k]), "l"(cu));
        asm volatile("sub.rn.f32x2 %0, %1, %2;" : "=l"(t1_) : "l"(u[(k + 1) & 7]), "l"(cu));
        asm volatile("sub.rn.f32x2 %0, %1, %2;" : "=l"(t2_) : "l"(u[(k + 2) & 7]), "l"(cu));
        asm volatile("mul.rn.f32x2 %0, %1, %1;" : "=l"(acc) : "l"(t0_));
        asm volatile("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc) : "l"(t1_));
        asm volatile("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc) : "l"(t2_));
        float lo = lo2(acc), hi = hi2(acc);
        asm volatile("min.f32 %0, %0, %1, %2;" : "+f"(f[k]) : "f"(c1), "f"(c2));
        asm volatile("max.f32 %0, %0, %1;" : "+f"(f[k]) : "f"(lo));
        asm volatile("min.f32 %0, %0, %1, %2;" : "+f"(f[(k + 4) & 7]) : "f"(c1), "f"(c2));
        asm volatile("max.f32 %0, %0, %1;" : "+f"(f[(k + 4) & 7]) : "f"(hi));
      } else if constexpr (OP == MB_MIX_I32D2) {
        long long d2;
        int dx, dy;
        asm volatile("sub.s32 %0, %1, %2;" : "=r"(dx) : "r"(iv[k]), "r"(it));
        asm volatile("sub.s32 %0, %1, %2;" : "=r"(dy) : "r"(iv[(k + 1) & 7]), "r"(it));
        asm volatile("mul.wide.s32 %0, %1, %1;" : "=l"(d2) : "r"(dx));
        asm volatile("mad.wide.s32 %0, %1, %1, %0;" : "+l"(d2) : "r"(dy));
        asm volatile("min.s64 %0, %0, %1;" : "+l"(lv[k]) : "l"(lv[(k + 1) & 7]));
        asm volatile("min.s64 %0, %0, %1;" : "+l"(lv[k]) : "l"(lv[(k + 2) & 7]));
        asm volatile("max.s64 %0, %0, %1;" : "+l"(lv[k]) : "l"(d2));
      } else if constexpr (OP == MB_DISTONLY_F32D3) {
        unsigned long long t0_, t1_, t2_, acc;
        asm volatile("sub.rn.f32x2 %0, %1, %2;" : "=l"(t0_) : "l"(u[k]), "l"(cu));
        asm volatile("sub.rn.f32x2 %0, %1, %2;" : "=l"(t1_) : "l"(u[(k + 1) & 7]), "l"(cu));
        asm volatile("sub.rn.f32x2 %0, %1, %2;" : "=l"(t2_) : "l"(u[(k + 2) & 7]), "l"(cu));
        asm volatile("mul.rn.f32x2 %0, %1, %1;" : "=l"(acc) : "l"(t0_));
        asm volatile("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc) : "l"(t1_));
        asm volatile("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc) : "l"(t2_));
        asm volatile("add.rn.f32x2 %0, %0, %1;" : "+l"(u[(k + 4) & 7]) : "l"(acc));
      }
    }
  }
  const unsigned long long t1 = clock64();
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += f[k] + lo2(u[k]) + (float)iv[k] + (float)lv[k];
  if (s == 1.2345f) sink[blockIdx.x] = s;
}

template <int OP>
dfd_status run_op(dfd_context* ctx, double* rate, double* mhz) {
  const int blocks = ctx->num_sms * MB_BLOCKS_PER_SM;
  unsigned long long* cyc = nullptr;
  float* sink = nullptr;
  if (cudaMalloc(&cyc, blocks * sizeof(unsigned long long)) != cudaSuccess) return DFD_ERR_OOM;
  if (cudaMalloc(&sink, blocks * sizeof(float)) != cudaSuccess) {
    cudaFree(cyc);
    return DFD_ERR_OOM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  micro_kernel<OP><<<blocks, MB_THREADS, 0, ctx->stream>>>(1.0f, cyc, sink);  // warm-up
  cudaEventRecord(e0, ctx->stream);
  micro_kernel<OP><<<blocks, MB_THREADS, 0, ctx->stream>>>(1.0f, cyc, sink);
  cudaEventRecord(e1, ctx->stream);
  dfd_status st = cuda_status(cudaStreamSynchronize(ctx->stream));
  if (st == DFD_OK) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    unsigned long long* h = new unsigned long long[blocks];
    cudaMemcpy(h, cyc, blocks * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    double mean_cyc = 0;
    for (int b = 0; b < blocks; ++b) mean_cyc += (double)h[b];
    mean_cyc /= blocks;
    delete[] h;
    // All blocks are resident together (4 x 256 threads per SM): per-SM
    // work over the mean per-block cycle count.
    const double ops_per_sm = (double)MB_BLOCKS_PER_SM * MB_THREADS * MB_ITERS * ops_per_iter(OP);
    *rate = ops_per_sm / mean_cyc;
    *mhz = mean_cyc / (ms * 1.0e3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(cyc);
  cudaFree(sink);
  return st;
}

}  // namespace
}  // namespace dfd

extern "C" dfd_status dfd_microbench(dfd_context* ctx, int op, double* per_clk_per_sm, double* sm_mhz) {
  using namespace dfd;
  if (!ctx || !per_clk_per_sm || !sm_mhz) return DFD_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DFD_ERR_CUDA;
  switch (op) {
    case MB_FFMA: return run_op<MB_FFMA>(ctx, per_clk_per_sm, sm_mhz);
    case MB_FFMA2: return run_op<MB_FFMA2>(ctx, per_clk_per_sm, sm_mhz);
    case MB_FMNMX: return run_op<MB_FMNMX>(ctx, per_clk_per_sm, sm_mhz);
    case MB_FMNMX3: return run_op<MB_FMNMX3>(ctx, per_clk_per_sm, sm_mhz);
    case MB_IMNMX: return run_op<MB_IMNMX>(ctx, per_clk_per_sm, sm_mhz);
    case MB_IMNMX64: return run_op<MB_IMNMX64>(ctx, per_clk_per_sm, sm_mhz);
    case MB_IMADWIDE: return run_op<MB_IMADWIDE>(ctx, per_clk_per_sm, sm_mhz);
    case MB_SHFL: return run_op<MB_SHFL>(ctx, per_clk_per_sm, sm_mhz);
    case MB_MIX_F32D3: return run_op<MB_MIX_F32D3>(ctx, per_clk_per_sm, sm_mhz);
    case MB_MIX_I32D2: return run_op<MB_MIX_I32D2>(ctx, per_clk_per_sm, sm_mhz);
    case MB_DISTONLY_F32D3: return run_op<MB_DISTONLY_F32D3>(ctx, per_clk_per_sm, sm_mhz);
    default: return DFD_ERR_INVALID_ARG;
  }
}
