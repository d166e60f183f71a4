// k_noalloc.cu -- dfd_pair for callers that cannot allocate device memory.
//
// Who needs it: processes whose device memory belongs to another allocator
// (a framework's caching pool, a serving engine that reserves its HBM budget
// up front) and latency-critical loops that must not call cudaMalloc /
// cudaFree, which can synchronise the device.  This entry point uses no
// context and allocates nothing: the band wavefront's scratch and the error
// word live in the fixed array below, part of the library's device image.
#include <cstring>
#include <mutex>

#include "dfd_device.cuh"
#include "dfd_internal.h"

namespace dfd {
namespace {

// Layout: [0, 256) error word (+ padding); [256, end) wavefront scratch
// (ticket, progress words, row buffer, packed q).  Every GPU that loads the
// library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DFD_NOALLOC_SCRATCH_BYTES];

constexpr size_t kErrBytes = 256;
constexpr int kMaxDevices = 64;

struct DeviceSetup {
  bool done = false;
  dfd_status status = DFD_OK;
  unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch
  int num_sms = 0;
  size_t smem_optin = 0;
};

std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

// Once per device, with that device current: the array's device address
// (in host code its name is only a host-side stand-in) and the SM count.
// Only a successful look-up is remembered; a failed one (for example a
// first call made inside a stream capture) is retried by the next call.
dfd_status setup_device(int device, DeviceSetup* out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceSetup& s = g_setup[device];
  if (!s.done) {
    void* ptr = nullptr;
    int sms = 0, optin = 0;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *out = s;
      return DFD_ERR_CUDA;
    }
    s.scratch = static_cast<unsigned char*>(ptr);
    s.num_sms = sms;
    s.smem_optin = (size_t)optin;
    s.status = DFD_OK;
    s.done = true;
  }
  *out = s;
  return s.status;
}

// Upper bound of the wavefront's scratch for (n, m) in this dtype / dim.
size_t scratch_needed(dfd_dtype dtype, int dim, int64_t n, int64_t m) {
  const int dk = dim_class(dim);
  // packed q bytes per column: float32 (and the narrow int32 class) 16-byte
  // planes of two coordinates, the exact int32 class planes of four; an
  // int32 pair packs both streams, and its prep kernel's bounding-box
  // partials (at most 128 blocks of dk (min, max) int pairs) sit beside them
  const size_t q_f = dk <= 4 ? 32 : dk == 8 ? 64 : 128;
  const size_t q_i = dk <= 4 ? 16 : dk == 8 ? 32 : 64;
  const size_t q_per_col = dtype == DFD_F32 ? q_f : q_f + q_i;
  const size_t box = dtype == DFD_F32 ? 0 : 128 * 2 * 16 * sizeof(int) + 256;
  const size_t vbytes = dtype == DFD_F32 ? 4 : 8;
  // packed q: m columns plus the skew and block padding, rounded up to whole
  // chunks of up to 512 columns (one front; two fronts are used only when
  // their doubled scratch also fits, else the wavefront runs one)
  return 2048 + box + 8 * (size_t)((n + 63) / 64) + (size_t)m * vbytes + ((size_t)m + 1024) * q_per_col;
}

}  // namespace
}  // namespace dfd

extern "C" dfd_status dfd_pair_noalloc(int device, dfd_dtype dtype, int dim, const void* p, int64_t n,
                                       const void* q, int64_t m, void* out_dist, void* out_dist2, void* stream) {
  using namespace dfd;
  if (dtype != DFD_F32 && dtype != DFD_I32) return DFD_ERR_INVALID_ARG;
  if (dim < 1 || !p || !q || n < 1 || m < 1 || (!out_dist && !out_dist2)) return DFD_ERR_INVALID_ARG;
  if (dim > 16) return DFD_ERR_UNSUPPORTED;
  if (device < 0 || device >= kMaxDevices) return DFD_ERR_INVALID_ARG;
  if (m > ((int64_t)1 << 29) || scratch_needed(dtype, dim, n, m) > DFD_NOALLOC_SCRATCH_BYTES - kErrBytes)
    return DFD_ERR_CAPACITY;

  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_CUDA;
  }
  DeviceSetup dev;
  dfd_status st = setup_device(device, &dev);
  if (st == DFD_OK) {
    // A context on the stack whose scratch IS the fixed array and whose
    // budget equals its size: the wavefront's grow-only scratch path returns
    // before it could ever free or allocate.
    dfd_context c;
    c.device = device;
    c.num_sms = dev.num_sms;
    c.smem_optin = dev.smem_optin;
    dfd_options_default(&c.opt);
    c.opt.mem_budget_bytes = DFD_NOALLOC_SCRATCH_BYTES - kErrBytes;
    c.d_err = reinterpret_cast<int*>(dev.scratch);
    c.scratch = dev.scratch + kErrBytes;
    c.scratch_bytes = DFD_NOALLOC_SCRATCH_BYTES - kErrBytes;
    c.attr_cache = false;   // no host-side cache either: nothing allocated
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Outputs start as NaN (float, double) / -1 (int64): all-ones bytes.
    const size_t vb = dtype == DFD_F32 ? 4 : 8;
    cudaError_t e = cudaSuccess;
    if (out_dist) e = cudaMemsetAsync(out_dist, 0xff, vb, s);
    if (e == cudaSuccess && out_dist2) e = cudaMemsetAsync(out_dist2, 0xff, vb, s);
    // The error word must start at zero for this call.
    if (e == cudaSuccess) e = cudaMemsetAsync(c.d_err, 0, sizeof(int), s);
    st = cuda_status(e);
    if (st == DFD_OK) st = launch_check_inputs2(dtype, dim, p, n * dim, q, m * dim, c.d_err, s);
    if (st == DFD_OK) {
      WaveShape sh;
      wave_plan(&c, dtype, dim, n, m, &sh);
      st = wave_run(&c, dtype, dim, p, n, q, m, out_dist, out_dist2, s, sh, false);   // checked above
      if (st == DFD_ERR_OOM) st = DFD_ERR_CAPACITY;
    }
    c.scratch = nullptr;   // not owned: nothing to release
    c.d_err = nullptr;
  }
  cudaSetDevice(prev);
  return st;
}
