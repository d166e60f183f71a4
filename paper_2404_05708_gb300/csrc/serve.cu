// serve.cu -- continuous-batching server for query-vs-candidates searches.
//
// Requests (a query curve and k candidate ids from a device-resident pool)
// arrive from any host thread.  A scheduler thread admits them while slots
// and device memory allow (a request's footprint is its query, O(n), plus an
// O(m) row state for each long pair in flight), and runs ticks: each tick is
// one persistent launch (per point dimension present) over (query,
// candidate) pairs drawn from every admitted request, costliest first, up to
// a cell budget.  Pairs longer than one stripe advance a few row stripes per
// tick and keep their bottom row in device memory between ticks (row i of
// the recurrence summarises rows 1..i, Sec. 3), so a long pair never blocks
// the requests that arrive behind it.  Two ticks are in flight at a time:
// while the GPU runs tick t the host prepares tick t+1 and retires t-1.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch_kernel.cuh"
#include "dfd_internal.h"

namespace dfd {
namespace serve {

struct Item {
  const float* P;   // rows curve (device)
  const float* Q;   // column curve (device)
  float* state;     // O(cols) row state (device) for multi-stripe pairs, else null
  int n, m;         // rows, columns
  int s0, s1;       // stripes run by this item
  int out;          // slot in the tick's output array if the pair finishes here, else -1
  int dim;          // point dimension (items are grouped by it)
};

template <int DK>
__global__ void __launch_bounds__(256, batch::kBlocksPerSM<DK>::value) serve_kernel(const Item* items, int n_items, int dim, int vec,
                                                       int* counter, float* out) {
  __shared__ uint4 stage_sm[8][batch::QStage<DK>::RECS];
  uint4* stage = stage_sm[threadIdx.x >> 5];
  const int L = threadIdx.x & 31;
  for (;;) {
    int i = 0;
    if (L == 0) i = atomicAdd(counter, 1);
    i = __shfl_sync(0xffffffffu, i, 0);
    if (i >= n_items) break;
    const Item it = items[i];
    const float r = batch::warp_dfd_any<F32, DK>(it.P, it.n, it.Q, it.m, dim, vec != 0, it.state, L, it.s0, it.s1,
                                                 static_cast<batch::NoAbandon<F32>*>(nullptr), stage);
    if (L == 0 && it.out >= 0) out[it.out] = sqrtf(r);
  }
}

inline double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit sub-allocator over one device region, 256-byte granularity.
class Arena {
 public:
  bool init(size_t bytes) {
    if (cudaMalloc(&base_, bytes) != cudaSuccess) {
      cudaGetLastError();
      base_ = nullptr;
      return false;
    }
    free_[0] = bytes;
    return true;
  }
  ~Arena() {
    if (base_) cudaFree(base_);
  }
  size_t alloc(size_t bytes) {   // offset or SIZE_MAX
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        used_ += bytes;
        return off;
      }
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  char* ptr(size_t off) const { return static_cast<char*>(base_) + off; }
  size_t used() const { return used_; }

 private:
  void* base_ = nullptr;
  size_t used_ = 0;
  std::map<size_t, size_t> free_;
};

struct Pool {
  float* points = nullptr;   // device
  std::vector<int64_t> offsets{0};
  ~Pool() {
    if (points) cudaFree(points);
  }
};

struct PairState {
  int rows = 0, cols = 0, nst = 1;
  bool query_is_rows = true;
  int issued = 0;             // stripes issued to ticks
  size_t state_off = SIZE_MAX;
};

struct Request {
  uint64_t ticket = 0;
  int dim = 0;
  int n = 0;
  std::vector<float> query;
  std::vector<int64_t> ids;
  float* host_out = nullptr;
  double t_arrival = 0, t_done = 0;
  dfd_status status = DFD_ERR_NOT_READY;
  bool cancelled = false;
  size_t q_off = SIZE_MAX;
  std::vector<PairState> pairs;
  int64_t remaining = 0;      // pairs without a result
  int64_t next_pair = 0;      // pairs before it have every stripe issued
  int inflight = 0;           // items of this request in ticks not yet retired
  double cells = 0;
};

struct Tick {
  std::vector<Item> items;
  std::vector<std::pair<Request*, int>> outs;   // output slot -> (request, pair)
  std::vector<Request*> members;                // one entry per item
  Item* h_items = nullptr;    // pinned
  float* h_out = nullptr;     // pinned
  Item* d_items = nullptr;
  float* d_out = nullptr;
  int* d_counter = nullptr;   // one counter per launch (one launch per dim)
  size_t cap_items = 0;
  char* h_stage = nullptr;    // pinned staging of the queries admitted with this tick
  size_t stage_used = 0;
  struct Upload {
    size_t arena_off, stage_off, bytes;
  };
  std::vector<Upload> uploads;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double cells = 0;
};

constexpr int MAX_DIM = 16;
constexpr size_t STAGE_BYTES = (size_t)32 << 20;   // pinned query staging per tick

}  // namespace serve
}  // namespace dfd

using namespace dfd;
using namespace dfd::serve;

struct dfd_server {
  dfd_context* ctx = nullptr;
  dfd_server_options opt{};
  cudaStream_t stream = nullptr;
  Arena arena;
  std::unordered_map<int, std::unique_ptr<Pool>> pools;   // by dim
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::vector<Request*> active;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> requests;
  uint64_t next_ticket = 1;
  Tick ticks[2];
  std::vector<int> sort_count, sort_key;   // build_tick's counting sort (reused buffers)
  std::vector<Item> sort_items;
  int next_tick = 0;
  std::deque<Tick*> inflight;
  std::thread worker;
  std::atomic<bool> stop{false};
  // statistics
  std::vector<double> latencies_ms;
  double busy_ms = 0, cells_done = 0, t_first = -1, t_last = 0;
  uint64_t completed = 0, n_cancelled = 0, n_ticks = 0;
  dfd_status fatal = DFD_OK;
};

namespace {

bool ensure_tick_capacity(Tick& t, size_t items) {
  if (items <= t.cap_items) return true;
  const size_t cap = std::max(items, t.cap_items * 2 + 1024);
  if (t.h_items) cudaFreeHost(t.h_items);
  if (t.h_out) cudaFreeHost(t.h_out);
  if (t.d_items) cudaFree(t.d_items);
  if (t.d_out) cudaFree(t.d_out);
  t.h_items = nullptr;
  t.h_out = nullptr;
  t.d_items = nullptr;
  t.d_out = nullptr;
  t.cap_items = 0;
  if (cudaMallocHost(&t.h_items, cap * sizeof(Item)) != cudaSuccess ||
      cudaMallocHost(&t.h_out, cap * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&t.d_items, cap * sizeof(Item)) != cudaSuccess ||
      cudaMalloc(&t.d_out, cap * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  t.cap_items = cap;
  return true;
}

int stripes_for(int dim, int rows) {
  switch (dim_class(dim)) {
    case 2: return batch::num_stripes<2>(rows);
    case 3: return batch::num_stripes<3>(rows);
    case 4: return batch::num_stripes<4>(rows);
    case 8: return batch::num_stripes<8>(rows);
    default: return batch::num_stripes<16>(rows);
  }
}

void release_request_memory(dfd_server* s, Request* r) {
  if (r->q_off != SIZE_MAX) {
    s->arena.release(r->q_off, (size_t)r->n * r->dim * sizeof(float));
    r->q_off = SIZE_MAX;
  }
  for (auto& p : r->pairs) {
    if (p.state_off != SIZE_MAX) {
      s->arena.release(p.state_off, (size_t)p.cols * sizeof(float));
      p.state_off = SIZE_MAX;
    }
  }
}

// Caller holds s->mu.
void finish_request(dfd_server* s, Request* r, dfd_status st, double t) {
  release_request_memory(s, r);
  r->status = st;
  r->t_done = t;
  s->active.erase(std::remove(s->active.begin(), s->active.end(), r), s->active.end());
  if (st == DFD_OK) {
    s->completed++;
    s->latencies_ms.push_back((t - r->t_arrival) * 1e3);
    s->cells_done += r->cells;
    s->t_last = t;
  } else {
    s->n_cancelled++;
  }
  s->cv_done.notify_all();
}

// Admit pending requests in arrival order while slots and memory allow; the
// admitted queries are staged in the tick's pinned buffer and copied to the
// device ahead of the tick's kernels (stream order).
void admit(dfd_server* s, Tick& t) {
  const int max_slots = s->opt.max_slots > 0 ? s->opt.max_slots : 256;
  t.uploads.clear();
  t.stage_used = 0;
  while (!s->pending.empty() && (int)s->active.size() < max_slots) {
    Request* r = s->pending.front();
    const size_t qb = (size_t)r->n * r->dim * sizeof(float);
    if (t.stage_used + qb > STAGE_BYTES) break;   // the next tick takes it
    const size_t off = s->arena.alloc(qb);
    if (off == SIZE_MAX) break;                   // wait for running requests to release memory
    s->pending.pop_front();
    r->q_off = off;
    std::memcpy(t.h_stage + t.stage_used, r->query.data(), qb);
    t.uploads.push_back({off, t.stage_used, qb});
    t.stage_used += (qb + 15) / 16 * 16;
    Pool& pool = *s->pools[r->dim];
    r->pairs.resize(r->ids.size());
    for (size_t k = 0; k < r->ids.size(); ++k) {
      const int64_t c = r->ids[k];
      const int len = (int)(pool.offsets[c + 1] - pool.offsets[c]);
      PairState& p = r->pairs[k];
      p.query_is_rows = r->n <= len;
      p.rows = std::min(r->n, len);
      p.cols = std::max(r->n, len);
      p.nst = stripes_for(r->dim, p.rows);
      r->cells += (double)p.rows * p.cols;
    }
    r->remaining = (int64_t)r->ids.size();
    s->active.push_back(r);
  }
}

// Fill `t` with the next slice of work of the admitted requests (oldest first).
void build_tick(dfd_server* s, Tick& t) {
  t.items.clear();
  t.outs.clear();
  t.members.clear();
  t.cells = 0;
  const double budget = s->opt.tick_cells > 0 ? s->opt.tick_cells : 2.0e9;
  const int max_st = s->opt.stripes_per_tick > 0 ? s->opt.stripes_per_tick : 4;
  for (Request* r : s->active) {
    if (t.cells >= budget) break;
    if (r->cancelled) continue;
    Pool& pool = *s->pools[r->dim];
    const float* qdev = reinterpret_cast<const float*>(s->arena.ptr(r->q_off));
    for (int64_t k = r->next_pair; k < (int64_t)r->pairs.size() && t.cells < budget; ++k) {
      PairState& p = r->pairs[k];
      if (p.issued >= p.nst) continue;
      if (p.nst > 1 && p.state_off == SIZE_MAX) {
        p.state_off = s->arena.alloc((size_t)p.cols * sizeof(float));
        if (p.state_off == SIZE_MAX) continue;   // no room for its row state in this tick
      }
      const float* cdev = pool.points + pool.offsets[r->ids[k]] * r->dim;
      Item it;
      it.P = p.query_is_rows ? qdev : cdev;
      it.Q = p.query_is_rows ? cdev : qdev;
      it.state = p.nst > 1 ? reinterpret_cast<float*>(s->arena.ptr(p.state_off)) : nullptr;
      it.n = p.rows;
      it.m = p.cols;
      it.s0 = p.issued;
      it.s1 = std::min(p.nst, p.issued + max_st);
      it.dim = r->dim;
      if (it.s1 == p.nst) {
        it.out = (int)t.outs.size();
        t.outs.emplace_back(r, (int)k);
      } else {
        it.out = -1;
      }
      t.cells += (double)(it.s1 - it.s0) / p.nst * p.rows * (double)p.cols;
      p.issued = it.s1;
      t.items.push_back(it);
      t.members.push_back(r);
      r->inflight++;
    }
    while (r->next_pair < (int64_t)r->pairs.size() && r->pairs[r->next_pair].issued >= r->pairs[r->next_pair].nst)
      r->next_pair++;
  }
  // One launch per dimension; costliest items first inside it (LPT by
  // power-of-two cost classes): a counting sort, linear in the items, where
  // a comparison sort of every pair was the scheduler's largest per-pair cost.
  constexpr int NCLS = 48;
  const size_t n_it = t.items.size();
  if (n_it > 1) {
    std::vector<int>& cnt = s->sort_count;
    cnt.assign((MAX_DIM + 1) * NCLS + 1, 0);
    std::vector<int>& key = s->sort_key;
    key.resize(n_it);
    for (size_t i = 0; i < n_it; ++i) {
      const Item& it = t.items[i];
      const unsigned long long c =
          (unsigned long long)(it.s1 - it.s0) * (unsigned long long)it.m * (unsigned long long)std::min(it.n, 256);
      const int b = c > 1 ? std::min(NCLS - 1, 63 - __builtin_clzll(c)) : 0;
      key[i] = std::min(it.dim, MAX_DIM) * NCLS + (NCLS - 1 - b);
      ++cnt[key[i] + 1];
    }
    for (size_t k = 1; k < cnt.size(); ++k) cnt[k] += cnt[k - 1];
    std::vector<Item>& out = s->sort_items;
    out.resize(n_it);
    for (size_t i = 0; i < n_it; ++i) out[cnt[key[i]]++] = t.items[i];
    t.items.swap(out);
  }
}

void launch_tick(dfd_server* s, Tick& t) {
  const size_t n = t.items.size();
  if (n) std::memcpy(t.h_items, t.items.data(), n * sizeof(Item));
  cudaEventRecord(t.ev0, s->stream);
  for (const auto& u : t.uploads)
    cudaMemcpyAsync(s->arena.ptr(u.arena_off), t.h_stage + u.stage_off, u.bytes, cudaMemcpyHostToDevice, s->stream);
  if (n) cudaMemcpyAsync(t.d_items, t.h_items, n * sizeof(Item), cudaMemcpyHostToDevice, s->stream);
  cudaMemsetAsync(t.d_counter, 0, (MAX_DIM + 1) * sizeof(int), s->stream);
  size_t b = 0;
  while (b < n) {
    size_t e = b;
    const int dim = t.items[b].dim;
    while (e < n && t.items[e].dim == dim) ++e;
    const int dk = dim_class(dim);
    const int vec = (dim == dk && dk != 3) ? 1 : 0;
    const int count = (int)(e - b);
    const int blocks = std::max(1, std::min((count + 7) / 8, 2 * s->ctx->num_sms));
    const Item* items = t.d_items + b;
    int* counter = t.d_counter + dim;
#define DFD_SERVE_CASE(K)                                                                                   \
  case K:                                                                                                   \
    serve_kernel<K><<<blocks, 256, 0, s->stream>>>(items, count, dim, vec, counter, t.d_out);              \
    break;
    switch (dk) {
      DFD_SERVE_CASE(2)
      DFD_SERVE_CASE(3)
      DFD_SERVE_CASE(4)
      DFD_SERVE_CASE(8)
      DFD_SERVE_CASE(16)
      default:
        break;
    }
#undef DFD_SERVE_CASE
    b = e;
  }
  if (!t.outs.empty())
    cudaMemcpyAsync(t.h_out, t.d_out, t.outs.size() * sizeof(float), cudaMemcpyDeviceToHost, s->stream);
  cudaEventRecord(t.ev1, s->stream);
  if (cudaGetLastError() != cudaSuccess) s->fatal = DFD_ERR_CUDA;
}

// Caller holds s->mu; the tick's ev1 has completed.
void retire_tick(dfd_server* s, Tick& t) {
  const double now = now_s();
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, t.ev0, t.ev1) == cudaSuccess) s->busy_ms += ms;
  s->n_ticks++;
  for (size_t i = 0; i < t.outs.size(); ++i) {
    Request* r = t.outs[i].first;
    if (!r->cancelled && r->host_out) r->host_out[t.outs[i].second] = t.h_out[i];
    r->remaining--;
  }
  for (Request* r : t.members) r->inflight--;
  // completion: every pair has a result, or a cancelled request has nothing in flight
  std::vector<Request*> done;
  for (Request* r : s->active) {
    if (r->inflight == 0 && (r->remaining == 0 || r->cancelled)) done.push_back(r);
  }
  for (Request* r : done) finish_request(s, r, r->cancelled ? DFD_ERR_CANCELLED : DFD_OK, now);
}

void worker_loop(dfd_server* s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    Tick& t = s->ticks[s->next_tick];
    bool launched = false;
    if (s->inflight.size() < 2) {
      admit(s, t);
      build_tick(s, t);
      if (!t.items.empty() || !t.uploads.empty()) {
        if (!ensure_tick_capacity(t, t.items.size())) {
          s->fatal = DFD_ERR_OOM;
        } else {
          launch_tick(s, t);
          s->inflight.push_back(&t);
          s->next_tick ^= 1;
          launched = true;
        }
      }
    }
    if (!s->inflight.empty() && (s->inflight.size() >= 2 || !launched)) {
      Tick* old = s->inflight.front();
      lk.unlock();
      cudaEventSynchronize(old->ev1);
      lk.lock();
      s->inflight.pop_front();
      retire_tick(s, *old);
      continue;
    }
    if (!launched) s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
  }
  // drain
  while (!s->inflight.empty()) {
    Tick* old = s->inflight.front();
    lk.unlock();
    cudaEventSynchronize(old->ev1);
    lk.lock();
    s->inflight.pop_front();
    retire_tick(s, *old);
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

dfd_status dfd_server_options_default(dfd_server_options* o) {
  if (!o) return DFD_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->struct_size = sizeof(dfd_server_options);
  o->mem_budget_bytes = (size_t)1 << 30;
  o->max_slots = 256;
  o->tick_cells = 2.0e9;
  o->stripes_per_tick = 4;
  return DFD_OK;
}

dfd_status dfd_server_create(dfd_context* ctx, const dfd_server_options* opt, dfd_server** out) {
  if (!ctx || !out) return DFD_ERR_INVALID_ARG;
  *out = nullptr;
  dfd_server_options o;
  dfd_server_options_default(&o);
  if (opt) {
    if (opt->struct_size != sizeof(dfd_server_options)) return DFD_ERR_INVALID_ARG;
    o = *opt;
  }
  if (o.mem_budget_bytes < ((size_t)1 << 20)) return DFD_ERR_INVALID_ARG;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return DFD_ERR_CUDA;
  dfd_server* s = new (std::nothrow) dfd_server();
  if (!s) return DFD_ERR_OOM;
  s->ctx = ctx;
  s->opt = o;
  bool ok = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && s->arena.init(o.mem_budget_bytes);
  for (auto& t : s->ticks) {
    ok = ok && cudaEventCreate(&t.ev0) == cudaSuccess && cudaEventCreate(&t.ev1) == cudaSuccess;
    ok = ok && cudaMalloc(&t.d_counter, (MAX_DIM + 1) * sizeof(int)) == cudaSuccess;
    ok = ok && cudaMallocHost(&t.h_stage, STAGE_BYTES) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    dfd_server_destroy(s);
    return DFD_ERR_OOM;
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return DFD_OK;
}

dfd_status dfd_server_destroy(dfd_server* s) {
  if (!s) return DFD_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->ctx->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (auto& t : s->ticks) {
    if (t.h_items) cudaFreeHost(t.h_items);
    if (t.h_out) cudaFreeHost(t.h_out);
    if (t.d_items) cudaFree(t.d_items);
    if (t.d_out) cudaFree(t.d_out);
    if (t.d_counter) cudaFree(t.d_counter);
    if (t.h_stage) cudaFreeHost(t.h_stage);
    if (t.ev0) cudaEventDestroy(t.ev0);
    if (t.ev1) cudaEventDestroy(t.ev1);
  }
  if (s->stream) cudaStreamDestroy(s->stream);
  cudaGetLastError();
  delete s;
  return DFD_OK;
}

dfd_status dfd_server_add_candidates(dfd_server* s, int dim, const float* host_points, const int64_t* host_offsets,
                                     int64_t n_curves, int64_t* first_id) {
  if (!s || !host_points || !host_offsets || n_curves < 1 || dim < 1) return DFD_ERR_INVALID_ARG;
  if (dim > MAX_DIM) return DFD_ERR_UNSUPPORTED;
  if (host_offsets[0] != 0) return DFD_ERR_INVALID_ARG;
  for (int64_t c = 0; c < n_curves; ++c) {
    const int64_t len = host_offsets[c + 1] - host_offsets[c];
    if (len < 1 || len > (1 << 24)) return DFD_ERR_INVALID_ARG;
  }
  const int64_t npts = host_offsets[n_curves];
  for (int64_t i = 0; i < npts * dim; ++i)
    if (!std::isfinite(host_points[i])) return DFD_ERR_NONFINITE;
  std::lock_guard<std::mutex> lk(s->mu);
  if (cudaSetDevice(s->ctx->device) != cudaSuccess) return DFD_ERR_CUDA;
  auto& slot = s->pools[dim];
  if (!slot) slot.reset(new Pool());
  Pool& pool = *slot;
  const int64_t old_pts = pool.offsets.back();
  // grow: new device array with old + new points (the worker is not using the
  // pool while we hold the lock, and the copy below is ordered on its stream)
  float* grown = nullptr;
  if (cudaMalloc(&grown, (size_t)(old_pts + npts) * dim * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_OOM;
  }
  cudaStreamSynchronize(s->stream);
  if (pool.points) cudaMemcpy(grown, pool.points, (size_t)old_pts * dim * sizeof(float), cudaMemcpyDeviceToDevice);
  cudaMemcpy(grown + old_pts * dim, host_points, (size_t)npts * dim * sizeof(float), cudaMemcpyHostToDevice);
  if (pool.points) cudaFree(pool.points);
  pool.points = grown;
  if (first_id) *first_id = (int64_t)pool.offsets.size() - 1;
  for (int64_t c = 0; c < n_curves; ++c) pool.offsets.push_back(old_pts + host_offsets[c + 1]);
  return cudaGetLastError() == cudaSuccess ? DFD_OK : DFD_ERR_CUDA;
}

dfd_status dfd_server_submit(dfd_server* s, int dim, const float* host_query, int64_t n, const int64_t* cand_ids,
                             int64_t k, float* host_out, double arrival_s, uint64_t* ticket) {
  if (!s || !host_query || n < 1 || !cand_ids || k < 1 || !host_out || !ticket) return DFD_ERR_INVALID_ARG;
  if (n > (1 << 24)) return DFD_ERR_UNSUPPORTED;
  for (int64_t i = 0; i < n * dim; ++i)
    if (!std::isfinite(host_query[i])) return DFD_ERR_NONFINITE;
  std::unique_ptr<Request> r(new (std::nothrow) Request());
  if (!r) return DFD_ERR_OOM;
  r->dim = dim;
  r->n = (int)n;
  r->query.assign(host_query, host_query + n * dim);
  r->ids.assign(cand_ids, cand_ids + k);
  r->host_out = host_out;
  r->t_arrival = arrival_s >= 0 ? arrival_s : now_s();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->fatal != DFD_OK) return s->fatal;
  auto pit = s->pools.find(dim);
  if (pit == s->pools.end()) return DFD_ERR_INVALID_ARG;
  const int64_t ncand = (int64_t)pit->second->offsets.size() - 1;
  for (int64_t i = 0; i < k; ++i)
    if (cand_ids[i] < 0 || cand_ids[i] >= ncand) return DFD_ERR_INVALID_ARG;
  const size_t qb = (size_t)n * dim * sizeof(float);
  if (qb > s->opt.mem_budget_bytes / 2) return DFD_ERR_BUSY;   // never admissible
  r->ticket = s->next_ticket++;
  *ticket = r->ticket;
  if (s->t_first < 0) s->t_first = r->t_arrival;
  s->pending.push_back(r.get());
  s->requests[r->ticket] = std::move(r);
  s->cv_work.notify_all();
  return DFD_OK;
}

dfd_status dfd_server_wait(dfd_server* s, uint64_t ticket, double timeout_ms) {
  if (!s) return DFD_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return DFD_ERR_INVALID_ARG;
  Request* r = it->second.get();
  auto ready = [&] { return r->status != DFD_ERR_NOT_READY || s->fatal != DFD_OK; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), ready)) {
    return DFD_ERR_NOT_READY;
  }
  if (r->status == DFD_ERR_NOT_READY) return s->fatal;
  const dfd_status st = r->status;
  s->requests.erase(it);
  return st;
}

dfd_status dfd_server_cancel(dfd_server* s, uint64_t ticket) {
  if (!s) return DFD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->requests.find(ticket);
  if (it == s->requests.end()) return DFD_ERR_INVALID_ARG;
  Request* r = it->second.get();
  if (r->status != DFD_ERR_NOT_READY) return DFD_OK;   // already finished
  r->cancelled = true;
  auto pit = std::find(s->pending.begin(), s->pending.end(), r);
  if (pit != s->pending.end()) {
    s->pending.erase(pit);
    r->status = DFD_ERR_CANCELLED;
    s->n_cancelled++;
    s->cv_done.notify_all();
  } else if (r->inflight == 0) {
    finish_request(s, r, DFD_ERR_CANCELLED, now_s());
  }
  s->cv_work.notify_all();
  return DFD_OK;
}

dfd_status dfd_server_stats(dfd_server* s, dfd_serving_stats* out) {
  if (!s || !out) return DFD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->completed = s->completed;
  out->cancelled = s->n_cancelled;
  out->ticks = s->n_ticks;
  out->cells = s->cells_done;
  out->p50_ms = percentile(s->latencies_ms, 0.50);
  out->p99_ms = percentile(s->latencies_ms, 0.99);
  double mean = 0;
  for (double v : s->latencies_ms) mean += v;
  out->mean_ms = s->latencies_ms.empty() ? 0 : mean / s->latencies_ms.size();
  out->gpu_busy_ms = s->busy_ms;
  out->gcups_busy = s->busy_ms > 0 ? s->cells_done / (s->busy_ms * 1e-3) / 1e9 : 0;
  const double wall = s->t_last - s->t_first;
  out->gcups_wall = wall > 0 ? s->cells_done / wall / 1e9 : 0;
  out->arena_used_bytes = s->arena.used();
  return DFD_OK;
}

dfd_status dfd_server_stats_reset(dfd_server* s) {
  if (!s) return DFD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  s->latencies_ms.clear();
  s->busy_ms = 0;
  s->cells_done = 0;
  s->t_first = -1;
  s->t_last = 0;
  s->completed = 0;
  s->n_cancelled = 0;
  s->n_ticks = 0;
  return DFD_OK;
}

double dfd_server_now(dfd_server* s) {
  (void)s;
  return now_s();
}

}  // extern "C"
