// serve.cu -- continuous-batching server for query-vs-candidates searches.
//
// Requests (a query curve and k candidate ids from a device-resident pool)
// arrive from any host thread.  A scheduler thread admits them while slots
// and device memory allow (a request's footprint is its query and candidate
// ids, O(n + k), plus an O(m) row state for each long pair in flight), and
// runs ticks: each tick is one persistent launch per point dimension present
// over (query, candidate) pairs drawn from every admitted request, oldest
// request first, up to a cell budget.
//
// Admission sorts a request's pairs by cost class (power-of-two cell count).
// Pairs that finish within one tick are handed to a tick as slices -- a run
// of consecutive positions in that order, one class per slice -- and
// expanded into pairs on the device: a warp takes a global pair index and
// finds its slice by a 32-way search of the slices' prefix sums.  So the
// host's work per tick grows with the requests, not with the pairs.  Only
// long pairs (more row stripes than a tick runs, or a row state wider than a
// warp's buffer) go out one by one as items: they advance a few stripes per
// tick and keep their bottom row in device memory between ticks (row i of
// the recurrence summarises rows 1..i, Sec. 3), so a long pair never blocks
// the requests behind it.  Inside a launch the items come first, then the
// slices in decreasing cost class (largest first, LPT).  Two ticks are in
// flight, each on its own stream: while tick t drains its last warps, tick
// t+1's blocks already take the SMs it frees (a long pair is in at most one
// tick in flight, so the two never share a row state), and the host
// prepares the next tick while it retires the oldest.
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

// One long pair's stripes [s0, s1).
struct Item {
  const float* P;   // rows curve (device)
  const float* Q;   // column curve (device)
  float* state;     // O(cols) row state (device) for multi-stripe pairs, else null
  int n, m;         // rows, columns
  int s0, s1;       // stripes run by this item
  int out;          // slot in the tick's output array if the pair finishes here, else -1
  int dim;          // point dimension (items are grouped by it)
};

// `count` pairs of one request, expanded on the device: pair li compares the
// query with candidate cids[li] and writes its distance to out[out_base + li].
struct Slice {
  const float* query;     // device, n x dim
  const int32_t* cids;    // device, candidate ids of the slice's pairs
  int n;                  // query points
  int count;              // pairs
  int out_base;           // output slot of the slice's first pair
  int pad;
};

struct ServeArgs {
  const Item* items;      // long pairs (first in the launch's index space)
  int n_items;
  int n_slices;
  const Slice* slices;
  const int* prefix;      // n_slices + 1 pair-count prefix sums (relative to prefix[0])
  const float* pool;      // candidate points of this dim (device)
  const int64_t* offsets; // candidate c spans points [offsets[c], offsets[c + 1])
  int dim, vec;
  int* counter;
  float* out;
  float* rowbuf;          // batch::BUF_COLS values per warp (multi-stripe short pairs)
};

template <int DK>
__global__ void __launch_bounds__(256, batch::kBlocksPerSM<DK>::value) serve_kernel(ServeArgs a) {
  __shared__ uint4 stage_sm[8][batch::QStage<DK>::RECS];
  uint4* stage = stage_sm[threadIdx.x >> 5];
  const int L = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  float* buf = a.rowbuf + gw * batch::BUF_COLS;
  const int base = a.n_slices > 0 ? a.prefix[0] : 0;
  const int total = a.n_items + (a.n_slices > 0 ? a.prefix[a.n_slices] - base : 0);
  for (;;) {
    int i = 0;
    if (L == 0) i = atomicAdd(a.counter, 1);
    i = __shfl_sync(0xffffffffu, i, 0);
    if (i >= total) break;
    const float *P, *Q;
    float* state;
    int n, m, s0 = 0, s1 = 1 << 30, out;
    if (i < a.n_items) {
      const Item it = a.items[i];
      P = it.P;
      Q = it.Q;
      state = it.state;
      n = it.n;
      m = it.m;
      s0 = it.s0;
      s1 = it.s1;
      out = it.out;
    } else {
      // the slice holding pair j: prefix[lo] - base <= j < prefix[hi] - base,
      // narrowed 32-fold per round (one probe per lane)
      const int j = i - a.n_items;
      int lo = 0, hi = a.n_slices;
      while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int p = lo + L * step;
        const bool le = p < hi && a.prefix[p] - base <= j;
        const int cnt = __popc(__ballot_sync(0xffffffffu, le));   // >= 1: position lo qualifies
        lo += (cnt - 1) * step;
        hi = min(hi, lo + step);
      }
      const Slice sl = a.slices[lo];
      const int li = j - (a.prefix[lo] - base);
      const int64_t o = a.offsets[sl.cids[li]];
      const int len = (int)(a.offsets[sl.cids[li] + 1] - o);
      const float* C = a.pool + o * a.dim;
      const bool qrows = sl.n <= len;
      P = qrows ? sl.query : C;
      Q = qrows ? C : sl.query;
      n = qrows ? sl.n : len;
      m = qrows ? len : sl.n;
      state = buf;
      out = sl.out_base + li;
      if (batch::num_stripes<DK>(n) > 1 && m > batch::BUF_COLS) {   // admission makes such pairs items
        if (L == 0) a.out[out] = -1.f;
        continue;
      }
    }
    const float r = batch::warp_dfd_any<F32, DK>(P, n, Q, m, a.dim, a.vec != 0, state, L, s0, s1,
                                                 static_cast<batch::NoAbandon<F32>*>(nullptr), stage);
    if (L == 0 && out >= 0) a.out[out] = sqrtf(r);
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
  float* points = nullptr;        // device
  int64_t* d_offsets = nullptr;   // device copy of `offsets`
  std::vector<int64_t> offsets{0};
  ~Pool() {
    if (points) cudaFree(points);
    if (d_offsets) cudaFree(d_offsets);
  }
};

// A pair that spans ticks.
struct LongPair {
  int k = 0;                  // pair index in the request
  int rows = 0, cols = 0, nst = 1;
  bool query_is_rows = true;
  int issued = 0;             // stripes issued to ticks
  bool busy = false;          // in a tick in flight
  size_t state_off = SIZE_MAX;
};

// A run of a request's cost-sorted short pairs that share one cost class.
struct ClassRun {
  int begin;                  // first position in `order`
  int cls;                    // rank: 0 = costliest class
};

struct Request {
  uint64_t ticket = 0;
  int dim = 0;
  int n = 0;
  std::vector<float> query;
  std::vector<int64_t> ids;
  float* host_out = nullptr;
  double t_arrival = 0, t_done = 0;
  double t_submit = 0, t_admit = 0, t_launch = 0;   // submission, admission, first tick launch
  double t_locked = 0;                                // submission: server lock taken
  dfd_status status = DFD_ERR_NOT_READY;
  bool cancelled = false;
  size_t q_off = SIZE_MAX;
  size_t cid_off = SIZE_MAX, cid_bytes = 0;   // candidate ids of the short pairs (int32, in `order`)
  std::vector<int32_t> order;       // short pairs (indices into ids), costliest class first
  std::vector<double> cells_pre;    // cells of order[0 .. i)
  std::vector<ClassRun> runs;
  std::vector<LongPair> longs;
  int64_t next_short = 0;     // positions of `order` before it are in a slice
  size_t next_long = 0;       // long pairs before it have every stripe issued
  int64_t remaining = 0;      // pairs without a result
  int inflight = 0;           // items and slices of this request in ticks not yet retired
  double cells = 0;
};

// Host record of a slice.
struct SliceRec {
  Slice d;
  Request* r;
  int first;                  // position of the slice's first pair in r->order
  int key;                    // dim * NCLS + class rank
};

// A tick's launches alternate between its two streams (forked after the
// tick's copies, joined before its results are read back), so the launches
// of different point dimensions overlap like consecutive ticks do.
constexpr int NSTREAM = 2;

struct Tick {
  double t_build = 0, t_launched = 0;   // host: build began, launch calls returned
  double t_admitted = 0, t_built = 0;   // host: admission and tick building done
  double t_sync0 = 0, t_sync1 = 0, t_locked = 0;   // host: wait for the tick's last event, lock retaken
  double slow_call_ms = 0;              // the slowest CUDA call of the launch, and which (1-9)
  int slow_call = 0;
  int n_admitted = 0;
  cudaStream_t stream[NSTREAM] = {};
  float* rowbuf[NSTREAM] = {};   // per-warp row buffers of the launches on each stream
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  std::vector<LongPair*> longs_issued;
  std::vector<Item> items;
  std::vector<std::pair<Request*, int>> outs;   // item output slot -> (request, pair)
  std::vector<Request*> members;                // one entry per item
  std::vector<SliceRec> slices;
  std::vector<int> prefix;                      // pair-count prefix sums of `slices`
  size_t n_outs = 0;          // item outputs, then the slices' pairs
  char* h_desc = nullptr;     // pinned: items | slices | prefix
  char* d_desc = nullptr;
  size_t cap_desc = 0;
  size_t off_slices = 0, off_prefix = 0, desc_bytes = 0;
  float* h_out = nullptr;     // pinned
  float* d_out = nullptr;
  size_t cap_out = 0;
  int* d_counter = nullptr;   // one counter per launch (one launch per dim)
  char* h_stage = nullptr;    // pinned staging of the queries and ids admitted with this tick
  size_t stage_used = 0;
  struct Upload {
    size_t arena_off, stage_off, bytes;
  };
  std::vector<Upload> uploads;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t ev_up = nullptr;   // this tick's uploads (and every earlier tick's) are done
  double cells = 0;
};

constexpr int MAX_DIM = 16;
constexpr int NTICK = 3;        // tick slots; at most NTICK - 1 in flight
constexpr int NCLS = 48;                           // cost classes: floor(log2(cells))
constexpr size_t STAGE_BYTES = (size_t)32 << 20;   // pinned query / id staging per tick

inline int cost_rank(unsigned long long cells) {   // 0 for the costliest class
  const int b = cells > 1 ? std::min(NCLS - 1, 63 - __builtin_clzll(cells)) : 0;
  return NCLS - 1 - b;
}

inline size_t align16(size_t b) { return (b + 15) / 16 * 16; }

}  // namespace serve
}  // namespace dfd

using namespace dfd;
using namespace dfd::serve;

struct dfd_server {
  dfd_context* ctx = nullptr;
  dfd_server_options opt{};
  Arena arena;
  std::unordered_map<int, std::unique_ptr<Pool>> pools;   // by dim
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> pending;
  std::vector<Request*> active;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> requests;
  uint64_t next_ticket = 1;
  Tick ticks[NTICK];
  Tick* last_launched = nullptr;
  Tick* last_retired = nullptr;
  std::vector<int> sort_count, sort_key;   // counting sorts (reused buffers)
  std::vector<Item> sort_items;
  std::vector<SliceRec> sort_slices;
  int next_tick = 0;
  std::deque<Tick*> inflight;
  std::thread worker;
  std::atomic<bool> stop{false};
  // statistics
  std::vector<double> latencies_ms;
  std::vector<dfd_request_record> log;   // completed requests (since the last stats reset)
  std::vector<dfd_tick_record> tick_log; // retired ticks (since the last stats reset)
  double busy_ms = 0, cells_done = 0, t_first = -1, t_last = 0;
  uint64_t completed = 0, n_cancelled = 0, n_ticks = 0;
  dfd_status fatal = DFD_OK;
};

namespace {

// Warps of the widest tick launch: blocks are capped at two per SM.
inline size_t max_tick_warps(const dfd_server* s) { return (size_t)2 * s->ctx->num_sms * 8; }

bool ensure_tick_capacity(Tick& t, size_t desc_bytes, size_t outs) {
  if (desc_bytes > t.cap_desc) {
    const size_t cap = std::max(desc_bytes, t.cap_desc * 2 + (64 << 10));
    if (t.h_desc) cudaFreeHost(t.h_desc);
    if (t.d_desc) cudaFree(t.d_desc);
    t.h_desc = t.d_desc = nullptr;
    t.cap_desc = 0;
    if (cudaMallocHost(&t.h_desc, cap) != cudaSuccess || cudaMalloc(&t.d_desc, cap) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    t.cap_desc = cap;
  }
  if (outs > t.cap_out) {
    const size_t cap = std::max(outs, t.cap_out * 2 + 4096);
    if (t.h_out) cudaFreeHost(t.h_out);
    if (t.d_out) cudaFree(t.d_out);
    t.h_out = nullptr;
    t.d_out = nullptr;
    t.cap_out = 0;
    if (cudaMallocHost(&t.h_out, cap * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&t.d_out, cap * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    t.cap_out = cap;
  }
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
  if (r->cid_off != SIZE_MAX) {
    s->arena.release(r->cid_off, r->cid_bytes);
    r->cid_off = SIZE_MAX;
  }
  for (auto& p : r->longs) {
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
    if (s->log.size() < ((size_t)1 << 22)) {
      dfd_request_record rec;
      rec.ticket = r->ticket;
      rec.arrival_s = r->t_arrival;
      rec.submit_s = r->t_submit;
      rec.admit_s = r->t_admit;
      rec.launch_s = r->t_launch;
      rec.done_s = t;
      rec.cells = r->cells;
      rec.locked_s = r->t_locked;
      rec.n = r->n;
      rec.k = (int)r->ids.size();
      rec.dim = r->dim;
      rec.pad = 0;
      s->log.push_back(rec);
    }
    s->cells_done += r->cells;
    s->t_last = t;
  } else {
    s->n_cancelled++;
  }
  s->cv_done.notify_all();
}

// Split a request's pairs into long pairs and short pairs, the short ones in
// decreasing cost class (a counting sort), with their cell prefix sums and
// class runs; the candidate ids in that order go to `cid_stage`.
void plan_request(dfd_server* s, Request* r, int32_t* cid_stage) {
  const int max_st = s->opt.stripes_per_tick > 0 ? s->opt.stripes_per_tick : 8;
  const Pool& pool = *s->pools[r->dim];
  const int k = (int)r->ids.size();
  std::vector<int>& key = s->sort_key;
  std::vector<int>& cnt = s->sort_count;
  key.resize(k);
  cnt.assign(NCLS + 1, 0);
  r->longs.clear();
  r->cells = 0;
  for (int x = 0; x < k; ++x) {
    const int64_t c = r->ids[x];
    const int len = (int)(pool.offsets[c + 1] - pool.offsets[c]);
    const int rows = std::min(r->n, len), cols = std::max(r->n, len);
    const int nst = stripes_for(r->dim, rows);
    r->cells += (double)rows * cols;
    if (nst > max_st || (nst > 1 && cols > batch::BUF_COLS)) {
      LongPair lp;
      lp.k = x;
      lp.rows = rows;
      lp.cols = cols;
      lp.nst = nst;
      lp.query_is_rows = r->n <= len;
      r->longs.push_back(lp);
      key[x] = -1;
    } else {
      key[x] = cost_rank((unsigned long long)rows * (unsigned long long)cols);
      ++cnt[key[x] + 1];
    }
  }
  for (int c = 1; c <= NCLS; ++c) cnt[c] += cnt[c - 1];
  const int n_short = cnt[NCLS];
  r->runs.clear();
  for (int c = 0; c < NCLS; ++c)
    if (cnt[c + 1] > cnt[c]) r->runs.push_back({cnt[c], c});
  r->order.resize(n_short);
  for (int x = 0; x < k; ++x)
    if (key[x] >= 0) r->order[cnt[key[x]]++] = x;
  r->cells_pre.resize(n_short + 1);
  r->cells_pre[0] = 0;
  for (int y = 0; y < n_short; ++y) {
    const int64_t c = r->ids[r->order[y]];
    const int len = (int)(pool.offsets[c + 1] - pool.offsets[c]);
    r->cells_pre[y + 1] = r->cells_pre[y] + (double)r->n * len;
    cid_stage[y] = (int32_t)c;
  }
  r->next_short = 0;
  r->next_long = 0;
  r->remaining = k;
}

// Admit pending requests in arrival order while slots and memory allow; the
// admitted queries and candidate ids are staged in the tick's pinned buffer
// and copied to the device ahead of the tick's kernels (stream order).
void admit(dfd_server* s, Tick& t) {
  const int max_slots = s->opt.max_slots > 0 ? s->opt.max_slots : 256;
  t.uploads.clear();
  t.stage_used = 0;
  while (!s->pending.empty() && (int)s->active.size() < max_slots) {
    Request* r = s->pending.front();
    const size_t qb = (size_t)r->n * r->dim * sizeof(float);
    const size_t ib = std::max<size_t>(r->ids.size() * sizeof(int32_t), 16);
    if (t.stage_used + align16(qb) + align16(ib) > STAGE_BYTES) break;   // the next tick takes it
    const size_t off = s->arena.alloc(qb);
    if (off == SIZE_MAX) break;                    // wait for running requests to release memory
    const size_t coff = s->arena.alloc(ib);
    if (coff == SIZE_MAX) {
      s->arena.release(off, qb);
      break;
    }
    s->pending.pop_front();
    r->t_admit = now_s();
    r->q_off = off;
    r->cid_off = coff;
    r->cid_bytes = ib;
    std::memcpy(t.h_stage + t.stage_used, r->query.data(), qb);
    t.uploads.push_back({off, t.stage_used, qb});
    t.stage_used += align16(qb);
    plan_request(s, r, reinterpret_cast<int32_t*>(t.h_stage + t.stage_used));
    if (!r->order.empty()) t.uploads.push_back({coff, t.stage_used, r->order.size() * sizeof(int32_t)});
    t.stage_used += align16(ib);
    s->active.push_back(r);
  }
}

// Fill `t` with the next work of the admitted requests (oldest first): the
// long pairs' next stripes, then a run of the short pairs.
void build_tick(dfd_server* s, Tick& t) {
  t.items.clear();
  t.outs.clear();
  t.members.clear();
  t.slices.clear();
  t.longs_issued.clear();
  t.cells = 0;
  const double budget = s->opt.tick_cells > 0 ? s->opt.tick_cells : 4.0e9;
  const int max_st = s->opt.stripes_per_tick > 0 ? s->opt.stripes_per_tick : 8;
  for (Request* r : s->active) {
    if (t.cells >= budget) break;
    if (r->cancelled) continue;
    Pool& pool = *s->pools[r->dim];
    const float* qdev = reinterpret_cast<const float*>(s->arena.ptr(r->q_off));
    for (size_t x = r->next_long; x < r->longs.size() && t.cells < budget; ++x) {
      LongPair& p = r->longs[x];
      if (p.issued >= p.nst || p.busy) continue;
      if (p.nst > 1 && p.state_off == SIZE_MAX) {
        p.state_off = s->arena.alloc((size_t)p.cols * sizeof(float));
        if (p.state_off == SIZE_MAX) continue;   // no room for its row state in this tick
      }
      const float* cdev = pool.points + pool.offsets[r->ids[p.k]] * r->dim;
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
        t.outs.emplace_back(r, p.k);
      } else {
        it.out = -1;
      }
      t.cells += (double)(it.s1 - it.s0) / p.nst * p.rows * (double)p.cols;
      p.issued = it.s1;
      p.busy = true;
      t.longs_issued.push_back(&p);
      t.items.push_back(it);
      t.members.push_back(r);
      r->inflight++;
    }
    while (r->next_long < r->longs.size() && r->longs[r->next_long].issued >= r->longs[r->next_long].nst)
      r->next_long++;
    const int64_t n_short = (int64_t)r->order.size();
    if (r->next_short < n_short && t.cells < budget) {
      // the longest run of positions whose cells fit the budget left (at least one)
      const double* cp = r->cells_pre.data();
      const double want = cp[r->next_short] + (budget - t.cells);
      int64_t e = std::upper_bound(cp + r->next_short + 1, cp + n_short + 1, want) - cp - 1;
      e = std::max<int64_t>(e, r->next_short + 1);
      t.cells += cp[e] - cp[r->next_short];
      const int32_t* cids = reinterpret_cast<const int32_t*>(s->arena.ptr(r->cid_off));
      // one slice per class run inside [next_short, e)
      auto run = std::upper_bound(r->runs.begin(), r->runs.end(), (int)r->next_short,
                                  [](int pos, const ClassRun& c) { return pos < c.begin; }) - 1;
      for (int64_t a = r->next_short; a < e; ++run) {
        const int64_t run_end = (run + 1 == r->runs.end()) ? n_short : (run + 1)->begin;
        const int64_t b = std::min(e, run_end);
        SliceRec sr;
        sr.d.query = qdev;
        sr.d.cids = cids + a;
        sr.d.n = r->n;
        sr.d.count = (int)(b - a);
        sr.d.out_base = 0;
        sr.d.pad = 0;
        sr.r = r;
        sr.first = (int)a;
        sr.key = std::min(r->dim, MAX_DIM) * NCLS + run->cls;
        t.slices.push_back(sr);
        r->inflight++;
        a = b;
      }
      r->next_short = e;
    }
  }
  // One launch per dimension; inside it the items costliest first, then the
  // slices costliest class first (counting sorts, linear in the items).
  const size_t n_it = t.items.size();
  if (n_it > 1) {
    std::vector<int>& cnt = s->sort_count;
    cnt.assign((MAX_DIM + 1) * NCLS + 1, 0);
    std::vector<int>& key = s->sort_key;
    key.resize(n_it);
    for (size_t i = 0; i < n_it; ++i) {
      const Item& it = t.items[i];
      key[i] = std::min(it.dim, MAX_DIM) * NCLS +
               cost_rank((unsigned long long)(it.s1 - it.s0) * (unsigned long long)it.m *
                         (unsigned long long)std::min(it.n, 256));
      ++cnt[key[i] + 1];
    }
    for (size_t k = 1; k < cnt.size(); ++k) cnt[k] += cnt[k - 1];
    std::vector<Item>& out = s->sort_items;
    out.resize(n_it);
    for (size_t i = 0; i < n_it; ++i) out[cnt[key[i]]++] = t.items[i];
    t.items.swap(out);
  }
  const size_t n_sl = t.slices.size();
  if (n_sl > 1) {
    std::vector<int>& cnt = s->sort_count;
    cnt.assign((MAX_DIM + 1) * NCLS + 1, 0);
    for (const SliceRec& sr : t.slices) ++cnt[sr.key + 1];
    for (size_t k = 1; k < cnt.size(); ++k) cnt[k] += cnt[k - 1];
    std::vector<SliceRec>& out = s->sort_slices;
    out.resize(n_sl);
    for (const SliceRec& sr : t.slices) out[cnt[sr.key]++] = sr;
    t.slices.swap(out);
  }
  t.prefix.resize(n_sl + 1);
  t.prefix[0] = 0;
  const int n_item_outs = (int)t.outs.size();
  for (size_t j = 0; j < n_sl; ++j) {
    t.slices[j].d.out_base = n_item_outs + t.prefix[j];
    t.prefix[j + 1] = t.prefix[j] + t.slices[j].d.count;
  }
  t.n_outs = (size_t)n_item_outs + t.prefix[n_sl];
  t.off_slices = align16(n_it * sizeof(Item));
  t.off_prefix = t.off_slices + align16(n_sl * sizeof(Slice));
  t.desc_bytes = t.off_prefix + (n_sl + 1) * sizeof(int);
}

void launch_tick(dfd_server* s, Tick& t) {
  const size_t n_it = t.items.size(), n_sl = t.slices.size();
  t.slow_call_ms = 0;
  t.slow_call = 0;
  double tc = now_s();
  // the slowest CUDA call of the launch (host time), for the tick log
  auto mark = [&](int id) {
    const double x = now_s();
    if ((x - tc) * 1e3 > t.slow_call_ms) {
      t.slow_call_ms = (x - tc) * 1e3;
      t.slow_call = id;
    }
    tc = x;
  };
  if (n_it) std::memcpy(t.h_desc, t.items.data(), n_it * sizeof(Item));
  Slice* hs = reinterpret_cast<Slice*>(t.h_desc + t.off_slices);
  for (size_t j = 0; j < n_sl; ++j) hs[j] = t.slices[j].d;
  std::memcpy(t.h_desc + t.off_prefix, t.prefix.data(), (n_sl + 1) * sizeof(int));
  cudaStream_t st = t.stream[0];
  tc = now_s();
  cudaEventRecord(t.ev0, st);
  mark(1);
  // queries and ids admitted with earlier ticks were uploaded on their
  // streams: order this tick after those copies (not after their kernels)
  if (s->last_launched) cudaStreamWaitEvent(st, s->last_launched->ev_up, 0);
  mark(2);
  for (const auto& u : t.uploads) {
    cudaMemcpyAsync(s->arena.ptr(u.arena_off), t.h_stage + u.stage_off, u.bytes, cudaMemcpyHostToDevice, st);
    mark(3);
  }
  cudaEventRecord(t.ev_up, st);
  mark(1);
  if (n_it || n_sl) cudaMemcpyAsync(t.d_desc, t.h_desc, t.desc_bytes, cudaMemcpyHostToDevice, st);
  mark(4);
  cudaMemsetAsync(t.d_counter, 0, (MAX_DIM + 1) * sizeof(int), st);
  mark(5);
  cudaEventRecord(t.ev_fork, st);   // the tick's inputs are in place
  mark(1);
  const Item* d_items = reinterpret_cast<const Item*>(t.d_desc);
  const Slice* d_slices = reinterpret_cast<const Slice*>(t.d_desc + t.off_slices);
  const int* d_prefix = reinterpret_cast<const int*>(t.d_desc + t.off_prefix);
  int n_launch = 0;
  size_t ib = 0, sb = 0;
  while (ib < n_it || sb < n_sl) {
    // items and slices are both sorted by dim: take the smaller dim next
    const int di = ib < n_it ? t.items[ib].dim : MAX_DIM + 1;
    const int ds = sb < n_sl ? t.slices[sb].r->dim : MAX_DIM + 1;
    const int dim = std::min(di, ds);
    size_t ie = ib, se = sb;
    while (ie < n_it && t.items[ie].dim == dim) ++ie;
    while (se < n_sl && t.slices[se].r->dim == dim) ++se;
    const int lane = n_launch++ % NSTREAM;
    cudaStream_t ls = t.stream[lane];
    if (n_launch == 2) cudaStreamWaitEvent(ls, t.ev_fork, 0);
    mark(2);
    ServeArgs a;
    a.items = d_items + ib;
    a.n_items = (int)(ie - ib);
    a.n_slices = (int)(se - sb);
    a.slices = d_slices + sb;
    a.prefix = d_prefix + sb;
    const Pool& pool = *s->pools[dim];
    a.pool = pool.points;
    a.offsets = pool.d_offsets;
    a.dim = dim;
    const int dk = dim_class(dim);
    a.vec = (dim == dk && dk != 3) ? 1 : 0;
    a.counter = t.d_counter + dim;
    a.out = t.d_out;
    a.rowbuf = t.rowbuf[lane];
    const int64_t count = (int64_t)a.n_items + (t.prefix[se] - t.prefix[sb]);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((count + 7) / 8, 2 * (int64_t)s->ctx->num_sms));
#define DFD_SERVE_CASE(K)                                 \
  case K:                                                 \
    serve_kernel<K><<<blocks, 256, 0, ls>>>(a);           \
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
    mark(6);
    ib = ie;
    sb = se;
  }
  if (n_launch > 1) {
    cudaEventRecord(t.ev_join, t.stream[1]);
    cudaStreamWaitEvent(st, t.ev_join, 0);
    mark(7);
  }
  if (t.n_outs)
    cudaMemcpyAsync(t.h_out, t.d_out, t.n_outs * sizeof(float), cudaMemcpyDeviceToHost, st);
  mark(8);
  cudaEventRecord(t.ev1, st);
  mark(9);
  s->last_launched = &t;
  const double now = now_s();
  for (Request* r : t.members)
    if (r->t_launch == 0) r->t_launch = now;
  for (const SliceRec& sr : t.slices)
    if (sr.r->t_launch == 0) sr.r->t_launch = now;
  if (cudaGetLastError() != cudaSuccess) s->fatal = DFD_ERR_CUDA;
}

// Caller holds s->mu; the tick's ev1 has completed.
void retire_tick(dfd_server* s, Tick& t) {
  const double now = now_s();
  // device busy time: the union of the tick intervals (consecutive ticks
  // overlap; the previous tick's slot is not reused while this one retires)
  float ms = 0.f, ov = 0.f;
  if (cudaEventElapsedTime(&ms, t.ev0, t.ev1) == cudaSuccess) {
    if (!s->last_retired || cudaEventElapsedTime(&ov, t.ev0, s->last_retired->ev1) != cudaSuccess) ov = 0.f;
    s->busy_ms += ms - std::min(ms, std::max(ov, 0.f));
  }
  cudaGetLastError();
  s->last_retired = &t;
  s->n_ticks++;
  if (s->tick_log.size() < ((size_t)1 << 20)) {
    dfd_tick_record tr;
    tr.build_s = t.t_build;
    tr.launched_s = t.t_launched;
    tr.retired_s = now;
    tr.gpu_ms = ms;
    tr.cells = t.cells;
    tr.n_items = (int)t.items.size();
    tr.n_slices = (int)t.slices.size();
    tr.n_outs = (int)t.n_outs;
    tr.n_admitted = t.n_admitted;
    tr.admit_ms = (t.t_admitted - t.t_build) * 1e3;
    tr.build_ms = (t.t_built - t.t_admitted) * 1e3;
    tr.slow_call_ms = t.slow_call_ms;
    tr.slow_call = t.slow_call;
    tr.pad = 0;
    tr.sync_s = t.t_sync0;
    tr.synced_s = t.t_sync1;
    tr.locked_s = t.t_locked;
    s->tick_log.push_back(tr);
  }
  for (LongPair* p : t.longs_issued) p->busy = false;
  for (size_t i = 0; i < t.outs.size(); ++i) {
    Request* r = t.outs[i].first;
    if (!r->cancelled && r->host_out) r->host_out[t.outs[i].second] = t.h_out[i];
    r->remaining--;
  }
  for (Request* r : t.members) r->inflight--;
  bool bad = false;
  for (const SliceRec& sr : t.slices) {
    Request* r = sr.r;
    const float* v = t.h_out + sr.d.out_base;
    const int32_t* ord = r->order.data() + sr.first;
    if (!r->cancelled && r->host_out) {
      for (int li = 0; li < sr.d.count; ++li) {
        bad |= v[li] < 0.f;
        r->host_out[ord[li]] = v[li];
      }
    }
    r->remaining -= sr.d.count;
    r->inflight--;
  }
  if (bad && s->fatal == DFD_OK) s->fatal = DFD_ERR_CAPACITY;   // a pair the kernel refused (not planned so)
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
    if (s->inflight.size() < NTICK - 1) {
      t.t_build = now_s();
      const size_t before = s->active.size();
      admit(s, t);
      t.t_admitted = now_s();
      t.n_admitted = (int)(s->active.size() - before);
      build_tick(s, t);
      t.t_built = now_s();
      if (!t.items.empty() || !t.slices.empty() || !t.uploads.empty()) {
        if (!ensure_tick_capacity(t, t.desc_bytes, t.n_outs)) {
          s->fatal = DFD_ERR_OOM;
        } else {
          launch_tick(s, t);
          t.t_launched = now_s();
          s->inflight.push_back(&t);
          s->next_tick = (s->next_tick + 1) % NTICK;
          launched = true;
        }
      }
    }
    if (!s->inflight.empty() && (s->inflight.size() >= NTICK - 1 || !launched)) {
      Tick* old = s->inflight.front();
      lk.unlock();
      const double w0 = now_s();
      cudaEventSynchronize(old->ev1);
      const double w1 = now_s();
      lk.lock();
      old->t_sync0 = w0;
      old->t_sync1 = w1;
      old->t_locked = now_s();
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
  o->tick_cells = 4.0e9;
  o->stripes_per_tick = 8;
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
  bool ok = s->arena.init(o.mem_budget_bytes);
  for (auto& t : s->ticks) {
    for (int k = 0; k < NSTREAM; ++k) {
      ok = ok && cudaStreamCreateWithFlags(&t.stream[k], cudaStreamNonBlocking) == cudaSuccess;
      ok = ok && cudaMalloc(&t.rowbuf[k], max_tick_warps(s) * batch::BUF_COLS * sizeof(float)) == cudaSuccess;
    }
    ok = ok && cudaEventCreateWithFlags(&t.ev_fork, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&t.ev_join, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreate(&t.ev0) == cudaSuccess && cudaEventCreate(&t.ev1) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&t.ev_up, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMalloc(&t.d_counter, (MAX_DIM + 1) * sizeof(int)) == cudaSuccess;
    ok = ok && cudaMallocHost(&t.h_stage, STAGE_BYTES) == cudaSuccess;
    // descriptors and results for ticks of up to ~256K pairs from the start:
    // growing them later allocates (synchronising) inside a tick's latency
    ok = ok && ensure_tick_capacity(t, (size_t)1 << 20, (size_t)1 << 18);
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
  for (auto& t : s->ticks)
    for (cudaStream_t x : t.stream)
      if (x) cudaStreamSynchronize(x);
  for (auto& t : s->ticks) {
    if (t.h_desc) cudaFreeHost(t.h_desc);
    if (t.h_out) cudaFreeHost(t.h_out);
    if (t.d_desc) cudaFree(t.d_desc);
    if (t.d_out) cudaFree(t.d_out);
    if (t.d_counter) cudaFree(t.d_counter);
    if (t.h_stage) cudaFreeHost(t.h_stage);
    if (t.ev0) cudaEventDestroy(t.ev0);
    if (t.ev1) cudaEventDestroy(t.ev1);
    if (t.ev_up) cudaEventDestroy(t.ev_up);
    if (t.ev_fork) cudaEventDestroy(t.ev_fork);
    if (t.ev_join) cudaEventDestroy(t.ev_join);
    for (int k = 0; k < NSTREAM; ++k) {
      if (t.rowbuf[k]) cudaFree(t.rowbuf[k]);
      if (t.stream[k]) cudaStreamDestroy(t.stream[k]);
    }
  }
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
  if ((int64_t)pool.offsets.size() - 1 + n_curves > INT32_MAX) return DFD_ERR_UNSUPPORTED;   // ids travel as int32
  const int64_t old_pts = pool.offsets.back();
  // grow: new device arrays with old + new curves (the worker launches no
  // tick while we hold the lock; the ticks in flight finish before the old
  // arrays are freed, and the copies finish before the lock is released)
  float* grown = nullptr;
  if (cudaMalloc(&grown, (size_t)(old_pts + npts) * dim * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return DFD_ERR_OOM;
  }
  for (auto& t : s->ticks)   // ticks in flight read the old arrays
    for (cudaStream_t x : t.stream) cudaStreamSynchronize(x);
  if (pool.points) cudaMemcpy(grown, pool.points, (size_t)old_pts * dim * sizeof(float), cudaMemcpyDeviceToDevice);
  cudaMemcpy(grown + old_pts * dim, host_points, (size_t)npts * dim * sizeof(float), cudaMemcpyHostToDevice);
  if (pool.points) cudaFree(pool.points);
  pool.points = grown;
  const size_t old_curves = pool.offsets.size() - 1;
  for (int64_t c = 0; c < n_curves; ++c) pool.offsets.push_back(old_pts + host_offsets[c + 1]);
  int64_t* offs = nullptr;
  if (cudaMalloc(&offs, pool.offsets.size() * sizeof(int64_t)) != cudaSuccess) {
    cudaGetLastError();
    pool.offsets.resize(old_curves + 1);
    return DFD_ERR_OOM;
  }
  cudaMemcpy(offs, pool.offsets.data(), pool.offsets.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
  cudaStreamSynchronize(0);
  if (pool.d_offsets) cudaFree(pool.d_offsets);
  pool.d_offsets = offs;
  if (first_id) *first_id = (int64_t)old_curves;
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
  r->t_submit = now_s();
  r->t_arrival = arrival_s >= 0 ? arrival_s : r->t_submit;
  std::lock_guard<std::mutex> lk(s->mu);
  r->t_locked = now_s();
  if (s->fatal != DFD_OK) return s->fatal;
  auto pit = s->pools.find(dim);
  if (pit == s->pools.end()) return DFD_ERR_INVALID_ARG;
  const int64_t ncand = (int64_t)pit->second->offsets.size() - 1;
  for (int64_t i = 0; i < k; ++i)
    if (cand_ids[i] < 0 || cand_ids[i] >= ncand) return DFD_ERR_INVALID_ARG;
  const size_t qb = (size_t)n * dim * sizeof(float);
  if (qb > s->opt.mem_budget_bytes / 2) return DFD_ERR_BUSY;   // never admissible
  if (align16(qb) + align16(std::max<size_t>((size_t)k * sizeof(int32_t), 16)) > STAGE_BYTES)
    return DFD_ERR_CAPACITY;
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
  s->log.clear();
  s->tick_log.clear();
  return DFD_OK;
}

dfd_status dfd_server_tick_log(dfd_server* s, dfd_tick_record* out, int64_t cap, int64_t* n) {
  if (!s || !n || cap < 0 || (cap > 0 && !out)) return DFD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  const int64_t m = std::min<int64_t>(cap, (int64_t)s->tick_log.size());
  if (m > 0) std::memcpy(out, s->tick_log.data(), (size_t)m * sizeof(dfd_tick_record));
  *n = (int64_t)s->tick_log.size();
  return DFD_OK;
}

dfd_status dfd_server_request_log(dfd_server* s, dfd_request_record* out, int64_t cap, int64_t* n) {
  if (!s || !n || cap < 0 || (cap > 0 && !out)) return DFD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  const int64_t m = std::min<int64_t>(cap, (int64_t)s->log.size());
  if (m > 0) std::memcpy(out, s->log.data(), (size_t)m * sizeof(dfd_request_record));
  *n = (int64_t)s->log.size();
  return DFD_OK;
}

double dfd_server_now(dfd_server* s) {
  (void)s;
  return now_s();
}

}  // extern "C"
