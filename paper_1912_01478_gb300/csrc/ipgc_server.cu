// Colouring server: continuous batching of independent requests.
//
// A request (a host CSR graph) is copied into pinned staging at submission
// and waits in a FIFO. A scheduler thread admits requests while the device
// arena (the HBM budget, one allocation) has room for the request's graph,
// colours and working set, and copies them in on a copy stream. Whenever
// one of `inflight` batch slots is free, every admitted request is coloured
// in one batched launch on that slot's stream (the phases of a single-graph
// colouring, so every result is the one the graph gets alone); slots run
// concurrently, and requests admitted while batches are running start in the
// next free slot. Each request completes on its own: the team that colours it
// writes the colours and the control block straight into pinned staging
// through its device mapping and then raises the request's flag, which the
// scheduler polls, so a small request does not wait for a large one in the
// same launch; its device memory returns to the arena at once, so waiting
// requests are admitted as memory frees up.
//
// Batches run as ordinary launches of at most 1/inflight of the device's
// resident CTAs each, so all CTAs of every in-flight batch fit on the GPU at
// the same time and the bounded team barriers always complete. Unless
// rescanning is asked for, every launch runs the pushing batched kernel
// (forbidden-colour bitmaps, as ipgc_color_batched), which also colours, by
// rescanning, the graphs without a node above t1: one kernel per launch, so
// a small request never waits for another kernel of its launch.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ipgc_internal.h"

using ipgc::Ctrl;
using ipgc::Params;

namespace {

using Clock = std::chrono::steady_clock;

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

// First-fit allocator over [0, cap) in 256-byte units, coalescing on free.
class Arena {
 public:
  void reset(size_t cap) {
    cap_ = cap;
    used_ = 0;
    peak_ = 0;
    free_.clear();
    if (cap) free_[0] = cap;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = al256(bytes ? bytes : 1);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = al256(bytes ? bytes : 1);
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
  size_t cap() const { return cap_; }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  size_t cap_ = 0, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;
};

enum class St { Pending, Ready, Running, Done, Failed };

struct Request {
  int32_t n = 0;
  int64_t nnz = 0;
  size_t h_off = 0, h_bytes = 0;  // staging: rowptr, col, colours (colours only by reference)
  size_t h_colors = 0;            // offset of the colours inside the staging block
  const int32_t* ref_rowptr = nullptr;  // caller's arrays (submission by reference)
  const int32_t* ref_col = nullptr;
  size_t d_off = 0, d_bytes = 0;  // device: rowptr, col, colours, working set
  St st = St::Pending;
  Clock::time_point t_submit, t_done;
  ipgc_stats stats{};
  int err = IPGC_OK;
};

struct Slot {
  bool busy = false;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  Params* d_params = nullptr;
  int32_t* d_lists = nullptr;
  size_t lists_cap = 0;
  Ctrl* d_ctrl = nullptr;
  // pinned, written by the kernel through their device mappings: each
  // graph's control block and its completion flag
  Ctrl* h_ctrl = nullptr;
  int32_t* h_done = nullptr;
  Ctrl* m_ctrl = nullptr;
  int32_t* m_done = nullptr;
  std::vector<Params> params;
  std::vector<int32_t> lists;
  std::vector<uint64_t> tickets;
  std::vector<char> finished;  // ticket i already completed from its flag
};

// Per-request device layout (offsets from the request's block); with
// pushing also the bitmaps, the two list buffers, the list counts and state,
// the push queue, the winners, the push targets and the list rewrite queue
// (offsets 0 without).
struct DevLayout {
  size_t rowptr, col, colors, tent, wl0, wl1, it0, it1, its, gbits, done_a, done_d, flag;
  size_t pbits = 0, alist0 = 0, alist1 = 0, flen0 = 0, flen1 = 0, fst = 0, fdead = 0, pq = 0,
         pw = 0, pinfo = 0, rq = 0;
  size_t total;
  int64_t icap, gcap;
};

DevLayout dev_layout(int32_t n, int64_t nnz, int t1, int chunk, bool push) {
  DevLayout L;
  int64_t nbig = nnz / (t1 + 1);
  if (nbig > n) nbig = n;
  L.icap = nnz / chunk + nbig + 1;
  L.gcap = nnz / ((int64_t)chunk + 1) + 1;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += al256(bytes);
    return at;
  };
  L.rowptr = take(4 * ((size_t)n + 1));
  L.col = take(4 * (size_t)(nnz > 0 ? nnz : 1));
  L.colors = take(4 * (size_t)n);
  L.tent = take(4 * (size_t)n);
  L.wl0 = take(4 * (size_t)n);
  L.wl1 = take(4 * (size_t)n);
  L.it0 = take(16 * (size_t)L.icap);
  L.it1 = take(16 * (size_t)L.icap);
  L.its = take(16 * (size_t)L.icap);
  L.gbits = take(4 * (size_t)ipgc::kGWords * (size_t)L.gcap);
  L.done_a = take(4 * (size_t)L.gcap);
  L.done_d = take(4 * (size_t)L.gcap);
  L.flag = take(4 * (size_t)L.gcap);
  if (push) {  // as the batched workspace: 12 bytes per entry, 16 per node, ...
    const size_t e = (size_t)(nnz > 0 ? nnz : 1);
    L.pbits = take(4 * e);
    L.alist0 = take(4 * e);
    L.alist1 = take(4 * e);
    L.flen0 = take(8 * (size_t)L.gcap);
    L.flen1 = take(8 * (size_t)L.gcap);
    L.fst = take(4 * (size_t)L.gcap);
    L.fdead = take(4 * (size_t)L.gcap);
    L.pq = take(16 * (size_t)(nnz / ipgc::kPushChunk + 2 * nbig + 1));
    L.pw = take(4 * (size_t)n);
    L.pinfo = take(8 * (size_t)n);
    L.rq = take(16 * (size_t)(nnz / ipgc::kPushChunk + 2 * L.gcap + 1));
  }
  L.total = o;
  return L;
}

size_t host_bytes(int32_t n, int64_t nnz) {
  return al256(4 * ((size_t)n + 1)) + al256(4 * (size_t)(nnz > 0 ? nnz : 1)) + al256(4 * (size_t)n);
}

}  // namespace

struct ipgc_server {
  int device = 0;
  ipgc_server_options opt{};
  int t1 = 0, chunk = 0, bs = 256, grid = 0, max_team = 1;
  bool push = false;  // forbidden-colour bitmaps: every launch runs the pushing batched kernel
  char* d_arena = nullptr;
  char* h_arena = nullptr;  // pinned
  char* m_arena = nullptr;  // h_arena's device mapping
  Arena dev, host;
  cudaStream_t copy_stream = nullptr;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> pending, ready, done_q;
  std::unordered_map<uint64_t, Request> reqs;
  uint64_t next_ticket = 1;
  bool stop = false;
  int fatal = IPGC_OK;
  std::thread worker;
  // learned mode switch: the current network (nullptr: none); every network
  // loaded stays allocated until the server is destroyed, since launches in
  // flight may still read an earlier one
  const float* d_mlp = nullptr;
  std::vector<float*> mlp_bufs;
  // counters
  uint64_t n_submitted = 0, n_completed = 0, n_batches = 0, graphs_in_batches = 0;
  int32_t max_batch_seen = 0;
};

namespace {

void fail_all_locked(ipgc_server* S, int err) {
  S->fatal = err;
  for (auto& kv : S->reqs) {
    if (kv.second.st == St::Done || kv.second.st == St::Failed) continue;
    kv.second.st = St::Failed;
    kv.second.err = err;
    kv.second.t_done = Clock::now();
    S->done_q.push_back(kv.first);
  }
  S->pending.clear();
  S->ready.clear();
  S->cv_done.notify_all();
}

// One request's result is in staging: statistics from its control block,
// its device memory back to the arena (no CTA touches it any more).
void complete_locked(ipgc_server* S, uint64_t ticket, const Ctrl& c, int err) {
  Request& r = S->reqs[ticket];
  r.stats.rounds = c.rounds;
  r.stats.num_colors = c.maxc;
  r.stats.rounds_topo = c.rounds_topo;
  r.stats.rounds_data = c.rounds_data;
  r.stats.edges_processed = (int64_t)c.edges;
  r.stats.ns = c.t_end >= c.t_start ? c.t_end - c.t_start : 0;
  r.stats.error = err != IPGC_OK ? err : c.status;
  r.err = r.stats.error;
  r.st = r.err == IPGC_OK ? St::Done : St::Failed;
  r.t_done = Clock::now();
  S->dev.release(r.d_off, r.d_bytes);
  S->done_q.push_back(ticket);
  ++S->n_completed;
}

// Completes every graph whose flag is up, and frees the slots of finished
// launches; returns true when something changed.
bool reap_locked(ipgc_server* S) {
  bool any = false;
  for (Slot& sl : S->slots) {
    if (!sl.busy) continue;
    for (size_t i = 0; i < sl.tickets.size(); ++i) {
      if (sl.finished[i] || __atomic_load_n(sl.h_done + i, __ATOMIC_ACQUIRE) == 0) continue;
      complete_locked(S, sl.tickets[i], sl.h_ctrl[i], IPGC_OK);
      sl.finished[i] = 1;
      any = true;
    }
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) continue;
    sl.busy = false;
    any = true;
    // a finished launch has raised every flag; anything else is a failure
    for (size_t i = 0; i < sl.tickets.size(); ++i) {
      if (sl.finished[i]) continue;
      const bool up = q == cudaSuccess && __atomic_load_n(sl.h_done + i, __ATOMIC_ACQUIRE) != 0;
      complete_locked(S, sl.tickets[i], sl.h_ctrl[i], up ? IPGC_OK : IPGC_ERR_CUDA);
    }
    sl.tickets.clear();
    sl.finished.clear();
    if (q != cudaSuccess) {
      fail_all_locked(S, IPGC_ERR_CUDA);
      return true;
    }
  }
  if (any) S->cv_done.notify_all();
  return any;
}

// Admits pending requests in order while device memory lasts.
bool admit_locked(ipgc_server* S) {
  bool any = false;
  while (!S->pending.empty()) {
    Request& r = S->reqs[S->pending.front()];
    size_t off = 0;
    if (!S->dev.alloc(r.d_bytes, &off)) break;
    r.d_off = off;
    const DevLayout L = dev_layout(r.n, r.nnz, S->t1, S->chunk, S->push);
    char* dbase = S->d_arena + off;
    const char* hbase = S->h_arena + r.h_off;
    const void* src_rp = r.ref_rowptr ? (const void*)r.ref_rowptr : (const void*)hbase;
    const void* src_col = r.ref_rowptr ? (const void*)r.ref_col
                                       : (const void*)(hbase + al256(4 * ((size_t)r.n + 1)));
    cudaError_t e = cudaMemcpyAsync(dbase + L.rowptr, src_rp, 4 * ((size_t)r.n + 1),
                                    cudaMemcpyHostToDevice, S->copy_stream);
    if (e == cudaSuccess && r.nnz > 0)
      e = cudaMemcpyAsync(dbase + L.col, src_col, 4 * (size_t)r.nnz, cudaMemcpyHostToDevice,
                          S->copy_stream);
    if (e != cudaSuccess) {
      fail_all_locked(S, IPGC_ERR_CUDA);
      return true;
    }
    r.st = St::Ready;
    S->ready.push_back(S->pending.front());
    S->pending.pop_front();
    any = true;
  }
  return any;
}

// Launches the admitted requests in a free slot.
bool launch_locked(ipgc_server* S) {
  if (S->ready.empty()) return false;
  Slot* sl = nullptr;
  for (Slot& s : S->slots)
    if (!s.busy) {
      sl = &s;
      break;
    }
  if (!sl) return false;
  cudaEvent_t copied;
  if (cudaEventCreateWithFlags(&copied, cudaEventDisableTiming) != cudaSuccess) {
    fail_all_locked(S, IPGC_ERR_CUDA);
    return true;
  }
  const int32_t G = (int32_t)std::min<size_t>(S->ready.size(), (size_t)S->opt.max_batch_graphs);
  sl->tickets.assign(S->ready.begin(), S->ready.begin() + G);
  sl->finished.assign(G, 0);
  S->ready.erase(S->ready.begin(), S->ready.begin() + G);
  sl->params.resize(G);
  std::memset(sl->h_done, 0, sizeof(int32_t) * (size_t)G);  // the slot's last launch is over
  for (int32_t i = 0; i < G; ++i) {
    Request& r = S->reqs[sl->tickets[i]];
    r.st = St::Running;
    const DevLayout L = dev_layout(r.n, r.nnz, S->t1, S->chunk, S->push);
    char* b = S->d_arena + r.d_off;
    Params& p = sl->params[i];
    std::memset(&p, 0, sizeof(p));
    p.rowptr = (const int32_t*)(b + L.rowptr);
    p.col = (const int32_t*)(b + L.col);
    p.n = r.n;
    p.nnz = r.nnz;
    p.color = (int32_t*)(b + L.colors);
    p.tent = (int32_t*)(b + L.tent);
    p.wl[0] = (int32_t*)(b + L.wl0);
    p.wl[1] = (int32_t*)(b + L.wl1);
    p.items[0] = (int4*)(b + L.it0);
    p.items[1] = (int4*)(b + L.it1);
    p.istat = (int4*)(b + L.its);
    p.gbits = (uint32_t*)(b + L.gbits);
    p.done_a = (int32_t*)(b + L.done_a);
    p.done_d = (int32_t*)(b + L.done_d);
    p.flag = (int32_t*)(b + L.flag);
    p.ctrl = sl->d_ctrl + i;
    p.t1 = S->t1;
    p.chunk = S->chunk;
    const double h = (double)S->opt.batch.base.threshold_frac * (double)r.n;
    p.H = (int64_t)(h > 0 ? h : 0);
    p.policy = S->opt.batch.base.mode;
    // the network loaded by ipgc_server_policy_load (none: the threshold rule)
    p.mlp = p.policy == IPGC_MODE_LEARNED ? S->d_mlp : nullptr;
    p.mlp_margin = S->opt.batch.base.policy_margin;
    p.max_rounds = r.n + 1;
    p.timeout_ns = S->opt.batch.base.timeout_ns ? S->opt.batch.base.timeout_ns : 10000000000ull;
    p.col_vec = 1;  // arena blocks are 256-byte aligned
    // the team publishes the result straight into staging (256-byte aligned)
    p.out_colors = (int32_t*)(S->m_arena + r.h_off + r.h_colors);
    p.out_ctrl = sl->m_ctrl + i;
    p.out_done = sl->m_done + i;
    if (S->push) {  // a graph's bitmaps and lists, in its own block
      p.push_stay = 1;  // one kernel per launch: graphs without bitmaps rescan in it
      p.pbits = (uint32_t*)(b + L.pbits);
      p.alist[0] = (int32_t*)(b + L.alist0);
      p.alist[1] = (int32_t*)(b + L.alist1);
      p.flen[0] = (int2*)(b + L.flen0);
      p.flen[1] = (int2*)(b + L.flen1);
      p.fst = (int32_t*)(b + L.fst);
      p.fdead = (int32_t*)(b + L.fdead);
      p.pq = (int4*)(b + L.pq);
      p.pw = (int32_t*)(b + L.pw);
      p.pinfo = (int2*)(b + L.pinfo);
      p.rq = (int4*)(b + L.rq);
    }
  }
  int rc = IPGC_OK;
  cudaError_t e = cudaEventRecord(copied, S->copy_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(sl->stream, copied, 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(sl->d_ctrl, 0, sizeof(Ctrl) * (size_t)G, sl->stream);
  if (e == cudaSuccess)
    e = ipgc::schedule_and_launch(sl->params.data(), G, S->bs, S->grid, S->max_team,
                                  S->opt.batch.nnz_per_cta, false, sl->d_params, sl->d_lists,
                                  sl->lists_cap, sl->lists, sl->stream, &rc, S->push);
  if (e == cudaSuccess) e = cudaEventRecord(sl->done, sl->stream);
  cudaEventDestroy(copied);
  if (e != cudaSuccess || rc != IPGC_OK) {
    fail_all_locked(S, e != cudaSuccess ? IPGC_ERR_CUDA : rc);
    return true;
  }
  sl->busy = true;
  ++S->n_batches;
  S->graphs_in_batches += (uint64_t)G;
  S->max_batch_seen = std::max(S->max_batch_seen, G);
  return true;
}

void worker_main(ipgc_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    bool progress = false;
    if (S->fatal == IPGC_OK) {
      progress |= reap_locked(S);
      progress |= admit_locked(S);
      progress |= launch_locked(S);
    }
    bool busy = false;
    for (const Slot& s : S->slots) busy |= s.busy;
    if (S->stop && !busy) break;
    if (progress) continue;
    // idle: poll in-flight batches often, otherwise wait for a submission
    if (busy || !S->ready.empty())
      S->cv_work.wait_for(lk, std::chrono::microseconds(20));
    else
      S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
  }
}

void destroy_resources(ipgc_server* S) {
  cudaSetDevice(S->device);
  for (Slot& s : S->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.done) cudaEventDestroy(s.done);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.d_params) cudaFree(s.d_params);
    if (s.h_ctrl) cudaFreeHost(s.h_ctrl);
    if (s.h_done) cudaFreeHost(s.h_done);
  }
  if (S->copy_stream) {
    cudaStreamSynchronize(S->copy_stream);
    cudaStreamDestroy(S->copy_stream);
  }
  if (S->d_arena) cudaFree(S->d_arena);
  if (S->h_arena) cudaFreeHost(S->h_arena);
  for (float* b : S->mlp_bufs) cudaFree(b);
  S->mlp_bufs.clear();
}

}  // namespace

extern "C" {

void ipgc_server_options_default(ipgc_server_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->hbm_budget = (size_t)8 << 30;
  o->host_budget = (size_t)4 << 30;
  o->inflight = 2;
  o->max_batch_graphs = 1024;
  o->max_pending = 1 << 16;
  ipgc_batch_options_default(&o->batch);
}

int ipgc_server_create(ipgc_server** out, int device, const ipgc_server_options* opt) {
  if (!out) return IPGC_ERR_INVALID;
  *out = nullptr;
  ipgc_server_options o;
  if (opt)
    o = *opt;
  else
    ipgc_server_options_default(&o);
  if (o.inflight < 1 || o.inflight > 8 || o.max_batch_graphs < 1 || o.max_pending < 1 ||
      o.hbm_budget < 4096 || o.host_budget < 4096 || o.batch.max_team < 0 ||
      o.batch.nnz_per_cta < 1 || o.batch.base.forbidden < IPGC_FORBIDDEN_AUTO ||
      o.batch.base.forbidden > IPGC_FORBIDDEN_PUSH)
    return IPGC_ERR_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return IPGC_ERR_INVALID;
  if (cudaSetDevice(device) != cudaSuccess) return IPGC_ERR_CUDA;
  ipgc_server* S = new (std::nothrow) ipgc_server();
  if (!S) return IPGC_ERR_OOM;
  S->device = device;
  S->opt = o;
  S->t1 = ipgc::effective_t1(o.batch.base);
  S->chunk = ipgc::effective_chunk(o.batch.base);
  S->bs = o.batch.base.block_size ? o.batch.base.block_size : ipgc::kBlock;
  S->push = o.batch.base.forbidden != IPGC_FORBIDDEN_RESCAN;
  int occ = 0, pocc = 0, sms = 0;
  int rc = IPGC_OK;
  if (ipgc::occupancy_batched(S->bs, &occ) != cudaSuccess ||
      (S->push && ipgc::occupancy_batched(S->bs, &pocc, true) != cudaSuccess) ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    rc = IPGC_ERR_CUDA;
  // with pushing every launch runs the pushing kernel (graphs without a node
  // above t1 rescan inside it), whose occupancy sizes the slots
  if (S->push) occ = pocc;
  S->grid = occ * sms / o.inflight;
  // largest team: max_team (0: the grid), at most the grid
  S->max_team = o.batch.max_team > 0 && o.batch.max_team < S->grid ? o.batch.max_team : S->grid;
  if (S->max_team < 1) S->max_team = 1;
  if (rc == IPGC_OK && S->grid < 1) rc = IPGC_ERR_UNSUPPORTED;
  if (rc == IPGC_OK && cudaMalloc((void**)&S->d_arena, o.hbm_budget) != cudaSuccess) rc = IPGC_ERR_OOM;
  if (rc == IPGC_OK && cudaMallocHost((void**)&S->h_arena, o.host_budget) != cudaSuccess)
    rc = IPGC_ERR_OOM;
  if (rc == IPGC_OK && cudaHostGetDevicePointer((void**)&S->m_arena, S->h_arena, 0) != cudaSuccess)
    rc = IPGC_ERR_CUDA;
  if (rc == IPGC_OK &&
      cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
    rc = IPGC_ERR_CUDA;
  S->slots.resize(o.inflight);
  for (Slot& s : S->slots) {
    if (rc != IPGC_OK) break;
    s.lists_cap = ipgc::schedule_lists_bound(o.max_batch_graphs, S->grid, S->max_team);
    const size_t b_params = al256(sizeof(Params) * (size_t)o.max_batch_graphs);
    const size_t b_lists = al256(sizeof(int32_t) * s.lists_cap);
    const size_t b_ctrl = al256(sizeof(Ctrl) * (size_t)o.max_batch_graphs);
    char* base = nullptr;
    if (cudaMalloc((void**)&base, b_params + b_lists + b_ctrl) != cudaSuccess ||
        cudaMallocHost((void**)&s.h_ctrl, sizeof(Ctrl) * (size_t)o.max_batch_graphs) != cudaSuccess ||
        cudaMallocHost((void**)&s.h_done, sizeof(int32_t) * (size_t)o.max_batch_graphs) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&s.m_ctrl, s.h_ctrl, 0) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&s.m_done, s.h_done, 0) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
      if (base) cudaFree(base);
      rc = IPGC_ERR_OOM;
      break;
    }
    s.d_params = (Params*)base;
    s.d_lists = (int32_t*)(base + b_params);
    s.d_ctrl = (Ctrl*)(base + b_params + b_lists);
  }
  if (rc != IPGC_OK) {
    destroy_resources(S);
    delete S;
    return rc;
  }
  S->dev.reset(o.hbm_budget);
  S->host.reset(o.host_budget);
  S->worker = std::thread(worker_main, S);
  *out = S;
  return IPGC_OK;
}

}  // extern "C"

namespace {

int submit_impl(ipgc_server* S, const int32_t* h_rowptr, const int32_t* h_col, int32_t n,
                int64_t nnz, uint64_t* ticket, bool by_ref) {
  if (!S || !ticket || n < 0 || nnz < 0 || nnz > INT32_MAX || n == INT32_MAX) return IPGC_ERR_INVALID;
  if ((n > 0 && !h_rowptr) || (nnz > 0 && !h_col) || (nnz > 0 && n == 0)) return IPGC_ERR_INVALID;
  if (n > 0 && (h_rowptr[0] != 0 || (int64_t)h_rowptr[n] != nnz)) return IPGC_ERR_INVALID;
  if (S->opt.batch.base.validate &&
      ipgc_validate_csr(nullptr, h_rowptr, h_col, n, nnz, 0, nullptr) != IPGC_OK)
    return IPGC_ERR_INVALID;
  const size_t hb = by_ref ? al256(4 * (size_t)(n > 0 ? n : 1)) : host_bytes(n, nnz);
  const size_t db = dev_layout(n, nnz, S->t1, S->chunk, S->push).total;
  if (hb > S->host.cap() || db > S->dev.cap()) return IPGC_ERR_TOO_LARGE;
  size_t h_off = 0;
  uint64_t t = 0;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->fatal != IPGC_OK) return S->fatal;
    if (S->stop) return IPGC_ERR_INVALID;
    if ((int64_t)S->pending.size() >= S->opt.max_pending) return IPGC_ERR_BUSY;
    if (!S->host.alloc(hb, &h_off)) return IPGC_ERR_BUSY;
    t = S->next_ticket++;
    Request& r = S->reqs[t];
    r.n = n;
    r.nnz = nnz;
    r.h_off = h_off;
    r.h_bytes = hb;
    r.h_colors = by_ref ? 0
                        : al256(4 * ((size_t)n + 1)) + al256(4 * (size_t)(nnz > 0 ? nnz : 1));
    r.d_bytes = db;
    r.st = St::Pending;
    r.t_submit = Clock::now();
    if (by_ref) {
      r.ref_rowptr = h_rowptr;
      r.ref_col = h_col;
    }
  }
  if (!by_ref) {  // copy the graph into staging outside the lock (the block is ours)
    char* hb_base = S->h_arena + h_off;
    if (n > 0) std::memcpy(hb_base, h_rowptr, 4 * ((size_t)n + 1));
    if (nnz > 0) std::memcpy(hb_base + al256(4 * ((size_t)n + 1)), h_col, 4 * (size_t)nnz);
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    Request& r = S->reqs[t];
    if (n == 0) {  // nothing to colour
      r.st = St::Done;
      r.t_done = Clock::now();
      S->done_q.push_back(t);
      ++S->n_completed;
      S->cv_done.notify_all();
    } else {
      S->pending.push_back(t);
    }
    ++S->n_submitted;
  }
  S->cv_work.notify_one();
  *ticket = t;
  return IPGC_OK;
}

}  // namespace

extern "C" {

int ipgc_server_submit(ipgc_server* S, const int32_t* h_rowptr, const int32_t* h_col, int32_t n,
                       int64_t nnz, uint64_t* ticket) {
  return submit_impl(S, h_rowptr, h_col, n, nnz, ticket, false);
}

int ipgc_server_submit_ref(ipgc_server* S, const int32_t* h_rowptr, const int32_t* h_col,
                           int32_t n, int64_t nnz, uint64_t* ticket) {
  return submit_impl(S, h_rowptr, h_col, n, nnz, ticket, true);
}

int ipgc_server_poll(ipgc_server* S, uint64_t ticket, int32_t* h_colors, ipgc_stats* stats,
                     int64_t* latency_ns) {
  if (!S) return IPGC_ERR_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return IPGC_ERR_NOT_FOUND;
  Request& r = it->second;
  if (r.st != St::Done && r.st != St::Failed) return IPGC_PENDING;
  const int err = r.st == St::Done ? IPGC_OK : (r.err != IPGC_OK ? r.err : IPGC_ERR_CUDA);
  if (err == IPGC_OK && h_colors && r.n > 0)
    std::memcpy(h_colors, S->h_arena + r.h_off + r.h_colors, 4 * (size_t)r.n);
  if (stats) *stats = r.stats;
  if (latency_ns)
    *latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(r.t_done - r.t_submit).count();
  S->host.release(r.h_off, r.h_bytes);
  S->reqs.erase(it);
  return err;
}

int ipgc_server_next_done(ipgc_server* S, uint64_t* ticket, uint64_t timeout_ns) {
  if (!S || !ticket) return IPGC_ERR_INVALID;
  std::unique_lock<std::mutex> lk(S->mu);
  // tickets already released by ipgc_server_poll are skipped
  auto drop_released = [&] {
    while (!S->done_q.empty() && S->reqs.find(S->done_q.front()) == S->reqs.end())
      S->done_q.pop_front();
    return !S->done_q.empty();
  };
  const bool got =
      S->cv_done.wait_for(lk, std::chrono::nanoseconds(timeout_ns), drop_released);
  if (!got) return IPGC_PENDING;
  *ticket = S->done_q.front();
  S->done_q.pop_front();
  return IPGC_OK;
}

int ipgc_server_query(ipgc_server* S, ipgc_server_counters* c) {
  if (!S || !c) return IPGC_ERR_INVALID;
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(c, 0, sizeof(*c));
  c->submitted = S->n_submitted;
  c->completed = S->n_completed;
  c->batches = S->n_batches;
  c->graphs_in_batches = S->graphs_in_batches;
  c->pending = (int64_t)S->pending.size();
  c->ready = (int64_t)S->ready.size();
  int busy = 0;
  for (const Slot& s : S->slots) busy += s.busy;
  c->running_batches = busy;
  c->max_batch = S->max_batch_seen;
  c->hbm_used = (int64_t)S->dev.used();
  c->hbm_peak = (int64_t)S->dev.peak();
  c->host_used = (int64_t)S->host.used();
  c->status = S->fatal;
  return IPGC_OK;
}

int ipgc_server_policy_load(ipgc_server* S, const float* w, int32_t len) {
  if (!S || len < 0 || (len > 0 && (!w || len != ipgc::kMlpParams))) return IPGC_ERR_INVALID;
  if (len == 0) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->d_mlp = nullptr;
    return IPGC_OK;
  }
  // a buffer of its own (launches in flight keep reading the previous one),
  // filled before it is handed to the scheduler
  float* buf = nullptr;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(S->device) != cudaSuccess) return IPGC_ERR_CUDA;
  int rc = IPGC_OK;
  if (cudaMalloc((void**)&buf, sizeof(float) * (size_t)len) != cudaSuccess)
    rc = IPGC_ERR_OOM;
  else if (cudaMemcpy(buf, w, sizeof(float) * (size_t)len, cudaMemcpyHostToDevice) != cudaSuccess)
    rc = IPGC_ERR_CUDA;
  cudaSetDevice(prev);
  if (rc != IPGC_OK) {
    if (buf) cudaFree(buf);
    return rc;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  S->mlp_bufs.push_back(buf);
  S->d_mlp = buf;
  return IPGC_OK;
}

int ipgc_server_destroy(ipgc_server* S) {
  if (!S) return IPGC_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->pending.clear();  // not admitted: dropped
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  destroy_resources(S);
  delete S;
  return IPGC_OK;
}

}  // extern "C"
