// Batched hybrid IPGC: thousands of independent graphs in one persistent
// cooperative launch.
//
// Every graph runs its own round loop (its own worklists, round counter, mode
// decision and control block) with exactly the single-graph phases of
// ipgc_phases.cuh, so each graph's colours equal those of colouring it alone.
// A graph with many entries is coloured by a team of CTAs (a power of two in
// size, growing with the graph) that separate its rounds with a bounded team
// barrier; the host gang-schedules the teams onto aligned blocks of CTAs.
// Every other graph is coloured by a single CTA that takes graphs, largest
// first, from a shared counter once its own team jobs are done, so the short
// graphs fill the tail.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <queue>
#include <vector>

#include "ipgc_internal.h"
#include "ipgc_phases.cuh"

namespace ipgc {

struct BatchParams {
  const Params* params;       // [G] per-graph parameters
  const int4* jobs;           // {graph, rank in its team, team size, 0}
  const int32_t* cta_off;     // CTA c runs jobs[cta_off[c] .. cta_off[c + 1]) in order
  const int32_t* solo_list;   // graphs coloured by one CTA each, largest first
  int32_t nsolo;
  int32_t* solo_next;         // shared counter over solo_list (zeroed before launch)
};

// Every CTA first runs its own list of team jobs. The lists are cut from one
// global job order, so the team of the earliest unfinished job can always
// meet at its barriers and no two teams wait on each other in a cycle. Then
// every CTA takes single-CTA graphs from the shared counter.
// The jobs of one CTA, then single-CTA graphs from the shared counter. With
// PUSH every graph is coloured with forbidden-colour bitmaps (Params::pbits),
// except those without a node above t1, which it leaves to the rescanning
// kernel launched after it (ctrl->push_off); without PUSH a graph given
// bitmaps is skipped unless the pushing kernel left it.
template <int BS, bool PUSH>
__device__ __forceinline__ void batched_jobs(const BatchParams& bp, Smem<BS>& sm, int* s_k) {
  // one call site of the round loop (two inlined copies cost registers)
  int j = bp.cta_off[blockIdx.x];
  const int jend = bp.cta_off[blockIdx.x + 1];
  for (;;) {
    int g;
    Team tm{0, 1};
    if (j < jend) {
      const int4 jb = bp.jobs[j++];
      g = jb.x;
      tm = Team{jb.y, jb.z};
    } else {
      __syncthreads();
      if (threadIdx.x == 0) *s_k = atomicAdd(bp.solo_next, 1);
      __syncthreads();
      const int k = *s_k;
      if (k >= bp.nsolo) break;
      g = bp.solo_list[k];
    }
    const Params& gp = bp.params[g];
    if (!PUSH && gp.pbits && ld_cg(&gp.ctrl->push_off) == 0) continue;  // coloured by pushing
    color_graph<BS, PUSH>(gp, sm, tm);
  }
}

template <int BS>
__global__ void __launch_bounds__(BS, min_blocks(BS)) batched_kernel(BatchParams bp) {
  __shared__ Smem<BS> sm;
  __shared__ int s_k;
  smem_clear<BS>(sm, 1);  // (the pushing batched kernel counts on counter 0)
  batched_jobs<BS, false>(bp, sm, &s_k);
}

// The pushing instantiation keeps 3 CTAs of 256 per SM (80 registers), as the
// single-graph pushing kernel does.
constexpr int batched_push_min_blocks(int bs) { return bs >= 512 ? 2 : 3; }

template <int BS>
__global__ void __launch_bounds__(BS, batched_push_min_blocks(BS)) batched_push_kernel(BatchParams bp) {
  __shared__ Smem<BS> sm;
  __shared__ int s_k;
  smem_clear<BS>(sm);
  batched_jobs<BS, true>(bp, sm, &s_k);
}

cudaError_t occupancy_batched(int bs, int* blocks_per_sm, bool push) {
  return with_block(bs, [&](auto B) {
    return push ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      blocks_per_sm, batched_push_kernel<decltype(B)::value>, decltype(B)::value, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      blocks_per_sm, batched_kernel<decltype(B)::value>, decltype(B)::value, 0);
  });
}

cudaError_t launch_batched(const BatchParams& bp, int bs, int blocks, bool cooperative,
                           cudaStream_t s, bool push) {
  return with_block(bs, [&](auto B) {
    BatchParams q = bp;
    const void* k = push ? (const void*)batched_push_kernel<decltype(B)::value>
                         : (const void*)batched_kernel<decltype(B)::value>;
    if (!cooperative) {
      if (push)
        batched_push_kernel<decltype(B)::value><<<blocks, decltype(B)::value, 0, s>>>(q);
      else
        batched_kernel<decltype(B)::value><<<blocks, decltype(B)::value, 0, s>>>(q);
      return cudaGetLastError();
    }
    void* args[] = {&q};
    return cudaLaunchCooperativeKernel(k, dim3(blocks), dim3(decltype(B)::value), args, 0, s);
  });
}

// Schedule of a batch on `grid` CTAs. A graph's team size k is the smallest
// power of two with k * nnz_per_cta >= nnz, or cap = min(max_team (0: the
// grid), grid) when that power is larger (cap itself need not be a power of
// two, so the largest graphs can use every CTA). Graphs with k = 1 go to the
// shared single-CTA queue, largest first. The others are gang-scheduled
// largest team first, then largest work first: each takes the block of k
// consecutive CTAs starting at a multiple of k whose busiest CTA is least
// loaded, and every CTA of the block is then busy until that load plus the
// graph's work / k (work = n + nnz). Since larger teams come first and all
// smaller sizes are powers of two, every candidate block is evenly loaded
// when a team is placed, so no CTA idles waiting for its team. Jobs are
// appended to the CTAs' lists in this one global order. Lists layout
// (int32): jobs as int4 (16-byte aligned first), cta_off[grid + 1], solo
// list, queue counter.
void build_schedule(const Params* h_params, int32_t G, int grid, int max_team,
                    int64_t nnz_per_cta, std::vector<int32_t>& lists, int32_t* njobs_out,
                    int32_t* nsolo_out, int32_t* seq_out) {
  const int cap = max_team > 0 && max_team < grid ? max_team : grid;
  std::vector<int32_t> order(G);
  std::iota(order.begin(), order.end(), 0);
  std::vector<int32_t> team(G, 0);
  for (int32_t g = 0; g < G; ++g) {
    if (h_params[g].n == 0) continue;
    const int64_t need = nnz_per_cta > 0 ? (h_params[g].nnz + nnz_per_cta - 1) / nnz_per_cta : 1;
    int64_t k = 1;
    while (k < need && k < cap) k *= 2;
    team[g] = (int32_t)std::min<int64_t>(k, cap);
  }
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    if (team[a] != team[b]) return team[a] > team[b];
    return h_params[a].nnz + h_params[a].n > h_params[b].nnz + h_params[b].n;
  });
  std::vector<double> load(grid, 0.0);
  std::vector<std::vector<int4>> per_cta(grid);
  std::vector<int32_t> solo;
  int32_t njobs = 0, nteam = 0;
  for (int32_t g : order) {
    const int k = team[g];
    if (seq_out) seq_out[g] = -1;
    if (k == 0) continue;
    if (k == 1) {
      if (seq_out) seq_out[g] = (int32_t)solo.size();
      solo.push_back(g);
      continue;
    }
    if (seq_out) seq_out[g] = nteam;
    ++nteam;
    int best = 0;
    double best_start = 1e300;
    for (int b = 0; b + k <= grid; b += k) {
      double m = 0;
      for (int c = b; c < b + k; ++c) m = std::max(m, load[c]);
      if (m < best_start) {
        best_start = m;
        best = b;
      }
    }
    const double finish = best_start + (double)(h_params[g].nnz + h_params[g].n) / k;
    for (int c = best; c < best + k; ++c) {
      load[c] = finish;
      per_cta[c].push_back(make_int4(g, c - best, k, 0));
    }
    njobs += k;
  }
  lists.clear();
  lists.reserve(4 * (size_t)njobs + grid + 1 + solo.size() + 1);
  std::vector<int32_t> cta_off(grid + 1, 0);
  for (int c = 0; c < grid; ++c) {
    cta_off[c + 1] = cta_off[c] + (int32_t)per_cta[c].size();
    for (const int4& j : per_cta[c]) {
      lists.push_back(j.x);
      lists.push_back(j.y);
      lists.push_back(j.z);
      lists.push_back(j.w);
    }
  }
  lists.insert(lists.end(), cta_off.begin(), cta_off.end());
  lists.insert(lists.end(), solo.begin(), solo.end());
  lists.push_back(0);  // solo queue counter
  *njobs_out = njobs;
  *nsolo_out = (int32_t)solo.size();
}

namespace {

// The kernel arguments of a schedule uploaded to d_lists (see build_schedule).
BatchParams batch_params(const Params* d_params, int32_t* d_lists, int32_t njobs, int32_t nsolo,
                         int grid) {
  BatchParams bp;
  bp.params = d_params;
  bp.jobs = reinterpret_cast<const int4*>(d_lists);
  bp.cta_off = d_lists + 4 * (size_t)njobs;
  bp.solo_list = bp.cta_off + grid + 1;
  bp.nsolo = nsolo;
  bp.solo_next = d_lists + 4 * (size_t)njobs + grid + 1 + nsolo;
  return bp;
}

}  // namespace

cudaError_t launch_schedule(const Params* h_params, int32_t G, int bs, int grid, bool cooperative,
                            const std::vector<int32_t>& lists, int32_t njobs, int32_t nsolo,
                            Params* d_params, int32_t* d_lists, cudaStream_t s, bool push) {
  cudaError_t e = h_params ? cudaMemcpyAsync(d_params, h_params, sizeof(Params) * (size_t)G,
                                             cudaMemcpyHostToDevice, s)
                           : cudaSuccess;  // (already on the device)
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_lists, lists.data(), sizeof(int32_t) * lists.size(),
                        cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return launch_batched(batch_params(d_params, d_lists, njobs, nsolo, grid), bs, grid, cooperative,
                        s, push);
}

cudaError_t schedule_and_launch(const Params* h_params, int32_t G, int bs, int grid, int max_team,
                                int64_t nnz_per_cta, bool cooperative, Params* d_params,
                                int32_t* d_lists, size_t lists_cap, std::vector<int32_t>& lists,
                                cudaStream_t s, int* rc, bool push) {
  *rc = IPGC_OK;
  int32_t njobs = 0, nsolo = 0;
  build_schedule(h_params, G, grid, max_team, nnz_per_cta, lists, &njobs, &nsolo, nullptr);
  if (lists.size() > lists_cap) {
    *rc = IPGC_ERR_UNSUPPORTED;
    return cudaSuccess;
  }
  return launch_schedule(h_params, G, bs, grid, cooperative, lists, njobs, nsolo, d_params, d_lists,
                         s, push);
}

}  // namespace ipgc

// ------------------------------------------------------------------ host --

using ipgc::BatchParams;
using ipgc::Ctrl;
using ipgc::Params;

namespace {

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

struct BatchWs {
  int device = -1;
  char* dev = nullptr;  // one device allocation, carved below
  size_t dev_bytes = 0;
  Ctrl* h_ctrl = nullptr;  // pinned copy of the per-graph control blocks
  size_t h_ctrl_cap = 0;
  int* h_err = nullptr;  // pinned
  std::vector<Params> params;
  std::vector<int32_t> lists;   // schedule of the rescanning kernel
  std::vector<int32_t> plists;  // ... of the pushing kernel
};

// workspace kept per context (one batch at a time per context)
struct BatchCtxSlot {
  ipgc_ctx* ctx;
  BatchWs ws;
};
std::vector<BatchCtxSlot*> g_slots;
std::mutex g_slots_mu;

BatchWs* ws_for(ipgc_ctx* ctx) {
  std::lock_guard<std::mutex> lk(g_slots_mu);
  for (BatchCtxSlot* s : g_slots)
    if (s->ctx == ctx) return &s->ws;
  BatchCtxSlot* s = new (std::nothrow) BatchCtxSlot{ctx, BatchWs()};
  if (!s) return nullptr;
  g_slots.push_back(s);
  return &s->ws;
}

int cuda_err(ipgc_ctx* ctx, cudaError_t e) {
  ipgc::ctx_note_cuda_error(ctx, (int)e);
  return e == cudaErrorMemoryAllocation ? IPGC_ERR_OOM : IPGC_ERR_CUDA;
}

#define BCUDA(call)                         \
  do {                                      \
    cudaError_t e_ = (call);                \
    if (e_ != cudaSuccess) return cuda_err(ctx, e_); \
  } while (0)

}  // namespace

extern "C" {

void ipgc_batch_options_default(ipgc_batch_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  ipgc_options_default(&o->base);
  o->base.validate = 0;
  o->max_team = 0;
  o->nnz_per_cta = 131072;
}

int ipgc_color_batched(ipgc_ctx* ctx, int32_t num_graphs, const int64_t* node_off,
                       const int64_t* edge_off, const int32_t* rowptr_cat, const int32_t* col_cat,
                       int32_t* colors_cat, ipgc_stats* per_graph_stats,
                       const ipgc_batch_options* opt, void* stream) {
  if (!ctx || num_graphs < 0 || (num_graphs > 0 && (!node_off || !edge_off))) return IPGC_ERR_INVALID;
  ipgc_batch_options o;
  if (opt)
    o = *opt;
  else
    ipgc_batch_options_default(&o);
  if (o.max_team < 0 || o.nnz_per_cta < 1) return IPGC_ERR_INVALID;
  if (o.base.mode < IPGC_MODE_THRESHOLD || o.base.mode > IPGC_MODE_LEARNED) return IPGC_ERR_INVALID;
  if (o.base.block_size != 0 && o.base.block_size != 256 && o.base.block_size != 512)
    return IPGC_ERR_UNSUPPORTED;
  if (num_graphs == 0) return IPGC_OK;
  // graph shapes (host offsets)
  if (node_off[0] != 0 || edge_off[0] != 0) return IPGC_ERR_INVALID;
  const int64_t total_n = node_off[num_graphs], total_e = edge_off[num_graphs];
  for (int32_t g = 0; g < num_graphs; ++g) {
    const int64_t n = node_off[g + 1] - node_off[g], e = edge_off[g + 1] - edge_off[g];
    if (n < 0 || e < 0 || n >= INT32_MAX || e > INT32_MAX) return IPGC_ERR_INVALID;
    if (e > 0 && n == 0) return IPGC_ERR_INVALID;
  }
  if (total_n > 0 && (!rowptr_cat || !colors_cat)) return IPGC_ERR_INVALID;
  if (total_e > 0 && !col_cat) return IPGC_ERR_INVALID;

  const int dev = ipgc::ctx_device(ctx);
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != dev) cudaSetDevice(dev);
  struct Restore {
    int prev, dev;
    ~Restore() {
      if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
  } restore{prev, dev};
  cudaStream_t s = (cudaStream_t)stream;

  BatchWs* W = ws_for(ctx);
  if (!W) return IPGC_ERR_OOM;
  const int t1 = ipgc::effective_t1(o.base), chunk = ipgc::effective_chunk(o.base);
  const int bs = o.base.block_size ? o.base.block_size : ipgc::kBlock;
  if (o.base.forbidden < IPGC_FORBIDDEN_AUTO || o.base.forbidden > IPGC_FORBIDDEN_PUSH)
    return IPGC_ERR_INVALID;
  // forbidden-colour bitmaps unless rescanning is asked for
  const bool push = o.base.forbidden != IPGC_FORBIDDEN_RESCAN;

  // per-graph slices of the workspace
  std::vector<int64_t> item_base(num_graphs + 1), gbase(num_graphs + 1), pq_base(num_graphs + 1),
      lbase(num_graphs + 1), rq_base(num_graphs + 1);
  item_base[0] = gbase[0] = pq_base[0] = lbase[0] = rq_base[0] = 0;
  for (int32_t g = 0; g < num_graphs; ++g) {
    const int64_t n = node_off[g + 1] - node_off[g], e = edge_off[g + 1] - edge_off[g];
    int64_t nbig = e / (t1 + 1);
    if (nbig > n) nbig = n;
    item_base[g + 1] = item_base[g] + e / chunk + nbig + 1;
    gbase[g + 1] = gbase[g] + e / ((int64_t)chunk + 1) + 1;
    pq_base[g + 1] = pq_base[g] + (push ? e / ipgc::kPushChunk + 2 * nbig + 1 : 0);
    // list rewrite units (one window each) of the graph's merge-state slots
    rq_base[g + 1] = rq_base[g] + (push ? e / ipgc::kPushChunk + 2 * (gbase[g + 1] - gbase[g]) + 1 : 0);
    // lists are read as int4 windows from their buffer's base: every graph's
    // slice starts on a 16-byte boundary
    lbase[g + 1] = lbase[g] + (push ? (e + 3) / 4 * 4 : 0);
  }
  // the schedule needs only the shapes, so it is built first and sizes its buffer
  W->params.assign(num_graphs, Params());
  for (int32_t g = 0; g < num_graphs; ++g) {
    W->params[g].n = (int32_t)(node_off[g + 1] - node_off[g]);
    W->params[g].nnz = edge_off[g + 1] - edge_off[g];
  }
  // one schedule per kernel, each for its own grid (occupancies differ): the
  // pushing kernel first, then the rescanning one, which colours only the
  // graphs the first left to it (or every graph, without pushing)
  int occ = 0, pocc = 0;
  BCUDA(ipgc::occupancy_batched(bs, &occ));
  if (push) BCUDA(ipgc::occupancy_batched(bs, &pocc, true));
  const int grid = occ * ipgc::ctx_num_sms(ctx), pgrid = pocc * ipgc::ctx_num_sms(ctx);
  int32_t njobs = 0, nsolo = 0, pnjobs = 0, pnsolo = 0;
  ipgc::build_schedule(W->params.data(), num_graphs, grid, o.max_team, o.nnz_per_cta, W->lists,
                       &njobs, &nsolo, nullptr);
  W->plists.clear();
  if (push)
    ipgc::build_schedule(W->params.data(), num_graphs, pgrid, o.max_team, o.nnz_per_cta,
                         W->plists, &pnjobs, &pnsolo, nullptr);
  const size_t b_params = al256(sizeof(Params) * (size_t)num_graphs);
  const size_t b_lists = al256(sizeof(int32_t) * W->lists.size());
  const size_t b_plists = al256(sizeof(int32_t) * W->plists.size());
  const size_t b_ctrl = al256(sizeof(Ctrl) * (size_t)num_graphs);
  const size_t b_node = al256(sizeof(int32_t) * (size_t)total_n);
  const size_t b_items = al256(sizeof(int4) * (size_t)item_base[num_graphs]);
  const size_t b_gbits = al256(sizeof(uint32_t) * ipgc::kGWords * (size_t)gbase[num_graphs]);
  const size_t b_gint = al256(sizeof(int32_t) * (size_t)gbase[num_graphs]);
  // pushing: bitmaps and two list buffers [entries], list counts (int2) x 2 and
  // state, dead counts [slots], push queues, winners [nodes]
  const size_t b_edge = push ? al256(sizeof(int32_t) * (size_t)total_e) : 0;
  const size_t b_lists_e = push ? al256(sizeof(int32_t) * (size_t)lbase[num_graphs]) : 0;
  const size_t b_gint2 = push ? al256(sizeof(int2) * (size_t)gbase[num_graphs]) : 0;
  const size_t b_gpint = push ? b_gint : 0;
  const size_t b_pq = al256(sizeof(int4) * (size_t)pq_base[num_graphs]);
  const size_t b_pw = push ? b_node : 0;
  // ... and per node {row start, degree while active and bitmapped} (push targets)
  const size_t b_pinfo = push ? al256(sizeof(int2) * (size_t)total_n) : 0;
  const size_t b_rq = al256(sizeof(int4) * (size_t)rq_base[num_graphs]);
  const size_t need = b_params + b_lists + b_plists + b_ctrl + 3 * b_node + 3 * b_items + b_gbits +
                      3 * b_gint + b_edge + 2 * b_lists_e + 2 * b_gint2 + 2 * b_gpint + b_pq +
                      b_pw + b_pinfo + b_rq + 256;
  if (W->dev_bytes < need || W->device != dev) {
    if (W->dev) cudaFree(W->dev);
    W->dev = nullptr;
    W->dev_bytes = 0;
    BCUDA(cudaMalloc((void**)&W->dev, need));
    W->dev_bytes = need;
    W->device = dev;
  }
  if (W->h_ctrl_cap < (size_t)num_graphs) {
    if (W->h_ctrl) cudaFreeHost(W->h_ctrl);
    W->h_ctrl = nullptr;
    W->h_ctrl_cap = 0;
    BCUDA(cudaMallocHost((void**)&W->h_ctrl, sizeof(Ctrl) * (size_t)num_graphs));
    W->h_ctrl_cap = num_graphs;
  }
  if (!W->h_err) BCUDA(cudaMallocHost((void**)&W->h_err, sizeof(int)));
  char* w = W->dev;
  Params* d_params = (Params*)w;
  w += b_params;
  int32_t* d_lists = (int32_t*)w;
  w += b_lists;
  int32_t* d_plists = (int32_t*)w;
  w += b_plists;
  Ctrl* d_ctrl = (Ctrl*)w;
  w += b_ctrl;
  int32_t* d_tent = (int32_t*)w;
  w += b_node;
  int32_t* d_wl0 = (int32_t*)w;
  w += b_node;
  int32_t* d_wl1 = (int32_t*)w;
  w += b_node;
  int4* d_it0 = (int4*)w;
  w += b_items;
  int4* d_it1 = (int4*)w;
  w += b_items;
  int4* d_its = (int4*)w;
  w += b_items;
  uint32_t* d_gbits = (uint32_t*)w;
  w += b_gbits;
  int32_t* d_done_a = (int32_t*)w;
  w += b_gint;
  int32_t* d_done_d = (int32_t*)w;
  w += b_gint;
  int32_t* d_flag = (int32_t*)w;
  w += b_gint;
  uint32_t* d_pbits = (uint32_t*)w;
  w += b_edge;
  int32_t* d_alist0 = (int32_t*)w;
  w += b_lists_e;
  int32_t* d_alist1 = (int32_t*)w;
  w += b_lists_e;
  int2* d_flen0 = (int2*)w;
  w += b_gint2;
  int2* d_flen1 = (int2*)w;
  w += b_gint2;
  int32_t* d_fst = (int32_t*)w;
  w += b_gpint;
  int32_t* d_fdead = (int32_t*)w;
  w += b_gpint;
  int4* d_pq = (int4*)w;
  w += b_pq;
  int32_t* d_pw = (int32_t*)w;
  w += b_pw;
  int2* d_pinfo = (int2*)w;
  w += b_pinfo;
  int4* d_rq = (int4*)w;
  w += b_rq;
  ipgc::ValidateState* d_err = (ipgc::ValidateState*)w;

  // optional validation of every graph (one launch per graph)
  if (o.base.validate) {
    BCUDA(cudaMemsetAsync(d_err, 0, sizeof(ipgc::ValidateState), s));
    for (int32_t g = 0; g < num_graphs; ++g) {
      const int64_t n = node_off[g + 1] - node_off[g], e = edge_off[g + 1] - edge_off[g];
      if (n == 0) continue;
      int blocks = (int)std::min<int64_t>(1024, (n * 32 + 255) / 256);
      BCUDA(ipgc::launch_validate(rowptr_cat + node_off[g] + g, col_cat + edge_off[g], (int32_t)n, e,
                                  d_err, blocks, s));
    }
    BCUDA(cudaMemcpyAsync(W->h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BCUDA(cudaStreamSynchronize(s));
    if (*W->h_err) return IPGC_ERR_INVALID;
  }

  // per-graph parameters
  const float* d_mlp = ipgc::ctx_policy_weights(ctx);
  for (int32_t g = 0; g < num_graphs; ++g) {
    Params& p = W->params[g];
    std::memset(&p, 0, sizeof(p));
    const int64_t n = node_off[g + 1] - node_off[g], e = edge_off[g + 1] - edge_off[g];
    p.rowptr = rowptr_cat + node_off[g] + g;
    p.col = col_cat + edge_off[g];
    p.n = (int32_t)n;
    p.nnz = e;
    p.color = colors_cat + node_off[g];
    p.tent = d_tent + node_off[g];
    p.wl[0] = d_wl0 + node_off[g];
    p.wl[1] = d_wl1 + node_off[g];
    p.items[0] = d_it0 + item_base[g];
    p.items[1] = d_it1 + item_base[g];
    p.istat = d_its + item_base[g];
    p.gbits = d_gbits + (size_t)gbase[g] * ipgc::kGWords;
    p.done_a = d_done_a + gbase[g];
    p.done_d = d_done_d + gbase[g];
    p.flag = d_flag + gbase[g];
    p.ctrl = d_ctrl + g;
    p.t1 = t1;
    p.chunk = chunk;
    double h = (double)o.base.threshold_frac * (double)n;
    p.H = (int64_t)(h > 0 ? h : 0);
    p.policy = o.base.mode;
    p.max_rounds = o.base.max_rounds > 0 ? o.base.max_rounds : (int32_t)n + 1;
    p.timeout_ns = o.base.timeout_ns ? o.base.timeout_ns : 10000000000ull;
    p.mlp = o.base.mode == IPGC_MODE_LEARNED ? d_mlp : nullptr;
    p.mlp_margin = o.base.policy_margin;
    p.col_vec = ((uintptr_t)p.col & 15u) == 0 ? 1 : 0;
    if (push) {  // a graph's bitmaps and lists live inside its own entry range
      p.pbits = d_pbits + edge_off[g];
      p.alist[0] = d_alist0 + lbase[g];
      p.alist[1] = d_alist1 + lbase[g];
      p.flen[0] = d_flen0 + gbase[g];
      p.flen[1] = d_flen1 + gbase[g];
      p.fst = d_fst + gbase[g];
      p.fdead = d_fdead + gbase[g];
      p.pq = d_pq + pq_base[g];
      p.pw = d_pw + node_off[g];
      p.pinfo = d_pinfo + node_off[g];
      p.rq = d_rq + rq_base[g];
    }
  }

  BCUDA(cudaMemsetAsync(d_ctrl, 0, sizeof(Ctrl) * (size_t)num_graphs, s));
  if (push)
    BCUDA(ipgc::launch_schedule(W->params.data(), num_graphs, bs, pgrid, true, W->plists, pnjobs,
                                pnsolo, d_params, d_plists, s, true));
  BCUDA(ipgc::launch_schedule(push ? nullptr : W->params.data(), num_graphs, bs, grid, true,
                              W->lists, njobs, nsolo, d_params, d_lists, s));

  if (!per_graph_stats) return IPGC_OK;
  BCUDA(cudaMemcpyAsync(W->h_ctrl, d_ctrl, sizeof(Ctrl) * (size_t)num_graphs,
                        cudaMemcpyDeviceToHost, s));
  BCUDA(cudaStreamSynchronize(s));
  int worst = IPGC_OK;
  for (int32_t g = 0; g < num_graphs; ++g) {
    const Ctrl& c = W->h_ctrl[g];
    ipgc_stats& st = per_graph_stats[g];
    std::memset(&st, 0, sizeof(st));
    if (node_off[g + 1] == node_off[g]) continue;
    st.rounds = c.rounds;
    st.num_colors = c.maxc;
    st.rounds_topo = c.rounds_topo;
    st.rounds_data = c.rounds_data;
    st.edges_processed = (int64_t)c.edges;
    st.ns = c.t_end >= c.t_start ? c.t_end - c.t_start : 0;
    st.error = c.status;
    if (c.status != IPGC_OK && worst == IPGC_OK) worst = c.status;
  }
  return worst;
}

int ipgc_batch_plan(int32_t num_graphs, const int32_t* n, const int64_t* nnz, int32_t grid,
                    int32_t max_team, int64_t nnz_per_cta, int32_t* team, int32_t* first_cta,
                    int32_t* seq) {
  if (num_graphs < 0 || grid < 1 || max_team < 0 || nnz_per_cta < 1) return IPGC_ERR_INVALID;
  if (num_graphs > 0 && (!n || !nnz || !team || !first_cta || !seq)) return IPGC_ERR_INVALID;
  std::vector<Params> ps(num_graphs, Params());
  for (int32_t g = 0; g < num_graphs; ++g) {
    if (n[g] < 0 || nnz[g] < 0) return IPGC_ERR_INVALID;
    ps[g].n = n[g];
    ps[g].nnz = nnz[g];
  }
  std::vector<int32_t> lists;
  int32_t njobs = 0, nsolo = 0;
  ipgc::build_schedule(ps.data(), num_graphs, grid, max_team, nnz_per_cta, lists, &njobs, &nsolo,
                       seq);
  for (int32_t g = 0; g < num_graphs; ++g) {
    team[g] = seq[g] < 0 ? 0 : 1;
    first_cta[g] = -1;
  }
  const int32_t* cta_off = lists.data() + 4 * (size_t)njobs;
  for (int32_t c = 0; c < grid; ++c)
    for (int32_t j = cta_off[c]; j < cta_off[c + 1]; ++j) {
      const int32_t* jb = lists.data() + 4 * (size_t)j;
      team[jb[0]] = jb[2];
      first_cta[jb[0]] = c - jb[1];
    }
  return IPGC_OK;
}

}  // extern "C"

void ipgc::batched_release(ipgc_ctx* ctx) {
  std::lock_guard<std::mutex> lk(g_slots_mu);
  for (size_t i = 0; i < g_slots.size(); ++i) {
    if (g_slots[i]->ctx != ctx) continue;
    BatchWs& W = g_slots[i]->ws;
    if (W.dev) cudaFree(W.dev);
    if (W.h_ctrl) cudaFreeHost(W.h_ctrl);
    if (W.h_err) cudaFreeHost(W.h_err);
    delete g_slots[i];
    g_slots.erase(g_slots.begin() + i);
    return;
  }
}
