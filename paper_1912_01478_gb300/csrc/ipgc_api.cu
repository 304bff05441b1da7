// C ABI of libipgc.so: contexts, workspace, argument checks, drivers.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "ipgc_internal.h"

using ipgc::Ctrl;
using ipgc::Params;

struct ipgc_ctx {
  int device = 0;
  int num_sms = 0;
  int occ256 = 0, occ512 = 0;  // resident CTAs per SM of the rescanning persistent kernels
  int pocc256 = 0, pocc512 = 0;  // ... of the pushing kernel
  // workspace for one colouring: tent, worklists, static lists
  char* ws = nullptr;
  size_t ws_bytes = 0;
  Ctrl* d_ctrl = nullptr;
  Ctrl* h_ctrl = nullptr;  // pinned
  ipgc::ValidateState* d_err = nullptr;
  int* h_err = nullptr;  // pinned
  // device copies for ipgc_color_host
  int32_t* d_rowptr = nullptr;
  int32_t* d_col = nullptr;
  int32_t* d_colors = nullptr;
  size_t cap_rowptr = 0, cap_col = 0, cap_colors = 0;
  // auxiliary device buffer (micro-benchmark worklists), grown on demand
  char* aux = nullptr;
  size_t aux_bytes = 0;
  // learned policy weights
  float* d_mlp = nullptr;
  int32_t mlp_len = 0;
  std::vector<float> h_mlp;  // host copy (host-loop driver)
  // state of the last colouring
  int last_cuda = 0;
  cudaStream_t last_stream = nullptr;
  int last_status = IPGC_OK;
  int last_valid = 0;  // h_ctrl holds a finished colouring
  int last_trivial = 0;  // n == 0
};

namespace ipgc {

int effective_t1(const ipgc_options& o) {
  return o.t1 > 0 ? (o.t1 < kMaxT1 ? o.t1 : kMaxT1) : kDefaultT1;
}

int effective_chunk(const ipgc_options& o) {
  if (o.chunk <= 0) return kDefaultChunk;
  if (o.chunk < kMinChunk) return kMinChunk;
  return o.chunk > kMaxChunk ? kMaxChunk : o.chunk;
}

int ctx_device(const ipgc_ctx* ctx) { return ctx->device; }
int ctx_num_sms(const ipgc_ctx* ctx) { return ctx->num_sms; }
void ctx_note_cuda_error(ipgc_ctx* ctx, int err) { ctx->last_cuda = err; }
const float* ctx_policy_weights(const ipgc_ctx* ctx) { return ctx->mlp_len ? ctx->d_mlp : nullptr; }
Ctrl* ctx_ctrl_dev(ipgc_ctx* ctx) { return ctx->d_ctrl; }
Ctrl* ctx_ctrl_host(ipgc_ctx* ctx) { return ctx->h_ctrl; }

void* ctx_aux(ipgc_ctx* ctx, size_t bytes, int* rc) {
  *rc = IPGC_OK;
  if (ctx->aux && ctx->aux_bytes >= bytes) return ctx->aux;
  if (ctx->aux) cudaFree(ctx->aux);
  ctx->aux = nullptr;
  ctx->aux_bytes = 0;
  const cudaError_t e = cudaMalloc((void**)&ctx->aux, bytes ? bytes : 1);
  if (e != cudaSuccess) {
    ctx->last_cuda = (int)e;
    *rc = e == cudaErrorMemoryAllocation ? IPGC_ERR_OOM : IPGC_ERR_CUDA;
    return nullptr;
  }
  ctx->aux_bytes = bytes;
  return ctx->aux;
}

}  // namespace ipgc

namespace {

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int cuda_fail(ipgc_ctx* ctx, cudaError_t e) {
  if (ctx) ctx->last_cuda = (int)e;
  return e == cudaErrorMemoryAllocation ? IPGC_ERR_OOM : IPGC_ERR_CUDA;
}

#define IPGC_CUDA(ctx, call)                      \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_); \
  } while (0)

// Workspace of one colouring, every array 256-byte aligned:
//   tent[n]; low-degree worklists [2 parities][n]; work items (int4) of the
//   high-degree nodes [2 parities + static][item_cap]; per-node state of
//   nodes with several items or with filtering: bits [gcap][kGWords],
//   done_a, done_d, flag [gcap]; with neighbour filtering, the filtered lists
//   [2 buffers][nnz], their counts (int2) [2 buffers][gcap], list state and
//   finalised-entry counts [gcap] each (contiguous after the counts), and
//   the work items of filtered nodes [2 parities][item_cap].
// A node of degree > t1 has more than t1 entries, so at most nnz / (t1 + 1)
// exist, with at most nnz / chunk + (their number) items; a node with several
// items has more than `chunk` entries and a filtered one more than filt_deg.
//   With pushing (IPGC_FORBIDDEN_PUSH), the list arrays of filtering (lower
//   parts only, no filtered items) and at the end the forbidden-colour
//   bitmaps [nnz] words (a node's bitmap inside its own row range), the push
//   queue, the winners list [n] and the push targets' {row start, degree}
//   [n] int2.
struct WsLayout {
  size_t a4n, items_bytes, gbits_bytes, gint_bytes, alist_bytes, flen_bytes, fst_bytes, pbits_bytes,
      pq_bytes, pinfo_bytes, rq_bytes, total;
};

using ipgc::effective_chunk;
using ipgc::effective_t1;

// Forbidden colours pushed into per-node bitmaps (else rows are rescanned).
bool effective_push(const ipgc_options& o) {
  return o.forbidden == IPGC_FORBIDDEN_PUSH ||
         (o.forbidden == IPGC_FORBIDDEN_AUTO && o.driver == IPGC_DRIVER_PERSISTENT);
}

// Degree above which a node is filtered (INT32_MAX: off); at least the
// chunk, so every such node has several work items and a merge-state slot.
// Forced pushing never filters; the automatic choice keeps filtering for the
// graphs it leaves to the rescanning kernels (the pushing kernel ignores it).
int effective_filt_deg(const ipgc_options& o) {
  if (o.filter_degree < 0 || o.worklist == IPGC_WORKLIST_REBUILD ||
      o.forbidden == IPGC_FORBIDDEN_PUSH)
    return INT32_MAX;
  const int f = o.filter_degree > 0 ? o.filter_degree : ipgc::kDefaultFiltDeg;
  const int lo = effective_chunk(o) > effective_t1(o) ? effective_chunk(o) : effective_t1(o);
  return f > lo ? f : lo;
}

WsLayout ws_layout(int32_t n, int64_t nnz, int t1, int chunk, int filt_deg, bool push) {
  WsLayout L;
  L.a4n = align256((size_t)n * sizeof(int32_t));
  int64_t nbig = nnz / ((int64_t)t1 + 1);
  if (nbig > n) nbig = n;
  const int64_t item_cap = nnz / chunk + nbig + 1;
  const bool filt = filt_deg != INT32_MAX;
  const bool lists = filt || push;
  const int64_t gcap = nnz / ((int64_t)chunk + 1) + 1;
  L.items_bytes = align256((size_t)item_cap * sizeof(int4));
  L.gbits_bytes = align256((size_t)gcap * ipgc::kGWords * sizeof(uint32_t));
  L.gint_bytes = align256((size_t)gcap * sizeof(int32_t));
  L.alist_bytes = lists ? align256((size_t)nnz * sizeof(int32_t)) : 0;
  L.flen_bytes = lists ? align256((size_t)gcap * sizeof(int2)) : 0;
  L.fst_bytes = lists ? align256((size_t)gcap * sizeof(int32_t)) : 0;
  L.pbits_bytes = push ? align256((size_t)nnz * sizeof(uint32_t)) : 0;
  // push items of one round: one-window items of the rows of nodes of degree > t1
  // (ceil(d / kPushChunk) + 1 at most for a row of d entries)
  L.pq_bytes = push ? align256((size_t)(nnz / ipgc::kPushChunk + 2 * nbig + 1) * sizeof(int4)) : 0;
  L.pinfo_bytes = push ? align256((size_t)n * sizeof(int2)) : 0;
  // list rewrite units of one round: one-window units of the lists of nodes
  // with a merge-state slot (ceil(L / kPushChunk) + 1 at most for L entries)
  L.rq_bytes = push ? align256((size_t)(nnz / ipgc::kPushChunk + 2 * gcap + 1) * sizeof(int4)) : 0;
  L.total = 3 * L.a4n + 3 * L.items_bytes + L.gbits_bytes + 3 * L.gint_bytes +
            2 * L.alist_bytes + 2 * L.flen_bytes + 2 * L.fst_bytes +
            (filt ? 2 * L.items_bytes : 0) +
            (push ? L.pbits_bytes + L.pq_bytes + L.a4n + L.pinfo_bytes + L.rq_bytes : 0);
  return L;
}

size_t ws_bytes_for(int32_t n, int64_t nnz, const ipgc_options& o) {
  return ws_layout(n, nnz, effective_t1(o), effective_chunk(o), effective_filt_deg(o),
                   effective_push(o))
      .total;
}

int ensure_ws(ipgc_ctx* ctx, int32_t n, int64_t nnz, const ipgc_options& o) {
  const size_t need = ws_bytes_for(n, nnz, o);
  if (ctx->ws_bytes >= need && ctx->ws) return IPGC_OK;
  if (ctx->ws) {
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  IPGC_CUDA(ctx, cudaMalloc((void**)&ctx->ws, need));
  ctx->ws_bytes = need;
  return IPGC_OK;
}

template <class T>
int ensure_buf(ipgc_ctx* ctx, T** p, size_t* cap, size_t count) {
  if (*cap >= count && *p) return IPGC_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  IPGC_CUDA(ctx, cudaMalloc((void**)p, (count > 0 ? count : 1) * sizeof(T)));
  *cap = count;
  return IPGC_OK;
}

void fill_params(ipgc_ctx* ctx, Params& p, const int32_t* rowptr, const int32_t* col, int32_t n,
                 int64_t nnz, int32_t* colors, const ipgc_options& o) {
  std::memset(&p, 0, sizeof(p));
  p.rowptr = rowptr;
  p.col = col;
  p.n = n;
  p.nnz = nnz;
  p.color = colors;
  p.t1 = effective_t1(o);
  p.chunk = effective_chunk(o);
  p.filt_deg = effective_filt_deg(o);
  const bool push = effective_push(o);
  const WsLayout L = ws_layout(n, nnz, p.t1, p.chunk, p.filt_deg, push);
  const size_t a = L.a4n;
  char* w = ctx->ws;
  p.tent = (int32_t*)w;
  w += a;
  p.wl[0] = (int32_t*)w;
  w += a;
  p.wl[1] = (int32_t*)w;
  w += a;
  p.items[0] = (int4*)w;
  w += L.items_bytes;
  p.items[1] = (int4*)w;
  w += L.items_bytes;
  p.istat = (int4*)w;
  w += L.items_bytes;
  p.gbits = (uint32_t*)w;
  w += L.gbits_bytes;
  p.done_a = (int32_t*)w;
  w += L.gint_bytes;
  p.done_d = (int32_t*)w;
  w += L.gint_bytes;
  p.flag = (int32_t*)w;
  w += L.gint_bytes;
  if (L.alist_bytes) {
    p.alist[0] = (int32_t*)w;
    w += L.alist_bytes;
    p.alist[1] = (int32_t*)w;
    w += L.alist_bytes;
    p.flen[0] = (int2*)w;
    w += L.flen_bytes;
    p.flen[1] = (int2*)w;
    w += L.flen_bytes;
    p.fst = (int32_t*)w;
    w += L.fst_bytes;
    p.fdead = (int32_t*)w;
    w += L.fst_bytes;
    if (p.filt_deg != INT32_MAX) {
      p.fitems[0] = (int4*)w;
      w += L.items_bytes;
      p.fitems[1] = (int4*)w;
      w += L.items_bytes;
      // hand over to filtering once |WL| <= filter_start * n
      const double fs = o.filter_start > 0 ? (double)o.filter_start : ipgc::kDefaultFiltStart;
      const double hw = fs * (double)n;
      p.handoff_wl = hw >= 1.0 ? (int64_t)hw : 1;
    }
  }
  if (push) {
    p.pbits = (uint32_t*)w;
    w += L.pbits_bytes;
    p.pq = (int4*)w;
    w += L.pq_bytes;
    p.pw = (int32_t*)w;
    w += L.a4n;
    p.pinfo = (int2*)w;
    w += L.pinfo_bytes;
    p.rq = (int4*)w;
  }
  p.ctrl = ctx->d_ctrl;
  p.trace = o.trace;
  p.fin = o.fin_round;
  p.trace_cap = o.trace ? o.trace_cap : 0;
  double h = (double)o.threshold_frac * (double)n;
  if (h < 0) h = 0;
  p.H = (int64_t)h;  // floor for h >= 0
  p.policy = o.mode;
  p.max_rounds = o.max_rounds > 0 ? o.max_rounds : (n < INT32_MAX ? n + 1 : INT32_MAX);
  p.timeout_ns = o.timeout_ns ? o.timeout_ns : 10000000000ull;
  p.mlp = (o.mode == IPGC_MODE_LEARNED && ctx->mlp_len) ? ctx->d_mlp : nullptr;
  p.bar_extra = o.fault_inject ? 1u : 0u;
  p.mlp_margin = o.policy_margin;
  p.col_vec = ((uintptr_t)col & 15u) == 0 ? 1 : 0;
  p.shrink = o.driver == IPGC_DRIVER_PERSISTENT ? 1 : 0;
  p.t1_auto = o.t1 <= 0 ? 1 : 0;  // default t1: chosen on the device
  p.push_auto = o.forbidden == IPGC_FORBIDDEN_AUTO ? 1 : 0;
  p.wl_rebuild = o.worklist == IPGC_WORKLIST_REBUILD ? 1 : 0;
}

void stats_from_ctrl(const Ctrl& c, ipgc_stats* st) {
  st->rounds = c.rounds;
  st->num_colors = c.maxc;
  st->rounds_topo = c.rounds_topo;
  st->rounds_data = c.rounds_data;
  st->edges_processed = (int64_t)c.edges;
  st->ns = c.t_end >= c.t_start ? c.t_end - c.t_start : 0;
  st->error = c.status;
  st->filter_round = c.handoff_round;
}

int check_graph_args(const int32_t* rowptr, const int32_t* col, int32_t n, int64_t nnz,
                     const int32_t* colors) {
  if (n < 0 || nnz < 0 || nnz > (int64_t)INT32_MAX) return IPGC_ERR_INVALID;
  if (n > 0 && (!rowptr || !colors)) return IPGC_ERR_INVALID;
  if (nnz > 0 && (!col || n == 0)) return IPGC_ERR_INVALID;
  if (n == INT32_MAX) return IPGC_ERR_INVALID;
  return IPGC_OK;
}

int run_validate(ipgc_ctx* ctx, const int32_t* rowptr, const int32_t* col, int32_t n, int64_t nnz,
                 cudaStream_t s) {
  IPGC_CUDA(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(ipgc::ValidateState), s));
  int blocks = ctx->num_sms * 8;
  IPGC_CUDA(ctx, ipgc::launch_validate(rowptr, col, n, nnz, ctx->d_err, blocks, s));
  IPGC_CUDA(ctx, cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  IPGC_CUDA(ctx, cudaStreamSynchronize(s));
  return *ctx->h_err ? IPGC_ERR_INVALID : IPGC_OK;
}

int run_hostloop(ipgc_ctx* ctx, const Params& p0, int bs, int blocks, cudaStream_t s) {
  Params p = p0;
  IPGC_CUDA(ctx, ipgc::launch_round1(p, bs, blocks, s));
  int r = 2;
  for (;; ++r) {
    IPGC_CUDA(ctx, cudaMemcpyAsync(ctx->h_ctrl, ctx->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    IPGC_CUDA(ctx, cudaStreamSynchronize(s));
    const int par = r & 1;
    const int64_t total =
        (int64_t)ctx->h_ctrl->cnt[par][ipgc::B_SMALL] + ctx->h_ctrl->cnt[par][ipgc::B_BIG];
    if (total == 0) break;
    if (r > p.max_rounds) {
      ctx->h_ctrl->status = IPGC_ERR_NO_CONVERGE;
      IPGC_CUDA(ctx, cudaMemcpyAsync(&ctx->d_ctrl->status, &ctx->h_ctrl->status, sizeof(int32_t),
                                     cudaMemcpyHostToDevice, s));
      break;
    }
    int mode;
    if (p.policy == IPGC_MODE_TOPO)
      mode = IPGC_MODE_TOPO;
    else if (p.policy == IPGC_MODE_DATA)
      mode = IPGC_MODE_DATA;
    else
      mode = total > p.H ? IPGC_MODE_TOPO : IPGC_MODE_DATA;
    if (p.policy == IPGC_MODE_LEARNED && p.mlp && !ctx->h_mlp.empty()) {
      // same network and inputs as the device decision, evaluated on the host
      const Ctrl& c = *ctx->h_ctrl;
      float f[ipgc::kMlpIn];
      ipgc::policy_features(p.n, p.nnz, r, total, c.cnt[par][ipgc::B_SMALL], (int64_t)c.dsum[par],
                            c.maxc, f);
      const float pr = 1.0f / (1.0f + std::exp(-ipgc::mlp_logit_host(ctx->h_mlp.data(), f)));
      if (std::fabs(pr - 0.5f) >= p.mlp_margin) mode = pr > 0.5f ? IPGC_MODE_TOPO : IPGC_MODE_DATA;
    }
    if (p.filt_r0 == 0 && ipgc::handoff_now(p, r, total, ctx->h_ctrl->dsum[par], ctx->h_ctrl->maxc)) {
      // hand over to neighbour filtering: list counts and states start at zero
      const WsLayout L = ws_layout(p.n, p.nnz, p.t1, p.chunk, p.filt_deg, false);
      IPGC_CUDA(ctx, cudaMemsetAsync(p.flen[0], 0, 2 * L.flen_bytes + 2 * L.fst_bytes, s));
      p.filt_r0 = r;
    }
    IPGC_CUDA(ctx, ipgc::launch_assign(p, bs, blocks, r, mode, s));
    IPGC_CUDA(ctx, ipgc::launch_detect(p, bs, blocks, r, mode, s));
  }
  IPGC_CUDA(ctx, ipgc::launch_finish(p, r - 1, s));
  return IPGC_OK;
}

}  // namespace

extern "C" {

void ipgc_options_default(ipgc_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->mode = IPGC_MODE_THRESHOLD;
  o->threshold_frac = 0.6f;
  o->driver = IPGC_DRIVER_PERSISTENT;
  o->max_rounds = 0;
  o->timeout_ns = 0;
  o->validate = 1;
  o->policy_margin = 0.05f;
}

const char* ipgc_strerror(int s) {
  switch (s) {
    case IPGC_OK: return "ok";
    case IPGC_PENDING: return "pending";
    case IPGC_ERR_INVALID: return "invalid argument or graph";
    case IPGC_ERR_OOM: return "out of memory";
    case IPGC_ERR_TIMEOUT: return "a bounded device-side wait timed out";
    case IPGC_ERR_NO_CONVERGE: return "did not converge within max_rounds";
    case IPGC_ERR_CUDA: return "CUDA error (see ipgc_ctx_cuda_error)";
    case IPGC_ERR_BUSY: return "not admissible now (busy)";
    case IPGC_ERR_UNSUPPORTED: return "unsupported option";
    case IPGC_ERR_NOT_FOUND: return "unknown ticket";
    case IPGC_ERR_TOO_LARGE: return "graph exceeds the fixed scratch of this entry point";
    default: return "unknown status";
  }
}

size_t ipgc_workspace_size(int32_t n, int64_t nnz, const ipgc_options* opt) {
  if (n <= 0 || nnz < 0) return 0;
  ipgc_options o;
  if (opt)
    o = *opt;
  else
    ipgc_options_default(&o);
  return ws_bytes_for(n, nnz, o) + align256(sizeof(Ctrl));
}

int ipgc_ctx_create(ipgc_ctx** out, int device) {
  if (!out) return IPGC_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return IPGC_ERR_INVALID;
  ipgc_ctx* ctx = new (std::nothrow) ipgc_ctx();
  if (!ctx) return IPGC_ERR_OOM;
  ctx->device = device;
  DeviceGuard g(device);
  int rc = IPGC_OK;
  int coop = 0;
  cudaError_t e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
  if (e == cudaSuccess) e = ipgc::occupancy_persistent(256, &ctx->occ256);
  if (e == cudaSuccess) e = ipgc::occupancy_persistent(512, &ctx->occ512);
  if (e == cudaSuccess) e = ipgc::occupancy_push(256, &ctx->pocc256);
  if (e == cudaSuccess) e = ipgc::occupancy_push(512, &ctx->pocc512);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_ctrl, sizeof(Ctrl));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_ctrl, sizeof(Ctrl));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_err, sizeof(ipgc::ValidateState));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_err, sizeof(int));
  if (e != cudaSuccess) rc = cuda_fail(ctx, e);
  if (rc == IPGC_OK && (!coop || ctx->occ256 < 1 || ctx->occ512 < 1 || ctx->pocc256 < 1 ||
                        ctx->pocc512 < 1))
    rc = IPGC_ERR_UNSUPPORTED;
  if (rc != IPGC_OK) {
    ipgc_ctx_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return IPGC_OK;
}

int ipgc_ctx_destroy(ipgc_ctx* ctx) {
  if (!ctx) return IPGC_OK;
  {
    DeviceGuard g(ctx->device);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->d_ctrl) cudaFree(ctx->d_ctrl);
    if (ctx->h_ctrl) cudaFreeHost(ctx->h_ctrl);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    if (ctx->d_rowptr) cudaFree(ctx->d_rowptr);
    if (ctx->d_col) cudaFree(ctx->d_col);
    if (ctx->d_colors) cudaFree(ctx->d_colors);
    if (ctx->d_mlp) cudaFree(ctx->d_mlp);
    if (ctx->aux) cudaFree(ctx->aux);
    ipgc::batched_release(ctx);
  }
  delete ctx;
  return IPGC_OK;
}

int ipgc_ctx_cuda_error(const ipgc_ctx* ctx) { return ctx ? ctx->last_cuda : 0; }

int ipgc_policy_load(ipgc_ctx* ctx, const float* w, int32_t len) {
  if (!ctx) return IPGC_ERR_INVALID;
  if (len == 0) {
    ctx->mlp_len = 0;
    ctx->h_mlp.clear();
    return IPGC_OK;  // the device copy stays allocated but unused
  }
  if (len != ipgc::kMlpParams || !w) return IPGC_ERR_INVALID;
  for (int32_t i = 0; i < len; ++i)
    if (!std::isfinite(w[i])) return IPGC_ERR_INVALID;
  DeviceGuard g(ctx->device);
  if (!ctx->d_mlp) IPGC_CUDA(ctx, cudaMalloc((void**)&ctx->d_mlp, sizeof(float) * ipgc::kMlpParams));
  IPGC_CUDA(ctx, cudaMemcpy(ctx->d_mlp, w, sizeof(float) * len, cudaMemcpyHostToDevice));
  ctx->h_mlp.assign(w, w + len);
  ctx->mlp_len = len;
  return IPGC_OK;
}

int ipgc_color_ex(ipgc_ctx* ctx, const int32_t* rowptr, const int32_t* col, int32_t n, int64_t nnz,
                  int32_t* colors_out, ipgc_stats* stats_out, const ipgc_options* opt,
                  void* stream) {
  if (!ctx) return IPGC_ERR_INVALID;
  int rc = check_graph_args(rowptr, col, n, nnz, colors_out);
  if (rc != IPGC_OK) return rc;
  ipgc_options o;
  if (opt)
    o = *opt;
  else
    ipgc_options_default(&o);
  if (o.mode < IPGC_MODE_THRESHOLD || o.mode > IPGC_MODE_LEARNED) return IPGC_ERR_INVALID;
  if (o.driver != IPGC_DRIVER_PERSISTENT && o.driver != IPGC_DRIVER_HOSTLOOP) return IPGC_ERR_INVALID;
  if (o.block_size != 0 && o.block_size != 256 && o.block_size != 512) return IPGC_ERR_UNSUPPORTED;
  if (o.trace && o.trace_cap < 0) return IPGC_ERR_INVALID;
  if (!(o.threshold_frac >= 0.0f)) return IPGC_ERR_INVALID;
  if (o.worklist != IPGC_WORKLIST_KEEP && o.worklist != IPGC_WORKLIST_REBUILD) return IPGC_ERR_INVALID;
  if (o.worklist == IPGC_WORKLIST_REBUILD && o.driver != IPGC_DRIVER_PERSISTENT)
    return IPGC_ERR_UNSUPPORTED;
  if (o.forbidden < IPGC_FORBIDDEN_AUTO || o.forbidden > IPGC_FORBIDDEN_PUSH) return IPGC_ERR_INVALID;
  if (o.forbidden == IPGC_FORBIDDEN_PUSH && o.driver != IPGC_DRIVER_PERSISTENT)
    return IPGC_ERR_UNSUPPORTED;
  cudaStream_t s = (cudaStream_t)stream;
  DeviceGuard g(ctx->device);
  if (!g.ok) return cuda_fail(ctx, cudaErrorInvalidDevice);
  ctx->last_valid = 0;
  ctx->last_stream = s;
  ctx->last_status = IPGC_OK;
  if (n == 0) {
    ctx->last_trivial = 1;
    ctx->last_valid = 1;
    if (stats_out) std::memset(stats_out, 0, sizeof(*stats_out));
    return IPGC_OK;
  }
  ctx->last_trivial = 0;
  rc = ensure_ws(ctx, n, nnz, o);
  if (rc != IPGC_OK) return rc;
  if (o.validate) {
    rc = run_validate(ctx, rowptr, col, n, nnz, s);
    if (rc != IPGC_OK) return rc;
  }
  Params p;
  fill_params(ctx, p, rowptr, col, n, nnz, colors_out, o);
  IPGC_CUDA(ctx, cudaMemsetAsync(ctx->d_ctrl, 0, sizeof(Ctrl), s));
  const int bs = o.block_size ? o.block_size : ipgc::kBlock;
  int bps = bs == 256 ? ctx->occ256 : ctx->occ512;
  int pbps = bs == 256 ? ctx->pocc256 : ctx->pocc512;
  if (o.blocks_per_sm > 0 && o.blocks_per_sm < bps) bps = o.blocks_per_sm;
  if (o.blocks_per_sm > 0 && o.blocks_per_sm < pbps) pbps = o.blocks_per_sm;
  const int blocks = bps * ctx->num_sms;
  if (o.driver == IPGC_DRIVER_PERSISTENT) {
    IPGC_CUDA(ctx, ipgc::launch_persistent(p, bs, blocks, pbps * ctx->num_sms, s));
  } else {
    rc = run_hostloop(ctx, p, bs, blocks, s);
    if (rc != IPGC_OK) return rc;
  }
  IPGC_CUDA(ctx, cudaMemcpyAsync(ctx->h_ctrl, ctx->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  ctx->last_valid = 1;
  if (!stats_out) return IPGC_OK;
  return ipgc_ctx_last_stats(ctx, stats_out);
}

int ipgc_ctx_last_stats(ipgc_ctx* ctx, ipgc_stats* st) {
  if (!ctx || !st) return IPGC_ERR_INVALID;
  if (!ctx->last_valid) return IPGC_ERR_INVALID;
  if (ctx->last_trivial) {
    std::memset(st, 0, sizeof(*st));
    return IPGC_OK;
  }
  DeviceGuard g(ctx->device);
  IPGC_CUDA(ctx, cudaStreamSynchronize(ctx->last_stream));
  stats_from_ctrl(*ctx->h_ctrl, st);
  return st->error;
}

namespace {
struct DefaultCtxs {
  std::vector<ipgc_ctx*> by_dev;
  ~DefaultCtxs() {
    for (ipgc_ctx* c : by_dev)
      if (c) ipgc_ctx_destroy(c);
  }
};
thread_local DefaultCtxs t_default;
}  // namespace

int ipgc_color(const int32_t* rowptr, const int32_t* col, int32_t n, int64_t nnz,
               int32_t* colors_out, ipgc_stats* stats_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return IPGC_ERR_CUDA;
  if ((int)t_default.by_dev.size() <= dev) t_default.by_dev.resize(dev + 1, nullptr);
  if (!t_default.by_dev[dev]) {
    int rc = ipgc_ctx_create(&t_default.by_dev[dev], dev);
    if (rc != IPGC_OK) return rc;
  }
  ipgc_stats local;
  return ipgc_color_ex(t_default.by_dev[dev], rowptr, col, n, nnz, colors_out,
                       stats_out ? stats_out : &local, nullptr, nullptr);
}

int ipgc_color_host(ipgc_ctx* ctx, const int32_t* rowptr, const int32_t* col, int32_t n,
                    int64_t nnz, int32_t* colors_out, ipgc_stats* stats_out,
                    const ipgc_options* opt, void* stream) {
  if (!ctx) return IPGC_ERR_INVALID;
  int rc = check_graph_args(rowptr, col, n, nnz, colors_out);
  if (rc != IPGC_OK) return rc;
  if (n == 0) {
    if (stats_out) std::memset(stats_out, 0, sizeof(*stats_out));
    return IPGC_OK;
  }
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  rc = ensure_buf(ctx, &ctx->d_rowptr, &ctx->cap_rowptr, (size_t)n + 1);
  if (rc == IPGC_OK) rc = ensure_buf(ctx, &ctx->d_col, &ctx->cap_col, (size_t)nnz);
  if (rc == IPGC_OK) rc = ensure_buf(ctx, &ctx->d_colors, &ctx->cap_colors, (size_t)n);
  if (rc != IPGC_OK) return rc;
  IPGC_CUDA(ctx, cudaMemcpyAsync(ctx->d_rowptr, rowptr, ((size_t)n + 1) * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, s));
  if (nnz > 0)
    IPGC_CUDA(ctx, cudaMemcpyAsync(ctx->d_col, col, (size_t)nnz * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, s));
  ipgc_stats local;
  ipgc_stats* st = stats_out ? stats_out : &local;
  rc = ipgc_color_ex(ctx, ctx->d_rowptr, ctx->d_col, n, nnz, ctx->d_colors, st, opt, stream);
  if (rc != IPGC_OK) return rc;
  IPGC_CUDA(ctx, cudaMemcpyAsync(colors_out, ctx->d_colors, (size_t)n * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, s));
  IPGC_CUDA(ctx, cudaStreamSynchronize(s));
  return IPGC_OK;
}

int ipgc_validate_csr(ipgc_ctx* ctx, const int32_t* rowptr, const int32_t* col, int32_t n,
                      int64_t nnz, int on_device, void* stream) {
  if (n < 0 || nnz < 0 || nnz > (int64_t)INT32_MAX || n == INT32_MAX) return IPGC_ERR_INVALID;
  if (!rowptr) return IPGC_ERR_INVALID;
  if (nnz > 0 && !col) return IPGC_ERR_INVALID;
  if (!on_device) {
    if (rowptr[0] != 0 || (int64_t)rowptr[n] != nnz) return IPGC_ERR_INVALID;
    for (int32_t v = 0; v < n; ++v) {
      const int32_t s = rowptr[v], e = rowptr[v + 1];
      if (s < 0 || e < s || (int64_t)e > nnz) return IPGC_ERR_INVALID;
    }
    for (int32_t v = 0; v < n; ++v) {
      for (int32_t k = rowptr[v]; k < rowptr[v + 1]; ++k) {
        const int32_t u = col[k];
        if (u < 0 || u >= n || u == v) return IPGC_ERR_INVALID;
        if (k > rowptr[v] && col[k - 1] >= u) return IPGC_ERR_INVALID;
        int32_t lo = rowptr[u], hi = rowptr[u + 1];
        const int32_t hi0 = hi;
        while (lo < hi) {
          const int32_t mid = lo + ((hi - lo) >> 1);
          if (col[mid] < v)
            lo = mid + 1;
          else
            hi = mid;
        }
        if (lo >= hi0 || col[lo] != v) return IPGC_ERR_INVALID;
      }
    }
    return IPGC_OK;
  }
  if (n == 0) return IPGC_OK;
  bool own = false;
  if (!ctx) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return IPGC_ERR_CUDA;
    int rc = ipgc_ctx_create(&ctx, dev);
    if (rc != IPGC_OK) return rc;
    own = true;
  }
  int rc;
  {
    DeviceGuard g(ctx->device);
    rc = run_validate(ctx, rowptr, col, n, nnz, (cudaStream_t)stream);
  }
  if (own) ipgc_ctx_destroy(ctx);
  return rc;
}

}  // extern "C"
