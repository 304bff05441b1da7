// The micro-benchmark of Section III on the device.
//
// The worklist starts as every node; iteration i deactivates the next
// `count` node IDs: node v stays active iff v >= count * (i + 1) (the text's
// reading of the listing's threshold). Push_WL iterates over the worklist
// (data-driven) and pushes the nodes that stay active; Push_NoWL iterates
// over every node of the graph (topology-driven) and pushes the active ones;
// both keep a worklist in every iteration and produce the same one. The
// hybrid runs Push_NoWL while |WL| > switch_wl, then Push_WL. The Pipe is one
// cooperative launch whose iterations are separated by the bounded team
// barrier; CTA 0 records each iteration's time (%globaltimer), so the time
// per iteration (TTI) of both kernels and their crossover can be measured.
//
// Pushes are aggregated per CTA: a tile of kPushTile entries is compacted
// with a block-wide prefix sum and one atomic reserves its room (a tile that
// keeps nothing skips both), so the worklist order differs between runs and
// modes while its contents do not.
#include <cstring>

#include "ipgc_internal.h"

namespace ipgc {

namespace {

constexpr int kPushBS = 256;
constexpr int kPushIPT = 16;                    // entries per thread per tile
constexpr int kPushTile = kPushBS * kPushIPT;  // entries per tile

struct PushParams {
  int64_t n;
  int32_t count;
  int32_t mode;        // IPGC_PUSH_*
  int64_t switch_wl;   // hybrid: Push_NoWL while |WL| > switch_wl
  int32_t* wl[2];      // worklists, per parity
  int64_t* cnt;        // [3] worklist lengths: cnt[i % 3] is iteration i's input
  int64_t* rec;        // [cap][4]: |WL| after, sum of its IDs, kernel used, TTI ns (or null)
  int64_t cap;
  Ctrl* ctrl;          // barrier, status, iterations (rounds)
  uint64_t timeout_ns;
};

// Exclusive prefix sum of x over the CTA; *total receives the sum.
__device__ __forceinline__ int block_exclusive_sum(int x, int* warp_tot, int* total) {
  const int lane = lane_id(), warp = threadIdx.x >> 5;
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int t = lane < kPushBS / 32 ? warp_tot[lane] : 0;
    int ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, ti, o);
      if (lane >= o) ti += y;
    }
    if (lane < kPushBS / 32) warp_tot[lane] = ti - t;  // exclusive per warp
    if (lane == 31) *total = ti;
  }
  __syncthreads();
  const int r = warp_tot[warp] + incl - x;
  __syncthreads();  // warp_tot is reused by the next call
  return r;
}

__global__ void __launch_bounds__(kPushBS) push_kernel(const __grid_constant__ PushParams q) {
  __shared__ int warp_tot[kPushBS / 32];
  __shared__ int s_total;
  __shared__ long long s_base;
  __shared__ unsigned long long s_sum[kPushBS / 32];
  const Team tm{(int)blockIdx.x, (int)gridDim.x};
  const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
  Ctrl* c = q.ctrl;
  uint64_t t_prev = gtime();
  for (int64_t i = 0;; ++i) {
    const int64_t len = ld_cg_i64(&q.cnt[i % 3]);
    const bool nowl = q.mode == IPGC_PUSH_NOWL || (q.mode == IPGC_PUSH_HYBRID && len > q.switch_wl);
    const int64_t thr = (int64_t)q.count * (i + 1);
    const int64_t dom = nowl ? q.n : len;  // ForAll node in graph.nodes / wlnode in WL
    const int32_t* in = q.wl[i & 1];
    int32_t* out = q.wl[(i + 1) & 1];
    int64_t* cnt_out = &q.cnt[(i + 1) % 3];
    if (lead) q.cnt[(i + 2) % 3] = 0;  // the counter of iteration i + 2's output
    unsigned long long sum = 0;
    for (int64_t base = (int64_t)tm.cta * kPushTile; base < dom;
         base += (int64_t)tm.ncta * kPushTile) {
      int32_t v[kPushIPT];
      int k = 0;
#pragma unroll
      for (int j = 0; j < kPushIPT; ++j) {
        const int64_t idx = base + (int64_t)j * kPushBS + threadIdx.x;  // coalesced
        int32_t x = -1;
        if (idx < dom) x = nowl ? (int32_t)idx : ld_cg(in + idx);
        v[j] = (x >= 0 && x >= thr) ? x : -1;
        k += v[j] >= 0;
      }
      if (!__syncthreads_or(k)) continue;  // nothing of this tile stays active
      const int off = block_exclusive_sum(k, warp_tot, &s_total);
      if (threadIdx.x == 0) s_base = s_total ? atomicAdd((unsigned long long*)cnt_out,
                                                         (unsigned long long)s_total) : 0;
      __syncthreads();
      int64_t o = s_base + off;
#pragma unroll
      for (int j = 0; j < kPushIPT; ++j) {
        if (v[j] < 0) continue;
        out[o++] = v[j];
        sum += (unsigned long long)v[j];
      }
      __syncthreads();  // s_base is reused
    }
    if (q.rec && i < q.cap) {  // the sum of the pushed IDs, one atomic per CTA
      sum = warp_sum_u64(sum);
      if (lane_id() == 0) s_sum[threadIdx.x >> 5] = sum;
      __syncthreads();
      if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kPushBS / 32; ++w) t += s_sum[w];
        if (t) atomicAdd((unsigned long long*)&q.rec[4 * i + 1], t);
      }
    }
    if (!team_barrier(c, tm.cta, tm.ncta, q.timeout_ns)) break;
    const int64_t next = ld_cg_i64(cnt_out);
    if (lead) {
      const uint64_t t = gtime();
      if (q.rec && i < q.cap) {
        q.rec[4 * i + 0] = next;
        q.rec[4 * i + 2] = nowl ? IPGC_PUSH_NOWL : IPGC_PUSH_WL;
        q.rec[4 * i + 3] = (int64_t)(t - t_prev);
      }
      t_prev = t;
      c->rounds = (int32_t)(i + 1);
    }
    if (next == 0) break;
  }
}

__global__ void push_init_kernel(int32_t* wl, int64_t n, int64_t* cnt) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = tid; v < n; v += stride) wl[v] = (int32_t)v;  // WL = graph.nodes
  if (tid == 0) {
    cnt[0] = n;
    cnt[1] = 0;
    cnt[2] = 0;
  }
}

inline size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

}  // namespace ipgc

extern "C" int ipgc_push_bench(ipgc_ctx* ctx, int64_t n, int32_t count, int32_t mode,
                               int64_t switch_wl, int64_t* rec, int64_t cap,
                               int64_t* iterations, void* stream) {
  using namespace ipgc;
  if (!ctx || n < 0 || n > INT32_MAX || count < 1) return IPGC_ERR_INVALID;
  if (mode != IPGC_PUSH_WL && mode != IPGC_PUSH_NOWL && mode != IPGC_PUSH_HYBRID)
    return IPGC_ERR_INVALID;
  if (cap < 0 || (cap > 0 && !rec)) return IPGC_ERR_INVALID;
  if (iterations) *iterations = 0;
  if (n == 0) return IPGC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = ctx_device(ctx), prev = -1;
  cudaGetDevice(&prev);
  if (prev != dev) cudaSetDevice(dev);
  struct Restore {
    int prev, dev;
    ~Restore() {
      if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
  } restore{prev, dev};

  const size_t b_wl = al256(sizeof(int32_t) * (size_t)n);
  int rc = IPGC_OK;
  char* w = (char*)ctx_aux(ctx, 2 * b_wl + 256, &rc);
  if (!w) return rc;
  PushParams q;
  std::memset(&q, 0, sizeof(q));
  q.n = n;
  q.count = count;
  q.mode = mode;
  q.switch_wl = switch_wl;
  q.wl[0] = (int32_t*)w;
  q.wl[1] = (int32_t*)(w + b_wl);
  q.cnt = (int64_t*)(w + 2 * b_wl);
  q.rec = cap > 0 ? rec : nullptr;
  q.cap = cap;
  q.ctrl = ctx_ctrl_dev(ctx);
  q.timeout_ns = 10000000000ull;

  auto fail = [&](cudaError_t e) {
    ctx_note_cuda_error(ctx, (int)e);
    return e == cudaErrorMemoryAllocation ? IPGC_ERR_OOM : IPGC_ERR_CUDA;
  };
  cudaError_t e = cudaMemsetAsync(q.ctrl, 0, sizeof(Ctrl), s);
  if (e == cudaSuccess && q.rec) e = cudaMemsetAsync(q.rec, 0, sizeof(int64_t) * 4 * (size_t)cap, s);
  if (e != cudaSuccess) return fail(e);
  push_init_kernel<<<4 * ctx_num_sms(ctx), 256, 0, s>>>(q.wl[0], n, q.cnt);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
  int occ = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, push_kernel, kPushBS, 0)) !=
      cudaSuccess)
    return fail(e);
  void* args[] = {&q};
  e = cudaLaunchCooperativeKernel((const void*)push_kernel, dim3(occ * ctx_num_sms(ctx)),
                                  dim3(kPushBS), args, 0, s);
  if (e != cudaSuccess) return fail(e);
  Ctrl* h = ctx_ctrl_host(ctx);
  if ((e = cudaMemcpyAsync(h, q.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return fail(e);
  if (iterations) *iterations = h->rounds;
  return h->status;
}
