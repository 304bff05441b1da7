// Hybrid IPGC colouring of one graph on sm_103a.
//
// One round of Section II-C's loop is two phases separated by grid barriers:
//   assign: every active node v takes tent[v] = the smallest colour c >= 1
//           not committed on a neighbour (first fit / mex, Section II-C);
//           committed colours (color[]) are not written in this phase, so all
//           nodes see the snapshot of the previous round;
//   detect: v loses iff a lower-ID neighbour u has tent[u] == tent[v] (a
//           conflict, Section II-C; the higher ID stays in the worklist).
//           Finalised neighbours keep tent == their colour, which assign
//           excluded, so they never match. Winners commit color[v] = tent[v];
//           losers are pushed to the next worklist with warp-aggregated
//           atomics (the paper's Cooperative Conversion, Section V).
// Each round runs topology-driven (sweep all nodes, active iff color == 0)
// or data-driven (sweep the worklist), chosen from |WL| (Section IV); losers
// are pushed in both modes so the worklist stays alive (Sections I, IV).
// Round 1 is always topology-driven (|WL| = n): every tentative colour is 1,
// so v loses iff its smallest neighbour ID is below v, and with sorted rows
// that is one load.
//
// Work per node follows its degree bucket (the paper's Nested Parallelism,
// Section V): a warp colours 32 low-degree nodes together with their edges
// spread evenly over the lanes, a warp takes each mid-degree node, a CTA
// each high-degree node. The whole round loop runs inside one cooperative
// launch (the paper's Iteration Outlining, Section V).
#include <climits>

#include "ipgc_internal.h"

namespace ipgc {

enum { MODE_TOPO = IPGC_MODE_TOPO, MODE_DATA = IPGC_MODE_DATA };

template <int BS>
struct Smem {
  unsigned small_w[BS / 32][64];  // per warp: two mask words per lane / loser flags
  unsigned mid_w[BS / 32][32];    // per warp: bitmap of colours 1..1024
  unsigned big_w[kBigWords];      // per CTA: bitmap window of 65536 colours
  int bcast[4];
  int red[BS / 32];
};

template <int BS>
__device__ __forceinline__ void smem_clear(Smem<BS>& sm) {
  unsigned* w = &sm.small_w[0][0];
  for (int i = threadIdx.x; i < (BS / 32) * 64; i += BS) w[i] = 0;
  w = &sm.mid_w[0][0];
  for (int i = threadIdx.x; i < (BS / 32) * 32; i += BS) w[i] = 0;
  for (int i = threadIdx.x; i < kBigWords; i += BS) sm.big_w[i] = 0;
  __syncthreads();
}

template <int BS>
__device__ __forceinline__ int block_max(Smem<BS>& sm, int x) {
  const int warp = threadIdx.x >> 5, lane = lane_id();
  x = __reduce_max_sync(FULL, x);
  __syncthreads();
  if (lane == 0) sm.red[warp] = x;
  __syncthreads();
  int y = lane < BS / 32 ? sm.red[lane] : INT_MIN;
  y = __reduce_max_sync(FULL, y);
  return y;
}

template <int BS>
__device__ __forceinline__ int block_min(Smem<BS>& sm, int x) {
  const int warp = threadIdx.x >> 5, lane = lane_id();
  x = __reduce_min_sync(FULL, x);
  __syncthreads();
  if (lane == 0) sm.red[warp] = x;
  __syncthreads();
  int y = lane < BS / 32 ? sm.red[lane] : INT_MAX;
  y = __reduce_min_sync(FULL, y);
  return y;
}

// ---------------------------------------------------------------- round 1 --

// Round 1: all nodes active, all tentative colours 1. v wins iff no
// neighbour has a lower ID. Builds the worklist of round 2 (parity 0) and
// the static lists of mid / big nodes used by later topology sweeps.
template <int BS>
__device__ void round1(const Params& p, int& my_maxc) {
  Ctrl* c = p.ctrl;
  const int lane = lane_id();
  for (int64_t base = (int64_t)blockIdx.x * BS; base < p.n; base += (int64_t)gridDim.x * BS) {
    const int v = (int)(base + threadIdx.x);
    const bool valid = v < p.n;
    int d = 0;
    bool lose = false;
    if (valid) {
      const int s = ld_ro(p.rowptr + v), e = ld_ro(p.rowptr + v + 1);
      d = e - s;
      lose = d > 0 && ld_ro(p.col + s) < v;
      p.color[v] = lose ? 0 : 1;
      p.tent[v] = lose ? 0 : 1;
      if (!lose) my_maxc = 1;
      if (p.fin) p.fin[v] = lose ? 0 : 1;
    }
    const int b = bucket_of(d, p.t1, p.t2);
#pragma unroll
    for (int k = 0; k < NB; ++k) warp_push(lose && b == k, v, p.wl[0][k], &c->cnt[0][k]);
    warp_push(valid && b == B_MID, v, p.stat[B_MID], &c->nstat[B_MID]);
    warp_push(valid && b == B_BIG, v, p.stat[B_BIG], &c->nstat[B_BIG]);
    const unsigned long long ds = warp_sum_u64(lose ? (unsigned long long)d : 0ull);
    if (lane == 0 && ds) atomicAdd(&c->dsum[0], ds);
  }
}

// ------------------------------------------------------- small-degree nodes --
//
// A warp handles up to 32 nodes of degree <= t1 (<= 63), one per lane (idle
// lanes: v = -1, d = 0). Their edge lists are laid end to end and dealt out
// to the lanes 32 at a time, so loads stay coalesced within a row and no lane
// idles while another walks a long row. The owner of edge e is the last lane
// whose exclusive prefix offset is <= e.

struct SmallSeg {
  int off;    // exclusive prefix of degrees over the warp
  int total;  // sum of degrees over the warp
};

__device__ __forceinline__ SmallSeg small_scan(int d) {
  const int lane = lane_id();
  int incl = d;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  SmallSeg g;
  g.off = incl - d;
  g.total = __shfl_sync(FULL, incl, 31);
  return g;
}

__device__ __forceinline__ int small_owner(int off, int e) {
  int j = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const int cand = j + step;
    const int oc = __shfl_sync(FULL, off, cand);
    if (oc <= e) j = cand;
  }
  return j;
}

constexpr int kSmallUnroll = 4;

// First-fit colour of each lane's node into tent[v]. wm: this warp's 64 words.
__device__ __forceinline__ void small_assign(const Params& p, int v, int s, int d, unsigned* wm) {
  const int lane = lane_id();
  const SmallSeg g = small_scan(d);
  wm[2 * lane] = 0;
  wm[2 * lane + 1] = 0;
  __syncwarp();
  for (int base = 0; base < g.total; base += 32 * kSmallUnroll) {
    int u[kSmallUnroll], j[kSmallUnroll];
#pragma unroll
    for (int q = 0; q < kSmallUnroll; ++q) {
      const int e = base + q * 32 + lane;
      const int jj = small_owner(g.off, e);
      const int sj = __shfl_sync(FULL, s, jj);
      const int oj = __shfl_sync(FULL, g.off, jj);
      j[q] = jj;
      u[q] = e < g.total ? ld_ro(p.col + sj + (e - oj)) : -1;
    }
    int cc[kSmallUnroll];
#pragma unroll
    for (int q = 0; q < kSmallUnroll; ++q) cc[q] = u[q] >= 0 ? ld_cg(p.color + u[q]) : 0;
#pragma unroll
    for (int q = 0; q < kSmallUnroll; ++q) {
      const int c = cc[q];
      if (c >= 1 && c <= 64) atomicOr(&wm[2 * j[q] + ((c - 1) >> 5)], 1u << ((c - 1) & 31));
    }
  }
  __syncwarp();
  if (v >= 0) {
    const unsigned long long m =
        (unsigned long long)wm[2 * lane] | ((unsigned long long)wm[2 * lane + 1] << 32);
    p.tent[v] = __ffsll((long long)~m);
  }
  __syncwarp();
}

// Loser flag of each lane's node (t = its tentative colour).
__device__ __forceinline__ bool small_lose(const Params& p, int v, int s, int d, int t,
                                           unsigned* wm) {
  const int lane = lane_id();
  const SmallSeg g = small_scan(d);
  wm[lane] = 0;
  __syncwarp();
  for (int base = 0; base < g.total; base += 32 * kSmallUnroll) {
    int u[kSmallUnroll], j[kSmallUnroll];
#pragma unroll
    for (int q = 0; q < kSmallUnroll; ++q) {
      const int e = base + q * 32 + lane;
      const int jj = small_owner(g.off, e);
      const int sj = __shfl_sync(FULL, s, jj);
      const int oj = __shfl_sync(FULL, g.off, jj);
      const int vj = __shfl_sync(FULL, v, jj);
      j[q] = jj;
      const int uu = e < g.total ? ld_ro(p.col + sj + (e - oj)) : INT_MAX;
      u[q] = uu < vj ? uu : -1;  // only lower-ID neighbours can beat v
    }
    int tt[kSmallUnroll];
#pragma unroll
    for (int q = 0; q < kSmallUnroll; ++q) tt[q] = u[q] >= 0 ? ld_cg(p.tent + u[q]) : 0;
#pragma unroll
    for (int q = 0; q < kSmallUnroll; ++q) {
      const int tj = __shfl_sync(FULL, t, j[q]);
      if (u[q] >= 0 && tt[q] == tj) wm[j[q]] = 1u;
    }
  }
  __syncwarp();
  const bool lose = wm[lane] != 0;
  __syncwarp();
  return lose;
}

// --------------------------------------------------------- mid-degree nodes --

// One warp, one node of degree t1 < d <= t2 (<= 1023): lane-private mask for
// colours 1..32, shared per-warp bitmap for 33..1024. wb is zero on entry and
// on exit.
__device__ __forceinline__ int mid_assign(const Params& p, int s, int d, unsigned* wb) {
  const int lane = lane_id();
  unsigned pm = 0;
  for (int k0 = 0; k0 < d; k0 += 32 * 4) {
    int u[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = k0 + q * 32 + lane;
      u[q] = k < d ? ld_ro(p.col + s + k) : -1;
    }
    int cc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) cc[q] = u[q] >= 0 ? ld_cg(p.color + u[q]) : 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = cc[q];
      if (c >= 1 && c <= 32)
        pm |= 1u << (c - 1);
      else if (c > 32 && c <= 1024)
        atomicOr(&wb[(c - 1) >> 5], 1u << ((c - 1) & 31));
    }
  }
  __syncwarp();
  pm = __reduce_or_sync(FULL, pm);
  const unsigned w = lane == 0 ? (pm | wb[0]) : wb[lane];
  const unsigned nf = __ballot_sync(FULL, w != FULL);  // non-zero: d <= 1023
  const int fl = __ffs(nf) - 1;
  const unsigned wf = __shfl_sync(FULL, w, fl);
  const int t = 32 * fl + __ffs(~wf);
  __syncwarp();
  wb[lane] = 0;
  __syncwarp();
  return t;
}

__device__ __forceinline__ bool mid_lose(const Params& p, int v, int s, int d, int t) {
  const int lane = lane_id();
  for (int k0 = 0; k0 < d; k0 += 32) {
    const int k = k0 + lane;
    const int u = k < d ? ld_ro(p.col + s + k) : INT_MAX;
    const bool hit = u < v && ld_cg(p.tent + u) == t;
    if (__any_sync(FULL, hit)) return true;
    if (__any_sync(FULL, u >= v)) return false;  // rows are sorted
  }
  return false;
}

// -------------------------------------------------------- high-degree nodes --

// One CTA, one node of degree d > t2. Only colours 1..lim with
// lim = min(d, maxc) + 1 can decide the first fit, since the answer is at
// most d + 1 and at most (largest committed colour) + 1. Colours are
// scanned in windows of 32 * kBigWords (one window unless lim exceeds it).
template <int BS>
__device__ int big_assign(const Params& p, Smem<BS>& sm, int s, int d, int maxc) {
  const int lane = lane_id();
  const int lim = min(d, maxc) + 1;
  for (int wbase = 0;; wbase += 32 * kBigWords) {
    const int wcols = min(lim - wbase, 32 * kBigWords);
    if (wcols <= 0) {  // unreachable for a valid graph: some colour <= lim is free
      if (threadIdx.x == 0) atomicCAS(&p.ctrl->status, 0, IPGC_ERR_INVALID);
      return lim;
    }
    const int nw = (wcols + 31) >> 5;
    unsigned pm = 0;
    for (int k0 = 0; k0 < d; k0 += BS * 4) {
      int u[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + q * BS + threadIdx.x;
        u[q] = k < d ? ld_ro(p.col + s + k) : -1;
      }
      int cc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) cc[q] = u[q] >= 0 ? ld_cg(p.color + u[q]) : 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = cc[q] - wbase;
        if (c >= 1 && c <= 32)
          pm |= 1u << (c - 1);
        else if (c > 32 && c <= wcols)
          atomicOr(&sm.big_w[(c - 1) >> 5], 1u << ((c - 1) & 31));
      }
    }
    pm = __reduce_or_sync(FULL, pm);
    if (lane == 0 && pm) atomicOr(&sm.big_w[0], pm);
    __syncthreads();
    int first = INT_MAX;
    for (int i = threadIdx.x; i < nw; i += BS)
      if (sm.big_w[i] != FULL) {
        first = i;
        break;
      }
    first = block_min<BS>(sm, first);
    int t = 0;
    if (first != INT_MAX) t = wbase + 32 * first + __ffs(~sm.big_w[first]);
    __syncthreads();
    for (int i = threadIdx.x; i < nw; i += BS) sm.big_w[i] = 0;
    __syncthreads();
    if (first != INT_MAX) return t;
  }
}

template <int BS>
__device__ bool big_lose(const Params& p, int v, int s, int d, int t) {
  for (int k0 = 0; k0 < d; k0 += BS) {
    const int k = k0 + threadIdx.x;
    const int u = k < d ? ld_ro(p.col + s + k) : INT_MAX;
    const bool hit = u < v && ld_cg(p.tent + u) == t;
    if (__syncthreads_or(hit)) return true;
    if (__syncthreads_or(u >= v)) return false;
  }
  return false;
}

// ------------------------------------------------------------------ phases --

struct RoundView {
  int round;     // 1-based round number
  int par;       // worklist parity read this round
  int mode;      // MODE_TOPO or MODE_DATA
  int cnt[NB];   // worklist sizes
  int nstat[NB]; // static list sizes
  int maxc;      // largest committed colour at round start
};

__device__ __forceinline__ RoundView read_round(const Params& p, int r) {
  RoundView rv;
  rv.round = r;
  rv.par = r & 1;
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    rv.cnt[k] = ld_cg(&p.ctrl->cnt[rv.par][k]);
    rv.nstat[k] = ld_cg(&p.ctrl->nstat[k]);
  }
  rv.maxc = ld_cg(&p.ctrl->maxc);
  rv.mode = MODE_DATA;
  return rv;
}

__device__ __forceinline__ int decide_mode(const Params& p, int64_t total) {
  if (p.policy == IPGC_MODE_TOPO) return MODE_TOPO;
  if (p.policy == IPGC_MODE_DATA) return MODE_DATA;
  return total > p.H ? MODE_TOPO : MODE_DATA;
}

// Bookkeeping by CTA 0 at the start of round r (after the previous barrier):
// clear the counters this round pushes into and the work counters of the
// next round, count the round.
__device__ __forceinline__ void round_begin(const Params& p, const RoundView& rv, int r,
                                            int64_t total) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  Ctrl* c = p.ctrl;
  const int nxt = rv.par ^ 1;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    c->cnt[nxt][k] = 0;
    c->grab[nxt][k] = 0;
  }
  c->dsum[nxt] = 0;
  c->rounds = r;
  if (rv.mode == MODE_TOPO)
    c->rounds_topo += 1;
  else
    c->rounds_data += 1;
  c->last_mode = rv.mode;
  const unsigned long long ds = __ldcg(&c->dsum[rv.par]);
  c->edges += ds;
  if (p.trace && r <= p.trace_cap) {
    ipgc_trace_rec& tr = p.trace[r - 1];
    tr.round = r;
    tr.mode = rv.mode;
    tr.wl_size = total;
    tr.deg_sum = (int64_t)ds;
    tr.max_color = rv.maxc;
    tr.shortcut = 0;
    tr.t_begin = gtime();
  }
  __threadfence();
}

template <int BS>
__device__ void assign_phase(const Params& p, Smem<BS>& sm, const RoundView& rv) {
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const int gwarp = blockIdx.x * (BS / 32) + warp, nwarps = gridDim.x * (BS / 32);
  const bool topo = rv.mode == MODE_TOPO;
  // high-degree nodes: one CTA each, taken from a shared counter
  {
    const int32_t* list = topo ? p.stat[B_BIG] : p.wl[rv.par][B_BIG];
    const int count = topo ? rv.nstat[B_BIG] : rv.cnt[B_BIG];
    for (;;) {
      __syncthreads();
      if (threadIdx.x == 0) sm.bcast[0] = (int)atomicAdd(&p.ctrl->grab[rv.par][G_ASSIGN_BIG], 1u);
      __syncthreads();
      const int idx = sm.bcast[0];
      if (idx >= count) break;
      const int v = ld_cg(list + idx);
      if (topo && ld_cg(p.color + v) != 0) continue;
      const int s = ld_ro(p.rowptr + v), d = ld_ro(p.rowptr + v + 1) - s;
      const int t = big_assign<BS>(p, sm, s, d, rv.maxc);
      if (threadIdx.x == 0) p.tent[v] = t;
    }
  }
  // mid-degree nodes: one warp each
  {
    const int32_t* list = topo ? p.stat[B_MID] : p.wl[rv.par][B_MID];
    const int count = topo ? rv.nstat[B_MID] : rv.cnt[B_MID];
    unsigned* wb = sm.mid_w[warp];
    for (int i = gwarp; i < count; i += nwarps) {
      const int v = ld_cg(list + i);
      if (topo && ld_cg(p.color + v) != 0) continue;
      const int s = ld_ro(p.rowptr + v), d = ld_ro(p.rowptr + v + 1) - s;
      const int t = mid_assign(p, s, d, wb);
      if (lane == 0) p.tent[v] = t;
    }
  }
  // low-degree nodes: 32 per warp
  {
    unsigned* wm = sm.small_w[warp];
    const int64_t span = topo ? (int64_t)p.n : (int64_t)rv.cnt[B_SMALL];
    for (int64_t base = (int64_t)gwarp * 32; base < span; base += (int64_t)nwarps * 32) {
      const int64_t i = base + lane;
      int v = -1, s = 0, d = 0;
      if (i < span) {
        v = topo ? (int)i : ld_cg(p.wl[rv.par][B_SMALL] + i);
        s = ld_ro(p.rowptr + v);
        d = ld_ro(p.rowptr + v + 1) - s;
        if (topo && (d > p.t1 || ld_cg(p.color + v) != 0)) {
          v = -1;
          d = 0;
        }
      }
      small_assign(p, v, s, d, wm);
    }
  }
}

template <int BS>
__device__ void detect_phase(const Params& p, Smem<BS>& sm, const RoundView& rv, int& my_maxc) {
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const int gwarp = blockIdx.x * (BS / 32) + warp, nwarps = gridDim.x * (BS / 32);
  const bool topo = rv.mode == MODE_TOPO;
  const int nxt = rv.par ^ 1;
  Ctrl* c = p.ctrl;
  {
    const int32_t* list = topo ? p.stat[B_BIG] : p.wl[rv.par][B_BIG];
    const int count = topo ? rv.nstat[B_BIG] : rv.cnt[B_BIG];
    for (;;) {
      __syncthreads();
      if (threadIdx.x == 0) sm.bcast[0] = (int)atomicAdd(&c->grab[rv.par][G_DETECT_BIG], 1u);
      __syncthreads();
      const int idx = sm.bcast[0];
      if (idx >= count) break;
      const int v = ld_cg(list + idx);
      if (topo && ld_cg(p.color + v) != 0) continue;
      const int s = ld_ro(p.rowptr + v), d = ld_ro(p.rowptr + v + 1) - s;
      const int t = ld_cg(p.tent + v);
      const bool lose = big_lose<BS>(p, v, s, d, t);
      if (threadIdx.x == 0) {
        if (lose) {
          const int pos = atomicAdd(&c->cnt[nxt][B_BIG], 1);
          p.wl[nxt][B_BIG][pos] = v;
          atomicAdd(&c->dsum[nxt], (unsigned long long)d);
        } else {
          p.color[v] = t;
          my_maxc = max(my_maxc, t);
          if (p.fin) p.fin[v] = rv.round;
        }
      }
    }
  }
  {
    const int32_t* list = topo ? p.stat[B_MID] : p.wl[rv.par][B_MID];
    const int count = topo ? rv.nstat[B_MID] : rv.cnt[B_MID];
    for (int i = gwarp; i < count; i += nwarps) {
      const int v = ld_cg(list + i);
      if (topo && ld_cg(p.color + v) != 0) continue;
      const int s = ld_ro(p.rowptr + v), d = ld_ro(p.rowptr + v + 1) - s;
      const int t = ld_cg(p.tent + v);
      const bool lose = mid_lose(p, v, s, d, t);
      if (lane == 0) {
        if (lose) {
          const int pos = atomicAdd(&c->cnt[nxt][B_MID], 1);
          p.wl[nxt][B_MID][pos] = v;
          atomicAdd(&c->dsum[nxt], (unsigned long long)d);
        } else {
          p.color[v] = t;
          my_maxc = max(my_maxc, t);
          if (p.fin) p.fin[v] = rv.round;
        }
      }
    }
  }
  {
    unsigned* wm = sm.small_w[warp];
    const int64_t span = topo ? (int64_t)p.n : (int64_t)rv.cnt[B_SMALL];
    for (int64_t base = (int64_t)gwarp * 32; base < span; base += (int64_t)nwarps * 32) {
      const int64_t i = base + lane;
      int v = -1, s = 0, d = 0, t = 0;
      if (i < span) {
        v = topo ? (int)i : ld_cg(p.wl[rv.par][B_SMALL] + i);
        s = ld_ro(p.rowptr + v);
        d = ld_ro(p.rowptr + v + 1) - s;
        if (topo && (d > p.t1 || ld_cg(p.color + v) != 0)) {
          v = -1;
          d = 0;
        }
      }
      if (v >= 0) t = ld_cg(p.tent + v);
      const bool lose = small_lose(p, v, s, d, t, wm);
      warp_push(v >= 0 && lose, v, p.wl[nxt][B_SMALL], &c->cnt[nxt][B_SMALL]);
      const unsigned long long ds = warp_sum_u64(v >= 0 && lose ? (unsigned long long)d : 0ull);
      if (lane == 0 && ds) atomicAdd(&c->dsum[nxt], ds);
      if (v >= 0 && !lose) {
        p.color[v] = t;
        my_maxc = max(my_maxc, t);
        if (p.fin) p.fin[v] = rv.round;
      }
    }
  }
}

template <int BS>
__device__ __forceinline__ void commit_maxc(const Params& p, Smem<BS>& sm, int my_maxc) {
  const int m = block_max<BS>(sm, my_maxc);
  if (threadIdx.x == 0 && m > 0) atomicMax(&p.ctrl->maxc, m);
}

__device__ __forceinline__ void trace_round1(const Params& p, uint64_t t0) {
  Ctrl* c = p.ctrl;
  c->rounds = 1;
  c->rounds_topo = 1;
  c->last_mode = MODE_TOPO;
  c->edges = (unsigned long long)p.nnz;
  if (p.trace && p.trace_cap >= 1) {
    const uint64_t t1 = gtime();
    ipgc_trace_rec& tr = p.trace[0];
    tr.round = 1;
    tr.mode = MODE_TOPO;
    tr.wl_size = p.n;
    tr.deg_sum = p.nnz;
    tr.max_color = 0;
    tr.shortcut = 1;
    tr.t_begin = t0;
    tr.t_assign = t0;
    tr.t_detect = t1;
  }
}

// ------------------------------------------------------- persistent kernel --

template <int BS>
__global__ void __launch_bounds__(BS, 2) persistent_kernel(Params p) {
  __shared__ Smem<BS> sm;
  smem_clear<BS>(sm);
  Ctrl* c = p.ctrl;
  const uint64_t t0 = gtime();
  if (blockIdx.x == 0 && threadIdx.x == 0) c->t_start = t0;
  int my_maxc = 0;
  round1<BS>(p, my_maxc);
  commit_maxc<BS>(p, sm, my_maxc);
  if (!grid_barrier(c, p.timeout_ns, p.bar_extra)) goto done;
  if (blockIdx.x == 0 && threadIdx.x == 0) trace_round1(p, t0);
  for (int r = 2;; ++r) {
    RoundView rv = read_round(p, r);
    const int64_t total = (int64_t)rv.cnt[0] + rv.cnt[1] + rv.cnt[2];
    if (total == 0) break;
    if (r > p.max_rounds) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&c->status, 0, IPGC_ERR_NO_CONVERGE);
      break;
    }
    rv.mode = decide_mode(p, total);
    round_begin(p, rv, r, total);
    assign_phase<BS>(p, sm, rv);
    if (!grid_barrier(c, p.timeout_ns, p.bar_extra)) break;
    if (blockIdx.x == 0 && threadIdx.x == 0 && p.trace && r <= p.trace_cap)
      p.trace[r - 1].t_assign = gtime();
    my_maxc = 0;
    detect_phase<BS>(p, sm, rv, my_maxc);
    commit_maxc<BS>(p, sm, my_maxc);
    if (!grid_barrier(c, p.timeout_ns, p.bar_extra)) break;
    if (blockIdx.x == 0 && threadIdx.x == 0 && p.trace && r <= p.trace_cap)
      p.trace[r - 1].t_detect = gtime();
  }
done:
  if (blockIdx.x == 0 && threadIdx.x == 0) c->t_end = gtime();
}

// ------------------------------------------------------ host-loop kernels --

template <int BS>
__global__ void __launch_bounds__(BS, 2) round1_kernel(Params p) {
  __shared__ Smem<BS> sm;
  const uint64_t t0 = gtime();
  if (blockIdx.x == 0 && threadIdx.x == 0) p.ctrl->t_start = t0;
  int my_maxc = 0;
  round1<BS>(p, my_maxc);
  commit_maxc<BS>(p, sm, my_maxc);
  if (blockIdx.x == 0 && threadIdx.x == 0) trace_round1(p, t0);
}

template <int BS>
__global__ void __launch_bounds__(BS, 2) assign_kernel(Params p, int r, int mode) {
  __shared__ Smem<BS> sm;
  smem_clear<BS>(sm);
  RoundView rv = read_round(p, r);
  rv.mode = mode;
  const int64_t total = (int64_t)rv.cnt[0] + rv.cnt[1] + rv.cnt[2];
  round_begin(p, rv, r, total);
  assign_phase<BS>(p, sm, rv);
}

template <int BS>
__global__ void __launch_bounds__(BS, 2) detect_kernel(Params p, int r, int mode) {
  __shared__ Smem<BS> sm;
  smem_clear<BS>(sm);
  if (blockIdx.x == 0 && threadIdx.x == 0 && p.trace && r <= p.trace_cap)
    p.trace[r - 1].t_assign = gtime();
  RoundView rv = read_round(p, r);
  rv.mode = mode;
  int my_maxc = 0;
  detect_phase<BS>(p, sm, rv, my_maxc);
  commit_maxc<BS>(p, sm, my_maxc);
}

__global__ void finish_kernel(Params p, int last_round) {
  if (p.trace && last_round >= 2 && last_round <= p.trace_cap) p.trace[last_round - 1].t_detect = gtime();
  p.ctrl->t_end = gtime();
}

// ------------------------------------------------------------- validation --

// One warp per row: offsets sane, entries in range, no self-loop, strictly
// ascending, and every (v, u) has its (u, v) (binary search in row u).
__global__ void validate_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                int32_t n, int64_t nnz, int* err) {
  const int lane = lane_id();
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (gw == 0 && lane == 0) {
    if (rowptr[0] != 0 || (int64_t)rowptr[n] != nnz) atomicOr(err, 1);
  }
  for (int64_t v = gw; v < n; v += nw) {
    const int s = rowptr[v], e = rowptr[v + 1];
    if (s < 0 || e < s || (int64_t)e > nnz) {
      if (lane == 0) atomicOr(err, 2);
      continue;
    }
    for (int k = s + lane; k < e; k += 32) {
      const int u = col[k];
      if (u < 0 || u >= n || u == (int)v) {
        atomicOr(err, 4);
        continue;
      }
      if (k > s && col[k - 1] >= u) atomicOr(err, 8);
      const int lo0 = rowptr[u], hi0 = rowptr[u + 1];
      if (lo0 < 0 || hi0 < lo0 || (int64_t)hi0 > nnz) {
        atomicOr(err, 2);
        continue;
      }
      int lo = lo0, hi = hi0;  // search v in col[lo, hi)
      while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        if (col[mid] < (int)v)
          lo = mid + 1;
        else
          hi = mid;
      }
      if (lo >= hi0 || col[lo] != (int)v) atomicOr(err, 16);
    }
  }
}

// ------------------------------------------------------------ host launch --

cudaError_t occupancy_persistent(int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, persistent_kernel<kBlock>,
                                                       kBlock, 0);
}

cudaError_t launch_persistent(const Params& p, int blocks, cudaStream_t s) {
  Params pp = p;
  void* args[] = {&pp};
  return cudaLaunchCooperativeKernel((const void*)persistent_kernel<kBlock>, dim3(blocks),
                                     dim3(kBlock), args, 0, s);
}

cudaError_t launch_round1(const Params& p, int blocks, cudaStream_t s) {
  round1_kernel<kBlock><<<blocks, kBlock, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_assign(const Params& p, int blocks, int round, int mode, cudaStream_t s) {
  assign_kernel<kBlock><<<blocks, kBlock, 0, s>>>(p, round, mode);
  return cudaGetLastError();
}

cudaError_t launch_detect(const Params& p, int blocks, int round, int mode, cudaStream_t s) {
  detect_kernel<kBlock><<<blocks, kBlock, 0, s>>>(p, round, mode);
  return cudaGetLastError();
}

cudaError_t launch_finish(const Params& p, int last_round, cudaStream_t s) {
  finish_kernel<<<1, 1, 0, s>>>(p, last_round);
  return cudaGetLastError();
}

cudaError_t launch_validate(const int32_t* rowptr, const int32_t* col, int32_t n, int64_t nnz,
                            int* d_err, int blocks, cudaStream_t s) {
  validate_kernel<<<blocks, 256, 0, s>>>(rowptr, col, n, nnz, d_err);
  return cudaGetLastError();
}

}  // namespace ipgc
