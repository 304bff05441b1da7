// The phases of the hybrid IPGC loop for one graph, shared by the
// single-graph kernels (ipgc_color.cu) and the batched kernel
// (ipgc_batched.cu). See ipgc_color.cu for the method.
#pragma once

#include <climits>
#include <type_traits>

#include "ipgc_device.cuh"

namespace ipgc {

enum { MODE_TOPO = IPGC_MODE_TOPO, MODE_DATA = IPGC_MODE_DATA };

// Resident CTAs per SM each block size is compiled for: 512 threads x 2 or
// 256 x 4 cap a thread at 64 registers. The rescanning kernels are mostly
// the packed low-degree loop, which wants warps (road 5.3 -> 3.6 ms going
// from 3 CTAs of 256 to 4, same GPU); the pushing kernel keeps 3 (its own
// bound, in ipgc_color.cu).
constexpr int min_blocks(int bs) { return bs >= 512 ? 2 : 4; }

template <int BS>
struct Smem {
  static constexpr int W = BS / 32;
  unsigned small_w[W][32 * kSmallWords];  // per warp: the lanes' colour masks / loser flags
  unsigned wbits[W][kGWords];       // per warp: bitmap of colours 1..2048 (work items)
  int32_t stage_s[W][kStageSmall];  // staged pushes: low-degree losers
  int4 stage_i[W][kStageItems];     // staged pushes: work items of high-degree losers
  int4 stage_t[W][kStageItems];     // staged pushes: static work items (round 1),
                                    // items of filtered nodes (conflict steps)
  unsigned long long red64[W];
  int red[W];
  int mode_b;  // broadcast of the round's mode (learned policy)
  unsigned red2[W];
  unsigned red3[W];
  unsigned red4[W];
  int rvb[24];  // round state read from the control block once per CTA
  int rvn[16];  // round rvn_round's state, read ahead (before a push phase)
  int rvn_round;
  BarMemo bar;  // the last team barrier this CTA passed (team_barrier)
};

// Whether team barriers count arrivals against the CTA's memo (BarMemo)
// instead of releasing generations: on in every kernel that colours graphs
// (a translation unit may turn it off by defining it as 0).
#ifndef IPGC_BAR_MEMO
#define IPGC_BAR_MEMO 1
#endif

template <int BS>
__device__ __forceinline__ BarMemo* bar_memo(Smem<BS>& sm) {
  return IPGC_BAR_MEMO ? &sm.bar : nullptr;
}

// bar_idx: the kernel's arrival counter for the counting barrier (one per
// single-graph kernel of a colouring: 0 pushing, 1 rescanning, 2 filtering).
template <int BS>
__device__ __forceinline__ void smem_clear(Smem<BS>& sm, int bar_idx = 0) {
  unsigned* w = &sm.small_w[0][0];
  for (int i = threadIdx.x; i < Smem<BS>::W * 32 * kSmallWords; i += BS) w[i] = 0;
  w = &sm.wbits[0][0];
  for (int i = threadIdx.x; i < Smem<BS>::W * kGWords; i += BS) w[i] = 0;
  if (threadIdx.x == 0) {
    sm.bar.ctrl = nullptr;
    sm.bar.idx = bar_idx;
    sm.rvn_round = 0;
  }
  __syncthreads();
}

template <int BS>
__device__ __forceinline__ int block_max(Smem<BS>& sm, int x) {
  const int warp = threadIdx.x >> 5, lane = lane_id();
  x = __reduce_max_sync(FULL, x);
  __syncthreads();
  if (lane == 0) sm.red[warp] = x;
  __syncthreads();
  int y = lane < Smem<BS>::W ? sm.red[lane] : INT_MIN;
  return __reduce_max_sync(FULL, y);
}

template <int BS>
__device__ __forceinline__ unsigned long long block_sum64(Smem<BS>& sm, unsigned long long x) {
  const int warp = threadIdx.x >> 5, lane = lane_id();
  x = warp_sum_u64(x);
  __syncthreads();
  if (lane == 0) sm.red64[warp] = x;
  __syncthreads();
  unsigned long long y = lane < Smem<BS>::W ? sm.red64[lane] : 0ull;
  return warp_sum_u64(y);
}

// Per-thread accumulators of one phase, merged once per CTA at its end.
struct PhaseAcc {
  int maxc = 0;                 // largest colour committed by this thread
  unsigned long long dsum = 0;  // degrees of the nodes this thread pushed
  unsigned long long nbig = 0;  // high-degree nodes this thread pushed
  unsigned long long nsm = 0;   // low-degree losers counted, not pushed (worklist rebuild)
  unsigned nodd = 0;            // pushing: losers that keep the next round from running late
};

// One CTA-wide reduction of the accumulators, then one atomic each.
template <int BS>
__device__ __forceinline__ void phase_commit(const Params& p, Smem<BS>& sm, const PhaseAcc& a,
                                             int nxt) {
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const int m = __reduce_max_sync(FULL, a.maxc);
  const unsigned long long ds = warp_sum_u64(a.dsum);
  const unsigned nb = __reduce_add_sync(FULL, (unsigned)a.nbig);
  const unsigned ns = __reduce_add_sync(FULL, (unsigned)a.nsm);
  const unsigned no = __reduce_add_sync(FULL, a.nodd);
  __syncthreads();  // previous users of the scratch slots are done
  if (lane == 0) {
    sm.red[warp] = m;
    sm.red64[warp] = ds;
    sm.red2[warp] = nb;
    sm.red3[warp] = ns;
    sm.red4[warp] = no;
  }
  __syncthreads();
  if (warp == 0) {
    const bool in = lane < Smem<BS>::W;
    const int mm = __reduce_max_sync(FULL, in ? sm.red[lane] : 0);
    const unsigned long long dd = warp_sum_u64(in ? sm.red64[lane] : 0ull);
    const unsigned bb = __reduce_add_sync(FULL, in ? sm.red2[lane] : 0u);
    const unsigned ss = __reduce_add_sync(FULL, in ? sm.red3[lane] : 0u);
    const unsigned oo = __reduce_add_sync(FULL, in ? sm.red4[lane] : 0u);
    if (lane == 0) {
      if (mm > 0) atomicMax(&p.ctrl->maxc, mm);
      if (dd) atomicAdd(&p.ctrl->dsum[nxt], dd);
      if (bb) atomicAdd(&p.ctrl->cnt[nxt][B_BIG], (int)bb);
      if (ss) atomicAdd(&p.ctrl->cnt[nxt][B_SMALL], (int)ss);
      if (oo) atomicAdd(&p.ctrl->cnt[nxt][2], (int)oo);
    }
  }
}

__device__ __forceinline__ int num_chunks(int d, int chunk) { return (d + chunk - 1) / chunk; }

// A node of degree > t1 committed: with pushing, it no longer receives pushes
// (round 1 writes pinfo for every node, and the degree of a node of degree
// <= t1 or committed in round 1 as 0; later commits retire their node here).
__device__ __forceinline__ void retire_push_target(const Params& p, int v) {
  if (p.pinfo) p.pinfo[v].y = 0;
}

// ---------------------------------------------------------------- round 1 --

__device__ __forceinline__ void small_push(const Params& p, int s, int d, int t, int t1,
                                           bool check_active);

// Round 1: all nodes active, all tentative colours 1. v wins iff no
// neighbour has a lower ID. Builds the worklist of round 2 (parity 0) and
// the static work items of every high-degree node used by later topology
// sweeps; hands out merge-state slots to nodes with several items.
template <int BS, bool PUSH = false>
__device__ void round1(const Params& p, Smem<BS>& sm, PhaseAcc& acc, Team tm, int t1,
                       bool pushing) {
  Ctrl* c = p.ctrl;
  const int warp = threadIdx.x >> 5, lane = lane_id();
  WarpStage ss{sm.stage_s[warp], 0};
  ItemStage si{sm.stage_i[warp], 0}, st{sm.stage_t[warp], 0};
  for (int64_t base = (int64_t)tm.cta * BS; base < p.n; base += (int64_t)tm.ncta * BS) {
    const int v = (int)(base + threadIdx.x);
    const bool valid = v < p.n;
    int d = 0, s = 0;
    bool lose = false;
    if (valid) {
      s = ld_ro(p.rowptr + v);
      const int e = ld_ro(p.rowptr + v + 1);
      d = e - s;
      lose = d > 0 && ld_ro(p.col + s) < v;
      p.color[v] = lose ? 0 : 1;
      p.tent[v] = lose ? 0 : 1;
      // push targets: the nodes above t1 that stay active (the pushes of this
      // pass do not read these; the push phase after it does)
      if (PUSH && pushing && p.pinfo) p.pinfo[v] = make_int2(s, lose && d > t1 ? d : 0);
      if (!lose) acc.maxc = 1;
      if (p.fin) p.fin[v] = lose ? 0 : 1;
      if (lose) acc.dsum += (unsigned long long)d;
    }
    const bool big = valid && bucket_of(d, t1) == B_BIG;
    // round 1 is topology-driven: with worklist rebuild its losers are counted, not pushed
    const bool keep = !p.wl_rebuild;
    stage_push(ss, kStageSmall, keep && lose && !big, v, p.wl[0], &c->cnt[0][B_SMALL]);
    if (!keep && lose && !big) acc.nsm += 1;
    const int nch = big ? num_chunks(d, p.chunk) : 0;
    const bool multi = nch > 1;  // (every node that can be filtered is one of them)
    const unsigned mm = __ballot_sync(FULL, multi);
    int gslot = -1;
    if (mm) {
      int gb = 0;
      if (lane == 0) gb = atomicAdd(&c->ngslot, __popc(mm));
      gb = __shfl_sync(FULL, gb, 0);
      if (multi) {
        gslot = gb + __popc(mm & ((1u << lane) - 1u));
        for (int i = 0; i < kGWords; ++i) p.gbits[(size_t)gslot * kGWords + i] = 0;
        p.done_a[gslot] = 0;
        p.done_d[gslot] = 0;
        p.flag[gslot] = 0;
        if (PUSH && p.alist[0]) {  // lower-neighbour list state
          p.flen[0][gslot] = make_int2(0, 0);
          p.flen[1][gslot] = make_int2(0, 0);
          p.fst[gslot] = 0;
          p.fdead[gslot] = 0;
        }
      }
    }
    items_push(st, v, nch, gslot, p.istat, &c->nistat);
    items_push(si, v, keep && lose ? nch : 0, gslot, p.items[0], &c->icnt[0]);
    if (big && lose) acc.nbig += 1;
    if (PUSH && pushing) {  // winners: colour 1 into their neighbours' bitmaps
      const bool win = valid && !lose;
      small_push(p, s, win && !big ? d : 0, 1, t1, false);
      // the others' rows: queued for the push phase after round 1, one lane at a time
      const int nq = win && big ? push_items_of(s, d) : 0;
      int incl = nq;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += y;
      }
      const int tot = __shfl_sync(FULL, incl, 31);
      if (tot) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&c->pqcnt, tot);
        base = __shfl_sync(FULL, base, 0) + incl - nq;
        for (int j = 0; j < nq; ++j) p.pq[base + j] = make_int4(s, d, 1, j);
      }
    }
  }
  stage_flush(ss, p.wl[0], &c->cnt[0][B_SMALL]);
  items_flush(st, p.istat, &c->nistat);
  items_flush(si, p.items[0], &c->icnt[0]);
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

// First-fit colour of each lane's node into tent[v]. wm: this warp's 32 * kSmallWords words.
__device__ __forceinline__ void small_assign(const Params& p, int v, int s, int d, unsigned* wm) {
  const int lane = lane_id();
  const uint64_t pol = l2_keep_policy();
  const SmallSeg g = small_scan(d);
#pragma unroll
  for (int k = 0; k < kSmallWords; ++k) wm[kSmallWords * lane + k] = 0;
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
    for (int q = 0; q < kSmallUnroll; ++q) cc[q] = u[q] >= 0 ? ld_keep(p.color + u[q], pol) : 0;
#pragma unroll
    for (int q = 0; q < kSmallUnroll; ++q) {
      const int c = cc[q];
      if (c >= 1 && c <= 32 * kSmallWords)
        atomicOr(&wm[kSmallWords * j[q] + ((c - 1) >> 5)], 1u << ((c - 1) & 31));
    }
  }
  __syncwarp();
  if (v >= 0) {
    // first free colour: degree <= t1 < 32 * kSmallWords keeps it in the mask
    int t = 0;
#pragma unroll
    for (int k = 0; k < kSmallWords; ++k) {
      const unsigned w = wm[kSmallWords * lane + k];
      if (t == 0 && w != FULL) t = 32 * k + __ffs(~w);
    }
    p.tent[v] = t;
  }
  __syncwarp();
}

// Loser flag of each lane's node (t = its tentative colour).
__device__ __forceinline__ bool small_lose(const Params& p, int v, int s, int d, int t,
                                           unsigned* wm) {
  const int lane = lane_id();
  const uint64_t pol = l2_keep_policy();
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
    for (int q = 0; q < kSmallUnroll; ++q) tt[q] = u[q] >= 0 ? ld_keep(p.tent + u[q], pol) : 0;
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

// -------------------------------------------------------- high-degree nodes --

// First zero bit among 64 words read by the whole warp through get(i) for
// i < nw: returns 32 * word + bit + 1 (a colour), or 0 when all are full.
template <class Get>
__device__ __forceinline__ int first_free_64(int nw, Get get) {
  const int lane = lane_id();
  const unsigned w0 = lane < nw ? get(lane) : FULL;
  const unsigned w1 = lane + 32 < nw ? get(lane + 32) : FULL;
  const unsigned b0 = __ballot_sync(FULL, w0 != FULL);
  const unsigned b1 = __ballot_sync(FULL, w1 != FULL);
  if (b0) {
    const int fl = __ffs(b0) - 1;
    return 32 * fl + __ffs(~__shfl_sync(FULL, w0, fl));
  }
  if (b1) {
    const int fl = __ffs(b1) - 1;
    return 32 * (32 + fl) + __ffs(~__shfl_sync(FULL, w1, fl));
  }
  return 0;
}

// Neighbour entries per lane per window: 4 (one int4). With 8 the loops
// needed more registers than 3 CTAs of 256 per SM leave (80 per thread) and
// spilled; 4 with 24 warps per SM beat 8 with 16 (RMAT scale 22: 23.9 ms
// against 25.6, road 5.3 against 6.3, same GPU).
constexpr int kGather = 4;
constexpr int kWindow = 32 * kGather;  // neighbour entries per warp per window

// One window of the neighbour array: the kWindow entries at absolute index
// a + i (a a multiple of 4), lane l holding entries 4l..4l+3 (and
// 128h+4l..128h+4l+3 for h < kGather / 4), read as int4 where the array is
// 16-byte aligned and the four entries all lie in [lo, hi); entries outside
// [lo, hi) read `none`.
__device__ __forceinline__ void load_window(const Params& p, int64_t a, int64_t lo, int64_t hi,
                                            int none, int (&u)[kGather]) {
  const int lane = lane_id();
#pragma unroll
  for (int h = 0; h < kGather / 4; ++h) {
    const int64_t q = a + 128 * h + 4 * lane;
    if (p.col_vec && q >= lo && q + 3 < hi) {
      const int4 x = __ldg(reinterpret_cast<const int4*>(p.col + q));
      u[4 * h + 0] = x.x;
      u[4 * h + 1] = x.y;
      u[4 * h + 2] = x.z;
      u[4 * h + 3] = x.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        u[4 * h + j] = (q + j >= lo && q + j < hi) ? ld_ro(p.col + q + j) : none;
    }
  }
}

// The same over a neighbour list written during the launch (16-byte aligned
// base; read through L2, not the read-only path).
__device__ __forceinline__ void load_window_rw(const int32_t* arr, int64_t a, int64_t lo, int64_t hi,
                                               int none, int (&u)[kGather]) {
  const int lane = lane_id();
#pragma unroll
  for (int h = 0; h < kGather / 4; ++h) {
    const int64_t q = a + 128 * h + 4 * lane;
    if (q >= lo && q + 3 < hi) {
      const int4 x = ld_cg4(reinterpret_cast<const int4*>(arr + q));
      u[4 * h + 0] = x.x;
      u[4 * h + 1] = x.y;
      u[4 * h + 2] = x.z;
      u[4 * h + 3] = x.w;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j)
        u[4 * h + j] = (q + j >= lo && q + j < hi) ? ld_cg(arr + q + j) : none;
    }
  }
}

// Asks L2 to fetch neighbour entries [lo, hi) ahead of their use (one lane).
__device__ __forceinline__ void prefetch_l2(const Params& p, int64_t lo, int64_t hi) {
  if (!p.col_vec) return;
  const int64_t a = lo & ~int64_t(3), z = hi & ~int64_t(3);  // 16-byte aligned, inside the array
  if (z <= a) return;
  const int64_t bytes = (z - a) * 4;
  const unsigned sz = (unsigned)(bytes < (1 << 20) ? bytes : (1 << 20));
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p.col + a), "r"(sz) : "memory");
}

// ------------------------------------------------- forbidden-colour bitmaps --
//
// With pushing on (Params::pbits), a node of degree > t1 finds its colour in
// a bitmap of its finalised neighbours' colours that those neighbours filled
// when they were committed, instead of rescanning its row every round. The
// colours are the same: the bitmap of v at the start of round r holds
// exactly the colours committed to v's neighbours before round r (every
// commit pushes before the round's last barrier; the assignment step only
// reads). Colours above min(d, kPushMaxC) are not kept: the first free
// colour of a node of degree d is at most d + 1, and at most maxc + 1 <=
// kPushMaxC while pushing is on.

__device__ __forceinline__ int push_words(int d) { return (min(d, kPushMaxC) + 31) >> 5; }

static_assert(kPushChunk == kWindow, "a push item is one window");

constexpr int kPushUnroll = 8;

// OR `bit` into bitmap word *w unless the word, as this SM's L1 may hold it,
// has the bit already. Bitmaps only gain bits during a colouring, and none
// is read through L1 before it is cleared, so a cached copy holds a subset
// of the word's bits: a stale copy costs a redundant atomic, never a missed
// bit. A high-degree node receives one push per committed neighbour, most
// of them for the few low colours of one word; the check keeps those off
// the L2 atomic unit of that word.
__device__ __forceinline__ void push_bit(uint32_t* w, unsigned bit) {
  if ((__ldca(w) & bit) == 0) atomicOr(w, bit);
}

// Colour t into the bitmap of neighbour u, whose row starts at s and has d
// entries (colours above d never decide u's first free colour).
__device__ __forceinline__ void push_to(const Params& p, int s, int d, int t) {
  if (d < t) return;
  uint32_t* w = p.pbits + s + ((t - 1) >> 5);
  const unsigned bit = 1u << ((t - 1) & 31);
  if (d > kDefaultChunk)  // many pushes reach a high-degree node
    push_bit(w, bit);
  else
    atomicOr(w, bit);
}


// Colour t into the bitmaps of the kGather nodes u[] (-1: none) that keep one
// (degree > t1) and are still active: with pinfo one 8-byte gather each,
// else their row offsets and colour (independent gathers: the pushes are
// latency-bound).
__device__ __forceinline__ void push_targets(const Params& p, const int (&u)[kGather], int t, int t1,
                                             uint64_t pol) {
  if (p.pinfo) {
    int2 pi[kGather];
#pragma unroll
    for (int q = 0; q < kGather; ++q) pi[q] = u[q] >= 0 ? __ldcg(p.pinfo + u[q]) : make_int2(0, 0);
    // the word of colour t in each target's bitmap; the L1 reads of the
    // high-degree targets' words (push_bit) are all issued before the atomics
    const int off = (t - 1) >> 5;
    const unsigned bit = 1u << ((t - 1) & 31);
    unsigned seen[kGather];
#pragma unroll
    for (int q = 0; q < kGather; ++q)
      seen[q] = pi[q].y > kDefaultChunk && pi[q].y >= t ? __ldca(p.pbits + pi[q].x + off) : 0u;
#pragma unroll
    for (int q = 0; q < kGather; ++q)
      if (pi[q].y >= t && (seen[q] & bit) == 0) atomicOr(p.pbits + pi[q].x + off, bit);
    return;
  }
  int sw[kGather], ew[kGather], cw[kGather];
#pragma unroll
  for (int q = 0; q < kGather; ++q) {
    sw[q] = 0;
    ew[q] = 0;
    cw[q] = 1;
    if (u[q] >= 0) {
      sw[q] = ld_ro(p.rowptr + u[q]);
      ew[q] = ld_ro(p.rowptr + u[q] + 1);
      cw[q] = ld_keep(p.color + u[q], pol);
    }
  }
#pragma unroll
  for (int q = 0; q < kGather; ++q)
    if (cw[q] == 0 && ew[q] - sw[q] > t1) push_to(p, sw[q], ew[q] - sw[q], t);
}

// Colour t (just committed) into the bitmaps of the neighbours in entries
// [lo, hi) of col that keep one (degree > t1) and are still active. One warp.
inline __device__ __noinline__ void push_range(const Params& p, int64_t lo, int64_t hi, int t,
                                               int t1) {
  const uint64_t pol = l2_keep_policy();
  for (int64_t a = lo & ~int64_t(3); a < hi; a += kWindow) {
    int u[kGather];
    load_window(p, a, lo, hi, -1, u);
    push_targets(p, u, t, t1, pol);
  }
}

// The window of queued push item it = {row start, degree, colour, j}
// (push_items_of): its entries, -1 outside the row. One warp.
__device__ __forceinline__ void load_push_item(const Params& p, int4 it, int (&u)[kGather]) {
  const int64_t s = it.x, a = (s & ~int64_t(3)) + (int64_t)it.w * kPushChunk;
  load_window(p, a, a > s ? a : s, min(s + it.y, a + kPushChunk), -1, u);
}

// The same for the 32 nodes of a warp, one per lane (colour t, entries
// [s, s + d); d = 0 for a lane that pushes nothing), their rows laid end to
// end as in the low-degree steps. In round 1 (check_active false) colours are
// being written while it pushes, and every neighbour of a winner is active.
__device__ __forceinline__ void small_push(const Params& p, int s, int d, int t, int t1,
                                           bool check_active) {
  const int lane = lane_id();
  const uint64_t pol = l2_keep_policy();
  const SmallSeg g = small_scan(d);
  for (int base = 0; base < g.total; base += 32 * kPushUnroll) {
    int u[kPushUnroll], tq[kPushUnroll];
#pragma unroll
    for (int q = 0; q < kPushUnroll; ++q) {
      const int e = base + q * 32 + lane;
      const int jj = small_owner(g.off, e);
      const int sj = __shfl_sync(FULL, s, jj);
      const int oj = __shfl_sync(FULL, g.off, jj);
      tq[q] = __shfl_sync(FULL, t, jj);
      u[q] = e < g.total ? ld_ro(p.col + sj + (e - oj)) : -1;
    }
    if (p.pinfo && check_active) {  // (round 1 writes pinfo while it pushes: not read then)
      int2 pi[kPushUnroll];
#pragma unroll
      for (int q = 0; q < kPushUnroll; ++q)
        pi[q] = u[q] >= 0 ? __ldcg(p.pinfo + u[q]) : make_int2(0, 0);
#pragma unroll
      for (int q = 0; q < kPushUnroll; ++q)
        if (pi[q].y > 0) push_to(p, pi[q].x, pi[q].y, tq[q]);
      continue;
    }
    int sw[kPushUnroll], ew[kPushUnroll], cw[kPushUnroll];
#pragma unroll
    for (int q = 0; q < kPushUnroll; ++q) {
      sw[q] = 0;
      ew[q] = 0;
      cw[q] = 1;
      if (u[q] >= 0) {
        sw[q] = ld_ro(p.rowptr + u[q]);
        ew[q] = ld_ro(p.rowptr + u[q] + 1);
        cw[q] = check_active ? ld_keep(p.color + u[q], pol) : 0;
      }
    }
#pragma unroll
    for (int q = 0; q < kPushUnroll; ++q)
      if (cw[q] == 0 && ew[q] - sw[q] > t1) push_to(p, sw[q], ew[q] - sw[q], tq[q]);
  }
}

// Colours of neighbours k in [b, e) of row s, shifted by -wbase, into the
// lane-private mask (1..32) and the warp's bitmap wb (33..lim). The next
// window's entries are loaded while the current window's colours are
// gathered.
__device__ __forceinline__ unsigned gather_colours(const Params& p, int64_t s, int b, int e,
                                                   int wbase, int lim, unsigned* wb) {
  const uint64_t pol = l2_keep_policy();
  const int64_t lo = s + b, hi = s + e;
  int64_t a = lo & ~int64_t(3);
  int u[kGather];
  load_window(p, a, lo, hi, -1, u);
  unsigned pm = 0;
  for (; a < hi; a += kWindow) {
    int un[kGather];
    const bool more = a + kWindow < hi;
    if (more) load_window(p, a + kWindow, lo, hi, -1, un);
    int cc[kGather];
#pragma unroll
    for (int q = 0; q < kGather; ++q) cc[q] = u[q] >= 0 ? ld_keep(p.color + u[q], pol) : 0;
#pragma unroll
    for (int q = 0; q < kGather; ++q) {
      const int c = cc[q] - wbase;
      if (c >= 1 && c <= 32)
        pm |= 1u << (c - 1);
      else if (c > 32 && c <= lim)
        atomicOr(&wb[(c - 1) >> 5], 1u << ((c - 1) & 31));
    }
    if (more) {
#pragma unroll
      for (int q = 0; q < kGather; ++q) u[q] = un[q];
    }
  }
  __syncwarp();
  return __reduce_or_sync(FULL, pm);
}

// A whole node by one warp in windows of 32 * kGWords colours: used when the
// colour bound of a node exceeds the merge bitmap (more than 2048 colours).
__device__ inline int item_assign_windowed(const Params& p, unsigned* wb, int s, int d, int lim) {
  const int lane = lane_id();
  for (int wbase = 0;; wbase += 32 * kGWords) {
    const int wcols = min(lim - wbase, 32 * kGWords);
    if (wcols <= 0) {  // unreachable for a valid graph: some colour <= lim is free
      if (lane == 0) record_error(p.ctrl, IPGC_ERR_INVALID);
      return lim;
    }
    const int nw = (wcols + 31) >> 5;
    const unsigned pm = gather_colours(p, s, 0, d, wbase, wcols, wb);
    const int t = first_free_64(nw, [&](int i) { return i == 0 ? (pm | wb[0]) : wb[i]; });
    __syncwarp();
    wb[lane] = 0;
    wb[lane + 32] = 0;
    __syncwarp();
    if (t > 0) return wbase + t;
  }
}

// Assignment step for work item (v, c) of a node with nch items.
__device__ __forceinline__ void item_assign(const Params& p, unsigned* wb, int v, int s, int d,
                                            int c, int nch, int gslot, int maxc) {
  const int lane = lane_id();
  const int lim = min(d, maxc) + 1;  // tent[v] <= d + 1 and <= maxc + 1
  if (lim > 32 * kGWords) {
    if (c == 0) {
      const int t = item_assign_windowed(p, wb, s, d, lim);
      if (lane == 0) p.tent[v] = t;
    }
    return;
  }
  const int nw = (lim + 31) >> 5;
  const int b = c * p.chunk, e = min(d, b + p.chunk);
  const unsigned pm = gather_colours(p, s, b, e, 0, lim, wb);
  if (nch == 1) {
    const int t = first_free_64(nw, [&](int i) { return i == 0 ? (pm | wb[0]) : wb[i]; });
    if (lane == 0) p.tent[v] = t;
    __syncwarp();
    wb[lane] = 0;
    wb[lane + 32] = 0;
    __syncwarp();
    return;
  }
  uint32_t* g = p.gbits + (size_t)gslot * kGWords;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    if (i < nw) {
      const unsigned w = (i == 0 ? pm : 0u) | wb[i];
      if (w) atomicOr(&g[i], w);
    }
  }
  __syncwarp();
  wb[lane] = 0;
  wb[lane + 32] = 0;
  __threadfence();
  __syncwarp();
  int last = 0;
  if (lane == 0) last = atomicAdd(&p.done_a[gslot], 1) == nch - 1;
  last = __shfl_sync(FULL, last, 0);
  if (last) {  // every other item of v has merged its bits
    __threadfence();
    const int t = first_free_64(nw, [&](int i) { return atomicExch(&g[i], 0u); });
    if (lane == 0) {
      p.tent[v] = t;
      p.done_a[gslot] = 0;
    }
  }
}

// Assignment step of node v (degree d > t1, row at s) from its bitmap: the
// first colour none of its finalised neighbours has. One warp.
__device__ __forceinline__ void item_assign_push(const Params& p, int v, int s, int d) {
  const int nw = push_words(d);
  const uint32_t* b = p.pbits + s;
  int t = first_free_64(nw, [&](int i) { return __ldcg(b + i); });
  if (t == 0) t = 32 * nw + 1;  // colours 1..d all taken (d = 32 * nw <= kPushMaxC)
  if (lane_id() == 0) p.tent[v] = t;
}

// The row of a node of degree d (entries from s) committed with colour t,
// queued for the push phase in one-window items {s, d, t, j} (push_items_of),
// and asked into L2 meanwhile. One warp, warp-uniform arguments.
__device__ __forceinline__ void push_queue(const Params& p, int s, int d, int t) {
  const int lane = lane_id();
  const int n = push_items_of(s, d);
  int base = 0;
  if (lane == 0) {
    base = atomicAdd(&p.ctrl->pqcnt, n);
    prefetch_l2(p, s, (int64_t)s + d);
  }
  base = __shfl_sync(FULL, base, 0);
  for (int j = lane; j < n; j += 32) p.pq[base + j] = make_int4(s, d, t, j);
}

// Colour t into the bitmaps of the still-active, bitmap-keeping entries of
// list range [lo, hi) of lst (a late round's winner pushing along its list
// of active lower-ID neighbours). One warp.
inline __device__ __noinline__ void push_list(const Params& p, const int32_t* lst, int64_t lo,
                                              int64_t hi, int t, int t1) {
  const uint64_t pol = l2_keep_policy();
  for (int64_t a = lo & ~int64_t(3); a < hi; a += kWindow) {
    int u[kGather];
    load_window_rw(lst, a, lo, hi, -1, u);
    push_targets(p, u, t, t1, pol);
  }
}

// Conflict step for work item (v, c); the warp that finishes v's last item
// commits v or pushes its items to the next worklist.
__device__ __forceinline__ void item_detect(const Params& p, ItemStage& stage, int v, int s, int d,
                                            int c, int nch, int gslot, int nxt, PhaseAcc& acc,
                                            int round, bool push = true,
                                            WarpStage* wst = nullptr) {
  const int lane = lane_id();
  const uint64_t pol = l2_keep_policy();
  const int t = ld_cg(p.tent + v);
  const int b = c * p.chunk, e = min(d, b + p.chunk);
  const int64_t lo = (int64_t)s + b, hi = (int64_t)s + e;
  bool hit = false;
  // another item of v found a conflict already: v loses whatever this one finds
  const bool lost = nch > 1 && ld_cg(p.flag + gslot) != 0;
  if (!lost) {
    int64_t a = lo & ~int64_t(3);
    int u[kGather];
    load_window(p, a, lo, hi, -1, u);
    for (; a < hi; a += kWindow) {
      int un[kGather];
      const bool more = a + kWindow < hi;
      if (more) load_window(p, a + kWindow, lo, hi, -1, un);
      int tt[kGather];
#pragma unroll
      for (int q = 0; q < kGather; ++q)
        tt[q] = (u[q] >= 0 && u[q] < v) ? ld_keep(p.tent + u[q], pol) : 0;
      bool passed = false;
#pragma unroll
      for (int q = 0; q < kGather; ++q) {
        hit |= (u[q] >= 0 && u[q] < v && tt[q] == t);
        passed |= u[q] >= v;
      }
      if (__any_sync(FULL, hit)) break;
      if (__any_sync(FULL, passed)) break;  // sorted rows: no lower ID follows
      if (more) {
#pragma unroll
        for (int q = 0; q < kGather; ++q) u[q] = un[q];
      }
    }
  }
  hit = __any_sync(FULL, hit);
  int finisher = 1, lose = hit;
  if (nch > 1) {
    if (lane == 0) {
      if (hit) atomicOr(&p.flag[gslot], 1);
      __threadfence();
      finisher = atomicAdd(&p.done_d[gslot], 1) == nch - 1;
      lose = 0;
      if (finisher) {
        __threadfence();
        lose = atomicExch(&p.flag[gslot], 0) != 0;
        p.done_d[gslot] = 0;
      }
    }
    finisher = __shfl_sync(FULL, finisher, 0);
    lose = __shfl_sync(FULL, lose, 0);
  }
  items_push(stage, v, (push && finisher && lose && lane == 0) ? nch : 0, gslot, p.items[nxt],
             &p.ctrl->icnt[nxt]);
  if (finisher && lane == 0) {
    if (lose) {
      acc.nbig += 1;
      acc.dsum += (unsigned long long)d;
    } else {
      p.color[v] = t;
      retire_push_target(p, v);
      acc.maxc = max(acc.maxc, t);
      if (p.fin) p.fin[v] = round;
    }
  }
  if (wst && finisher && !lose)  // pushing: the push phase after this step ORs t into the
    push_queue(p, s, d, t);        // neighbours' bitmaps
  if (wst && finisher && lose && lane == 0) acc.nodd += 1;  // not a list node
}

// ------------------------------------- lower-neighbour lists (with pushing) --
//
// Under pushing a node with several work items (a merge-state slot) keeps
// the list of its lower-ID neighbours that are still active, in alist[b]
// at [rowptr[v], rowptr[v] + flen[b][gslot].x); fst[gslot]: bit 0 b, bit 1
// "rewrite in the next assignment step", bit 2 "built". Its conflict step
// reads the list instead of the lower part of its row: every active
// lower-ID neighbour is on it, and the finalised ones it may still hold
// cannot clash (tent[v] excludes their colours). The first assignment step
// after round 1 builds it from the row. Once a quarter of the entries the
// conflict step sampled were finalised, the list is rewritten without its
// finalised entries into the other buffer: by the push phase that follows
// that conflict step (queue_rewrite, spread over the team), or, after a late
// round, which has no push phase, by the node's next assignment step.

// Entries [lo, hi) of src (the sorted row when from_col): those of ID < v
// whose colour is 0 appended to v's list at dst[s + *len...]. One warp.
__device__ __forceinline__ void plist_append(const Params& p, const int32_t* src, bool from_col,
                                             int64_t lo, int64_t hi, int v, int64_t s,
                                             int32_t* dst, int* len) {
  const int lane = lane_id();
  const uint64_t pol = l2_keep_policy();
  for (int64_t a = lo & ~int64_t(3); a < hi; a += kWindow) {
    int u[kGather];
    if (from_col)
      load_window(p, a, lo, hi, -1, u);
    else
      load_window_rw(src, a, lo, hi, -1, u);
    int cc[kGather];
#pragma unroll
    for (int q = 0; q < kGather; ++q)
      cc[q] = (u[q] >= 0 && u[q] < v) ? ld_keep(p.color + u[q], pol) : 1;
    int k = 0;
    bool above = false;
#pragma unroll
    for (int q = 0; q < kGather; ++q) {
      k += cc[q] == 0;
      above |= u[q] >= v;
    }
    int x = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    const int tot = __shfl_sync(FULL, x, 31);
    if (tot) {
      int base = 0;
      if (lane == 0) base = atomicAdd(len, tot);
      int o = __shfl_sync(FULL, base, 0) + x - k;
#pragma unroll
      for (int q = 0; q < kGather; ++q)
        if (cc[q] == 0) dst[s + o++] = u[q];
    }
    if (from_col && __any_sync(FULL, above)) break;  // sorted row: no lower ID follows
  }
}

// Entries [lo, hi) of v's list src after a late round: the colours of the
// finalised ones into v's bitmap (those <= min(d, kPushMaxC)); with dst, the
// active ones appended to the list there (the rewrite). One warp.
__device__ __forceinline__ void plist_pull(const Params& p, const int32_t* src, int64_t lo,
                                           int64_t hi, int64_t s, int d, int32_t* dst, int* len) {
  const int lane = lane_id();
  const uint64_t pol = l2_keep_policy();
  const int lim = min(d, kPushMaxC);
  for (int64_t a = lo & ~int64_t(3); a < hi; a += kWindow) {
    int u[kGather];
    load_window_rw(src, a, lo, hi, -1, u);
    int cc[kGather];
#pragma unroll
    for (int q = 0; q < kGather; ++q) cc[q] = u[q] >= 0 ? ld_keep(p.color + u[q], pol) : -1;
    int k = 0;
#pragma unroll
    for (int q = 0; q < kGather; ++q) {
      if (cc[q] > 0 && cc[q] <= lim)
        atomicOr(p.pbits + s + ((cc[q] - 1) >> 5), 1u << ((cc[q] - 1) & 31));
      k += cc[q] == 0;
    }
    if (!dst) continue;
    int x = k;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    const int tot = __shfl_sync(FULL, x, 31);
    if (tot) {
      int base = 0;
      if (lane == 0) base = atomicAdd(len, tot);
      int o = __shfl_sync(FULL, base, 0) + x - k;
#pragma unroll
      for (int q = 0; q < kGather; ++q)
        if (cc[q] == 0) dst[s + o++] = u[q];
    }
  }
}

// Assignment step for work item c of nch of node v with a merge-state slot:
// item 0 takes tent[v] from the bitmap; every item builds or rewrites its
// share of the list.
__device__ __forceinline__ void item_assign_plist(const Params& p, int v, int s, int d, int c,
                                                  int nch, int gslot, bool pull) {
  const int st = ld_cg(p.fst + gslot);
  const int L0 = ld_cg(&p.flen[0][gslot].x), L1 = ld_cg(&p.flen[1][gslot].x);
  if (pull && (st & 4)) {  // after a late round: collect its lower-ID winners from the list
    const int cur = st & 1;
    const int L = cur ? L1 : L0;
    const int64_t lo = s + (int64_t)L * c / nch, hi = s + (int64_t)L * (c + 1) / nch;
    plist_pull(p, p.alist[cur], lo, hi, s, d, (st & 2) ? p.alist[cur ^ 1] : nullptr,
               &p.flen[cur ^ 1][gslot].x);
    __syncwarp();
    __threadfence();
    __syncwarp();
    if (nch == 1) {
      item_assign_push(p, v, s, d);
      return;
    }
    int last = 0;  // every item of v has collected its share: the last one takes tent[v]
    if (lane_id() == 0) last = atomicAdd(&p.done_a[gslot], 1) == nch - 1;
    last = __shfl_sync(FULL, last, 0);
    if (last) {
      __threadfence();
      item_assign_push(p, v, s, d);
      if (lane_id() == 0) p.done_a[gslot] = 0;
    }
    return;
  }
  if (c == 0) item_assign_push(p, v, s, d);
  if (!(st & 4)) {  // built from row chunk c (the items of a node without a list are its row's)
    const int64_t lo = (int64_t)s + (int64_t)c * p.chunk;
    const int64_t hi = min((int64_t)s + d, lo + p.chunk);
    if (lo < hi && ld_ro(p.col + lo) < v)
      plist_append(p, p.col, true, lo, hi, v, s, p.alist[0], &p.flen[0][gslot].x);
  } else if (st & 2) {
    const int cur = st & 1;
    const int L = cur ? L1 : L0;
    const int64_t lo = s + (int64_t)L * c / nch, hi = s + (int64_t)L * (c + 1) / nch;
    plist_append(p, p.alist[cur], false, lo, hi, v, s, p.alist[cur ^ 1],
                 &p.flen[cur ^ 1][gslot].x);
  }
}

// The one-window units {row start, slot, length, window | buffer << 31} of
// the rewrite of list buffer nb (L entries from s) of the node with slot
// gslot, queued for the push phase. One warp (out of line: it runs rarely).
inline __device__ __noinline__ void queue_rewrite(const Params& p, int s, int gslot, int L,
                                                  int nb) {
  const int lane = lane_id();
  const int n = push_items_of(s, L);
  int base = 0;
  if (lane == 0) base = atomicAdd(&p.ctrl->rqcnt, n);
  base = __shfl_sync(FULL, base, 0);
  for (int j = lane; j < n; j += 32)
    p.rq[base + j] = make_int4(s, gslot, L, (int)((unsigned)j | ((unsigned)nb << 31)));
}

// Conflict step for work item c of nch of node v with a merge-state slot:
// its share of the list up to the first clash. The warp that finishes v's
// last item commits v (queueing its row for the push phase) or pushes its
// items for round r + 1 (chunks of the list while the next round pushes,
// else of the row), and sets the list state. In odd rounds the finalised
// entries among the first window of each item are counted in fdead, all
// entries of those windows in done_a (idle in this mode).
__device__ __forceinline__ void item_detect_plist(const Params& p, ItemStage& stage, int v, int s,
                                                  int d, int c, int nch, int gslot, int nxt,
                                                  PhaseAcc& acc, int round, bool push,
                                                  bool lists_next, bool late, int t1) {
  const int lane = lane_id();
  const uint64_t pol = l2_keep_policy();
  const int t = ld_cg(p.tent + v);
  const int st = ld_cg(p.fst + gslot);
  // both buffers' lengths and the clash flag together with the state: one
  // round trip (the flag only for a node of several items: no other item
  // sets it otherwise)
  const int L0 = ld_cg(&p.flen[0][gslot].x), L1 = ld_cg(&p.flen[1][gslot].x);
  const int clashed = nch > 1 ? ld_cg(p.flag + gslot) : 0;
  const int cur = st & 1;
  const int nb = !(st & 4) ? 0 : ((st & 2) ? cur ^ 1 : cur);
  const int L = nb ? L1 : L0;
  const int32_t* lst = p.alist[nb];
  const int64_t lo = s + (int64_t)L * c / nch, hi = s + (int64_t)L * (c + 1) / nch;
  bool hit = false;
  int dead = 0, seen = 0;
  if (lo < hi && clashed == 0) {  // else another item found a clash already
    int64_t a = lo & ~int64_t(3);
    int u[kGather];
    load_window_rw(lst, a, lo, hi, -1, u);
    for (; a < hi; a += kWindow) {
      int un[kGather];
      const bool more = a + kWindow < hi;
      if (more) load_window_rw(lst, a + kWindow, lo, hi, -1, un);  // the next window ahead
      int tt[kGather];
#pragma unroll
      for (int q = 0; q < kGather; ++q) tt[q] = u[q] >= 0 ? ld_keep(p.tent + u[q], pol) : 0;
#pragma unroll
      for (int q = 0; q < kGather; ++q) hit |= u[q] >= 0 && tt[q] == t;
      // in odd rounds the item's first window samples how much of the list is
      // finalised (each sample is a second gather per entry; every other
      // round is often enough for the rewrites it triggers)
      if ((round & 1) && a < lo + kWindow) {
        int cc[kGather];
#pragma unroll
        for (int q = 0; q < kGather; ++q) cc[q] = u[q] >= 0 ? ld_keep(p.color + u[q], pol) : 0;
#pragma unroll
        for (int q = 0; q < kGather; ++q) {
          seen += u[q] >= 0;
          dead += u[q] >= 0 && cc[q] != 0;
        }
      }
      if (__any_sync(FULL, hit)) break;
      if (more) {
#pragma unroll
        for (int q = 0; q < kGather; ++q) u[q] = un[q];
      }
    }
  }
  hit = __any_sync(FULL, hit);
  dead = __reduce_add_sync(FULL, dead);
  seen = __reduce_add_sync(FULL, seen);
  int finisher = 0, lose = 0, requeue = 0;
  if (lane == 0) {
    int D = dead, S = seen;
    if (nch == 1) {  // the only item: nothing to merge
      finisher = 1;
      lose = hit;
    } else {
      if (hit) atomicOr(&p.flag[gslot], 1);
      if (dead) atomicAdd(p.fdead + gslot, dead);
      if (seen) atomicAdd(p.done_a + gslot, seen);
      __threadfence();
      finisher = atomicAdd(&p.done_d[gslot], 1) == nch - 1;
      if (finisher) {
        __threadfence();
        lose = atomicExch(&p.flag[gslot], 0) != 0;
        p.done_d[gslot] = 0;
        D = atomicExch(p.fdead + gslot, 0);
        S = atomicExch(p.done_a + gslot, 0);
      }
    }
    if (finisher) {
      const bool rw = D > 0 && 4 * (int64_t)D >= (int64_t)S;
      if ((st & 6) == 6) p.flen[cur][gslot] = make_int2(0, 0);  // rewritten: the old buffer is free
      // a loser due for a rewrite in a round with a push phase: that phase
      // rewrites the list into the other buffer, which round r + 1 reads
      // (in a late round, or without a queue, its next assignment step does).
      // Both lengths start again from zero: the units carry the old one, and
      // no item of this node reads it any more (this is its last item of the
      // round, and round r + 1 reads the other buffer), so the old buffer is
      // empty when a later rewrite appends to it.
      requeue = rw && lose && p.rq != nullptr && !late && lists_next;
      if (requeue) {
        p.flen[nb ^ 1][gslot] = make_int2(0, 0);
        p.flen[nb][gslot] = make_int2(0, 0);
      }
      p.fst[gslot] = requeue ? ((nb ^ 1) | 4) : (nb | 4 | (rw ? 2 : 0));
    }
  }
  finisher = __shfl_sync(FULL, finisher, 0);
  lose = __shfl_sync(FULL, lose, 0);
  if (__shfl_sync(FULL, requeue, 0)) queue_rewrite(p, s, gslot, L, nb);
  const int nxt_items = lists_next ? max(1, num_chunks(L, p.chunk)) : num_chunks(d, p.chunk);
  items_push(stage, v, (push && finisher && lose && lane == 0) ? nxt_items : 0, gslot,
             p.items[nxt], &p.ctrl->icnt[nxt]);
  if (finisher && !lose) {
    if (late && nch == 1)  // the list is v's active lower-ID neighbours: push along it
      push_list(p, lst, lo, hi, t, t1);
    else
      push_queue(p, s, d, t);
  }
  if (finisher && lose && lane == 0 && nxt_items > 1) acc.nodd += 1;
  if (finisher && lane == 0) {
    if (lose) {
      acc.nbig += 1;
      acc.dsum += (unsigned long long)d;
    } else {
      p.color[v] = t;
      retire_push_target(p, v);
      acc.maxc = max(acc.maxc, t);
      if (p.fin) p.fin[v] = round;
    }
  }
}

// ------------------------------------------------------ neighbour filtering --
//
// Filtering starts at round r0 (the hand-over round, see continue_graph).
// A filtered node v keeps a list of neighbours that holds every neighbour
// still active, in one of two buffers (state fst[gslot]: bit 0 the buffer,
// bit 1 "rewrite in the next round"). In round r0 the list is built from the
// row. Later rounds read the list: a neighbour found committed is finalised
// for good, its colour goes into v's persistent bitmap. Most neighbours of a
// long-lived high-degree node stay active from round to round, so the list
// is rewritten (into the other buffer, without its finalised entries) only
// once a quarter of it was found finalised; until then the finalised
// entries are read again, harmlessly (their colours are in the bitmap
// already and cannot clash: tent[v] excludes them). The conflict step scans
// the lower-ID part of the list. Colours, rounds and worklists are those of
// rescanning the whole row; only the entries read shrink.

// Work items of filtered node v in round r: chunks of its list.
__device__ __forceinline__ int filt_items(const Params& p, int round, int r0, int gslot, int d) {
  if (round == r0) return num_chunks(d, p.chunk);
  const int cur = ld_cg(p.fst + gslot) & 1;
  const int2 L = __ldcg(p.flen[cur] + gslot);
  return max(1, num_chunks(L.x + L.y, p.chunk));
}

// Entries [lo, hi) of v's list (absolute indexes into src; src is col in
// round r0): colours of committed neighbours into pm (1..32, lane-private)
// and wb (33..2048), their number added to dead. With `write`, active
// neighbours are appended to the list dst within v's row range [s, s + d),
// lower IDs from the front and higher IDs from the back, counted in *nlen.
__device__ __forceinline__ void filt_assign_range(const Params& p, const int32_t* src, bool from_col,
                                                  int64_t lo, int64_t hi, int v, int64_t s, int d,
                                                  bool write, int32_t* dst, int2* nlen,
                                                  unsigned& pm, int& dead, unsigned* wb) {
  // one window at a time: the lists are mostly in L2, and the registers a
  // second window would take are worth more than the overlap
  const int lane = lane_id();
  const uint64_t pol = l2_keep_policy();
  for (int64_t a = lo & ~int64_t(3); a < hi; a += kWindow) {
    int u[kGather];
    if (from_col)
      load_window(p, a, lo, hi, -1, u);
    else
      load_window_rw(src, a, lo, hi, -1, u);
    int cc[kGather];
#pragma unroll
    for (int q = 0; q < kGather; ++q) cc[q] = u[q] >= 0 ? ld_keep(p.color + u[q], pol) : 0;
    int klo = 0, khi = 0;
#pragma unroll
    for (int q = 0; q < kGather; ++q) {
      if (u[q] < 0) continue;
      const int c = cc[q];
      if (c == 0) {
        if (u[q] < v)
          ++klo;
        else
          ++khi;
      } else {
        ++dead;
        if (c <= 32)
          pm |= 1u << (c - 1);
        else if (c <= 32 * kGWords)
          atomicOr(&wb[(c - 1) >> 5], 1u << ((c - 1) & 31));
      }
    }
    if (!write) continue;
    // both counts in one prefix sum: a window holds at most 256 entries
    int x = klo | (khi << 16);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, x, o);
      if (lane >= o) x += y;
    }
    const int tot = __shfl_sync(FULL, x, 31);
    if (tot == 0) continue;
    int blo = 0, bhi = 0;
    if (lane == 0) {
      if (tot & 0xffff) blo = atomicAdd(&nlen->x, tot & 0xffff);
      if (tot >> 16) bhi = atomicAdd(&nlen->y, tot >> 16);
    }
    const int xe = x - (klo | (khi << 16));  // exclusive prefix of this lane
    int olo = __shfl_sync(FULL, blo, 0) + (xe & 0xffff);
    int ohi = __shfl_sync(FULL, bhi, 0) + (xe >> 16);
#pragma unroll
    for (int q = 0; q < kGather; ++q) {
      if (u[q] < 0 || cc[q] != 0) continue;
      if (u[q] < v)
        dst[s + olo++] = u[q];
      else
        dst[s + d - 1 - ohi++] = u[q];
    }
  }
}

// Assignment step for work item c of nch of filtered node v in round r: the
// item's share of the list, then the persistent bitmap gives tent[v].
__device__ __forceinline__ void item_assign_filtered(const Params& p, unsigned* wb, int v, int s,
                                                     int d, int c, int nch, int gslot, int round,
                                                     int r0, int maxc) {
  const int lane = lane_id();
  unsigned pm = 0;
  int dead = 0;
  if (round == r0) {  // the first filtered round builds the list (buffer 0) from the row
    const int b = c * p.chunk, e = min(d, b + p.chunk);
    filt_assign_range(p, p.col, true, (int64_t)s + b, (int64_t)s + e, v, s, d, true, p.alist[0],
                      p.flen[0] + gslot, pm, dead, wb);
  } else {
    // the list in buffer cur: [0, L.x) at s + k, [L.x, L.x + L.y) at s + d - L.y + (k - L.x)
    const int st = ld_cg(p.fst + gslot), cur = st & 1;
    const bool rewrite = (st >> 1) & 1;
    const int32_t* src = p.alist[cur];
    int32_t* dst = p.alist[cur ^ 1];
    int2* nlen = p.flen[cur ^ 1] + gslot;
    const int2 L = __ldcg(p.flen[cur] + gslot);
    const int b = c * p.chunk, e = min(L.x + L.y, b + p.chunk);
    if (b < L.x)
      filt_assign_range(p, src, false, (int64_t)s + b, (int64_t)s + min(e, L.x), v, s, d, rewrite,
                        dst, nlen, pm, dead, wb);
    if (e > L.x) {
      const int64_t h0 = (int64_t)s + d - L.y - L.x;
      filt_assign_range(p, src, false, h0 + max(b, L.x), h0 + e, v, s, d, rewrite, dst, nlen, pm,
                        dead, wb);
    }
    dead = __reduce_add_sync(FULL, dead);
    if (!rewrite && dead && lane == 0) atomicAdd(p.fdead + gslot, dead);
  }
  pm = __reduce_or_sync(FULL, pm);
  __syncwarp();
  const int lim = min(d, maxc) + 1;  // <= 2048 while filtering
  const int nw = (lim + 31) >> 5;
  uint32_t* g = p.gbits + (size_t)gslot * kGWords;
  unsigned nv[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    const unsigned w = (i == 0 ? pm : 0u) | wb[i];
    nv[h] = w ? (atomicOr(&g[i], w) | w) : (nch == 1 ? __ldcg(g + i) : 0u);
  }
  __syncwarp();
  wb[lane] = 0;
  wb[lane + 32] = 0;
  __syncwarp();
  if (nch == 1) {
    const int t = first_free_64(nw, [&](int i) { return i >= 32 ? nv[1] : nv[0]; });
    if (lane == 0) p.tent[v] = t;
    return;
  }
  __threadfence();
  __syncwarp();
  int last = 0;
  if (lane == 0) last = atomicAdd(&p.done_a[gslot], 1) == nch - 1;
  last = __shfl_sync(FULL, last, 0);
  if (last) {  // every other item of v has merged its bits
    __threadfence();
    const int t = first_free_64(nw, [&](int i) { return __ldcg(g + i); });
    if (lane == 0) {
      p.tent[v] = t;
      p.done_a[gslot] = 0;
    }
  }
}

// Conflict step for work item c of nch of filtered node v in round r: its
// share of the lower-ID part of v's list as the assignment step left it. The
// warp that finishes v's last item commits v or pushes its items for round
// r + 1 (shaped for filtering when filt_next) and updates v's list state.
__device__ __forceinline__ void item_detect_filtered(const Params& p, ItemStage& lstage,
                                                     ItemStage& fstage, int v, int s, int d, int c,
                                                     int nch, int gslot, int nxt, PhaseAcc& acc,
                                                     int round, int r0, bool filt_next) {
  const int lane = lane_id();
  const uint64_t pol = l2_keep_policy();
  const int t = ld_cg(p.tent + v);
  // the list after this round's assignment step: buffer 0 in round r0, the
  // other buffer after a rewrite, else the same one
  int cur = 0, nb = 0;
  bool rewrote = true;
  if (round != r0) {
    const int st = ld_cg(p.fst + gslot);
    cur = st & 1;
    rewrote = (st >> 1) & 1;
    nb = rewrote ? cur ^ 1 : cur;
  }
  const int2 L1 = __ldcg(p.flen[nb] + gslot);
  const int32_t* lst = p.alist[nb];
  const int64_t lo = (int64_t)s + (int64_t)L1.x * c / nch;
  const int64_t hi = (int64_t)s + (int64_t)L1.x * (c + 1) / nch;
  bool hit = false;
  for (int64_t a = lo & ~int64_t(3); a < hi; a += kWindow) {
    int u[kGather];
    load_window_rw(lst, a, lo, hi, -1, u);
    int tt[kGather];
#pragma unroll
    for (int q = 0; q < kGather; ++q) tt[q] = u[q] >= 0 ? ld_keep(p.tent + u[q], pol) : 0;
#pragma unroll
    for (int q = 0; q < kGather; ++q) hit |= (u[q] >= 0 && tt[q] == t);
    if (__any_sync(FULL, hit)) break;
  }
  hit = __any_sync(FULL, hit);
  int finisher = 1, lose = hit;
  if (nch > 1) {
    if (lane == 0) {
      if (hit) atomicOr(&p.flag[gslot], 1);
      __threadfence();
      finisher = atomicAdd(&p.done_d[gslot], 1) == nch - 1;
      lose = 0;
      if (finisher) {
        __threadfence();
        lose = atomicExch(&p.flag[gslot], 0) != 0;
        p.done_d[gslot] = 0;
      }
    }
    finisher = __shfl_sync(FULL, finisher, 0);
    lose = __shfl_sync(FULL, lose, 0);
  }
  const bool push = finisher && lose && lane == 0;
  if (filt_next)  // the next round reads the list
    items_push(fstage, v, push ? max(1, num_chunks(L1.x + L1.y, p.chunk)) : 0, gslot,
               p.fitems[nxt], &p.ctrl->ficnt[nxt]);
  else  // hand-over: back to reading the row
    items_push(lstage, v, push ? num_chunks(d, p.chunk) : 0, gslot, p.items[nxt],
               &p.ctrl->icnt[nxt]);
  if (finisher && lane == 0) {
    // list state for round r + 1: rewrite it once a quarter of it is finalised
    const int dead = rewrote ? 0 : ld_cg(p.fdead + gslot);
    const bool rw_next = 4 * (int64_t)dead >= (int64_t)(L1.x + L1.y) && dead > 0;
    if (round != r0 && rewrote) p.flen[cur][gslot] = make_int2(0, 0);  // the old buffer is free
    p.fst[gslot] = nb | (rw_next ? 2 : 0);
    p.fdead[gslot] = 0;
    if (lose) {
      acc.nbig += 1;
      acc.dsum += (unsigned long long)d;
    } else {
      p.color[v] = t;
      retire_push_target(p, v);
      acc.maxc = max(acc.maxc, t);
      if (p.fin) p.fin[v] = round;
    }
  }
}

// ------------------------------------------------------------ work walkers --
//
// Both walkers hand a warp its share of the work in a fixed stride and load
// the next two shares' records (and the next share's row offsets) before
// working on the current one, so their latency overlaps the gathers.

// Work items k = start, start + stride, ... < count: calls
// f(v, chunk, gslot, nch, s, d) for every item whose node is active. The
// next item's share of its row is prefetched into L2 when its node's degree
// is <= pf_max_deg (above it the node reads a filtered list, not the row).
template <class F>
__device__ __forceinline__ void for_items(const Params& p, const int4* items, int64_t count,
                                          bool topo, int64_t start, int64_t stride, int pf_max_deg,
                                          F f) {
  if (start >= count) return;
  const int4 none = make_int4(0, 0, -1, 0);
  int4 A = ld_cg4(items + start);
  int4 B = start + stride < count ? ld_cg4(items + start + stride) : none;
  int sA = ld_ro(p.rowptr + A.x), eA = ld_ro(p.rowptr + A.x + 1);
  int cA = topo ? ld_cg(p.color + A.x) : 0;
  for (int64_t k = start; k < count; k += stride) {
    int sB = 0, eB = 0, cB = 0;
    if (k + stride < count) {
      sB = ld_ro(p.rowptr + B.x);
      eB = ld_ro(p.rowptr + B.x + 1);
      if (topo) cB = ld_cg(p.color + B.x);
    }
    const int4 C = k + 2 * stride < count ? ld_cg4(items + k + 2 * stride) : none;
    if (cA == 0) f(A.x, A.y, A.z, A.w, sA, eA - sA);
    if (k + stride < count && cB == 0 && eB - sB <= pf_max_deg &&
        lane_id() == 0) {  // B's neighbours, into L2
      const int64_t lo = (int64_t)sB + (int64_t)B.y * p.chunk;
      prefetch_l2(p, lo, min((int64_t)eB, lo + p.chunk));
    }
    A = B;
    sA = sB;
    eA = eB;
    cA = cB;
    B = C;
  }
}

// The same without loading ahead (fewer registers), for the short item
// lists of filtered nodes; every item's node is active (data-driven).
template <class F>
__device__ __forceinline__ void for_items_plain(const Params& p, const int4* items, int64_t count,
                                                int64_t start, int64_t stride, F f) {
  for (int64_t k = start; k < count; k += stride) {
    const int4 A = ld_cg4(items + k);
    const int sA = ld_ro(p.rowptr + A.x), eA = ld_ro(p.rowptr + A.x + 1);
    f(A.x, A.y, A.z, A.w, sA, eA - sA);
  }
}

// Low-degree nodes, 32 per share: the worklist entries [base, base + 32) or,
// topology-driven, node IDs [base, base + 32) of degree <= t1 and colour 0.
// Calls f(v, s, d, t) per share for all lanes (v = -1, d = 0 on idle lanes;
// t = tent[v] when WithTent).
template <bool WithTent, class F>
__device__ __forceinline__ void for_small(const Params& p, const int32_t* list, int64_t span,
                                          bool topo, int t1, int64_t start, int64_t stride, F f) {
  if (start >= span) return;
  const int lane = lane_id();
  auto node_at = [&](int64_t i) -> int {
    return i < span ? (topo ? (int)i : ld_cg(list + i)) : -1;
  };
  int vA = node_at(start + lane);
  int vB = node_at(start + stride + lane);
  int sA = 0, eA = 0, cA = 0, tA = 0;
  if (vA >= 0) {
    sA = ld_ro(p.rowptr + vA);
    eA = ld_ro(p.rowptr + vA + 1);
    if (topo) cA = ld_cg(p.color + vA);
    if (WithTent) tA = ld_cg(p.tent + vA);
  }
  for (int64_t base = start; base < span; base += stride) {
    int sB = 0, eB = 0, cB = 0, tB = 0;
    if (vB >= 0) {
      sB = ld_ro(p.rowptr + vB);
      eB = ld_ro(p.rowptr + vB + 1);
      if (topo) cB = ld_cg(p.color + vB);
      if (WithTent) tB = ld_cg(p.tent + vB);
    }
    const int vC = node_at(base + 2 * stride + lane);
    int v = vA, d = eA - sA;
    if (v >= 0 && topo && (d > t1 || cA != 0)) v = -1;
    if (v < 0) d = 0;
    f(v, sA, d, tA);
    vA = vB;
    sA = sB;
    eA = eB;
    cA = cB;
    tA = tB;
    vB = vC;
  }
}

// ------------------------------------------------------------------ phases --

struct RoundView {
  int round;   // 1-based round number
  int par;     // worklist parity read this round
  int mode;    // MODE_TOPO or MODE_DATA
  int nsmall;  // low-degree nodes in the worklist
  int nbig;    // high-degree nodes in the worklist
  int icnt;    // work items of the worklist's high-degree nodes (not filtered)
  int nistat;  // work items of every high-degree node (not filtered)
  int ficnt;   // work items of the worklist's filtered nodes
  int maxc;    // largest committed colour at round start
  int r0;      // first round of neighbour filtering (0: not started)
  int t1;      // the low-degree bound in use
  int filt;    // nodes of degree > filt_deg read filtered lists this round
  int push;    // nodes of degree > t1 read their forbidden-colour bitmaps this round
  int odd;     // pushing: worklist nodes that are not list nodes with one work item
  int late;    // pushing: this round runs late (winners push along their lists, no push phase)
  int pull;    // pushing: the previous round ran late (list nodes collect lower-ID winners)
  unsigned long long dsum;  // degree sum of the worklist
};

// The state of round r, read from the control block by warp 0 (one field
// per lane) into shared memory and handed to every thread of the CTA: all
// warps of a large team loading the same few lines at once would queue at
// one L2 slice after every barrier. Called by every thread of the CTA.
// The 14 control-block words of round r's state into dst (warp 0). All of
// them are final once round r - 1's conflict step is over: its push phase
// writes none of them.
__device__ __forceinline__ void load_round_words(const Params& p, int r, int* dst) {
  const int par = r & 1;
  const Ctrl* c = p.ctrl;
  const int32_t* dsum = reinterpret_cast<const int32_t*>(&c->dsum[par]);
  const int32_t* src[14] = {&c->cnt[par][B_SMALL], &c->cnt[par][B_BIG], &c->icnt[par], &c->nistat,
                            &c->ficnt[par],        &c->t1,             &c->maxc,       dsum,
                            dsum + 1,              &c->handoff_round,  &c->maxc_start[(r - 1) & 1],
                            &c->push_on,           &c->cnt[par][2],    &c->late_at[(r - 1) & 1]};
  const int lane = lane_id();
  if (lane < 14) dst[lane] = ld_cg(src[lane]);
}

template <int BS>
__device__ __forceinline__ RoundView read_round(const Params& p, int r, Smem<BS>& sm) {
  const int par = r & 1;
  if (sm.rvn_round == r) {  // read ahead, before the previous round's push phase
    if (threadIdx.x < 14) sm.rvb[threadIdx.x] = sm.rvn[threadIdx.x];
  } else if (threadIdx.x < 32) {
    load_round_words(p, r, sm.rvb);
  }
  __syncthreads();
  RoundView rv;
  rv.round = r;
  rv.par = par;
  rv.nsmall = sm.rvb[0];
  rv.nbig = sm.rvb[1];
  rv.icnt = sm.rvb[2];
  rv.nistat = sm.rvb[3];
  rv.ficnt = sm.rvb[4];
  rv.t1 = sm.rvb[5];
  rv.maxc = sm.rvb[6];
  rv.dsum = (unsigned long long)(uint32_t)sm.rvb[7] | ((unsigned long long)(uint32_t)sm.rvb[8] << 32);
  rv.mode = MODE_DATA;
  const int maxc_prev = sm.rvb[10];
  // filtering in round r >= r0 iff the colours committed before round r - 1
  // fit the bitmap with room for round r - 1's (a round adds at most 1 to maxc)
  rv.r0 = p.filt_r0 > 0 ? p.filt_r0 : sm.rvb[9];
  rv.filt = p.alist[0] != nullptr && rv.r0 > 0 && r >= rv.r0 && maxc_prev <= kFiltMaxC;
  // pushing in round r iff the colours committed before round r - 1 are
  // <= kPushMaxC - 2: round r - 1 adds at most 1, so every tentative colour of
  // round r is <= kPushMaxC and the bitmaps hold it
  rv.push = p.pbits != nullptr && sm.rvb[11] != 0 && maxc_prev <= kPushMaxC - 2;
  rv.odd = sm.rvb[12];
  rv.late = 0;  // decided with the mode
  rv.pull = rv.push && r >= 3 && sm.rvb[13] != 0;
  return rv;
}

// One control-block word for every thread of the CTA (read by thread 0).
template <int BS>
__device__ __forceinline__ int read_shared_word(const int32_t* w, Smem<BS>& sm) {
  __syncthreads();  // earlier readers of the slot are done
  if (threadIdx.x == 0) sm.rvb[23] = ld_cg(w);
  __syncthreads();
  return sm.rvb[23];
}

__device__ __forceinline__ int decide_mode(const Params& p, int64_t total) {
  if (p.policy == IPGC_MODE_TOPO) return MODE_TOPO;
  if (p.policy == IPGC_MODE_DATA) return MODE_DATA;
  return total > p.H ? MODE_TOPO : MODE_DATA;
}

// Mode of the round for every thread of the CTA. With IPGC_MODE_LEARNED and
// a loaded network, warp 0 evaluates it (every CTA of the team computes the
// same value from the same inputs); the threshold rule decides when the
// network is unsure (|p - 0.5| < margin) or absent. A round after a late
// round (see run_rounds) collects its list nodes' lower-ID winners from the
// lists, which only the data-driven round does: the learned switch is not
// asked then (the threshold and data rules give data-driven there anyway).
template <int BS>
__device__ __forceinline__ int decide_mode_block(const Params& p, const RoundView& rv,
                                                 int64_t total, Smem<BS>& sm) {
  if (p.policy != IPGC_MODE_LEARNED || !p.mlp) return decide_mode(p, total);
  if (rv.pull) return MODE_DATA;
  if (threadIdx.x < 32) {
    float f[kMlpIn];
    policy_features(p.n, p.nnz, rv.round, total, rv.nsmall, (int64_t)rv.dsum, rv.maxc, f);
    const float z = mlp_logit_warp(p.mlp, f);
    if (threadIdx.x == 0) {
      const float pr = 1.0f / (1.0f + expf(-z));
      int mode = total > p.H ? MODE_TOPO : MODE_DATA;
      if (fabsf(pr - 0.5f) >= p.mlp_margin) mode = pr > 0.5f ? MODE_TOPO : MODE_DATA;
      sm.mode_b = mode;
    }
  }
  __syncthreads();
  return sm.mode_b;
}

// Bookkeeping by CTA 0 at the start of round r (after the previous barrier):
// clear the counters this round pushes into and count the round.
__device__ __forceinline__ void round_begin(const Params& p, const RoundView& rv, int r,
                                            int64_t total, Team tm) {
  if (tm.cta != 0 || threadIdx.x != 0) return;
  Ctrl* c = p.ctrl;
  const int nxt = rv.par ^ 1;
#pragma unroll
  for (int k = 0; k < 4; ++k) c->cnt[nxt][k] = 0;
  c->icnt[nxt] = 0;
  c->ficnt[nxt] = 0;
  c->dsum[nxt] = 0;
  c->pqcnt = 0;
  c->pwcnt = 0;
  c->rqcnt = 0;
  c->late_at[r & 1] = rv.late ? 1 : 0;
  c->rounds = r;
  c->maxc_start[r & 1] = rv.maxc;
  c->mode_at[r & 1] = rv.mode;
  if (rv.mode == MODE_TOPO) {  // a later rebuild counts from zero
    c->rbcnt[0] = 0;
    c->rbcnt[1] = 0;
  }
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
    tr.wl_small = rv.nsmall;
    tr.push_ns = 0;
    tr.t_begin = gtime();
  }
  __threadfence();
}

// The loops that involve filtered nodes are functions of their own (not
// inlined), so the register budget of the other loops stays as it is
// without them; they run once per phase. From round r0 on, filtered nodes
// have work items of their own (fitems); in round r0 (built from the items
// of the unfiltered rounds) and in topology sweeps (static items) they are
// mixed with the others.

// Assignment step of work items [k = gwarp, gwarp + nwarps, ...) of a list.
template <int BS>
__device__ __forceinline__ void assign_items(const Params& p, Smem<BS>& sm, const int4* items,
                                             int count, bool topo, int maxc, bool pushing,
                                             bool pull, Team tm) {
  const int warp = threadIdx.x >> 5;
  const int gwarp = tm.cta * (BS / 32) + warp, nwarps = tm.ncta * (BS / 32);
  unsigned* wb = sm.wbits[warp];
  for_items(p, items, count, topo, gwarp, nwarps, pushing ? -1 : INT_MAX,
            [&](int v, int c, int gslot, int nch, int s, int d) {
              if (pushing) {
                if (gslot >= 0)
                  item_assign_plist(p, v, s, d, c, nch, gslot, pull);
                else if (c == 0)
                  item_assign_push(p, v, s, d);
              } else {
                item_assign(p, wb, v, s, d, c, nch, gslot, maxc);
              }
            });
}

// Filtered or not, by degree (round r0 and topology sweeps while filtering).
template <int BS>
__device__ __noinline__ void assign_mixed(const Params& p, Smem<BS>& sm, const int4* items,
                                          int count, const RoundView& rv, Team tm) {
  const int warp = threadIdx.x >> 5;
  const int gwarp = tm.cta * (BS / 32) + warp, nwarps = tm.ncta * (BS / 32);
  const bool topo = rv.mode == MODE_TOPO;
  const int round = rv.round, r0 = rv.r0, maxc = rv.maxc;
  unsigned* wb = sm.wbits[warp];
  for_items(p, items, count, topo, gwarp, nwarps, round == r0 ? INT_MAX : p.filt_deg,
            [&](int v, int c, int gslot, int nch, int s, int d) {
              if (d > p.filt_deg) {
                const int ne = filt_items(p, round, r0, gslot, d);
                if (c < ne) item_assign_filtered(p, wb, v, s, d, c, ne, gslot, round, r0, maxc);
              } else {
                item_assign(p, wb, v, s, d, c, nch, gslot, maxc);
              }
            });
}

// The worklist's filtered nodes in a data-driven round after r0.
template <int BS>
__device__ __noinline__ void assign_fitems(const Params& p, Smem<BS>& sm, const RoundView& rv,
                                           Team tm) {
  const int warp = threadIdx.x >> 5;
  const int gwarp = tm.cta * (BS / 32) + warp, nwarps = tm.ncta * (BS / 32);
  unsigned* wb = sm.wbits[warp];
  const int round = rv.round, r0 = rv.r0, maxc = rv.maxc;
  for_items_plain(p, p.fitems[rv.par], rv.ficnt, gwarp, nwarps,
                  [&](int v, int c, int gslot, int nch, int s, int d) {
                    item_assign_filtered(p, wb, v, s, d, c, nch, gslot, round, r0, maxc);
                  });
}

template <int BS>
__device__ __forceinline__ void assign_small_nodes(const Params& p, Smem<BS>& sm,
                                                   const RoundView& rv, Team tm) {
  const int warp = threadIdx.x >> 5;
  const int gwarp = tm.cta * (BS / 32) + warp, nwarps = tm.ncta * (BS / 32);
  const bool topo = rv.mode == MODE_TOPO;
  unsigned* wm = sm.small_w[warp];
  const int64_t span = topo ? (int64_t)p.n : (int64_t)rv.nsmall;
  for_small<false>(p, p.wl[rv.par], span, topo, rv.t1, (int64_t)gwarp * 32, (int64_t)nwarps * 32,
                   [&](int v, int s, int d, int) { small_assign(p, v, s, d, wm); });
}

template <int BS, bool FILT, bool PUSH = false>
__device__ void assign_phase(const Params& p, Smem<BS>& sm, const RoundView& rv, Team tm) {
  const bool topo = rv.mode == MODE_TOPO;
  const int4* items = topo ? p.istat : p.items[rv.par];
  const int count = topo ? rv.nistat : rv.icnt;
  // (a call saves and restores registers in every thread, so warps without
  // an item of a list skip it)
  const int gwarp = tm.cta * (BS / 32) + (threadIdx.x >> 5);
  if (FILT && rv.filt && (topo || rv.round == rv.r0)) {
    if (gwarp < count) assign_mixed<BS>(p, sm, items, count, rv, tm);
  } else {
    assign_items<BS>(p, sm, items, count, topo, rv.maxc, PUSH && rv.push, PUSH && rv.pull, tm);
    if (FILT && rv.filt && gwarp < rv.ficnt) assign_fitems<BS>(p, sm, rv, tm);
  }
  assign_small_nodes<BS>(p, sm, rv, tm);
}

// Conflict step of work items of a list; pushes through `stage`.
template <int BS>
__device__ __forceinline__ PhaseAcc detect_items(const Params& p, ItemStage& stage,
                                                 const int4* items, int count, bool topo,
                                                 int round, int nxt, WarpStage* wst,
                                                 bool lists_next, bool late, int t1, Team tm) {
  const int warp = threadIdx.x >> 5;
  const int gwarp = tm.cta * (BS / 32) + warp, nwarps = tm.ncta * (BS / 32);
  PhaseAcc acc;
  const bool push = !(topo && p.wl_rebuild);  // rebuild: topology sweeps keep no worklist
  // (with pushing, nodes with a merge-state slot read their lists, not their rows)
  for_items(p, items, count, topo, gwarp, nwarps, wst ? p.chunk : INT_MAX,
            [&](int v, int cidx, int gslot, int nch, int s, int d) {
              if (wst && gslot >= 0)
                item_detect_plist(p, stage, v, s, d, cidx, nch, gslot, nxt, acc, round, push,
                                  lists_next, late, t1);
              else
                item_detect(p, stage, v, s, d, cidx, nch, gslot, nxt, acc, round, push, wst);
            });
  return acc;
}

// Conflict step, filtered or not by degree (round r0 and topology sweeps
// while filtering).
template <int BS>
__device__ __noinline__ PhaseAcc detect_mixed(const Params& p, Smem<BS>& sm, ItemStage& stage,
                                              const int4* items, int count, const RoundView& rv,
                                              Team tm) {
  const int warp = threadIdx.x >> 5;
  const int gwarp = tm.cta * (BS / 32) + warp, nwarps = tm.ncta * (BS / 32);
  const bool topo = rv.mode == MODE_TOPO;
  const int nxt = rv.par ^ 1, round = rv.round, r0 = rv.r0;
  Ctrl* c = p.ctrl;
  PhaseAcc acc;
  // the next round filters iff this round's starting maxc leaves room
  const bool filt_next = ld_cg(&c->maxc_start[round & 1]) <= kFiltMaxC;
  ItemStage st = stage;
  ItemStage fstage{sm.stage_t[warp], 0};
  for_items(p, items, count, topo, gwarp, nwarps, -1,
            [&](int v, int cidx, int gslot, int nch, int s, int d) {
              if (d > p.filt_deg) {
                const int ne = filt_items(p, round, r0, gslot, d);
                if (cidx < ne)
                  item_detect_filtered(p, st, fstage, v, s, d, cidx, ne, gslot, nxt, acc, round,
                                       r0, filt_next);
              } else {
                item_detect(p, st, v, s, d, cidx, nch, gslot, nxt, acc, round);
              }
            });
  items_flush(fstage, p.fitems[nxt], &c->ficnt[nxt]);
  stage = st;
  return acc;
}

// Conflict step of the worklist's filtered nodes in a data-driven round
// after r0.
template <int BS>
__device__ __noinline__ PhaseAcc detect_fitems(const Params& p, Smem<BS>& sm, ItemStage& stage,
                                               const RoundView& rv, Team tm) {
  const int warp = threadIdx.x >> 5;
  const int gwarp = tm.cta * (BS / 32) + warp, nwarps = tm.ncta * (BS / 32);
  const int nxt = rv.par ^ 1, round = rv.round, r0 = rv.r0;
  Ctrl* c = p.ctrl;
  PhaseAcc acc;
  const bool filt_next = ld_cg(&c->maxc_start[round & 1]) <= kFiltMaxC;
  ItemStage st = stage;
  ItemStage fstage{sm.stage_t[warp], 0};
  for_items_plain(p, p.fitems[rv.par], rv.ficnt, gwarp, nwarps,
                  [&](int v, int cidx, int gslot, int nch, int s, int d) {
                    item_detect_filtered(p, st, fstage, v, s, d, cidx, nch, gslot, nxt, acc,
                                         round, r0, filt_next);
                  });
  items_flush(fstage, p.fitems[nxt], &c->ficnt[nxt]);
  stage = st;
  return acc;
}

template <int BS>
__device__ __forceinline__ PhaseAcc detect_small_nodes(const Params& p, Smem<BS>& sm,
                                                       const RoundView& rv, WarpStage* wst,
                                                       Team tm) {
  const int warp = threadIdx.x >> 5;
  const int gwarp = tm.cta * (BS / 32) + warp, nwarps = tm.ncta * (BS / 32);
  const bool topo = rv.mode == MODE_TOPO;
  const int nxt = rv.par ^ 1;
  Ctrl* c = p.ctrl;
  PhaseAcc acc;
  unsigned* wm = sm.small_w[warp];
  WarpStage sg{sm.stage_s[warp], 0};
  const int64_t span = topo ? (int64_t)p.n : (int64_t)rv.nsmall;
  const bool push = !(topo && p.wl_rebuild);  // rebuild: topology sweeps keep no worklist
  for_small<true>(p, p.wl[rv.par], span, topo, rv.t1, (int64_t)gwarp * 32, (int64_t)nwarps * 32,
                  [&](int v, int s, int d, int t) {
                    const bool lose = small_lose(p, v, s, d, t, wm);
                    stage_push(sg, kStageSmall, push && v >= 0 && lose, v, p.wl[nxt],
                               &c->cnt[nxt][B_SMALL]);
                    if (v >= 0) {
                      if (lose) {
                        if (!push) acc.nsm += 1;
                        acc.dsum += (unsigned long long)d;
                      } else {
                        p.color[v] = t;  // (a node of degree <= t1 is never a push target)
                        acc.maxc = max(acc.maxc, t);
                        if (p.fin) p.fin[v] = rv.round;
                      }
                    }
                    if (wst)  // pushing: winners for the push phase
                      stage_push(*wst, kStageSmall, v >= 0 && !lose, v, p.pw, &c->pwcnt);
                  });
  stage_flush(sg, p.wl[nxt], &c->cnt[nxt][B_SMALL]);
  return acc;
}

__device__ __forceinline__ void acc_merge(PhaseAcc& a, const PhaseAcc& b) {
  a.maxc = max(a.maxc, b.maxc);
  a.dsum += b.dsum;
  a.nbig += b.nbig;
  a.nsm += b.nsm;
  a.nodd += b.nodd;
}

// Worklist rebuild (the discard-and-rebuild hybrid of Nasre et al., which the
// paper contrasts with its own, Section I): a data-driven round that follows
// a topology-driven one, which kept no worklist, first collects the active
// nodes: every low-degree node of colour 0 into the low-degree list, every
// static work item of an active high-degree node into the item list, with
// counts in rbcnt; a team barrier follows.
template <int BS>
__device__ __noinline__ void rebuild_worklists(const Params& p, Smem<BS>& sm, const RoundView& rv,
                                               Team tm) {
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const int gwarp = tm.cta * (BS / 32) + warp, nwarps = tm.ncta * (BS / 32);
  Ctrl* c = p.ctrl;
  WarpStage sg{sm.stage_s[warp], 0};
  for (int64_t base = (int64_t)gwarp * 32; base < p.n; base += (int64_t)nwarps * 32) {
    const int v = (int)(base + lane);
    bool act = false;
    if (v < p.n && ld_cg(p.color + v) == 0) {
      const int d = ld_ro(p.rowptr + v + 1) - ld_ro(p.rowptr + v);
      act = bucket_of(d, rv.t1) == B_SMALL;
    }
    stage_push(sg, kStageSmall, act, v, p.wl[rv.par], &c->rbcnt[0]);
  }
  stage_flush(sg, p.wl[rv.par], &c->rbcnt[0]);
  ItemStage st{sm.stage_i[warp], 0};
  for (int64_t k0 = (int64_t)gwarp * 32; k0 < rv.nistat; k0 += (int64_t)nwarps * 32) {
    const int64_t k = k0 + lane;
    int4 it = make_int4(0, 0, -1, 0);
    bool act = false;
    if (k < rv.nistat) {
      it = ld_cg4(p.istat + k);
      act = ld_cg(p.color + it.x) == 0;
    }
    // one item at a time, in the static list's order (items of a node are
    // pushed by its item 0 together, so each node's items stay one group)
    items_push(st, it.x, act && it.y == 0 ? it.w : 0, it.z, p.items[rv.par], &c->rbcnt[1]);
  }
  items_flush(st, p.items[rv.par], &c->rbcnt[1]);
}

template <int BS, bool FILT, bool PUSH = false>
__device__ void detect_phase(const Params& p, Smem<BS>& sm, const RoundView& rv, PhaseAcc& acc,
                             Team tm) {
  const int warp = threadIdx.x >> 5;
  const bool topo = rv.mode == MODE_TOPO;
  const int nxt = rv.par ^ 1;
  const int4* items = topo ? p.istat : p.items[rv.par];
  const int count = topo ? rv.nistat : rv.icnt;
  ItemStage stage{sm.stage_i[warp], 0};
  // with pushing, the winners are staged in the (then idle) filtered-item buffer
  static_assert(sizeof(sm.stage_t[0]) >= kStageSmall * sizeof(int32_t), "winner stage");
  WarpStage wst_buf{reinterpret_cast<int32_t*>(sm.stage_t[warp]), 0};
  WarpStage* wst = PUSH && rv.push ? &wst_buf : nullptr;
  const int gwarp = tm.cta * (BS / 32) + warp;
  if (FILT && rv.filt && (topo || rv.round == rv.r0)) {
    if (gwarp < count) acc_merge(acc, detect_mixed<BS>(p, sm, stage, items, count, rv, tm));
  } else {
    acc_merge(acc, detect_items<BS>(p, stage, items, count, topo, rv.round, nxt, wst,
                                    rv.maxc <= kPushMaxC - 2, PUSH && rv.late, rv.t1, tm));
    if (FILT && rv.filt && gwarp < rv.ficnt)
      acc_merge(acc, detect_fitems<BS>(p, sm, stage, rv, tm));
  }
  items_flush(stage, p.items[nxt], &p.ctrl->icnt[nxt]);
  acc_merge(acc, detect_small_nodes<BS>(p, sm, rv, wst, tm));
  if (wst) stage_flush(*wst, p.pw, &p.ctrl->pwcnt);
}

// The push phase that follows a conflict step (or round 1) with pushing:
// the colours of the nodes committed in it into their active neighbours'
// bitmaps. Work units: the queued one-window items of the rows of winners of
// degree > t1 (one warp each; a warp loads its next item's window and the
// record after that before it pushes the current one, so their latency
// overlaps the pushes' gathers), then the listed low-degree winners 32 at a
// time (their rows laid end to end, at most 32 * t1 entries), then the
// one-window units of the list rewrites the conflict step queued (the
// entries still active after it, appended to the node's other list buffer).
// A team barrier follows.
template <int BS>
__device__ __noinline__ void push_phase(const Params& p, int nq, int nw, int nr, int t1, Team tm) {
  const int gwarp = tm.cta * (BS / 32) + (threadIdx.x >> 5), nwarps = tm.ncta * (BS / 32);
  const int lane = lane_id();
  const int units = nq + (nw + 31) / 32;
  int k = gwarp;
  if (k < nq) {
    const uint64_t pol = l2_keep_policy();
    const int4 none = make_int4(0, 0, 0, 0);
    int4 A = ld_cg4(p.pq + k);
    int4 B = k + nwarps < nq ? ld_cg4(p.pq + k + nwarps) : none;
    int u[kGather];
    load_push_item(p, A, u);
    for (; k < nq; k += nwarps) {
      const bool more = k + nwarps < nq;
      const int4 C = k + 2 * nwarps < nq ? ld_cg4(p.pq + k + 2 * nwarps) : none;
      int un[kGather];
      if (more) load_push_item(p, B, un);
      push_targets(p, u, A.z, t1, pol);
      if (more) {
#pragma unroll
        for (int q = 0; q < kGather; ++q) u[q] = un[q];
      }
      A = B;
      B = C;
    }
  }
  // the low-degree winners: the next share's rows are located while the
  // current share pushes
  auto locate = [&](int kk, int& s, int& d, int& t) {
    const int i = (kk - nq) * 32 + lane;
    s = 0;
    d = 0;
    t = 1;
    if (kk < units && i < nw) {
      const int v = ld_cg(p.pw + i);
      s = ld_ro(p.rowptr + v);
      d = ld_ro(p.rowptr + v + 1) - s;
      t = ld_cg(p.color + v);
    }
  };
  if (k < units) {
    int s, d, t;
    locate(k, s, d, t);
    for (; k < units; k += nwarps) {
      int sn, dn, tn;
      locate(k + nwarps, sn, dn, tn);
      small_push(p, s, d, t, t1, true);
      s = sn;
      d = dn;
      t = tn;
    }
  }
  for (; k < units + nr; k += nwarps) {  // list rewrites {row start, slot, length, window | buffer}
    const int4 it = ld_cg4(p.rq + (k - units));
    const int src = (int)((unsigned)it.w >> 31), j = it.w & 0x7fffffff;
    const int64_t s = it.x, a = (s & ~int64_t(3)) + (int64_t)j * kPushChunk;
    plist_append(p, p.alist[src], false, a > s ? a : s, min(s + it.z, a + kPushChunk), INT_MAX, s,
                 p.alist[src ^ 1], &p.flen[src ^ 1][it.y].x);
  }
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
    tr.wl_small = 0;
    tr.push_ns = 0;
    tr.t_begin = t0;
    tr.t_assign = t0;
    tr.t_detect = t1;
  }
}


// ----------------------------------------------------------- one colouring --

// Result publication into host-mapped memory. Every CTA of the team copies
// its slice of the final colours (read from L2: other CTAs wrote them) and
// fences at system scope before it counts itself done; the CTA that counts
// last copies the control block and then raises the host flag, so a host that
// sees the flag sees the whole result.
template <int BS>
__device__ void publish_result(const Params& p, Team tm) {
  const int64_t n = p.n;
  int64_t lo = n * tm.cta / tm.ncta, hi = n * (tm.cta + 1) / tm.ncta;
  const bool vec = (((uintptr_t)p.color | (uintptr_t)p.out_colors) & 15u) == 0;
  if (vec) {
    // slices rounded to multiples of 4 nodes: int4 copies, scalar tail
    lo &= ~int64_t(3);
    hi = tm.cta + 1 == tm.ncta ? n : (hi & ~int64_t(3));
    const int64_t v_hi = lo + ((hi - lo) & ~int64_t(3));
    const int4* src = reinterpret_cast<const int4*>(p.color);
    int4* dst = reinterpret_cast<int4*>(p.out_colors);
    for (int64_t i = lo / 4 + threadIdx.x; i < v_hi / 4; i += BS) dst[i] = ld_cg4(src + i);
    for (int64_t i = v_hi + threadIdx.x; i < hi; i += BS) p.out_colors[i] = ld_cg(p.color + i);
  } else {
    for (int64_t i = lo + threadIdx.x; i < hi; i += BS) p.out_colors[i] = ld_cg(p.color + i);
  }
  __threadfence_system();
  __syncthreads();
  if (threadIdx.x == 0) {
    const int prev = atomicAdd(&p.ctrl->ctas_done, 1);
    if (prev == tm.ncta - 1) {
      __threadfence();
      const volatile uint32_t* s = reinterpret_cast<const volatile uint32_t*>(p.ctrl);
      volatile uint32_t* d = reinterpret_cast<volatile uint32_t*>(p.out_ctrl);
      for (int i = 0; i < (int)(sizeof(Ctrl) / 4); ++i) d[i] = s[i];
      __threadfence_system();
      *reinterpret_cast<volatile int32_t*>(p.out_done) = 1;
    }
  }
}

// The whole round loop of one graph by a team of CTAs (the whole grid for the
// single-graph kernel, a few CTAs or one CTA for a graph of a batch), the
// rounds separated by the team's bounded barrier.
// The low-degree bound when it is chosen on the device: every node when all
// degrees fit the low-degree path (regular graphs: a warp then colours 32
// nodes with their edges balanced over its lanes), else the given t1.
__device__ __forceinline__ int auto_t1(const Params& p, int maxdeg) {
  return maxdeg <= kMaxT1 ? (maxdeg > 0 ? maxdeg : 1) : p.t1;
}

// The largest degree of the graph into ctrl->maxdeg and, with pushing, the
// forbidden-colour bitmaps of every node that may keep one (degree > the
// given t1, which the t1 in use never undercuts where such nodes exist)
// cleared and the entries of their rows counted into ctrl->bigsum; then a
// team barrier.
template <int BS>
__device__ bool team_max_degree(const Params& p, Smem<BS>& sm, Team tm, bool zero) {
  int m = 0;
  unsigned long long big = 0;
  // four nodes per thread and step: one int4 of row offsets (16-byte aligned
  // rowptr) and the next offset, so a pass over a large graph keeps many
  // loads in flight
  const bool vec = ((uintptr_t)p.rowptr & 15u) == 0;
  const int64_t n = p.n;
  for (int64_t v0 = ((int64_t)tm.cta * BS + threadIdx.x) * 4; v0 < n;
       v0 += (int64_t)tm.ncta * BS * 4) {
    int r[5];
    if (vec && v0 + 4 <= n) {
      const int4 x = __ldg(reinterpret_cast<const int4*>(p.rowptr + v0));
      r[0] = x.x;
      r[1] = x.y;
      r[2] = x.z;
      r[3] = x.w;
      r[4] = ld_ro(p.rowptr + v0 + 4);
    } else {
#pragma unroll
      for (int j = 0; j < 5; ++j) r[j] = v0 + j <= n ? ld_ro(p.rowptr + v0 + j) : 0;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (v0 + j >= n) break;
      const int s = r[j], d = r[j + 1] - s;
      m = max(m, d);
      if (zero && d > p.t1) {
        big += (unsigned long long)d;
        for (int i = 0, nw = push_words(d); i < nw; ++i) p.pbits[s + i] = 0u;
      }
    }
  }
  m = block_max<BS>(sm, m);
  if (threadIdx.x == 0 && m > 0) atomicMax(&p.ctrl->maxdeg, m);
  if (zero) {
    big = block_sum64<BS>(sm, big);
    if (threadIdx.x == 0 && big) atomicAdd(&p.ctrl->bigsum, big);
  }
  return team_barrier(p.ctrl, tm.cta, tm.ncta, p.timeout_ns, p.bar_extra, bar_memo<BS>(sm));
}

// Rounds r_start, r_start + 1, ... of one graph by a team of CTAs, separated
// by the team's bounded barrier, until the worklist is empty. Without FILT
// the loop stops early at the hand-over round (handoff_now), which it
// records for continue_graph.
template <int BS, bool FILT, bool PUSH = false>
__device__ void run_rounds(const Params& p, Smem<BS>& sm, Team tm, int r_start) {
  Ctrl* c = p.ctrl;
  const bool lead = tm.cta == 0 && threadIdx.x == 0;
  for (int r = r_start;; ++r) {
    RoundView rv = read_round<BS>(p, r, sm);
    const int64_t total = (int64_t)rv.nsmall + rv.nbig;
    if (total == 0) break;
    if (r > p.max_rounds) {
      if (lead) record_error(c, IPGC_ERR_NO_CONVERGE);
      break;
    }
    if (!FILT && !PUSH && handoff_now(p, r, total, rv.dsum, rv.maxc)) {
      if (lead) c->handoff_round = r;
      break;
    }
    rv.mode = decide_mode_block<BS>(p, rv, total, sm);
    // pushing runs a round late when every active node keeps a list of one
    // work item (rounds after 2, data-driven; the round after a late one is
    // data-driven too: the threshold and data rules never go back to
    // topology-driven once |WL| is small, and the learned rule is overruled
    // there): the active edges are then all on the lists, a winner pushes
    // along its own list (its active lower-ID neighbours) and the next
    // round's list nodes collect their lower-ID winners from theirs, so no
    // push phase is needed
    rv.late = PUSH && rv.push && r >= 3 && rv.mode == MODE_DATA && rv.nsmall == 0 &&
              rv.odd == 0 && p.policy != IPGC_MODE_TOPO && !p.wl_rebuild;
    if (p.wl_rebuild && rv.mode == MODE_DATA &&
        (r == 2 || ld_cg(&c->mode_at[(r - 1) & 1]) == MODE_TOPO)) {
      rebuild_worklists<BS>(p, sm, rv, tm);
      if (!team_barrier(c, tm.cta, tm.ncta, p.timeout_ns, p.bar_extra, bar_memo<BS>(sm))) break;
      rv.nsmall = ld_cg(&c->rbcnt[0]);
      rv.icnt = ld_cg(&c->rbcnt[1]);
    }
    if (p.shrink && rv.mode == MODE_DATA && tm.ncta > kShrinkMin) {
      // a small round on a big team costs mostly barriers and idle passes:
      // once a quarter of the team would do with one work unit (an item or
      // 32 low-degree nodes) per warp, the CTAs beyond that leave for good
      // (the worklist only shrinks)
      const int64_t units = (int64_t)rv.icnt + (FILT ? rv.ficnt : 0) + ((int64_t)rv.nsmall + 31) / 32;
      const int64_t want = (units + (BS / 32) - 1) / (BS / 32);
      // (with pushing a high-degree winner's whole row is pushed after the
      // conflict step, one warp per kPushChunk entries: keep more CTAs, except
      // in late rounds, whose winners push along their short lists)
      const int kmin = PUSH && rv.push && !rv.late ? kShrinkMinPush : kShrinkMin;
      const int k = (int)(want > kmin ? want : kmin);
      if (4 * k <= tm.ncta) {
        if (tm.cta >= k) break;
        tm.ncta = k;
      }
    }
    round_begin(p, rv, r, total, tm);
    assign_phase<BS, FILT, PUSH>(p, sm, rv, tm);
    if (!team_barrier(c, tm.cta, tm.ncta, p.timeout_ns, p.bar_extra, bar_memo<BS>(sm))) break;
    if (lead && p.trace && r <= p.trace_cap) p.trace[r - 1].t_assign = gtime();
    {
      PhaseAcc acc;
      detect_phase<BS, FILT, PUSH>(p, sm, rv, acc, tm);
      phase_commit<BS>(p, sm, acc, rv.par ^ 1);
    }
    if (!team_barrier(c, tm.cta, tm.ncta, p.timeout_ns, p.bar_extra, bar_memo<BS>(sm))) break;
    if (PUSH && rv.push) {
      __syncthreads();  // the previous readers of the slots are done
      if (threadIdx.x == 0) {
        sm.rvb[20] = ld_cg(&c->pqcnt);
        sm.rvb[21] = ld_cg(&c->pwcnt);
        sm.rvb[22] = ld_cg(&c->rqcnt);
        sm.rvn_round = r + 1;
      }
      // the next round's state in the same round trip (final after this
      // conflict step), so the next round starts without reading it
      if (threadIdx.x < 32) load_round_words(p, r + 1, sm.rvn);
      __syncthreads();
      const int q = sm.rvb[20], w = sm.rvb[21], nr = sm.rvb[22];
      if (q > 0 || w > 0 || nr > 0) {
        const uint64_t tp = lead && p.trace && r <= p.trace_cap ? gtime() : 0;
        push_phase<BS>(p, q, w, nr, rv.t1, tm);
        if (!team_barrier(c, tm.cta, tm.ncta, p.timeout_ns, p.bar_extra, bar_memo<BS>(sm))) break;
        if (tp) p.trace[r - 1].push_ns = (int32_t)(gtime() - tp);
      }
    }
    if (lead && p.trace && r <= p.trace_cap) p.trace[r - 1].t_detect = gtime();
  }
}

// The whole colouring of one graph by a team of CTAs (the whole grid for the
// single-graph kernel, a few CTAs or one CTA for a graph of a batch). With
// neighbour filtering enabled it may stop at the hand-over round, and
// continue_graph (a second launch) finishes it.
template <int BS, bool PUSH = false>
__device__ void color_graph(const Params& p, Smem<BS>& sm, Team tm) {
  Ctrl* c = p.ctrl;
  const bool lead = tm.cta == 0 && threadIdx.x == 0;
  const uint64_t t0 = gtime();
  if (lead && c->t_start == 0) c->t_start = t0;  // (a pushing kernel before this one may have set it)
  if (threadIdx.x == 0) sm.rvn_round = 0;  // nothing read ahead for this graph yet
  int t1 = p.t1;
  bool pushing = false;
  // a pushing kernel that left the colouring to this one found the largest degree already
  const bool known = !PUSH && p.pbits != nullptr && read_shared_word<BS>(&c->push_off, sm) != 0;
  if (p.t1_auto || PUSH) {  // one pass over the row offsets: the largest degree decides t1
    if (!known && !team_max_degree<BS>(p, sm, tm, PUSH && p.pbits != nullptr)) {
      if (lead) c->t_end = gtime();
      return;
    }
    const int md = ld_cg(&c->maxdeg);
    if (p.t1_auto) t1 = auto_t1(p, md);
    pushing = PUSH && p.pbits != nullptr && md > t1;  // some node keeps a bitmap
    // chosen automatically, bitmaps are used only when the rows they stand
    // for hold at least half of the entries: otherwise the pushes of every
    // committed row cost more than the rescans of the few long rows they
    // save (a graph with a few giant hubs and few rounds)
    if (pushing && p.push_auto)
      pushing = 2 * __ldcg(&c->bigsum) >= (unsigned long long)p.nnz;
  }
  if (PUSH && !pushing && !p.push_stay) {  // nothing to push: the rescanning kernel colours it
    if (lead) c->push_off = 1;
    return;
  }
  if (lead) {
    c->t1 = t1;
    c->push_on = pushing ? 1 : 0;
  }
  {
    PhaseAcc acc;
    round1<BS, PUSH>(p, sm, acc, tm, t1, pushing);
    phase_commit<BS>(p, sm, acc, 0);
  }
  bool ok = team_barrier(c, tm.cta, tm.ncta, p.timeout_ns, p.bar_extra, bar_memo<BS>(sm));
  if (PUSH && ok && pushing) {
    const int q = read_shared_word<BS>(&c->pqcnt, sm);
    if (q > 0) {
      push_phase<BS>(p, q, 0, 0, t1, tm);
      ok = team_barrier(c, tm.cta, tm.ncta, p.timeout_ns, p.bar_extra, bar_memo<BS>(sm));
    }
  }
  if (ok) {
    if (lead) trace_round1(p, t0);
    run_rounds<BS, false, PUSH>(p, sm, tm, 2);
  }
  if (lead) c->t_end = gtime();
  if (p.out_done) publish_result<BS>(p, tm);
}

// The rounds from the hand-over round r0 on, with neighbour filtering; does
// nothing when color_graph finished the colouring itself.
template <int BS>
__device__ void continue_graph(const Params& p, Smem<BS>& sm, Team tm) {
  Ctrl* c = p.ctrl;
  const int r0 = ld_cg(&c->handoff_round);
  if (r0 == 0) return;
  if (threadIdx.x == 0) sm.rvn_round = 0;
  const bool lead = tm.cta == 0 && threadIdx.x == 0;
  // list counts of every merge-state slot start at zero
  const int ng = ld_cg(&c->ngslot);
  for (int i = tm.cta * BS + threadIdx.x; i < ng; i += tm.ncta * BS) {
    p.flen[0][i] = make_int2(0, 0);
    p.flen[1][i] = make_int2(0, 0);
    p.fst[i] = 0;
    p.fdead[i] = 0;
  }
  if (team_barrier(c, tm.cta, tm.ncta, p.timeout_ns, p.bar_extra, bar_memo<BS>(sm))) run_rounds<BS, true>(p, sm, tm, r0);
  if (lead) c->t_end = gtime();
}

}  // namespace ipgc
