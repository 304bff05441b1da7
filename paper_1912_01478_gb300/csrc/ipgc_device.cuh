// Device-side building blocks of the hybrid IPGC loop: control block, kernel
// parameters, bounded grid barrier, warp-aggregated worklist pushes and the
// degree buckets. Shared by the single-graph kernels and the host-loop driver.
#pragma once

#include <cstdint>

#include "../../include/ipgc.h"

namespace ipgc {

constexpr unsigned FULL = 0xffffffffu;

// Degree buckets (the paper's Nested Parallelism, Section V): a node of
// degree <= t1 is handled by one lane of a warp that colours 32 such nodes
// together; a node of higher degree is cut into work items of `chunk`
// neighbours, one warp each, and the warp that finishes its last item
// completes it.
enum Bucket : int { B_SMALL = 0, B_BIG = 1, NB = 2 };

constexpr int kSmallWords = 8;   // mask words per low-degree node: colours 1..256
constexpr int kMaxT1 = 32 * kSmallWords - 1;  // degree <= t1 has mex <= 256
constexpr int kDefaultT1 = 64;  // when some degree exceeds kMaxT1 (t1 chosen automatically)
constexpr int kDefaultChunk = 1024;
constexpr int kMinChunk = 32;
constexpr int kMaxChunk = 4096;
constexpr int kGWords = 64;      // per-warp / per-node bitmap: colours 1..2048
constexpr int kFiltMaxC = 32 * kGWords - 2;  // neighbour filtering while maxc <= this
constexpr int kDefaultFiltDeg = 1024;
constexpr double kDefaultFiltStart = 1.0 / 32;  // hand over once |WL| <= n / 32
constexpr int kBarGroups = 16;   // grid barrier: CTAs arrive in this many groups
constexpr int kBarFlat = 1024;   // ... when the team has more CTAs than this (none on GB300)
constexpr int kShrinkMin = 8;    // a shrinking team keeps at least this many CTAs
constexpr int kShrinkMinPush = 64;  // ... with pushing
constexpr int kStageSmall = 128; // per-warp staging of low-degree pushes
constexpr int kStageItems = 32;  // per-warp staging of work-item pushes
constexpr int kPushMaxC = 32 * kGWords;  // forbidden-colour bitmaps hold colours 1..2048
constexpr int kPushChunk = 128;  // row entries per queued push item (one warp window)

// A committed row of d entries from s is pushed in items of one aligned
// window each: item j covers entries [max(s, a), min(s + d, a + kPushChunk))
// with a = (s & ~3) + j * kPushChunk (at most ceil(d / kPushChunk) + 1 items).
__device__ __forceinline__ int push_items_of(int s, int d) {
  return ((s & 3) + d + kPushChunk - 1) / kPushChunk;
}

// State of the CSR check (launch_validate): the failed checks' bits (cleared
// by the caller) and the count of entries whose reverse was searched (reset by
// the check's last launch).
struct ValidateState {
  int32_t err;
  int32_t pad;
  unsigned long long resp;
};

// Per-colouring control block in device memory. Zeroed before every launch.
struct Ctrl {
  int32_t cnt[2][4];               // worklist size per parity: [B_SMALL] nodes, [B_BIG] nodes
  int32_t icnt[2];                 // work items of the worklist's high-degree nodes, per parity
  int32_t nistat;                  // work items of every high-degree node (topology sweeps)
  int32_t ngslot;                  // merge-state slots handed out (multi-item nodes)
  unsigned long long dsum[2];      // sum of degrees of the worklist being built
  int32_t maxc;                    // largest committed colour
  int32_t status;                  // IPGC_OK or an IPGC_ERR_* code
  uint32_t bar_count;              // grid barrier arrivals
  uint32_t bar_gen;                // grid barrier generation
  int32_t rounds, rounds_topo, rounds_data, last_mode;
  unsigned long long edges;        // sum over rounds of the worklist degree sums
  unsigned long long t_start, t_end;
  unsigned long long t_prev_assign, t_prev_detect;  // previous round's phase times
  int32_t ctas_done;               // team CTAs that have published their share of the result
  int32_t maxc_start[2];           // largest committed colour at the start of a round, per parity
  int32_t ficnt[2];                // work items of the worklist's filtered nodes, per parity
  int32_t handoff_round;           // first round of neighbour filtering (0: none)
  int32_t mode_at[2];              // mode of the latest round of each parity
  int32_t rbcnt[2];                // worklist rebuild: low-degree nodes, work items
  int32_t t1;                      // the low-degree bound in use (set before round 1)
  int32_t maxdeg;                  // largest degree (when t1 is chosen from it)
  unsigned long long bigsum;       // entries in the rows of degree > t1 (pushing kernel)
  int32_t pqcnt;                   // push items queued by the current conflict step
  int32_t pwcnt;                   // winners of the current conflict step still to push
  int32_t rqcnt;                   // list rewrite units queued by the current conflict step
  int32_t push_off;                // the pushing kernel found no node of degree > t1 and left
                                   // the colouring to the rescanning kernel launched after it
  int32_t late_at[2];              // pushing: the latest round of each parity ran late (no push
                                   // phase); parity slots, like maxc_start: CTA 0 writes round
                                   // r's while slower CTAs may still read round r - 1's
  int32_t push_on;                 // forbidden-colour bitmaps in use (some degree > t1)
  // arrival counters of the grid barrier's groups, one 32-byte sector each
  uint32_t bar_grp[kBarGroups][8];
  // arrival counts of the counting barrier (team_barrier with a memo), one
  // per single-graph kernel of a colouring (pushing, rescanning, filtering),
  // each starting from zero with the control block; bit 63: error
  unsigned long long bar_arrive[3];
};

struct Params {
  const int32_t* __restrict__ rowptr;
  const int32_t* __restrict__ col;
  int32_t n;
  int64_t nnz;
  int32_t* color;    // committed colours (the caller's output buffer)
  int32_t* tent;     // tentative colours
  int32_t* wl[2];    // worklist of low-degree nodes, per parity
  // high-degree nodes are held as work items {v, chunk index, gslot, #chunks}
  // where gslot indexes the merge state of a node with more than one chunk
  // (-1 otherwise)
  int4* items[2];     // the worklist's items, per parity
  int4* istat;        // items of every high-degree node (topology sweeps)
  uint32_t* gbits;    // [gslot][kGWords] colours seen by finished chunks (kept zero)
  int32_t* done_a;    // [gslot] chunks finished in the assignment step (kept zero)
  int32_t* done_d;    // [gslot] chunks finished in the conflict step (kept zero)
  int32_t* flag;      // [gslot] a chunk found a conflict (kept zero)
  Ctrl* ctrl;
  ipgc_trace_rec* trace;
  int32_t* fin;       // optional: round in which each node's colour was committed
  int32_t trace_cap;
  int32_t t1, chunk;
  int64_t H;          // topology-driven iff |WL| > H
  int32_t policy;     // IPGC_MODE_*
  int32_t max_rounds;
  uint64_t timeout_ns;
  const float* mlp;   // learned policy weights (device) or nullptr
  uint32_t bar_extra; // tests only: phantom CTAs every grid barrier waits for
  int32_t col_vec;    // col is 16-byte aligned: int4 loads and bulk L2 prefetches allowed
  float mlp_margin;   // learned policy: threshold rule when |p - 0.5| < margin
  // Neighbour filtering (alist[0] == nullptr: off). From the hand-over round
  // r0 on, a node of degree > filt_deg (>= chunk, so it has a merge-state
  // slot) reads a list that holds every neighbour still active (round r0: the
  // row itself), kept in alist[b] inside the node's own row range
  // [rowptr[v], rowptr[v + 1]): lower IDs from the front, higher IDs from the
  // back, their counts in flen[b][gslot]; b = fst[gslot] & 1, and bit 1 of
  // fst asks for a rewrite without finalised entries in the next round
  // (fdead counts the finalised entries the last reading found). Colours of
  // its finalised neighbours accumulate in gbits[gslot] across rounds. Used
  // in round r iff every colour committed before round r - 1 is <=
  // kFiltMaxC, so the bitmap holds every colour.
  int32_t* alist[2];
  int2* flen[2];
  int32_t* fst;
  int32_t* fdead;
  int4* fitems[2];    // work items of filtered nodes, per parity (as items[])
  int32_t filt_deg;
  int32_t filt_r0;    // host-loop driver: the hand-over round once reached (0: not yet)
  int32_t shrink;     // the team may drop CTAs in small data-driven rounds (single graph)
  int32_t wl_rebuild; // topology-driven rounds keep no worklist; it is rebuilt on the way back
  int32_t t1_auto;    // choose t1 on the device: the largest degree if <= kMaxT1, else t1
  int32_t push_auto;  // pushing kernel: colour with bitmaps only when the rows of degree > t1
                      // hold at least half of the entries (else leave it to rescanning)
  int32_t push_stay;  // pushing kernel: a graph it would leave to the rescanning kernel is
                      // coloured here by rescanning (the server runs one kernel per launch)
  int64_t handoff_wl; // hand over when |WL| <= handoff_wl (0: never)
  // Forbidden-colour bitmaps (pbits == nullptr: off). A node v of degree
  // d > t1 keeps the colours of its finalised neighbours as a bitmap of
  // ceil(min(d, kPushMaxC) / 32) words at pbits[rowptr[v]] (inside its own
  // row range of an nnz-word buffer; bit c - 1 = colour c): every node ORs
  // its colour into the bitmaps of its neighbours when it is committed, so
  // the assignment step of v reads the bitmap instead of the row. The
  // conflict step lists its winners (pw: nodes of degree <= t1; pq: the
  // one-window items {row start, degree, colour, window} of the rows of
  // the others), and a push phase of the whole team follows it. A node with
  // several items also keeps the list of its lower-ID neighbours that are
  // still active (alist/flen/fst/fdead as for neighbour filtering, lower
  // part only; built in round 2, rewritten without finalised entries by the
  // assignment step once a quarter of what the conflict step read was
  // finalised), which its conflict step reads instead of the row. Used in
  // round r while every colour committed before round r - 1 is
  // <= kPushMaxC - 2, so every colour of round r fits the bitmaps.
  uint32_t* pbits;
  int4* pq;
  int32_t* pw;
  // With pushing, optional: a loser of a conflict step that is not late and
  // whose list is due for a rewrite queues it here, in one-window units
  // {row start, slot, window, list buffer | length << 1}, and the push phase
  // that follows rewrites it, spread over the whole team (nullptr: the node's
  // own warps rewrite it in the next assignment step).
  int4* rq;
  // With pushing, optional: per node {row start, degree} while the node keeps
  // a bitmap and is active, {row start, 0} otherwise (written by round 1, the
  // degree cleared when the node is committed), so a push after round 1
  // learns whether and where to OR from one 8-byte gather instead of the row
  // offsets and the colour. nullptr: pushes read rowptr and color.
  int2* pinfo;
  // Optional result publication into host-mapped pinned memory (nullptr:
  // none). When a graph is done its team copies the colours to out_colors
  // and the control block to out_ctrl, then sets *out_done = 1, so the host
  // sees each graph complete while the rest of its launch still runs.
  int32_t* out_colors;
  Ctrl* out_ctrl;
  int32_t* out_done;
};

// Neighbour filtering takes over at the first round r >= 3 whose worklist
// has at most handoff_wl nodes of mean degree > filt_deg (by then most of
// their neighbours are finalised), while every colour fits the bitmap.
// Evaluated by the kernel and by the host-loop driver alike.
__host__ __device__ inline bool handoff_now(const Params& p, int r, int64_t total,
                                            unsigned long long dsum, int maxc) {
  return p.handoff_wl > 0 && r >= 3 && total <= p.handoff_wl &&
         dsum > (unsigned long long)total * (unsigned long long)p.filt_deg && maxc <= kFiltMaxC;
}

// ------------------------------------------------------- learned policy --

constexpr int kMlpIn = IPGC_MLP_INPUTS;
constexpr int kMlpH = IPGC_MLP_HIDDEN;
constexpr int kMlpParams = kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;
static_assert(kMlpParams == IPGC_MLP_PARAMS, "parameter count");
// offsets of W1[16][8], b1, W2[16][16], b2, w3, b3
constexpr int kW1 = 0, kB1 = kW1 + kMlpH * kMlpIn, kW2 = kB1 + kMlpH, kB2 = kW2 + kMlpH * kMlpH,
              kW3 = kB2 + kMlpH, kB3 = kW3 + kMlpH;

// The 8 inputs of the mode decision for a round with worklist size wl (of
// which wl_small low-degree nodes) and worklist degree sum deg_sum; all of
// them are known at the start of the round and none depends on the mode.
__host__ __device__ inline void policy_features(int64_t n, int64_t nnz, int round, int64_t wl,
                                                int64_t wl_small, int64_t deg_sum, int maxc,
                                                float f[kMlpIn]) {
  const float fn = (float)(n > 0 ? n : 1), fe = (float)(nnz > 0 ? nnz : 1);
  const float fwl = (float)(wl > 0 ? wl : 1);
  f[0] = (float)wl / fn;
  f[1] = (float)deg_sum / fe;
  f[2] = (float)wl_small / fwl;
  f[3] = log2f(fn + 1.0f) / 32.0f;
  f[4] = log2f((float)nnz / fn + 1.0f) / 8.0f;
  f[5] = log2f((float)(round > 0 ? round : 1)) / 16.0f;
  f[6] = log2f((float)deg_sum / fwl + 1.0f) / 16.0f;
  f[7] = (float)maxc / ((float)maxc + 64.0f);
}

// Network logit for inputs f, by one warp (all 32 lanes call; lanes j and
// j + 16 compute hidden unit j); every lane returns the same value, summed
// in a fixed order.
__device__ __forceinline__ float mlp_logit_warp(const float* __restrict__ w, const float f[kMlpIn]) {
  const int j = threadIdx.x & 15;
  float a = w[kB1 + j];
#pragma unroll
  for (int k = 0; k < kMlpIn; ++k) a += w[kW1 + j * kMlpIn + k] * f[k];
  const float h1 = tanhf(a);
  float a2 = w[kB2 + j];
#pragma unroll
  for (int k = 0; k < kMlpH; ++k) a2 += w[kW2 + j * kMlpH + k] * __shfl_sync(FULL, h1, k);
  const float h2 = tanhf(a2);
  float z = (threadIdx.x & 31) < 16 ? w[kW3 + j] * h2 : 0.0f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(FULL, z, o);
  return z + w[kB3];
}

// The same on the host (host-loop driver).
inline float mlp_logit_host(const float* w, const float f[kMlpIn]) {
  float h1[kMlpH], z = w[kB3];
  for (int j = 0; j < kMlpH; ++j) {
    float a = w[kB1 + j];
    for (int k = 0; k < kMlpIn; ++k) a += w[kW1 + j * kMlpIn + k] * f[k];
    h1[j] = tanhf(a);
  }
  for (int j = 0; j < kMlpH; ++j) {
    float a = w[kB2 + j];
    for (int k = 0; k < kMlpH; ++k) a += w[kW2 + j * kMlpH + k] * h1[k];
    z += w[kW3 + j] * tanhf(a);
  }
  return z;
}

__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Loads of data written by other CTAs during this launch bypass L1.
__device__ __forceinline__ int32_t ld_cg(const int32_t* p) { return __ldcg(p); }

// The same for the colour arrays gathered at random (committed and tentative
// colours, 4n bytes each): L1 bypassed, and the L2 line marked evict-last so
// the streamed neighbour lists do not push the colours out of L2.
__device__ __forceinline__ uint64_t l2_keep_policy() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ int32_t ld_keep(const int32_t* p, uint64_t pol) {
  int32_t v;
  asm volatile("ld.global.cg.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ int4 ld_cg4(const int4* p) { return __ldcg(p); }
__device__ __forceinline__ int64_t ld_cg_i64(const int64_t* p) {
  return (int64_t)__ldcg(reinterpret_cast<const long long*>(p));
}
// Loads of the read-only graph.
__device__ __forceinline__ int32_t ld_ro(const int32_t* p) { return __ldg(p); }

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ int bucket_of(int d, int t1) { return d <= t1 ? B_SMALL : B_BIG; }

// The CTAs that colour one graph together: this CTA's rank and their number.
struct Team {
  int cta;
  int ncta;
};

// Device-scope atomics and loads with the ordering a barrier needs (PTX
// memory model): an arrival releases the CTA's writes (ordered before it by
// __syncthreads) and acquires those of the CTAs that arrived before it; a
// waiter acquires them all through the generation word.
__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t* a, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(a), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* a) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* a, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(a), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* a) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* a) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}

// The top bit of the barrier's generation word: an error has been recorded,
// so every CTA leaves its barrier (the count lives in the low 31 bits).
constexpr uint32_t kBarErr = 0x80000000u;

// What a CTA remembers of its team's barrier (kept in shared memory): the
// generation the last barrier it passed on control block `ctrl` released
// (ctrl == nullptr: nothing yet).
struct BarMemo {
  const Ctrl* ctrl;
  int idx;                     // the kernel's arrival counter (Ctrl::bar_arrive)
  unsigned long long target;   // arrivals at which that barrier completed
};

// Records an error of the colouring (the first one wins) and raises the
// barrier's error bit, so that CTAs waiting in a barrier leave it at once.
__device__ __forceinline__ void record_error(Ctrl* c, int code) {
  atomicCAS(&c->status, 0, code);
  atomicOr(&c->bar_gen, kBarErr);
#pragma unroll
  for (int k = 0; k < 3; ++k) atomicOr(&c->bar_arrive[k], 1ull << 63);
}

// Barrier of a team of co-resident CTAs (a cooperative launch guarantees
// residency), bounded by timeout_ns: a CTA that waits longer records
// IPGC_ERR_TIMEOUT and leaves the barrier. Returns false when the team must
// stop (timeout here or an error recorded elsewhere, seen as the error bit of
// the generation word). The counters live in the graph's control block. A
// team of more than kBarFlat CTAs arrives in kBarGroups groups; every team
// on a GB300 (at most 608 CTAs) arrives on one counter: the arrivals are
// spread out in time, and the group level's extra dependent atomic cost more
// than the serialised arrivals (RMAT scale 22 1.8 % and kron's stand-in 3.3 %
// faster flat than in 16 groups, same GPU). `extra` phantom CTAs never arrive
// (tests).
//
// Thread 0 reads the generation before the CTA's warps meet (the barrier
// cannot complete before this CTA arrives, and this thread has seen the
// previous one complete, so the value is the current generation); arrivals
// are acquire-release atomics and the last arrival releases the next
// generation with an atomic add, which waiters acquire: no separate fences
// and no further read after the wait.
//
// With a memo (the single-graph kernels) the barrier counts instead: each
// CTA adds its arrival to the kernel's 64-bit arrival count with a release
// reduction (no reply to wait for) and waits, acquiring, until the count
// reaches the barrier's target, which the CTA keeps in its memo: the previous
// barrier's target plus the team's size (the count starts at zero with the
// control block, every barrier of the team adds exactly its size, and a team
// that shrinks does so between barriers, the same for every CTA). No CTA
// waits on a reply to its arrival and no generation is released: one
// dependent round trip fewer than the generation barrier. An error sets bit
// 63 of the count, and a waiter that sees it leaves with false.
__device__ __forceinline__ bool team_barrier(Ctrl* c, int cta, int ncta, uint64_t timeout_ns,
                                             uint32_t extra = 0, BarMemo* memo = nullptr) {
  __shared__ int s_ok;
  if (memo) {  // the counting barrier
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long* w = &c->bar_arrive[memo->idx];
      const unsigned long long target =
          (memo->ctrl == c ? memo->target : 0ull) + (unsigned long long)ncta + extra;
      red_release_add_u64(w, 1ull);
      bool ok = true;
      const uint64_t t0 = gtime();
      while (true) {
        const unsigned long long now = ld_acquire_u64(w);
        if (now >> 63) {
          ok = false;
          break;
        }
        if (now >= target) break;
        if (gtime() - t0 > timeout_ns) {
          record_error(c, IPGC_ERR_TIMEOUT);
          ok = false;
          break;
        }
        __nanosleep(32);
      }
      memo->ctrl = ok ? c : nullptr;  // a failed barrier is the team's last
      memo->target = target;
      s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
  }
  uint32_t gen = 0;
  if (threadIdx.x == 0) gen = ld_relaxed_u32(&c->bar_gen);
  __syncthreads();
  if (threadIdx.x == 0) {
    bool ok = (gen & kBarErr) == 0;
    if (ok) {
      bool last;
      if (ncta > kBarFlat) {
        // CTAs arrive on kBarGroups counters (CTA i in group i % kBarGroups);
        // the last of a group resets its counter and arrives on the top one
        const int g = cta % kBarGroups;
        const uint32_t gsz = (uint32_t)(ncta / kBarGroups + (g < ncta % kBarGroups ? 1 : 0));
        last = false;
        if (atom_add_acq_rel(&c->bar_grp[g][0], 1u) == gsz - 1) {
          c->bar_grp[g][0] = 0;  // ordered before the arrival below
          last = atom_add_acq_rel(&c->bar_count, 1u) == (uint32_t)kBarGroups + extra - 1;
        }
      } else {
        last = atom_add_acq_rel(&c->bar_count, 1u) == (uint32_t)ncta + extra - 1;
      }
      if (last) {
        c->bar_count = 0;  // ordered before the release below
        ok = (atom_add_acq_rel(&c->bar_gen, 1u) & kBarErr) == 0;
      } else {
        const uint64_t t0 = gtime();
        while (true) {
          const uint32_t now = ld_acquire_u32(&c->bar_gen);
          if (now != gen) {
            ok = (now & kBarErr) == 0;
            break;
          }
          if (gtime() - t0 > timeout_ns) {
            record_error(c, IPGC_ERR_TIMEOUT);
            ok = false;
            break;
          }
          __nanosleep(64);
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Warp-aggregated append (the paper's Cooperative Conversion, Section V): one
// atomicAdd per warp reserves the slots of every lane with pred set. All 32
// lanes must call it.
__device__ __forceinline__ void warp_push(bool pred, int32_t v, int32_t* list, int32_t* counter) {
  const unsigned m = __ballot_sync(FULL, pred);
  if (m == 0) return;
  const int lane = lane_id();
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(m));
  base = __shfl_sync(FULL, base, leader);
  if (pred) list[base + __popc(m & ((1u << lane) - 1u))] = v;
}

// The same, staged: lanes append to a per-warp buffer in shared memory and
// the warp reserves space in the global list once per buffer-full (and at
// the end of the phase), so one atomic serves up to `cap` pushes.
struct WarpStage {
  int32_t* buf;  // this warp's shared buffer
  int fill;      // entries in buf (warp-uniform)
};

__device__ __forceinline__ void stage_flush(WarpStage& st, int32_t* list, int32_t* counter) {
  if (st.fill == 0) return;
  __syncwarp();
  const int lane = lane_id();
  int base = 0;
  if (lane == 0) base = atomicAdd(counter, st.fill);
  base = __shfl_sync(FULL, base, 0);
  for (int i = lane; i < st.fill; i += 32) list[base + i] = st.buf[i];
  __syncwarp();
  st.fill = 0;
}

__device__ __forceinline__ void stage_push(WarpStage& st, int cap, bool pred, int32_t v,
                                           int32_t* list, int32_t* counter) {
  const unsigned m = __ballot_sync(FULL, pred);
  if (m == 0) return;
  const int lane = lane_id();
  if (pred) st.buf[st.fill + __popc(m & ((1u << lane) - 1u))] = v;
  st.fill += __popc(m);
  if (st.fill > cap - 32) stage_flush(st, list, counter);
}

// Staged append of work items: every lane may add the `cnt` items
// {v, j, gslot, cnt}, j < cnt, of one node (cnt = 0: none); one atomic per
// stage-full. All 32 lanes must call it.
struct ItemStage {
  int4* buf;  // this warp's shared buffer of kStageItems entries
  int fill;   // entries in buf (warp-uniform)
};

__device__ __forceinline__ void items_flush(ItemStage& st, int4* list, int32_t* counter) {
  if (st.fill == 0) return;
  __syncwarp();
  const int lane = lane_id();
  int base = 0;
  if (lane == 0) base = atomicAdd(counter, st.fill);
  base = __shfl_sync(FULL, base, 0);
  for (int i = lane; i < st.fill; i += 32) list[base + i] = st.buf[i];
  __syncwarp();
  st.fill = 0;
}

__device__ __forceinline__ void items_push(ItemStage& st, int v, int cnt, int gslot, int4* list,
                                           int32_t* counter) {
  const int lane = lane_id();
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  const int tot = __shfl_sync(FULL, incl, 31);
  if (tot == 0) return;
  const int excl = incl - cnt;
  if (tot > kStageItems) {  // more than a stage: reserve room directly
    int base = 0;
    if (lane == 0) base = atomicAdd(counter, tot);
    base = __shfl_sync(FULL, base, 0);
    for (int j = 0; j < cnt; ++j) list[base + excl + j] = make_int4(v, j, gslot, cnt);
    return;
  }
  if (st.fill + tot > kStageItems) items_flush(st, list, counter);
  for (int j = 0; j < cnt; ++j) st.buf[st.fill + excl + j] = make_int4(v, j, gslot, cnt);
  __syncwarp();
  st.fill += tot;
}

// items_push without staging: one warp-aggregated reservation per call.
__device__ __forceinline__ void items_push_direct(int v, int cnt, int gslot, int4* list,
                                                  int32_t* counter) {
  const int lane = lane_id();
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  const int tot = __shfl_sync(FULL, incl, 31);
  if (tot == 0) return;
  int base = 0;
  if (lane == 0) base = atomicAdd(counter, tot);
  base = __shfl_sync(FULL, base, 0) + incl - cnt;
  for (int j = 0; j < cnt; ++j) list[base + j] = make_int4(v, j, gslot, cnt);
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}

}  // namespace ipgc
