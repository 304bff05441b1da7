// Device-side building blocks of the hybrid IPGC loop: control block, kernel
// parameters, bounded grid barrier, warp-aggregated worklist push and the
// degree buckets. Shared by the single-graph colouring kernel and the
// host-loop driver.
#pragma once

#include <cstdint>

#include "../../include/ipgc.h"

namespace ipgc {

constexpr unsigned FULL = 0xffffffffu;

// Degree buckets (the paper's Nested Parallelism, Section V): a node of
// degree <= t1 is handled by one lane of a warp that colours 32 such nodes
// together, t1 < degree <= t2 by one warp, above t2 by one CTA.
enum Bucket : int { B_SMALL = 0, B_MID = 1, B_BIG = 2, NB = 3 };

constexpr int kMaxT1 = 63;     // 64-bit lane mask covers colours 1..64
constexpr int kMaxT2 = 1023;   // per-warp bitmap covers colours 1..1024
constexpr int kDefaultT1 = 24;
constexpr int kDefaultT2 = 1023;
constexpr int kBigWords = 2048;  // CTA bitmap window: 65536 colours

// Per-colouring control block in device memory. Zeroed before every launch.
struct Ctrl {
  int32_t cnt[2][4];               // worklist size per parity and bucket
  int32_t nstat[4];                // static lists of mid / big nodes (topology sweeps)
  uint32_t grab[2][4];             // dynamic work counters per parity
  unsigned long long dsum[2];      // sum of degrees of the worklist being built
  int32_t maxc;                    // largest committed colour
  int32_t status;                  // IPGC_OK or an IPGC_ERR_* code
  uint32_t bar_count;              // grid barrier arrivals
  uint32_t bar_gen;                // grid barrier generation
  int32_t rounds, rounds_topo, rounds_data, last_mode;
  unsigned long long edges;        // sum over rounds of the worklist degree sums
  unsigned long long t_start, t_end;
  unsigned long long t_prev_assign, t_prev_detect;  // previous round's phase times
  int32_t pad[8];
};

// grab[] slots
enum { G_ASSIGN_BIG = 0, G_DETECT_BIG = 1 };

struct Params {
  const int32_t* __restrict__ rowptr;
  const int32_t* __restrict__ col;
  int32_t n;
  int64_t nnz;
  int32_t* color;    // committed colours (the caller's output buffer)
  int32_t* tent;     // tentative colours
  int32_t* wl[2][NB];
  int32_t* stat[NB];  // [B_MID], [B_BIG]: every node of that bucket
  Ctrl* ctrl;
  ipgc_trace_rec* trace;
  int32_t* fin;       // optional: round in which each node's colour was committed
  int32_t trace_cap;
  int32_t t1, t2;
  int64_t H;          // topology-driven iff |WL| > H
  int32_t policy;     // IPGC_MODE_*
  int32_t max_rounds;
  uint64_t timeout_ns;
  const float* mlp;   // learned policy weights (device) or nullptr
  uint32_t bar_extra; // tests only: phantom CTAs every grid barrier waits for
};

__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Loads of data written by other CTAs during this launch bypass L1.
__device__ __forceinline__ int32_t ld_cg(const int32_t* p) { return __ldcg(p); }
// Loads of the read-only graph.
__device__ __forceinline__ int32_t ld_ro(const int32_t* p) { return __ldg(p); }

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ int bucket_of(int d, int t1, int t2) {
  return d <= t1 ? B_SMALL : (d <= t2 ? B_MID : B_BIG);
}

// Grid-wide barrier for a cooperative launch, bounded by timeout_ns: a CTA
// that waits longer records IPGC_ERR_TIMEOUT and leaves the barrier. Returns
// false when the launch must stop (timeout here or an error elsewhere).
__device__ __forceinline__ bool grid_barrier(Ctrl* c, uint64_t timeout_ns, uint32_t extra = 0) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t* genp = &c->bar_gen;
    const uint32_t gen = *genp;
    __threadfence();
    const uint32_t arrived = atomicAdd(&c->bar_count, 1u);
    if (arrived == gridDim.x + extra - 1) {
      c->bar_count = 0;
      __threadfence();
      atomicAdd(&c->bar_gen, 1u);
    } else {
      const uint64_t t0 = gtime();
      while (*genp == gen) {
        if (gtime() - t0 > timeout_ns) {
          atomicCAS(&c->status, 0, IPGC_ERR_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = (*(volatile int32_t*)&c->status) == 0;
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

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
  return x;
}

__device__ __forceinline__ int warp_max(int x) { return __reduce_max_sync(FULL, x); }

}  // namespace ipgc
