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
// Work per node follows its degree (the paper's Nested Parallelism, Section
// V): a warp colours 32 low-degree nodes together, their edges spread evenly
// over the lanes; a node of higher degree is cut into work items of `chunk`
// neighbours, one warp each, dealt to the warps in a fixed stride. A node
// with several items merges their colour bitmaps (assign) or conflict flags
// (detect) in global memory, and the warp that finishes its last item
// completes it. The round loop runs inside one cooperative launch (the
// paper's Iteration Outlining, Section V).
#include <climits>
#include <type_traits>

#include "ipgc_internal.h"
#include "ipgc_phases.cuh"

namespace ipgc {

// ------------------------------------------------------- persistent kernel --

template <int BS>
__global__ void __launch_bounds__(BS, min_blocks(BS)) persistent_kernel(const __grid_constant__ Params p) {
  // after a pushing kernel (p.pbits set) only when that one left the colouring to this one
  if (p.pbits && ld_cg(&p.ctrl->push_off) == 0) return;
  __shared__ Smem<BS> sm;
  smem_clear<BS>(sm, 1);
  color_graph<BS>(p, sm, Team{(int)blockIdx.x, (int)gridDim.x});
}

// The whole colouring with forbidden-colour bitmaps (Params::pbits): a
// separate instantiation, so the kernels that rescan rows keep their
// register budget (the occupancy of each kernel sets its own grid size):
// 3 CTAs of 256 per SM (80 registers), where 4 (64 registers) spilled and
// lost 4 % on RMAT scale 22.
constexpr int push_min_blocks(int bs) { return bs >= 512 ? 2 : 3; }

template <int BS>
__global__ void __launch_bounds__(BS, push_min_blocks(BS)) persistent_push_kernel(const __grid_constant__ Params p) {
  __shared__ Smem<BS> sm;
  smem_clear<BS>(sm);
  color_graph<BS, true>(p, sm, Team{(int)blockIdx.x, (int)gridDim.x});
}

// The rounds after the hand-over to neighbour filtering (enqueued right after
// persistent_kernel; returns at once when no hand-over happened).
template <int BS>
__global__ void __launch_bounds__(BS, min_blocks(BS)) persistent_filt_kernel(const __grid_constant__ Params p) {
  __shared__ Smem<BS> sm;
  smem_clear<BS>(sm, 2);
  continue_graph<BS>(p, sm, Team{(int)blockIdx.x, (int)gridDim.x});
}

// ------------------------------------------------------ host-loop kernels --

template <int BS>
__global__ void __launch_bounds__(BS, min_blocks(BS)) round1_kernel(const __grid_constant__ Params p) {
  __shared__ Smem<BS> sm;
  const uint64_t t0 = gtime();
  if (blockIdx.x == 0 && threadIdx.x == 0) p.ctrl->t_start = t0;
  PhaseAcc acc;
  // with t1 chosen on the device, maxdeg_kernel ran before this launch
  const int t1 = p.t1_auto ? auto_t1(p, ld_cg(&p.ctrl->maxdeg)) : p.t1;
  if (blockIdx.x == 0 && threadIdx.x == 0) p.ctrl->t1 = t1;
  round1<BS>(p, sm, acc, Team{(int)blockIdx.x, (int)gridDim.x}, t1, false);
  phase_commit<BS>(p, sm, acc, 0);
  if (blockIdx.x == 0 && threadIdx.x == 0) trace_round1(p, t0);
}

template <int BS, bool FILT>
__global__ void __launch_bounds__(BS, min_blocks(BS)) assign_kernel(const __grid_constant__ Params p, int r, int mode) {
  __shared__ Smem<BS> sm;
  smem_clear<BS>(sm);
  // the previous round ended when this launch began
  if (blockIdx.x == 0 && threadIdx.x == 0 && p.trace && r - 1 <= p.trace_cap)
    p.trace[r - 2].t_detect = gtime();
  RoundView rv = read_round<BS>(p, r, sm);
  rv.mode = mode;
  const int64_t total = (int64_t)rv.nsmall + rv.nbig;
  const Team tm{(int)blockIdx.x, (int)gridDim.x};
  round_begin(p, rv, r, total, tm);
  assign_phase<BS, FILT>(p, sm, rv, tm);
}

template <int BS, bool FILT>
__global__ void __launch_bounds__(BS, min_blocks(BS)) detect_kernel(const __grid_constant__ Params p, int r, int mode) {
  __shared__ Smem<BS> sm;
  smem_clear<BS>(sm);
  if (blockIdx.x == 0 && threadIdx.x == 0 && p.trace && r <= p.trace_cap)
    p.trace[r - 1].t_assign = gtime();
  RoundView rv = read_round<BS>(p, r, sm);
  rv.mode = mode;
  PhaseAcc acc;
  detect_phase<BS, FILT>(p, sm, rv, acc, Team{(int)blockIdx.x, (int)gridDim.x});
  phase_commit<BS>(p, sm, acc, rv.par ^ 1);
}

// The largest degree into ctrl->maxdeg (host-loop driver, before round 1).
__global__ void maxdeg_kernel(Params p) {
  int m = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < p.n;
       v += (int64_t)gridDim.x * blockDim.x)
    m = max(m, ld_ro(p.rowptr + v + 1) - ld_ro(p.rowptr + v));
  m = __reduce_max_sync(FULL, m);
  if (lane_id() == 0 && m > 0) atomicMax(&p.ctrl->maxdeg, m);
}

__global__ void finish_kernel(Params p, int last_round) {
  if (p.trace && last_round >= 2 && last_round <= p.trace_cap)
    p.trace[last_round - 1].t_detect = gtime();
  p.ctrl->t_end = gtime();
}

// ------------------------------------------------------------- validation --
//
// The input check of Section V's preprocessing (no self-loop, no multi-edge)
// and of the undirected graph of Section II-A (symmetric CSR), in three
// launches on one stream. The state is ValidateState: `err` collects the
// failed checks' bits (the caller clears it), `resp` counts the entries whose
// reverse was searched and is reset by the last launch.
//
// 1. validate_rowptr_kernel: rowptr[0] == 0, rowptr[n] == nnz, rowptr
//    non-decreasing (so every later index is in bounds).
// 2. validate_entries_kernel, skipped when (1) failed: every entry (v, u) is in
//    range, not a self-loop and above its left neighbour in the row (rows
//    strictly ascending: sorted, no duplicates). For symmetry each undirected
//    pair is searched once, from the end whose (degree, ID) is larger, in the
//    other end's (no longer) row; those entries are counted in `resp`.
// 3. validate_count_kernel: with every row free of duplicates and every
//    searched reverse found, the map (v, u) -> (u, v) sends the counted
//    entries one to one into the uncounted ones, so the CSR is symmetric iff
//    also 2 resp == nnz.
//
// Entries are dealt to warps edge-balanced along the merge path of the row
// ends and the entry indices (n + nnz items), so a hub's row is spread over
// many warps and a run of short or empty rows over few. Each warp takes a
// contiguous range of tiles of 32 consecutive items, one per lane; it finds
// the row its first tile starts in with a 32-way search of rowptr, and every
// later tile starts where the previous one ended. Per tile the warp stages
// the row offsets and entries in shared memory with coalesced loads.
//
// The lookups in the other end's rows are scattered reads of a 513 MB array
// (RMAT scale 22): their DRAM sectors, not the entries, set the cost, so
// each lookup reads whole sectors and guesses the first from the ID
// (row_has): most rows are short and one sector decides.

constexpr int kValTile = 32;     // items per warp tile (one per lane)
constexpr int kValBlock = 256;
constexpr int kValMinBlocks = 8; // resident CTAs per SM (a full SM: 64 warps)

__global__ void validate_rowptr_kernel(const int32_t* __restrict__ rowptr, int32_t n, int64_t nnz,
                                       ValidateState* st) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int bad = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += stride) {
    const int32_t a = __ldg(rowptr + v);
    if (v == 0 && a != 0) bad |= 1;
    if (v == n && (int64_t)a != nnz) bad |= 1;
    if (a < 0 || (int64_t)a > nnz) bad |= 2;
    if (v < n && __ldg(rowptr + v + 1) < a) bad |= 2;
  }
  bad = __reduce_or_sync(FULL, bad);
  if (bad && lane_id() == 0) atomicOr(&st->err, bad);
}

// Rows consumed on the merge path after the first d items: the row end of
// row j comes after entry rowptr[j + 1] - 1 and before entry rowptr[j + 1],
// so it is item j + rowptr[j + 1]; count the j in [0, n) with that item < d
// (a prefix of the rows). All 32 lanes call it and get the same value.
__device__ __forceinline__ int64_t merge_rows_before(const int32_t* rowptr, int32_t n, int64_t nnz,
                                                     int64_t d) {
  const int lane = lane_id();
  int64_t lo = d - nnz > 0 ? d - nnz : 0;  // rows [0, lo) are certainly consumed
  int64_t hi = d < n ? d : n;              // rows [hi, n) certainly not
  while (hi - lo > 32) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t j = lo + lane * step;
    const bool p = j < hi && (int64_t)__ldg(rowptr + j + 1) + j < d;
    const int c = __popc(__ballot_sync(FULL, p));  // the true probes are a prefix
    if (c == 0) {
      hi = lo;
    } else {
      const int64_t nlo = lo + (int64_t)(c - 1) * step + 1;
      hi = hi < lo + (int64_t)c * step ? hi : lo + (int64_t)c * step;
      lo = nlo;
    }
  }
  const int64_t j = lo + lane;
  const bool p = j < hi && (int64_t)__ldg(rowptr + j + 1) + j < d;
  return lo + __popc(__ballot_sync(FULL, p));
}

// Is v in col[a, b) (sorted ascending, b > a)? The lookup reads whole
// 32-byte sectors (8 entries, two int4 loads of one aligned block; vec: col
// is 16-byte aligned, else plain loads of the block's valid entries) and
// places the first one by the ID: neighbour IDs are spread over [0, n), so v
// sits near a + v (b - a) / n. Each block read either settles the answer
// (v among its entries, or between two of them) or narrows the range
// [lo, hi), whose bounding values vlo < v < vhi (-1 and n outside the row)
// place the next block by interpolation; after three, halving takes over to
// bound the worst case. A block may extend past the row or the array; only
// its entries inside [lo, hi) are used (the 32-byte block of an entry lies
// in the same page as the entry).
__device__ __forceinline__ bool row_has(const int32_t* __restrict__ col, int32_t a, int32_t b,
                                        int32_t v, int32_t n, bool vec) {
  int32_t lo = a, hi = b;
  int64_t vlo = -1, vhi = n;
  for (int step = 0; lo < hi; ++step) {
    int32_t g = step < 3 ? lo + (int32_t)(((int64_t)v - vlo) * (hi - lo) / (vhi - vlo))
                         : lo + ((hi - lo) >> 1);
    g = max(lo, min(hi - 1, g));
    const int32_t blk = g & ~7;
    int32_t e[8];
    if (vec) {
      const int4 x = __ldg(reinterpret_cast<const int4*>(col + blk));
      const int4 y = __ldg(reinterpret_cast<const int4*>(col + blk + 4));
      e[0] = x.x; e[1] = x.y; e[2] = x.z; e[3] = x.w;
      e[4] = y.x; e[5] = y.y; e[6] = y.z; e[7] = y.w;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) e[q] = blk + q >= lo && blk + q < hi ? __ldg(col + blk + q) : 0;
    }
    const int32_t f = max(lo, blk), l = min(hi, blk + 8) - 1;  // the block's entries in range
    int32_t first = 0, last = 0;
    bool hit = false;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const bool in = blk + q >= f && blk + q <= l;
      hit |= in && e[q] == v;
      if (blk + q == f) first = e[q];
      if (blk + q == l) last = e[q];
    }
    if (hit) return true;
    if (v < first) {
      hi = f;
      vhi = first;
    } else if (v > last) {
      lo = l + 1;
      vlo = last;
    } else {
      return false;  // between two entries of the block
    }
  }
  return false;
}

__global__ void __launch_bounds__(kValBlock, kValMinBlocks)
validate_entries_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                        int32_t n, int64_t nnz, ValidateState* st) {
  constexpr int kWarps = kValBlock / 32;
  __shared__ int32_t s_row[kWarps][kValTile + 2];  // rowptr[i0 .. i0 + kValTile + 1]
  __shared__ int32_t s_col[kWarps][kValTile];      // col[k0 .. k0 + kValTile)
  __shared__ unsigned long long s_resp[kWarps];
  if (*reinterpret_cast<volatile int*>(&st->err) != 0) return;  // rowptr is not safe to follow
  const int warp = threadIdx.x >> 5, lane = lane_id();
  const bool cvec = ((uintptr_t)col & 15u) == 0;
  int32_t* sr = s_row[warp];
  int32_t* sc = s_col[warp];
  const int64_t total = (int64_t)n + nnz;
  const int64_t ntiles = (total + kValTile - 1) / kValTile;
  // each warp walks a contiguous range of tiles: one search for its start,
  // then every tile starts where the previous one ended
  const int64_t nw = (int64_t)gridDim.x * kWarps, gw = (int64_t)blockIdx.x * kWarps + warp;
  const int64_t t_lo = ntiles * gw / nw, t_hi = ntiles * (gw + 1) / nw;
  unsigned long long resp = 0;
  int bad = 0;
  int64_t i0 = t_lo < t_hi ? merge_rows_before(rowptr, n, nnz, t_lo * kValTile) : 0;
  for (int64_t tile = t_lo; tile < t_hi; ++tile) {
    const int64_t d0 = tile * kValTile;
    const int64_t k0 = d0 - i0;
    const int nr = (int)min((int64_t)kValTile + 2, (int64_t)n + 1 - i0);
    const int nc = (int)min((int64_t)kValTile, nnz - k0);
    __syncwarp();  // the previous tile's readers are done
    for (int j = lane; j < nr; j += 32) sr[j] = __ldg(rowptr + i0 + j);
    if (lane < nc) sc[lane] = __ldg(col + k0 + lane);
    __syncwarp();
    // this lane's item d0 + lane: its row from the staged offsets
    const int64_t td = d0 + lane;
    int64_t i = i0;
    bool entry = false;
    int32_t v = 0, u = 0, sv = 0, dv = 0;
    int64_t k = 0;
    if (td < total) {
      int lo = 0, hi = (int)min((int64_t)kValTile, (int64_t)n - i0);
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int64_t)sr[mid + 1] + i0 + mid < td)
          lo = mid + 1;
        else
          hi = mid;
      }
      i = i0 + lo;
      k = td - i;
      const int ri = lo;
      if (i < n && (int64_t)sr[ri + 1] > k) {  // entry k of row i (else the end of row i)
        entry = true;
        v = (int32_t)i;
        sv = sr[ri];
        dv = sr[ri + 1] - sv;
        u = sc[k - k0];
      }
    }
    // the next tile starts after the rows whose ends lie in this one
    i0 = i0 + __popc(__ballot_sync(FULL, td < total && !entry));
    if (entry) {
      if (u < 0 || u >= n || u == v) {
        bad |= 4;
      } else {
        if (k > sv && (k - 1 >= k0 ? sc[k - 1 - k0] : __ldg(col + k - 1)) >= u) bad |= 8;
        const int32_t su = __ldg(rowptr + u), eu = __ldg(rowptr + u + 1);
        const int32_t du = eu - su;
        if (du < dv || (du == dv && u < v)) {  // this end looks the pair up in the other's row
          ++resp;
          if (du == 0 || !row_has(col, su, eu, v, n, cvec)) bad |= 16;
        }
      }
    }
  }
  // one atomic per CTA for the count, one per warp for a failure
  bad = __reduce_or_sync(FULL, bad);
  if (bad && lane == 0) atomicOr(&st->err, bad);
  for (int o = 16; o > 0; o >>= 1) resp += __shfl_down_sync(FULL, resp, o);
  if (lane == 0) s_resp[warp] = resp;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long sum = 0;
    for (int w = 0; w < kWarps; ++w) sum += s_resp[w];
    if (sum) atomicAdd(&st->resp, sum);
  }
}

__global__ void validate_count_kernel(int64_t nnz, ValidateState* st) {
  if (st->err == 0 && 2 * (int64_t)st->resp != nnz) st->err |= 32;
  st->resp = 0;
}

// ------------------------------------------------------------ host launch --

// The phases with neighbour filtering (FILT) are separate instantiations, so
// the kernels without it keep their register budget.
template <class F>
cudaError_t with_block_filt(int bs, bool filt, F f) {
  return with_block(bs, [&](auto B) {
    return filt ? f(B, std::true_type()) : f(B, std::false_type());
  });
}

cudaError_t occupancy_persistent(int bs, int* blocks_per_sm) {
  // the smaller of the rescanning kernels' occupancies
  int a = 0, b = 0;
  cudaError_t e = with_block(bs, [&](auto B) {
    cudaError_t r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &a, persistent_kernel<decltype(B)::value>, decltype(B)::value, 0);
    if (r == cudaSuccess)
      r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
          &b, persistent_filt_kernel<decltype(B)::value>, decltype(B)::value, 0);
    return r;
  });
  *blocks_per_sm = a < b ? a : b;
  return e;
}

cudaError_t occupancy_push(int bs, int* blocks_per_sm) {
  return with_block(bs, [&](auto B) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        blocks_per_sm, persistent_push_kernel<decltype(B)::value>, decltype(B)::value, 0);
  });
}

cudaError_t launch_persistent(const Params& p, int bs, int blocks, int push_blocks,
                              cudaStream_t s) {
  return with_block(bs, [&](auto B) {
    Params pp = p;
    void* args[] = {&pp};
    cudaError_t e = cudaSuccess;
    if (p.pbits)  // pushing; it leaves graphs without a node of degree > t1 to the next kernel
      e = cudaLaunchCooperativeKernel((const void*)persistent_push_kernel<decltype(B)::value>,
                                      dim3(push_blocks), dim3(decltype(B)::value), args, 0, s);
    if (e == cudaSuccess)
      e = cudaLaunchCooperativeKernel((const void*)persistent_kernel<decltype(B)::value>,
                                      dim3(blocks), dim3(decltype(B)::value), args, 0, s);
    if (e == cudaSuccess && p.handoff_wl > 0)
      e = cudaLaunchCooperativeKernel((const void*)persistent_filt_kernel<decltype(B)::value>,
                                      dim3(blocks), dim3(decltype(B)::value), args, 0, s);
    return e;
  });
}

cudaError_t launch_round1(const Params& p, int bs, int blocks, cudaStream_t s) {
  if (p.t1_auto) {
    maxdeg_kernel<<<blocks, 256, 0, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return with_block(bs, [&](auto B) {
    round1_kernel<decltype(B)::value><<<blocks, decltype(B)::value, 0, s>>>(p);
    return cudaGetLastError();
  });
}

cudaError_t launch_assign(const Params& p, int bs, int blocks, int round, int mode, cudaStream_t s) {
  return with_block_filt(bs, p.filt_r0 > 0, [&](auto B, auto F) {
    assign_kernel<decltype(B)::value, decltype(F)::value>
        <<<blocks, decltype(B)::value, 0, s>>>(p, round, mode);
    return cudaGetLastError();
  });
}

cudaError_t launch_detect(const Params& p, int bs, int blocks, int round, int mode, cudaStream_t s) {
  return with_block_filt(bs, p.filt_r0 > 0, [&](auto B, auto F) {
    detect_kernel<decltype(B)::value, decltype(F)::value>
        <<<blocks, decltype(B)::value, 0, s>>>(p, round, mode);
    return cudaGetLastError();
  });
}

cudaError_t launch_finish(const Params& p, int last_round, cudaStream_t s) {
  finish_kernel<<<1, 1, 0, s>>>(p, last_round);
  return cudaGetLastError();
}

cudaError_t launch_validate(const int32_t* rowptr, const int32_t* col, int32_t n, int64_t nnz,
                            ValidateState* st, int blocks, cudaStream_t s) {
  if (blocks < 1) blocks = 1;
  // the row offsets: four per thread and launch at most
  const int64_t want = ((int64_t)n + 1 + 4 * kValBlock - 1) / (4 * kValBlock);
  validate_rowptr_kernel<<<(int)(want < blocks ? want : blocks), kValBlock, 0, s>>>(rowptr, n, nnz, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t tiles = ((int64_t)n + nnz + kValTile - 1) / kValTile;
  const int64_t eb = (tiles + kValBlock / 32 - 1) / (kValBlock / 32);
  // (at most kValMinBlocks CTAs per SM are resident; more only queue)
  validate_entries_kernel<<<(int)(eb < blocks ? eb : blocks), kValBlock, 0, s>>>(rowptr, col, n, nnz,
                                                                               st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  validate_count_kernel<<<1, 1, 0, s>>>(nnz, st);
  return cudaGetLastError();
}

}  // namespace ipgc
