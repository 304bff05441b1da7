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
  smem_clear<BS>(sm);
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
  smem_clear<BS>(sm);
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
                            int* d_err, int blocks, cudaStream_t s) {
  validate_kernel<<<blocks, 256, 0, s>>>(rowptr, col, n, nnz, d_err);
  return cudaGetLastError();
}

}  // namespace ipgc
