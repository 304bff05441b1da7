// Host-side declarations shared by the library's translation units (not
// exported: the library is built with hidden visibility).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <vector>

#include "ipgc_device.cuh"

namespace ipgc {

constexpr int kBlock = 256;  // default threads per CTA of the colouring kernels (256 or 512)

// Calls f(std::integral_constant<int, bs>) for a supported block size.
template <class F>
cudaError_t with_block(int bs, F f) {
  switch (bs) {
    case 256: return f(std::integral_constant<int, 256>());
    case 512: return f(std::integral_constant<int, 512>());
    default: return cudaErrorInvalidValue;
  }
}

// Single-graph colouring (ipgc_color.cu); bs = threads per CTA.
cudaError_t occupancy_persistent(int bs, int* blocks_per_sm);  // the rescanning kernels
cudaError_t occupancy_push(int bs, int* blocks_per_sm);        // the pushing kernel
// The pushing kernel (when p.pbits) on push_blocks CTAs, then the rescanning
// kernels on `blocks` CTAs (they return at once when it coloured the graph).
cudaError_t launch_persistent(const Params& p, int bs, int blocks, int push_blocks,
                              cudaStream_t s);
cudaError_t launch_round1(const Params& p, int bs, int blocks, cudaStream_t s);
cudaError_t launch_assign(const Params& p, int bs, int blocks, int round, int mode, cudaStream_t s);
cudaError_t launch_detect(const Params& p, int bs, int blocks, int round, int mode, cudaStream_t s);
cudaError_t launch_finish(const Params& p, int last_round, cudaStream_t s);
cudaError_t launch_validate(const int32_t* rowptr, const int32_t* col, int32_t n, int64_t nnz,
                            ValidateState* st, int blocks, cudaStream_t s);

// Batched colouring (ipgc_batched.cu).
cudaError_t occupancy_batched(int bs, int* blocks_per_sm, bool push = false);
// Schedule of a batch on `grid` CTAs (int32 lists, see build_schedule), then
// its upload and launch; lists_cap bounds the device list buffer (rc =
// IPGC_ERR_UNSUPPORTED when the schedule does not fit).
void build_schedule(const Params* h_params, int32_t G, int grid, int max_team,
                    int64_t nnz_per_cta, std::vector<int32_t>& lists, int32_t* njobs_out,
                    int32_t* nsolo_out, int32_t* seq_out);
// Uploads the parameters (unless h_params is null: already there) and the
// lists, then launches the batched kernel: the pushing one when `push`.
cudaError_t launch_schedule(const Params* h_params, int32_t G, int bs, int grid, bool cooperative,
                            const std::vector<int32_t>& lists, int32_t njobs, int32_t nsolo,
                            Params* d_params, int32_t* d_lists, cudaStream_t s, bool push = false);
// With `push` the pushing kernel runs the schedule (graphs it would leave to
// the rescanning kernel need Params::push_stay).
cudaError_t schedule_and_launch(const Params* h_params, int32_t G, int bs, int grid, int max_team,
                                int64_t nnz_per_cta, bool cooperative, Params* d_params,
                                int32_t* d_lists, size_t lists_cap, std::vector<int32_t>& lists,
                                cudaStream_t s, int* rc, bool push = false);
// Upper bound on the list length build_schedule makes for G graphs with
// teams of at most kmax CTAs each on `grid` CTAs.
inline size_t schedule_lists_bound(int32_t G, int grid, int kmax) {
  return 4 * (size_t)G * (size_t)kmax + (size_t)grid + 1 + (size_t)G + 1;
}

// Context accessors (ipgc_api.cu).
int ctx_device(const ipgc_ctx* ctx);
int ctx_num_sms(const ipgc_ctx* ctx);
void ctx_note_cuda_error(ipgc_ctx* ctx, int err);
const float* ctx_policy_weights(const ipgc_ctx* ctx);
Ctrl* ctx_ctrl_dev(ipgc_ctx* ctx);
Ctrl* ctx_ctrl_host(ipgc_ctx* ctx);  // pinned
// The context's auxiliary device buffer of at least `bytes` (grown on demand);
// nullptr with *rc = IPGC_ERR_OOM / IPGC_ERR_CUDA on failure.
void* ctx_aux(ipgc_ctx* ctx, size_t bytes, int* rc);
int effective_t1(const ipgc_options& o);
int effective_chunk(const ipgc_options& o);

// Release the batched workspace held for a context (ipgc_batched.cu).
void batched_release(ipgc_ctx* ctx);

}  // namespace ipgc
