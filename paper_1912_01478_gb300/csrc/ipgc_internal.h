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
cudaError_t occupancy_persistent(int bs, int* blocks_per_sm);
cudaError_t launch_persistent(const Params& p, int bs, int blocks, cudaStream_t s);
cudaError_t launch_round1(const Params& p, int bs, int blocks, cudaStream_t s);
cudaError_t launch_assign(const Params& p, int bs, int blocks, int round, int mode, cudaStream_t s);
cudaError_t launch_detect(const Params& p, int bs, int blocks, int round, int mode, cudaStream_t s);
cudaError_t launch_finish(const Params& p, int last_round, cudaStream_t s);
cudaError_t launch_validate(const int32_t* rowptr, const int32_t* col, int32_t n, int64_t nnz,
                            int* d_err, int blocks, cudaStream_t s);

// Batched colouring (ipgc_batched.cu).
cudaError_t occupancy_batched(int bs, int* blocks_per_sm);
cudaError_t schedule_and_launch(const Params* h_params, int32_t G, int bs, int grid, int team_size,
                                int64_t team_min_nnz, bool cooperative, Params* d_params,
                                int32_t* d_lists, size_t lists_cap, std::vector<int32_t>& lists,
                                cudaStream_t s, int* rc);

// Context accessors (ipgc_api.cu).
int ctx_device(const ipgc_ctx* ctx);
int ctx_num_sms(const ipgc_ctx* ctx);
void ctx_note_cuda_error(ipgc_ctx* ctx, int err);
const float* ctx_policy_weights(const ipgc_ctx* ctx);
int effective_t1(const ipgc_options& o);
int effective_chunk(const ipgc_options& o);

// Release the batched workspace held for a context (ipgc_batched.cu).
void batched_release(ipgc_ctx* ctx);

}  // namespace ipgc
