// Host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include "ipgc_device.cuh"

namespace ipgc {

constexpr int kBlock = 256;  // default threads per CTA of the colouring kernels (256 or 512)

// Single-graph colouring (ipgc_color.cu); bs = threads per CTA.
cudaError_t occupancy_persistent(int bs, int* blocks_per_sm);
cudaError_t launch_persistent(const Params& p, int bs, int blocks, cudaStream_t s);
cudaError_t launch_round1(const Params& p, int bs, int blocks, cudaStream_t s);
cudaError_t launch_assign(const Params& p, int bs, int blocks, int round, int mode, cudaStream_t s);
cudaError_t launch_detect(const Params& p, int bs, int blocks, int round, int mode, cudaStream_t s);
cudaError_t launch_finish(const Params& p, int last_round, cudaStream_t s);
cudaError_t launch_validate(const int32_t* rowptr, const int32_t* col, int32_t n, int64_t nnz,
                            int* d_err, int blocks, cudaStream_t s);

}  // namespace ipgc
