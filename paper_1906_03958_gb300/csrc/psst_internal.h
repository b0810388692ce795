// Host-side declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include "psst_device.cuh"

namespace psst {

// CTA-resident batched kernel (psst_cta.cu).
int cta_max_smem(int device);
cudaError_t cta_occupancy(int block, int smem, int *blocks_per_sm);
cudaError_t cta_launch(const NetView &v, long long step0, int nsteps, int grid, int block, int G,
                       int smem, cudaStream_t stream);

}  // namespace psst
