// Host launch helpers of the batched phase kernels (k_batch.cu).
#pragma once
#include "batch_types.h"
#include "kernels.h"

namespace ader {

size_t batch_predict_smem_bytes(Precision p);
cudaError_t batch_configure(Precision p);
cudaError_t batch_occupancy(Precision p, int* blocks_per_sm);
// One step: predictor, Riemann, corrector (work-queue slots slot0..slot0+2),
// then the per-instance dt update.
cudaError_t batch_launch_step(Precision p, const BatchArgs& a, int grid, int slot0, cudaStream_t s);
// Rate of the current state and dt (work-queue slot `slot`).
cudaError_t batch_launch_rate(const BatchArgs& a, int grid, int slot, cudaStream_t s);

}  // namespace ader
