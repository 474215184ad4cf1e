// Batched persistent phase kernels, 2D Euler, orders 1..7, FP64 and FP32
// predictor; host-side launch helpers.
#include "batch.cuh"
#include <algorithm>

#include "batch_launch.h"

namespace ader {

template <class Real>
static size_t batch_predict_smem() {
  size_t m = 0;
  m = std::max(m, PredictSmem<2, 1, Euler<2>, Real>::bytes());
  m = std::max(m, PredictSmem<2, 2, Euler<2>, Real>::bytes());
  m = std::max(m, PredictSmem<2, 3, Euler<2>, Real>::bytes());
  m = std::max(m, PredictSmem<2, 4, Euler<2>, Real>::bytes());
  m = std::max(m, PredictSmem<2, 5, Euler<2>, Real>::bytes());
  m = std::max(m, PredictSmem<2, 6, Euler<2>, Real>::bytes());
  m = std::max(m, PredictSmem<2, 7, Euler<2>, Real>::bytes());
  return m;
}

size_t batch_predict_smem_bytes(Precision p) {
  return p == Precision::kFP64 ? batch_predict_smem<double>() : batch_predict_smem<float>();
}

cudaError_t batch_configure(Precision p) {
  const int smem = int(batch_predict_smem_bytes(p));
  return p == Precision::kFP64
             ? cudaFuncSetAttribute(batch_predict_kernel<2, Euler<2>, double>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem)
             : cudaFuncSetAttribute(batch_predict_kernel<2, Euler<2>, float>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t batch_occupancy(Precision p, int* blocks_per_sm) {
  const size_t smem = batch_predict_smem_bytes(p);
  return p == Precision::kFP64
             ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                   blocks_per_sm, batch_predict_kernel<2, Euler<2>, double>, 256, smem)
             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                   blocks_per_sm, batch_predict_kernel<2, Euler<2>, float>, 256, smem);
}

cudaError_t batch_launch_step(Precision p, const BatchArgs& a, int grid, int slot0, cudaStream_t s) {
  const size_t smem = batch_predict_smem_bytes(p);
  if (p == Precision::kFP64)
    batch_predict_kernel<2, Euler<2>, double><<<grid, 256, smem, s>>>(a, slot0);
  else
    batch_predict_kernel<2, Euler<2>, float><<<grid, 256, smem, s>>>(a, slot0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_face_kernel<2, Euler<2>><<<grid, 256, 0, s>>>(a, slot0 + 1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_correct_kernel<2, Euler<2>, true><<<grid, 256, 0, s>>>(a, slot0 + 2);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_finalize_kernel<<<(a.ninst + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t batch_launch_rate(const BatchArgs& a, int grid, int slot, cudaStream_t s) {
  batch_correct_kernel<2, Euler<2>, false><<<grid, 256, 0, s>>>(a, slot);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_finalize_kernel<<<(a.ninst + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ader
