// Kernels shared by every dimension and PDE.
#include "kernels.h"

namespace ader {

// dt_next = cfl / rate with rate = max sum_d lambda_d / h_d (stored as FP64
// bits); resets the accumulator for the next reduction.
__global__ void finalize_dt_kernel(unsigned long long* rate_max, double cfl, double* dt_next,
                                   uint32_t* status) {
  const double r = __longlong_as_double(static_cast<long long>(*rate_max));
  if (!(r > 0.0) || !isfinite(r))
    atomicOr(status, kStatusNonFiniteRate);
  else
    *dt_next = cfl / r;
  *rate_max = 0ull;
}

cudaError_t launch_finalize_dt(unsigned long long* rate_max, double cfl, double* dt_next,
                               uint32_t* status, cudaStream_t s) {
  finalize_dt_kernel<<<1, 1, 0, s>>>(rate_max, cfl, dt_next, status);
  return cudaGetLastError();
}

// Halo exchange of a partitioned mesh.  Entry e of `slots` names one face
// slot, local cell * 2d + (2 dir + side); its block in the buffer is the
// slot's M NF values of Q-bar followed by its M NF values of F-bar
// (blk = M NF).  Grid-stride over the count * 2 blk buffer values.
__global__ void halo_pack_kernel(const double* faceQ, const double* faceF, const int32_t* slots,
                                 int64_t count, int blk, double* buf) {
  const int64_t total = count * 2 * blk;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t e = i / (2 * blk);
    const int r = int(i - e * 2 * blk);
    const int64_t off = int64_t(slots[e]) * blk;
    buf[i] = r < blk ? faceQ[off + r] : faceF[off + r - blk];
  }
}

__global__ void halo_unpack_kernel(double* faceQ, double* faceF, const int32_t* slots, int64_t count,
                                   int blk, const double* buf) {
  const int64_t total = count * 2 * blk;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t e = i / (2 * blk);
    const int r = int(i - e * 2 * blk);
    const int64_t off = int64_t(slots[e]) * blk;
    if (r < blk)
      faceQ[off + r] = buf[i];
    else
      faceF[off + r - blk] = buf[i];
  }
}

namespace {
unsigned halo_grid(int64_t total) {
  const int64_t b = (total + 255) / 256;
  return unsigned(b < 4096 ? (b > 0 ? b : 1) : 4096);
}
}  // namespace

cudaError_t launch_halo_pack(const double* faceQ, const double* faceF, const int32_t* slots,
                             int64_t count, int blk, double* buf, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  halo_pack_kernel<<<halo_grid(count * 2 * blk), 256, 0, s>>>(faceQ, faceF, slots, count, blk, buf);
  return cudaGetLastError();
}

cudaError_t launch_halo_unpack(double* faceQ, double* faceF, const int32_t* slots, int64_t count,
                               int blk, const double* buf, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  halo_unpack_kernel<<<halo_grid(count * 2 * blk), 256, 0, s>>>(faceQ, faceF, slots, count, blk, buf);
  return cudaGetLastError();
}

}  // namespace ader
