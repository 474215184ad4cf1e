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

}  // namespace ader
