// Adjoint step kernels for linear acoustics, 2D and 3D, orders 1..7.
#include "adjoint.cuh"
#include "instantiate.cuh"

namespace ader {

cudaError_t launch_adjoint(int dim, int order, const AdjointArgs& a, cudaStream_t s) {
  if (dim == 2)
    return with_order(order, [&](auto N) { return launch_adjoint_t<2, N.value, 3>(a, s); });
  return with_order(order, [&](auto N) { return launch_adjoint_t<3, N.value, 4>(a, s); });
}

}  // namespace ader

namespace ader {

// out[p] = sum_node w[p][node] field[cell_p][var][node]; one CTA per point.
__global__ void sample_kernel(const double* field, int M, int NS, int var, int npts,
                              const int32_t* cells, const double* weights, double* out) {
  const int p = blockIdx.x;
  if (p >= npts) return;
  const int64_t c = cells[p];
  double s = 0.0;
  for (int i = threadIdx.x; i < NS; i += blockDim.x)
    s = fma(weights[int64_t(p) * NS + i], field[(c * M + var) * NS + i], s);
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x + 31) / 32; ++w) t += red[w];
    out[p] = t;
  }
}

// field[cell_p][var][node] += w[p][node] values[p], points in order (one CTA,
// so points sharing a cell accumulate deterministically).
__global__ void sample_adjoint_kernel(double* field, int M, int NS, int var, int npts,
                                      const int32_t* cells, const double* weights,
                                      const double* values) {
  for (int p = 0; p < npts; ++p) {
    const int64_t c = cells[p];
    const double v = values[p];
    for (int i = threadIdx.x; i < NS; i += blockDim.x)
      field[(c * M + var) * NS + i] = fma(weights[int64_t(p) * NS + i], v, field[(c * M + var) * NS + i]);
    __syncthreads();
  }
}

cudaError_t launch_sample(const double* field, int M, int NS, int var, int npts,
                          const int32_t* cells, const double* weights, double* out, cudaStream_t s) {
  if (npts == 0) return cudaSuccess;
  sample_kernel<<<npts, 128, 0, s>>>(field, M, NS, var, npts, cells, weights, out);
  return cudaGetLastError();
}

cudaError_t launch_sample_adjoint(double* field, int M, int NS, int var, int npts,
                                  const int32_t* cells, const double* weights, const double* values,
                                  cudaStream_t s) {
  if (npts == 0) return cudaSuccess;
  sample_adjoint_kernel<<<1, 256, 0, s>>>(field, M, NS, var, npts, cells, weights, values);
  return cudaGetLastError();
}

}  // namespace ader
