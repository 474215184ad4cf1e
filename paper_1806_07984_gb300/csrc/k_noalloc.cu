// Allocation-free time-step entry point (ader_compute_dt_static).
//
// Some callers cannot allocate device memory: code that runs inside a
// memory pool or arena it does not own (a host framework that forbids
// cudaMalloc after start-up, or that must not fragment its pool), or code on a
// path that must never fail for lack of memory.  For them this file computes
// the global time step dt = cfl / max_cells max_nodes sum_d lambda_d(u) / h_d
// without any allocation: the per-CTA partial maxima live in a file-scope
// device array of fixed size, reserved when the library is loaded and kept by
// every GPU that loads it until the process exits.
#include <mutex>

#include "../../include/ader.h"
#include "instantiate.cuh"

namespace ader {
namespace {

constexpr int64_t kStaticPartials = ADER_DT_STATIC_MAX_CELLS;

// One FP64 partial maximum per CTA of the first pass.  Every call overwrites
// the slots it uses and reads only those, so nothing has to be cleared.
static __device__ __align__(256) double g_dt_partials[kStaticPartials];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_partials_addr[kMaxDevices] = {nullptr};

// Maximum that propagates NaN (a NaN rate marks a non-physical state).
__device__ __forceinline__ double nan_max(double a, double b) {
  return (a != a || b != b) ? __longlong_as_double(0x7ff8000000000000ll) : fmax(a, b);
}

// Butterfly maximum over a full warp (every CTA of this file is whole warps).
__device__ __forceinline__ double warp_nan_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nan_max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// First pass: per node sum_d lambda_d / h_d, CTA maximum into partials[cta].
// inv_h per level and direction, passed by value.
struct InvH {
  double v[kMaxLevels][3];
};

// Threads of the first pass: the shape's threads rounded up to whole warps.
// The extra lanes hold the neutral rate 0 and load nothing, so every warp of
// the CTA is full and the butterfly shuffles read only existing lanes.
template <int DIM, int N>
struct PartialsShape {
  static constexpr int THREADS = (PredictShape<DIM, N>::THREADS + 31) / 32 * 32;
};

template <int DIM, int N, class PDE>
__global__ void __launch_bounds__(PartialsShape<DIM, N>::THREADS)
    dt_partials_kernel(const double* u, const int8_t* level, int64_t ncells, double gamma,
                       const InvH inv_h, double* partials) {
  using SH = PredictShape<DIM, N>;
  constexpr int NS = SH::NS, CPB = SH::CPB, M = PDE::M;
  const int tid = threadIdx.x;
  const int cl = tid / NS;
  const int node = tid - cl * NS;
  const int64_t cell = int64_t(blockIdx.x) * CPB + cl;
  double rate = 0.0;
  if (tid < SH::THREADS && cell < ncells) {
    const int lv_raw = int(level[cell]);
    const bool lv_ok = lv_raw >= 0 && lv_raw < kMaxLevels;
    const int lv = lv_ok ? lv_raw : 0;
    double q[M];
#pragma unroll
    for (int v = 0; v < M; ++v) q[v] = u[(cell * M + v) * NS + node];
    bool ok_all = lv_ok;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      bool ok;
      rate += PDE::max_speed(q, d, gamma, &ok) * inv_h.v[lv][d];
      ok_all = ok_all && ok;
    }
    if (!ok_all) rate = __longlong_as_double(0x7ff8000000000000ll);
  }
  __shared__ double red[32];
  rate = warp_nan_max(rate);
  const int lane = tid & 31, warp = tid >> 5;
  if (lane == 0) red[warp] = rate;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    double x = lane < nw ? red[lane] : 0.0;
    x = warp_nan_max(x);
    if (lane == 0) partials[blockIdx.x] = x;
  }
}

// Second pass: one CTA of 1024 threads (whole warps) reduces the partials
// and writes dt.
__global__ void dt_finish_kernel(const double* partials, int64_t count, double cfl, double* dt) {
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) m = nan_max(m, partials[i]);
  __shared__ double red[32];
  m = warp_nan_max(m);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = m;
  __syncthreads();
  if (warp == 0) {
    double x = lane < int(blockDim.x >> 5) ? red[lane] : 0.0;
    x = warp_nan_max(x);
    // a zero, infinite or NaN maximum rate has no time step: NaN, like the
    // non-finite-rate failure of the context path
    if (lane == 0) *dt = (x > 0.0 && isfinite(x)) ? cfl / x : __longlong_as_double(0x7ff8000000000000ll);
  }
}

template <int DIM, class PDE>
cudaError_t launch_partials(int order, const double* u, const int8_t* level, int64_t ncells,
                            double gamma, const InvH& inv_h, double* partials, int64_t* nblocks,
                            cudaStream_t s) {
  return with_order(order, [&](auto Nc) {
    constexpr int N = decltype(Nc)::value;
    using SH = PredictShape<DIM, N>;
    *nblocks = (ncells + SH::CPB - 1) / SH::CPB;
    dt_partials_kernel<DIM, N, PDE><<<unsigned(*nblocks), PartialsShape<DIM, N>::THREADS, 0, s>>>(
        u, level, ncells, gamma, inv_h, partials);
    return cudaGetLastError();
  });
}

// Device address of g_dt_partials for the current device, looked up once per
// device and kept for the life of the process (it names the primary
// context's copy of the array, so it is stale after cudaDeviceReset).
cudaError_t partials_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_partials_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_dt_partials);
    if (e != cudaSuccess) return e;
    g_partials_addr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace ader

extern "C" ader_status ader_compute_dt_static(int dim, int order, ader_pde pde, double gamma,
                                              double cfl, const int base[3], const double lo[3],
                                              const double hi[3], int64_t ncells,
                                              const double* u_dev, const int8_t* level_dev,
                                              double* dt_dev, void* stream) {
  using namespace ader;
  if ((dim != 2 && dim != 3) || order < 1 || order > 7 || !(cfl > 0.0) || !base || !lo || !hi ||
      !u_dev || !level_dev || !dt_dev || ncells < 1)
    return ADER_ERR_ARG;
  if (pde != ADER_EULER && pde != ADER_ACOUSTICS) return ADER_ERR_ARG;
  if (ncells > ADER_DT_STATIC_MAX_CELLS) return ADER_ERR_ARG;
  InvH ih{};
  for (int d = 0; d < dim; ++d) {
    if (base[d] < 1 || !(hi[d] > lo[d])) return ADER_ERR_ARG;
    double cells = double(base[d]);
    for (int l = 0; l < kMaxLevels; ++l) {
      ih.v[l][d] = cells / (hi[d] - lo[d]);
      cells *= 3.0;
    }
  }
  double* partials = nullptr;
  if (partials_address(&partials) != cudaSuccess) return ADER_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t nblocks = 0;
  cudaError_t e;
  if (pde == ADER_EULER)
    e = dim == 2 ? launch_partials<2, Euler<2>>(order, u_dev, level_dev, ncells, gamma, ih,
                                                partials, &nblocks, s)
                 : launch_partials<3, Euler<3>>(order, u_dev, level_dev, ncells, gamma, ih,
                                                partials, &nblocks, s);
  else
    e = dim == 2 ? launch_partials<2, Acoustics<2>>(order, u_dev, level_dev, ncells, gamma, ih,
                                                    partials, &nblocks, s)
                 : launch_partials<3, Acoustics<3>>(order, u_dev, level_dev, ncells, gamma, ih,
                                                    partials, &nblocks, s);
  if (e != cudaSuccess) return ADER_ERR_CUDA;
  dt_finish_kernel<<<1, 1024, 0, s>>>(partials, nblocks, cfl, dt_dev);
  return cudaGetLastError() == cudaSuccess ? ADER_OK : ADER_ERR_CUDA;
}
