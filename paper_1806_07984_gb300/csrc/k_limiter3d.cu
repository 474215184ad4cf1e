// Instantiations of the subcell FV limiter for 3D: orders 1..5
// (a 3D patch of (2N+1)^3 subcells with its halo stays in shared memory).
#include <type_traits>

#include "limiter.cuh"

namespace ader {

template <class PDE>
static cudaError_t dispatch(int order, LimiterKernel which, const LimiterArgs& a, int grid,
                            cudaStream_t s) {
  auto go = [&](auto N) { return launch_limiter_t<3, decltype(N)::value, PDE>(which, a, grid, s); };
  switch (order) {
    case 1: return go(std::integral_constant<int, 1>{});
    case 2: return go(std::integral_constant<int, 2>{});
    case 3: return go(std::integral_constant<int, 3>{});
    case 4: return go(std::integral_constant<int, 4>{});
    case 5: return go(std::integral_constant<int, 5>{});

    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_limiter_3d(int order, int pde, LimiterKernel which, const LimiterArgs& a, int grid,
                              cudaStream_t s) {
  return pde == 0 ? dispatch<Euler<3>>(order, which, a, grid, s)
                  : dispatch<Acoustics<3>>(order, which, a, grid, s);
}

}  // namespace ader
