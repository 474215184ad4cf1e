// Instantiations of the subcell FV limiter for 2D: orders 1..7
// (one translation unit per dimension so that they compile in parallel).
#include <type_traits>

#include "limiter.cuh"

namespace ader {

template <class PDE>
static cudaError_t dispatch(int order, LimiterKernel which, const LimiterArgs& a, int grid,
                            cudaStream_t s) {
  auto go = [&](auto N) { return launch_limiter_t<2, decltype(N)::value, PDE>(which, a, grid, s); };
  switch (order) {
    case 1: return go(std::integral_constant<int, 1>{});
    case 2: return go(std::integral_constant<int, 2>{});
    case 3: return go(std::integral_constant<int, 3>{});
    case 4: return go(std::integral_constant<int, 4>{});
    case 5: return go(std::integral_constant<int, 5>{});
    case 6: return go(std::integral_constant<int, 6>{});
    case 7: return go(std::integral_constant<int, 7>{});
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_limiter_2d(int order, int pde, LimiterKernel which, const LimiterArgs& a, int grid,
                              cudaStream_t s) {
  return pde == 0 ? dispatch<Euler<2>>(order, which, a, grid, s)
                  : dispatch<Acoustics<2>>(order, which, a, grid, s);
}

}  // namespace ader
