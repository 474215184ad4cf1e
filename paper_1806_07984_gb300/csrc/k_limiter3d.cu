// Instantiations of the subcell FV limiter for 3D, orders 1..7 (up to N=5
// the (2N+1)^3 patch and its halo stay in shared memory; at N=6, 7 in a
// global scratch slot per CTA).
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
    case 6: return go(std::integral_constant<int, 6>{});
    case 7: return go(std::integral_constant<int, 7>{});
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_limiter_3d(int order, int pde, LimiterKernel which, const LimiterArgs& a, int grid,
                              cudaStream_t s) {
  return pde == 0 ? dispatch<Euler<3>>(order, which, a, grid, s)
                  : dispatch<Acoustics<3>>(order, which, a, grid, s);
}

int64_t limiter_fv_scratch_3d(int order, int pde) {
  const int M = pde == 0 ? 5 : 4;
  if (order == 6) return M == 5 ? fv_scratch_slot<3, 6, 5>() : fv_scratch_slot<3, 6, 4>();
  if (order == 7) return M == 5 ? fv_scratch_slot<3, 7, 5>() : fv_scratch_slot<3, 7, 4>();
  return 0;
}

}  // namespace ader
