// Per-(dimension, PDE) instantiation of all kernels for orders 1..7, one
// translation unit each so that they compile in parallel.
#pragma once
#include <type_traits>

#include "faces.cuh"
#include "predict.cuh"

namespace ader {

template <class F>
cudaError_t with_order(int order, F&& f) {
  switch (order) {
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    case 3: return f(std::integral_constant<int, 3>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 5: return f(std::integral_constant<int, 5>{});
    case 6: return f(std::integral_constant<int, 6>{});
    case 7: return f(std::integral_constant<int, 7>{});
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ader

#define ADER_INSTANTIATE(TAG, DIM, PDE)                                                        \
  namespace ader {                                                                             \
  cudaError_t predict_##TAG(int order, Precision prec, const PredictArgs& a, cudaStream_t s) { \
    return with_order(order, [&](auto N) {                                                     \
      return prec == Precision::kFP64   ? launch_predict_t<DIM, N.value, PDE, double>(a, s)    \
             : prec == Precision::kDF64 ? launch_predict_t<DIM, N.value, PDE, df64>(a, s)      \
                                        : launch_predict_t<DIM, N.value, PDE, float>(a, s);    \
    });                                                                                        \
  }                                                                                            \
  cudaError_t faces_##TAG(int order, int which, const RiemannArgs& a, cudaStream_t s) {        \
    return with_order(order,                                                                   \
                      [&](auto N) { return launch_faces_t<DIM, N.value, PDE>(which, a, s); }); \
  }                                                                                            \
  cudaError_t correct_##TAG(int order, bool update, const CorrectArgs& a, cudaStream_t s) {    \
    return with_order(order, [&](auto N) {                                                     \
      return update ? launch_correct_t<DIM, N.value, PDE, true>(a, s)                          \
                    : launch_correct_t<DIM, N.value, PDE, false>(a, s);                        \
    });                                                                                        \
  }                                                                                            \
  cudaError_t transfer_##TAG(int order, const TransferArgs& a, cudaStream_t s) {               \
    return with_order(order,                                                                   \
                      [&](auto N) { return launch_transfer_t<DIM, N.value, PDE::M>(a, s); });  \
  }                                                                                            \
  cudaError_t indicator_##TAG(int order, const IndicatorArgs& a, cudaStream_t s) {             \
    return with_order(order,                                                                   \
                      [&](auto N) { return launch_indicator_t<DIM, N.value, PDE::M>(a, s); }); \
  }                                                                                            \
  }

// Cauchy-Kowalevski predictor (linear PDEs only).
#define ADER_INSTANTIATE_CK(TAG, DIM, PDE)                                                       \
  namespace ader {                                                                               \
  cudaError_t predict_ck_##TAG(int order, Precision prec, const PredictArgs& a, cudaStream_t s) { \
    return with_order(order, [&](auto N) {                                                       \
      return prec == Precision::kFP64 ? launch_predict_t<DIM, N.value, PDE, double, 1>(a, s)     \
                                      : launch_predict_t<DIM, N.value, PDE, float, 1>(a, s);     \
    });                                                                                          \
  }                                                                                              \
  }
