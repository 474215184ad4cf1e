// Tensor-core (tcgen05) predictor kernels: 3D Euler, orders 5..7, TF32,
// 3xTF32 and 3xBF16 derivative contractions.
#include "instantiate.cuh"

namespace ader {

cudaError_t predict_tc_euler3d(int order, Precision p, const PredictArgs& a, cudaStream_t s) {
  const int mode = p == Precision::kTF32 ? kTcTF32 : p == Precision::kTF32x3 ? kTcTF32x3
                   : p == Precision::kBF16x3 ? kTcBF16x3 : kTcNone;
  auto go = [&](auto Nc) -> cudaError_t {
    constexpr int N = decltype(Nc)::value;
    if constexpr (N >= 5) {
      switch (mode) {
        case kTcTF32: return launch_predict_tc_t<N, Euler<3>, kTcTF32>(a, s);
        case kTcTF32x3: return launch_predict_tc_t<N, Euler<3>, kTcTF32x3>(a, s);
        case kTcBF16x3: return launch_predict_tc_t<N, Euler<3>, kTcBF16x3>(a, s);
        default: return cudaErrorInvalidValue;
      }
    } else {
      return cudaErrorInvalidValue;
    }
  };
  return with_order(order, go);
}

}  // namespace ader
