// Per-(dimension, PDE) kernel entry points defined in k_*.cu.
#pragma once
#include "kernels.h"

namespace ader {

#define ADER_DECLARE(TAG)                                                                      \
  cudaError_t predict_##TAG(int order, Precision prec, const PredictArgs& a, cudaStream_t s); \
  cudaError_t faces_##TAG(int order, int which, const RiemannArgs& a, cudaStream_t s);        \
  cudaError_t correct_##TAG(int order, bool update, const CorrectArgs& a, cudaStream_t s);    \
  cudaError_t transfer_##TAG(int order, const TransferArgs& a, cudaStream_t s);              \
  cudaError_t indicator_##TAG(int order, const IndicatorArgs& a, cudaStream_t s);

ADER_DECLARE(euler2d)
ADER_DECLARE(euler3d)
ADER_DECLARE(acoustics2d)
ADER_DECLARE(acoustics3d)
#undef ADER_DECLARE
cudaError_t predict_ck_acoustics2d(int order, Precision prec, const PredictArgs& a, cudaStream_t s);
cudaError_t predict_ck_acoustics3d(int order, Precision prec, const PredictArgs& a, cudaStream_t s);
cudaError_t predict_tc_euler3d(int order, Precision p, const PredictArgs& a, cudaStream_t s);

}  // namespace ader
