// Kernels for Acoustics<2> (orders 1..7).
#include "instantiate.cuh"
ADER_INSTANTIATE(acoustics2d, 2, ader::Acoustics<2>)
ADER_INSTANTIATE_CK(acoustics2d, 2, ader::Acoustics<2>)
