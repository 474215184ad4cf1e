// Kernels for Acoustics<3> (orders 1..7).
#include "instantiate.cuh"
ADER_INSTANTIATE(acoustics3d, 3, ader::Acoustics<3>)
ADER_INSTANTIATE_CK(acoustics3d, 3, ader::Acoustics<3>)
