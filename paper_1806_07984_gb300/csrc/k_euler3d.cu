// Kernels for Euler<3> (orders 1..7).
#include "instantiate.cuh"
ADER_INSTANTIATE(euler3d, 3, ader::Euler<3>)
