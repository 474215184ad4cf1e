// Kernels for Euler<2> (orders 1..7).
#include "instantiate.cuh"
ADER_INSTANTIATE(euler2d, 2, ader::Euler<2>)
