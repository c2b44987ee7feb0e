// Element and face kernels instantiated for velocity degree k = 2.
#define STOKES_K 2
#include "elem_body.cuh"
STOKES_DEFINE_DEGREE(2)
