// Element and face kernels instantiated for velocity degree k = 3.
#define STOKES_K 3
#include "elem_body.cuh"
STOKES_DEFINE_DEGREE(3)
