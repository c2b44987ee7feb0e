// Element and face kernels instantiated for velocity degree k = 4.
#define STOKES_K 4
#include "elem_body.cuh"
STOKES_DEFINE_DEGREE(4)
