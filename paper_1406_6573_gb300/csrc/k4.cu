// Element, face and preconditioner-assembly kernels for velocity degree k = 4.
#define STOKES_K 4
#include "elem_body.cuh"
#include "precond_body.cuh"
STOKES_DEFINE_DEGREE(4)
STOKES_DEFINE_PRECOND(4)
