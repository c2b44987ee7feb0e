// Element, face and preconditioner-assembly kernels for velocity degree k = 3.
#define STOKES_K 3
#include "elem_body.cuh"
#include "precond_body.cuh"
STOKES_DEFINE_DEGREE(3)
STOKES_DEFINE_PRECOND(3)
