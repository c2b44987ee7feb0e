// Element, face and preconditioner-assembly kernels for velocity degree k = 2.
#define STOKES_K 2
#include "elem_body.cuh"
#include "precond_body.cuh"
STOKES_DEFINE_DEGREE(2)
STOKES_DEFINE_PRECOND(2)
