// Kernels for the velocity degrees k = 5 .. 9 (khigh.cu): one block per
// element or basal face, run-time degree, shared-memory sum factorisation.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "kernels.h"
#include "precond.h"

namespace stokes {

// degree-k tables on device dev (built once, kept for the process)
int high_tables(int dev, int k, const void** out);
// values per element of the linearised state (element-major layout)
int64_t high_state_stride(int k);
// partial sums written by the fixed-order A-gradient launch
int64_t high_grad_a_partials(int64_t E);
// element modes: residual, linearisation, stored-state apply and pressure
// block, A-gradient (a.htab, a.htab_k, a.state_stride set); cudaError_t value
int launch_elem_high(int mode, int prec, int state_prec, const ElemArgs& a, cudaStream_t s);
int launch_face_high(int mode, int prec, const FaceArgs& a, cudaStream_t s);
int launch_precond_assembly_high(int prec, const ColArgs& a, cudaStream_t s);

}  // namespace stokes
