// Vector kernels for the Newton-Krylov driver.  prec codes: 0 = double, 1 = float.
// All return a cudaError_t value.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace stokes {

// out[j] = sum_i V[j ld + i] w[i], j < m, and out[m] = ||w||^2 if self_norm
// (FP64-accurate accumulation; out overwritten; m <= 32)
int vec_multidot(int64_t n, int vprec, const void* V, int64_t ld, int m, int wprec, const void* w,
                 double* out, int self_norm, cudaStream_t s);
// w = scale (w - sum_j h[j] V[j ld + .]) (h on the device, m <= 32); if dots
// (device, may be NULL): dots[j] = V_j . w (j < m) and dots[m] = ||w||^2 of
// the updated w (a second pass)
int vec_multiaxpy(int64_t n, int prec, void* w, const void* V, int64_t ld, int m, const double* h, double scale,
                  double* dots, cudaStream_t s);
// y = a (* da[0] if da) x + b y
int vec_axpby(int64_t n, double a, const double* da, int xprec, const void* x, double b, int yprec, void* y,
              cudaStream_t s);
// x /= sqrt(nrm2[0])
int vec_normalize(int64_t n, int prec, void* x, const double* nrm2, cudaStream_t s);
// y += sum_j c[j] Z[j ld + .]   (c on the device)
int vec_combine(int64_t n, int zprec, const void* Z, int64_t ld, int m, const double* c, int yprec, void* y,
                cudaStream_t s);

}  // namespace stokes
