// Degree-independent kernels: the identity part of the constrained operator.
#include <cuda_runtime.h>

#include "kernels.h"

namespace stokes {
namespace {

// y[g] += s (x[g] - P_b x[g]) at every basal node b (g its global node): the
// s (I - P) term of the constrained residual P r(P u) + s (I - P) u and of the
// constrained Jacobian P J P + s (I - P).
template <typename T>
__global__ void constraint_kernel(int64_t Nb, const int32_t* __restrict__ nodes,
                                  const double* __restrict__ P, double scale, const T* __restrict__ x,
                                  T* __restrict__ y) {
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= Nb) return;
    const int64_t g = nodes[b];
    const double* p = P + 6 * b;
    const T x0 = x[3 * g], x1 = x[3 * g + 1], x2 = x[3 * g + 2];
    const T p00 = T(p[0]), p11 = T(p[1]), p22 = T(p[2]), p01 = T(p[3]), p02 = T(p[4]), p12 = T(p[5]);
    const T sc = T(scale);
    y[3 * g] += sc * (x0 - (p00 * x0 + p01 * x1 + p02 * x2));
    y[3 * g + 1] += sc * (x1 - (p01 * x0 + p11 * x1 + p12 * x2));
    y[3 * g + 2] += sc * (x2 - (p02 * x0 + p12 * x1 + p22 * x2));
}

}  // namespace

int launch_constraint(int prec, int64_t Nb, const int32_t* basal_nodes, const double* basal_P, double scale,
                      const void* x, void* y, cudaStream_t s) {
    if (Nb == 0) return int(cudaSuccess);
    const int threads = 256;
    const unsigned blocks = unsigned((Nb + threads - 1) / threads);
    if (prec == 1)
        constraint_kernel<float><<<blocks, threads, 0, s>>>(Nb, basal_nodes, basal_P, scale,
                                                            static_cast<const float*>(x), static_cast<float*>(y));
    else
        constraint_kernel<double><<<blocks, threads, 0, s>>>(Nb, basal_nodes, basal_P, scale,
                                                             static_cast<const double*>(x), static_cast<double*>(y));
    return int(cudaGetLastError());
}

}  // namespace stokes
