// Krylov / Newton vector kernels (HBM-bound, FP64 accumulation of every
// reduction).  Section 4: the outer Newton iteration and the Krylov
// orthogonalisation run on device vectors; inner products accumulate in FP64
// whatever the storage precision.
#include <cuda_runtime.h>

#include "vec.h"

namespace stokes {
namespace {

constexpr int VT = 256;

__device__ __forceinline__ double warp_sum(double v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// out[j] += sum_i V[j*ld + i] * w[i]   for j < m (grid.y = j); V rows may be of
// type TV, w of type TW.  out must be cleared by the caller.
template <typename TV, typename TW>
__global__ void multidot_kernel(int64_t n, const TV* __restrict__ V, int64_t ld, const TW* __restrict__ w,
                                double* __restrict__ out) {
    __shared__ double red[VT / 32];
    const int j = blockIdx.y;
    const TV* v = V + ld * j;
    double s = 0;
    for (int64_t i = int64_t(blockIdx.x) * VT + threadIdx.x; i < n; i += int64_t(gridDim.x) * VT)
        s += double(v[i]) * double(w[i]);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < VT / 32 ? red[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) atomicAdd(out + j, t);
    }
}

// w[i] -= sum_j h[j] V[j*ld + i];  nrm2 += ||w||^2 after the update
template <typename T>
__global__ void multiaxpy_kernel(int64_t n, T* __restrict__ w, const T* __restrict__ V, int64_t ld, int m,
                                 const double* __restrict__ h, double* __restrict__ nrm2) {
    __shared__ double red[VT / 32];
    double s = 0;
    for (int64_t i = int64_t(blockIdx.x) * VT + threadIdx.x; i < n; i += int64_t(gridDim.x) * VT) {
        double acc = double(w[i]);
        for (int j = 0; j < m; ++j) acc -= h[j] * double(V[ld * j + i]);
        const T r = T(acc);
        w[i] = r;
        s += double(r) * double(r);
    }
    if (nrm2) {
        s = warp_sum(s);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x < 32) {
            double t = threadIdx.x < VT / 32 ? red[threadIdx.x] : 0.0;
            t = warp_sum(t);
            if (threadIdx.x == 0) atomicAdd(nrm2, t);
        }
    }
}

// y = a * x + b * y  (types may differ; a, b from device scalars or host values)
template <typename TX, typename TY>
__global__ void axpby_kernel(int64_t n, double a, const double* __restrict__ da, const TX* __restrict__ x,
                             double b, TY* __restrict__ y) {
    const double aa = da ? a * da[0] : a;
    for (int64_t i = int64_t(blockIdx.x) * VT + threadIdx.x; i < n; i += int64_t(gridDim.x) * VT)
        y[i] = TY(aa * double(x[i]) + (b == 0.0 ? 0.0 : b * double(y[i])));
}

// x *= 1 / sqrt(nrm2[0])  (normalise in place from a device norm^2)
template <typename T>
__global__ void normalize_kernel(int64_t n, T* __restrict__ x, const double* __restrict__ nrm2) {
    const double s = 1.0 / sqrt(nrm2[0]);
    for (int64_t i = int64_t(blockIdx.x) * VT + threadIdx.x; i < n; i += int64_t(gridDim.x) * VT)
        x[i] = T(double(x[i]) * s);
}

// y += sum_j c[j] Z[j*ld + i]   (c host-side, passed by value as device array)
template <typename TZ, typename TY>
__global__ void combine_kernel(int64_t n, TY* __restrict__ y, const TZ* __restrict__ Z, int64_t ld, int m,
                               const double* __restrict__ c) {
    for (int64_t i = int64_t(blockIdx.x) * VT + threadIdx.x; i < n; i += int64_t(gridDim.x) * VT) {
        double acc = double(y[i]);
        for (int j = 0; j < m; ++j) acc += c[j] * double(Z[ld * j + i]);
        y[i] = TY(acc);
    }
}

int grid_for(int64_t n) {
    int64_t b = (n + VT - 1) / VT;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return int(b);
}

}  // namespace

#define DISPATCH2(prec_a, prec_b, CALL)                                   \
    if ((prec_a) == 1 && (prec_b) == 1) { using TA = float; using TB = float; CALL; }         \
    else if ((prec_a) == 1) { using TA = float; using TB = double; CALL; }                     \
    else if ((prec_b) == 1) { using TA = double; using TB = float; CALL; }                    \
    else { using TA = double; using TB = double; CALL; }

int vec_multidot(int64_t n, int vprec, const void* V, int64_t ld, int m, int wprec, const void* w,
                 double* out, cudaStream_t s) {
    if (m <= 0) return 0;
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * m, s);
    if (e != cudaSuccess) return int(e);
    dim3 grid(unsigned(grid_for(n) / 4 + 1), unsigned(m));
    DISPATCH2(vprec, wprec, (multidot_kernel<TA, TB><<<grid, VT, 0, s>>>(n, static_cast<const TA*>(V), ld,
                                                                         static_cast<const TB*>(w), out)));
    return int(cudaGetLastError());
}

int vec_multiaxpy(int64_t n, int prec, void* w, const void* V, int64_t ld, int m, const double* h,
                  double* nrm2, cudaStream_t s) {
    if (nrm2) {
        cudaError_t e = cudaMemsetAsync(nrm2, 0, sizeof(double), s);
        if (e != cudaSuccess) return int(e);
    }
    if (prec == 1)
        multiaxpy_kernel<float><<<grid_for(n), VT, 0, s>>>(n, static_cast<float*>(w), static_cast<const float*>(V),
                                                            ld, m, h, nrm2);
    else
        multiaxpy_kernel<double><<<grid_for(n), VT, 0, s>>>(n, static_cast<double*>(w),
                                                             static_cast<const double*>(V), ld, m, h, nrm2);
    return int(cudaGetLastError());
}

int vec_axpby(int64_t n, double a, const double* da, int xprec, const void* x, double b, int yprec, void* y,
              cudaStream_t s) {
    DISPATCH2(xprec, yprec, (axpby_kernel<TA, TB><<<grid_for(n), VT, 0, s>>>(n, a, da, static_cast<const TA*>(x), b,
                                                                            static_cast<TB*>(y))));
    return int(cudaGetLastError());
}

int vec_normalize(int64_t n, int prec, void* x, const double* nrm2, cudaStream_t s) {
    if (prec == 1)
        normalize_kernel<float><<<grid_for(n), VT, 0, s>>>(n, static_cast<float*>(x), nrm2);
    else
        normalize_kernel<double><<<grid_for(n), VT, 0, s>>>(n, static_cast<double*>(x), nrm2);
    return int(cudaGetLastError());
}

int vec_combine(int64_t n, int zprec, const void* Z, int64_t ld, int m, const double* c, int yprec, void* y,
                cudaStream_t s) {
    DISPATCH2(zprec, yprec, (combine_kernel<TA, TB><<<grid_for(n), VT, 0, s>>>(n, static_cast<TB*>(y),
                                                                              static_cast<const TA*>(Z), ld, m, c)));
    return int(cudaGetLastError());
}

}  // namespace stokes
