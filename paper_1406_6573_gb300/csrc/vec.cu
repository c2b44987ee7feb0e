// Krylov / Newton vector kernels (HBM-bound).  Section 4: the outer Newton
// iteration and the Krylov orthogonalisation run on device vectors.
//
// Inner products are accumulated to FP64 accuracy whatever the storage
// precision.  For FP32 vectors every product a*b is split exactly into
// p + e (p = a*b rounded, e = fma(a, b, -p)) and accumulated as a
// double-float pair (two FP32 words, about 48 significant bits) with
// error-free two-sums: GB300 runs FP32 at many times its FP64 rate, so this
// keeps the reductions memory-bound.  Per-thread partial sums are combined
// in FP64.  FP64 vectors use FP64 arithmetic.
#include <type_traits>

#include <cuda_runtime.h>

#include "vec.h"

namespace stokes {
namespace {

constexpr int VT = 256;
constexpr int MAXV = 32;   // most vectors in one multi-dot / multi-axpy

__device__ __forceinline__ double warp_sum(double v) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// double-float accumulator (hi + lo)
struct DF {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = a * b;
        const float e = fmaf(a, b, -p);          // exact: a*b = p + e
        const float s = hi + p;                  // two-sum(hi, p)
        const float bb = s - hi;
        const float err = (hi - (s - bb)) + (p - bb);
        hi = s;
        lo += err + e;
    }
    __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

template <typename T>
__device__ __forceinline__ void block_add(double v, double* out, double* red) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < VT / 32 ? red[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) atomicAdd(out, t);
    }
}

// out[j] += sum_i V[j*ld + i] * w[i], j < m: one pass reading w once and every
// V_j once.
__global__ void __launch_bounds__(VT) multidot_f32(int64_t n, const float* __restrict__ V, int64_t ld, int m,
                                                   const float* __restrict__ w, double* __restrict__ out) {
    __shared__ double red[VT / 32];
    DF acc[MAXV];
    for (int64_t i = int64_t(blockIdx.x) * VT + threadIdx.x; i < n; i += int64_t(gridDim.x) * VT) {
        const float wi = w[i];
        #pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < m) acc[j].add_prod(__ldcs(V + ld * j + i), wi);
    }
    #pragma unroll
    for (int j = 0; j < MAXV; ++j)
        if (j < m) block_add<float>(acc[j].value(), out + j, red);
}

__global__ void __launch_bounds__(VT) multidot_f64(int64_t n, const double* __restrict__ V, int64_t ld, int m,
                                                   const double* __restrict__ w, double* __restrict__ out) {
    __shared__ double red[VT / 32];
    double acc[MAXV];
    #pragma unroll
    for (int j = 0; j < MAXV; ++j) acc[j] = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * VT + threadIdx.x; i < n; i += int64_t(gridDim.x) * VT) {
        const double wi = w[i];
        #pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < m) acc[j] = fma(V[ld * j + i], wi, acc[j]);
    }
    #pragma unroll
    for (int j = 0; j < MAXV; ++j)
        if (j < m) block_add<double>(acc[j], out + j, red);
}

// w[i] -= sum_j h[j] V[j*ld + i];  nrm2 += ||w||^2 after the update
__global__ void __launch_bounds__(VT) multiaxpy_f32(int64_t n, float* __restrict__ w, const float* __restrict__ V,
                                                    int64_t ld, int m, const double* __restrict__ h,
                                                    double* __restrict__ nrm2) {
    __shared__ double red[VT / 32];
    __shared__ float hs[MAXV];
    if (threadIdx.x < MAXV) hs[threadIdx.x] = threadIdx.x < m ? float(h[threadIdx.x]) : 0.f;
    __syncthreads();
    DF acc;
    for (int64_t i = int64_t(blockIdx.x) * VT + threadIdx.x; i < n; i += int64_t(gridDim.x) * VT) {
        float r = w[i];
        #pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < m) r = fmaf(-hs[j], __ldcs(V + ld * j + i), r);
        w[i] = r;
        acc.add_prod(r, r);
    }
    if (nrm2) block_add<float>(acc.value(), nrm2, red);
}

__global__ void __launch_bounds__(VT) multiaxpy_f64(int64_t n, double* __restrict__ w, const double* __restrict__ V,
                                                    int64_t ld, int m, const double* __restrict__ h,
                                                    double* __restrict__ nrm2) {
    __shared__ double red[VT / 32];
    __shared__ double hs[MAXV];
    if (threadIdx.x < MAXV) hs[threadIdx.x] = threadIdx.x < m ? h[threadIdx.x] : 0.0;
    __syncthreads();
    double s = 0;
    for (int64_t i = int64_t(blockIdx.x) * VT + threadIdx.x; i < n; i += int64_t(gridDim.x) * VT) {
        double r = w[i];
        #pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < m) r = fma(-hs[j], V[ld * j + i], r);
        w[i] = r;
        s = fma(r, r, s);
    }
    if (nrm2) block_add<double>(s, nrm2, red);
}

// y = a x + b y in the arithmetic of the narrower operand type
template <typename TX, typename TY>
__global__ void axpby_kernel(int64_t n, double a, const double* __restrict__ da, const TX* __restrict__ x,
                             double b, TY* __restrict__ y) {
    const double aa = da ? a * da[0] : a;
    using C = typename std::conditional<(sizeof(TX) == 4 && sizeof(TY) == 4), float, double>::type;
    const C ca = C(aa), cb = C(b);
    for (int64_t i = int64_t(blockIdx.x) * VT + threadIdx.x; i < n; i += int64_t(gridDim.x) * VT) {
        const C xv = C(x[i]);
        y[i] = TY(b == 0.0 ? ca * xv : ca * xv + cb * C(y[i]));
    }
}

// x *= 1 / sqrt(nrm2[0])
template <typename T>
__global__ void normalize_kernel(int64_t n, T* __restrict__ x, const double* __restrict__ nrm2) {
    const T s = T(1.0 / sqrt(nrm2[0]));
    for (int64_t i = int64_t(blockIdx.x) * VT + threadIdx.x; i < n; i += int64_t(gridDim.x) * VT) x[i] *= s;
}

// y += sum_j c[j] Z[j*ld + i]   (c on the device; FP64 accumulation into y)
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
    if (b > 152 * 8) b = 152 * 8;
    if (b < 1) b = 1;
    return int(b);
}

}  // namespace

#define DISPATCH2(prec_a, prec_b, CALL)                                                        \
    if ((prec_a) == 1 && (prec_b) == 1) { using TA = float; using TB = float; CALL; }         \
    else if ((prec_a) == 1) { using TA = float; using TB = double; CALL; }                     \
    else if ((prec_b) == 1) { using TA = double; using TB = float; CALL; }                    \
    else { using TA = double; using TB = double; CALL; }

int vec_multidot(int64_t n, int vprec, const void* V, int64_t ld, int m, int wprec, const void* w,
                 double* out, cudaStream_t s) {
    if (m <= 0) return 0;
    if (m > MAXV || vprec != wprec) return int(cudaErrorInvalidValue);
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * m, s);
    if (e != cudaSuccess) return int(e);
    if (vprec == 1)
        multidot_f32<<<grid_for(n), VT, 0, s>>>(n, static_cast<const float*>(V), ld, m, static_cast<const float*>(w), out);
    else
        multidot_f64<<<grid_for(n), VT, 0, s>>>(n, static_cast<const double*>(V), ld, m,
                                                 static_cast<const double*>(w), out);
    return int(cudaGetLastError());
}

int vec_multiaxpy(int64_t n, int prec, void* w, const void* V, int64_t ld, int m, const double* h,
                  double* nrm2, cudaStream_t s) {
    if (m > MAXV) return int(cudaErrorInvalidValue);
    if (nrm2) {
        cudaError_t e = cudaMemsetAsync(nrm2, 0, sizeof(double), s);
        if (e != cudaSuccess) return int(e);
    }
    if (prec == 1)
        multiaxpy_f32<<<grid_for(n), VT, 0, s>>>(n, static_cast<float*>(w), static_cast<const float*>(V), ld, m, h, nrm2);
    else
        multiaxpy_f64<<<grid_for(n), VT, 0, s>>>(n, static_cast<double*>(w), static_cast<const double*>(V), ld, m, h,
                                                  nrm2);
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
