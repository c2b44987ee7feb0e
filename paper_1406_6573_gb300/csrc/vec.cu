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
#include <mutex>
#include <type_traits>
#include <utility>
#include <vector>

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

// out[j] += sum_i V[j*ld + i] * w[i], j < m, and with SELF also out[m] +=
// ||w||^2: one pass reading w once and every V_j once.
template <bool SELF>
__global__ void __launch_bounds__(VT) multidot_f32(int64_t n, const float* __restrict__ V, int64_t ld, int m,
                                                   const float* __restrict__ w, double* __restrict__ out) {
    __shared__ double red[VT / 32];
    DF acc[MAXV], an;
    for (int64_t i = int64_t(blockIdx.x) * VT + threadIdx.x; i < n; i += int64_t(gridDim.x) * VT) {
        const float wi = w[i];
        #pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < m) acc[j].add_prod(__ldcs(V + ld * j + i), wi);
        if (SELF) an.add_prod(wi, wi);
    }
    #pragma unroll
    for (int j = 0; j < MAXV; ++j)
        if (j < m) block_add(acc[j].value(), out + j, red);
    if (SELF) block_add(an.value(), out + m, red);
}

template <bool SELF>
__global__ void __launch_bounds__(VT) multidot_f64(int64_t n, const double* __restrict__ V, int64_t ld, int m,
                                                   const double* __restrict__ w, double* __restrict__ out) {
    __shared__ double red[VT / 32];
    double acc[MAXV], an = 0.0;
    #pragma unroll
    for (int j = 0; j < MAXV; ++j) acc[j] = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * VT + threadIdx.x; i < n; i += int64_t(gridDim.x) * VT) {
        const double wi = w[i];
        #pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < m) acc[j] = fma(__ldcs(V + ld * j + i), wi, acc[j]);
        if (SELF) an = fma(wi, wi, an);
    }
    #pragma unroll
    for (int j = 0; j < MAXV; ++j)
        if (j < m) block_add(acc[j], out + j, red);
    if (SELF) block_add(an, out + m, red);
}

// w[i] = scale (w[i] - sum_j h[j] V[j*ld + i]); with DOTS also
// out[j] += V_j . w_new (j < m) and out[m] += ||w_new||^2 in the same pass
// (the second classical Gram-Schmidt sweep reads every V_j once for both).
template <bool DOTS>
__global__ void __launch_bounds__(VT) multiaxpy_f32(int64_t n, float* __restrict__ w, const float* __restrict__ V,
                                                    int64_t ld, int m, const double* __restrict__ h, double scale,
                                                    double* __restrict__ out) {
    __shared__ double red[VT / 32];
    __shared__ float hs[MAXV];
    if (threadIdx.x < MAXV) hs[threadIdx.x] = threadIdx.x < m ? float(h[threadIdx.x]) : 0.f;
    __syncthreads();
    const float sc = float(scale);
    DF acc[DOTS ? MAXV : 1], an;
    for (int64_t i = int64_t(blockIdx.x) * VT + threadIdx.x; i < n; i += int64_t(gridDim.x) * VT) {
        float v[MAXV];
        float r = w[i];
        #pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < m) {
                v[j] = __ldcs(V + ld * j + i);
                r = fmaf(-hs[j], v[j], r);
            }
        r *= sc;
        w[i] = r;
        if (DOTS) {
            #pragma unroll
            for (int j = 0; j < MAXV; ++j)
                if (j < m) acc[DOTS ? j : 0].add_prod(v[j], r);
            an.add_prod(r, r);
        }
    }
    if (DOTS) {
        #pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < m) block_add(acc[DOTS ? j : 0].value(), out + j, red);
        block_add(an.value(), out + m, red);
    }
}

template <bool DOTS>
__global__ void __launch_bounds__(VT) multiaxpy_f64(int64_t n, double* __restrict__ w, const double* __restrict__ V,
                                                    int64_t ld, int m, const double* __restrict__ h, double scale,
                                                    double* __restrict__ out) {
    __shared__ double red[VT / 32];
    __shared__ double hs[MAXV];
    if (threadIdx.x < MAXV) hs[threadIdx.x] = threadIdx.x < m ? h[threadIdx.x] : 0.0;
    __syncthreads();
    double acc[DOTS ? MAXV : 1], an = 0.0;
    #pragma unroll
    for (int j = 0; j < (DOTS ? MAXV : 1); ++j) acc[j] = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * VT + threadIdx.x; i < n; i += int64_t(gridDim.x) * VT) {
        double v[MAXV];
        double r = w[i];
        #pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < m) {
                v[j] = __ldcs(V + ld * j + i);
                r = fma(-hs[j], v[j], r);
            }
        r *= scale;
        w[i] = r;
        if (DOTS) {
            #pragma unroll
            for (int j = 0; j < MAXV; ++j)
                if (j < m) acc[DOTS ? j : 0] = fma(v[j], r, acc[DOTS ? j : 0]);
            an = fma(r, r, an);
        }
    }
    if (DOTS) {
        #pragma unroll
        for (int j = 0; j < MAXV; ++j)
            if (j < m) block_add(acc[DOTS ? j : 0], out + j, red);
        block_add(an, out + m, red);
    }
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

// grid of a grid-stride reduction kernel: at most one wave of resident blocks
// (SM count x blocks per SM at the kernel's register footprint), so that no
// block starts after the others have finished their share.  The occupancy of
// each kernel is queried once per process (first device seen).
int resident_blocks(const void* kernel) {
    static std::mutex mu;
    static std::vector<std::pair<const void*, int>> cache;
    std::lock_guard<std::mutex> lock(mu);
    for (const auto& c : cache)
        if (c.first == kernel) return c.second;
    int dev = 0, sms = 0, b = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, VT, 0);
    const int total = (b > 0 ? b : 1) * (sms > 0 ? sms : 1);
    cache.emplace_back(kernel, total);
    return total;
}

template <typename F>
int grid_resident(F kernel, int64_t n) {
    int64_t b = (n + VT - 1) / VT;
    const int64_t cap = resident_blocks(reinterpret_cast<const void*>(kernel));
    if (b > cap) b = cap;
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
                 double* out, int self_norm, cudaStream_t s) {
    const int mo = m + (self_norm ? 1 : 0);
    if (mo <= 0) return 0;
    if (m < 0 || m > MAXV || vprec != wprec) return int(cudaErrorInvalidValue);
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * mo, s);
    if (e != cudaSuccess) return int(e);
    const float* vf = static_cast<const float*>(V);
    const double* vd = static_cast<const double*>(V);
    const float* wf = static_cast<const float*>(w);
    const double* wd = static_cast<const double*>(w);
    if (vprec == 1) {
        if (self_norm) multidot_f32<true><<<grid_resident(multidot_f32<true>, n), VT, 0, s>>>(n, vf, ld, m, wf, out);
        else multidot_f32<false><<<grid_resident(multidot_f32<false>, n), VT, 0, s>>>(n, vf, ld, m, wf, out);
    } else {
        if (self_norm) multidot_f64<true><<<grid_resident(multidot_f64<true>, n), VT, 0, s>>>(n, vd, ld, m, wd, out);
        else multidot_f64<false><<<grid_resident(multidot_f64<false>, n), VT, 0, s>>>(n, vd, ld, m, wd, out);
    }
    return int(cudaGetLastError());
}

int vec_multiaxpy(int64_t n, int prec, void* w, const void* V, int64_t ld, int m, const double* h, double scale,
                  double* dots, cudaStream_t s) {
    if (m < 0 || m > MAXV) return int(cudaErrorInvalidValue);
    if (dots) {
        cudaError_t e = cudaMemsetAsync(dots, 0, sizeof(double) * (m + 1), s);
        if (e != cudaSuccess) return int(e);
    }
    const float* vf = static_cast<const float*>(V);
    const double* vd = static_cast<const double*>(V);
    if (prec == 1) {
        float* wf = static_cast<float*>(w);
        if (dots) multiaxpy_f32<true><<<grid_resident(multiaxpy_f32<true>, n), VT, 0, s>>>(n, wf, vf, ld, m, h, scale, dots);
        else multiaxpy_f32<false><<<grid_resident(multiaxpy_f32<false>, n), VT, 0, s>>>(n, wf, vf, ld, m, h, scale, nullptr);
    } else {
        double* wd = static_cast<double*>(w);
        if (dots) multiaxpy_f64<true><<<grid_resident(multiaxpy_f64<true>, n), VT, 0, s>>>(n, wd, vd, ld, m, h, scale, dots);
        else multiaxpy_f64<false><<<grid_resident(multiaxpy_f64<false>, n), VT, 0, s>>>(n, wd, vd, ld, m, h, scale, nullptr);
    }
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
