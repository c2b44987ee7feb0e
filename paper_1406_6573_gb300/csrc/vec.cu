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
#include <algorithm>
#include <cstdint>
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

// FP64 accumulator with the interface of DF
struct D1 {
    double s = 0.0;
    __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <typename T> using Acc = typename std::conditional<sizeof(T) == 4, DF, D1>::type;

// VEC consecutive values starting at p (16-byte aligned when VEC > 1), streamed
template <typename T, int VEC>
__device__ __forceinline__ void load_vec(const T* p, T (&o)[VEC]) {
    if constexpr (VEC == 4) {
        const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    } else if constexpr (VEC == 2) {
        const double2 v = __ldcs(reinterpret_cast<const double2*>(p));
        o[0] = v.x; o[1] = v.y;
    } else {
        o[0] = __ldcs(p);
    }
}
template <typename T, int VEC>
__device__ __forceinline__ void store_vec(T* p, const T (&o)[VEC]) {
    if constexpr (VEC == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else if constexpr (VEC == 2) {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    } else {
        p[0] = o[0];
    }
}

constexpr int MD_ROW = 16;   // vectors per grid row of the multi-dot

// out[j] += sum_i V[j*ld + i] w[i] for the MD_ROW vectors j of grid row
// blockIdx.y (j < m); with SELF, grid row 0 also adds ||w||^2 to out[m].
// Values are read in VEC-wide chunks (16-byte loads); the n % VEC tail is
// read by the first threads of block (0, y).
template <typename T, bool SELF, int VEC>
__global__ void __launch_bounds__(VT, 2) multidot_kernel(int64_t n, const T* __restrict__ V, int64_t ld, int m,
                                                         const T* __restrict__ w, double* __restrict__ out) {
    __shared__ double red[VT / 32];
    const int j0 = int(blockIdx.y) * MD_ROW;
    const int mc = min(MD_ROW, m - j0);
    const bool self = SELF && blockIdx.y == 0;
    const T* Vr = V + ld * j0;
    Acc<T> acc[MD_ROW], an;
    const int64_t nv = n / VEC;
    for (int64_t c = int64_t(blockIdx.x) * VT + threadIdx.x; c < nv; c += int64_t(gridDim.x) * VT) {
        T wv[VEC], vv[MD_ROW][VEC];
        load_vec<T, VEC>(w + c * VEC, wv);
        // all loads first (predicated, independent), then the arithmetic
        #pragma unroll
        for (int jj = 0; jj < MD_ROW; ++jj)
            if (jj < mc) load_vec<T, VEC>(Vr + ld * jj + c * VEC, vv[jj]);
        #pragma unroll
        for (int jj = 0; jj < MD_ROW; ++jj)
            if (jj < mc) {
                #pragma unroll
                for (int q = 0; q < VEC; ++q) acc[jj].add_prod(vv[jj][q], wv[q]);
            }
        if (self) {
            #pragma unroll
            for (int q = 0; q < VEC; ++q) an.add_prod(wv[q], wv[q]);
        }
    }
    if (VEC > 1 && blockIdx.x == 0) {
        const int64_t i = nv * VEC + threadIdx.x;
        if (i < n) {
            const T wi = w[i];
            #pragma unroll
            for (int jj = 0; jj < MD_ROW; ++jj)
                if (jj < mc) acc[jj].add_prod(Vr[ld * jj + i], wi);
            if (self) an.add_prod(wi, wi);
        }
    }
    #pragma unroll
    for (int jj = 0; jj < MD_ROW; ++jj)
        if (jj < mc) block_add(acc[jj].value(), out + j0 + jj, red);
    if (self) block_add(an.value(), out + m, red);
}

// w[i] = scale (w[i] - sum_j h[j] V[j*ld + i]), VEC-wide chunks; the vectors
// are read in groups of 8 (bounded registers, 8 loads in flight per thread).
template <typename T, int VEC>
__global__ void __launch_bounds__(VT, 2) multiaxpy_kernel(int64_t n, T* __restrict__ w, const T* __restrict__ V,
                                                          int64_t ld, int m, const double* __restrict__ h,
                                                          double scale) {
    __shared__ T hs[MAXV];
    if (threadIdx.x < MAXV) hs[threadIdx.x] = threadIdx.x < m ? T(h[threadIdx.x]) : T(0);
    __syncthreads();
    const T sc = T(scale);
    const int64_t nv = n / VEC;
    auto body = [&](int64_t off, auto tag) {
        constexpr int W = decltype(tag)::value;
        T r[W];
        load_vec<T, W>(w + off, r);
        #pragma unroll 1
        for (int g = 0; g < m; g += 8) {
            T vv[8][W];
            #pragma unroll
            for (int jj = 0; jj < 8; ++jj)
                if (g + jj < m) load_vec<T, W>(V + ld * (g + jj) + off, vv[jj]);
            #pragma unroll
            for (int jj = 0; jj < 8; ++jj)
                if (g + jj < m) {
                    const T hj = hs[g + jj];
                    #pragma unroll
                    for (int q = 0; q < W; ++q) r[q] = fma(-hj, vv[jj][q], r[q]);
                }
        }
        #pragma unroll
        for (int q = 0; q < W; ++q) r[q] *= sc;
        store_vec<T, W>(w + off, r);
    };
    for (int64_t c = int64_t(blockIdx.x) * VT + threadIdx.x; c < nv; c += int64_t(gridDim.x) * VT)
        body(c * VEC, std::integral_constant<int, VEC>());
    if (VEC > 1 && blockIdx.x == 0) {
        const int64_t i = nv * VEC + threadIdx.x;
        if (i < n) body(i, std::integral_constant<int, 1>());
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

template <typename T>
bool aligned16(const T* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <typename T>
int multidot_t(int64_t n, const T* V, int64_t ld, int m, const T* w, double* out, bool self, cudaStream_t s) {
    constexpr int VEC = sizeof(T) == 4 ? 4 : 2;
    const bool vec = aligned16(V) && aligned16(w) && (m <= 1 || ld % VEC == 0);
    const int rows = std::max(1, (m + MD_ROW - 1) / MD_ROW);
    auto go = [&](auto kernel, int width) {
        const int gx = grid_resident(kernel, (n + width - 1) / width);
        const int gxr = std::max(1, gx / rows);
        kernel<<<dim3(unsigned(gxr), unsigned(rows)), VT, 0, s>>>(n, V, ld, m, w, out);
    };
    if (vec) {
        if (self) go(multidot_kernel<T, true, VEC>, VEC); else go(multidot_kernel<T, false, VEC>, VEC);
    } else {
        if (self) go(multidot_kernel<T, true, 1>, 1); else go(multidot_kernel<T, false, 1>, 1);
    }
    return int(cudaGetLastError());
}

template <typename T>
int multiaxpy_t(int64_t n, T* w, const T* V, int64_t ld, int m, const double* h, double scale, cudaStream_t s) {
    constexpr int VEC = sizeof(T) == 4 ? 4 : 2;
    if (aligned16(V) && aligned16(w) && (m <= 1 || ld % VEC == 0))
        multiaxpy_kernel<T, VEC><<<grid_resident(multiaxpy_kernel<T, VEC>, (n + VEC - 1) / VEC), VT, 0, s>>>(
            n, w, V, ld, m, h, scale);
    else
        multiaxpy_kernel<T, 1><<<grid_resident(multiaxpy_kernel<T, 1>, n), VT, 0, s>>>(n, w, V, ld, m, h, scale);
    return int(cudaGetLastError());
}

int vec_multidot(int64_t n, int vprec, const void* V, int64_t ld, int m, int wprec, const void* w,
                 double* out, int self_norm, cudaStream_t s) {
    const int mo = m + (self_norm ? 1 : 0);
    if (mo <= 0) return 0;
    if (m < 0 || m > MAXV || vprec != wprec) return int(cudaErrorInvalidValue);
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * mo, s);
    if (e != cudaSuccess) return int(e);
    if (vprec == 1)
        return multidot_t(n, static_cast<const float*>(V), ld, m, static_cast<const float*>(w), out, self_norm != 0, s);
    return multidot_t(n, static_cast<const double*>(V), ld, m, static_cast<const double*>(w), out, self_norm != 0, s);
}

int vec_multiaxpy(int64_t n, int prec, void* w, const void* V, int64_t ld, int m, const double* h, double scale,
                  double* dots, cudaStream_t s) {
    if (m < 0 || m > MAXV) return int(cudaErrorInvalidValue);
    // the dots of the updated w are a second pass (a multi-dot with its norm):
    // two bandwidth-bound sweeps measured faster than one sweep that holds
    // all m values of V per thread for the dots
    int e = prec == 1 ? multiaxpy_t(n, static_cast<float*>(w), static_cast<const float*>(V), ld, m, h, scale, s)
                      : multiaxpy_t(n, static_cast<double*>(w), static_cast<const double*>(V), ld, m, h, scale, s);
    if (e || !dots) return e;
    return vec_multidot(n, prec, V, ld, m, prec, w, dots, 1, s);
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
