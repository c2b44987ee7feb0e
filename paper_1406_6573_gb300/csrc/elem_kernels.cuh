// Sum-factorised element kernels of the nonlinear Stokes operator (sm_103a):
// shared layout, tables and device helpers.
//
// One thread owns one (i, j) column of GLL nodes / Gauss points of an element
// and loops over the third index l: contractions along zeta run in registers,
// contractions along xi and eta exchange through shared memory (Section 3.3:
// every element operation is a sequence of 1-D kernels).  The N1^2 threads of
// an element always sit in one warp (EPW = 32 / N1^2 elements per warp), so
// every exchange is warp-synchronous: there is no block-wide barrier in the
// element loop and each warp streams through its own element groups.
// Per element:
//   gather (R_i: global node per slot, basal projector P, hanging-node 1-D
//   interpolation) -> reference gradients at the Gauss points (3 interpolation
//   sweeps + 3 collocated derivative sweeps per field) -> pointwise physics
//   (Glen viscosity Eq. 2.2, Newton tensor Eq. 2.7, pressure / divergence
//   terms of Eq. 2.5) -> transposed sweeps -> R_i^T -> atomic scatter-add.
// Each translation unit includes this header with STOKES_K defined and gets
// its own constant-memory tables for that degree.
#pragma once

#include <cuda_runtime.h>

#include "common.h"
#include "hanging.h"
#include "kernels.h"

#ifndef STOKES_K
#error "STOKES_K must be defined before including elem_kernels.cuh"
#endif

// Every degree lives in its own namespace: the kernels, device helpers and
// constant tables of different degrees share names and must not be merged
// across translation units by the linker.
#define STOKES_NS_CAT(a, b) a##b
#define STOKES_NS_NAME(k) STOKES_NS_CAT(degree, k)
#define STOKES_NS STOKES_NS_NAME(STOKES_K)

namespace stokes {
namespace dev {
namespace STOKES_NS {

constexpr int K = STOKES_K;
constexpr int N1 = K + 1;
constexpr int Q = N1;
constexpr int N2 = N1 * N1;
constexpr int N3 = N1 * N1 * N1;
constexpr int Q3 = N3;
constexpr int WARPS = 8;
constexpr int THREADS = 32 * WARPS;
constexpr int EPW = 32 / N2;          // elements per warp
constexpr int EPB = WARPS * EPW;      // elements per block (face kernels)
// warps per block of the generic element kernel: fewer in FP64 so that the
// static exchange buffers stay within 48 KB
template <typename T> constexpr int GW = sizeof(T) == 8 ? 4 : 8;
static_assert(EPW >= 1, "an element's columns must fit in one warp");
// padded length of a contraction line in shared memory: a 16-byte multiple,
// so that one line is read with vector loads
template <typename T> struct LineLen { static constexpr int v = (N1 + (16 / int(sizeof(T))) - 1) / (16 / int(sizeof(T))) * (16 / int(sizeof(T))); };
template <typename T> constexpr int LP = LineLen<T>::v;
// one exchange buffer holds an N1 x N1 x N1 tensor as N1^2 padded lines
template <typename T> constexpr int BUFLEN = LP<T> * N2;
constexpr int NPRK = (K - 1) * (K - 1) * (K - 1) > K * (K + 1) * (K + 2) / 6
                         ? (K - 1) * (K - 1) * (K - 1) : K * (K + 1) * (K + 2) / 6;
// Per-element block of the linearised state: 2 element constants, a shift
// of STATE_SHIFT(e) values, STATE_FIELDS values per quadrature point, padding
// to a 16-byte multiple.  The stride and the shift place the q^2 values that
// the lanes of a warp's EPW elements read together on distinct shared-memory
// banks once a group of blocks is staged: for EPW = 3 (k = 2) the shift is 1
// for the first two elements of each group (windows at banks 3, 15 and 26
// mod 32); for EPW = 2 (k = 3) the stride is 16 mod 32.
constexpr int STATE_USED = 2 + STATE_FIELDS * Q3;
constexpr int sstride_calc() {
    int s = (STATE_USED + 1 + 3) / 4 * 4;
    if (EPW == 2)
        while (s % 32 != 16) s += 4;
    return s;
}
constexpr int SSTRIDE = sstride_calc();
__host__ __device__ constexpr int state_shift(int64_t e) { return (EPW == 3 && e % 3 != 2) ? 1 : 0; }

// ---------------------------------------------------------------- tables
__constant__ double cB[Q][N1];        // GLL Lagrange at Gauss points
__constant__ double cDg[Q][Q];        // Gauss collocation derivative
__constant__ double cI[2][N1][N1];    // hanging interpolation, per half
__constant__ double cP1[2][Q][N1];    // pressure 1-D factors [pspace][iq][a]
__constant__ int cPm[2][NPRK > 0 ? NPRK : 1][3];
__constant__ int cNpr[2];
__constant__ float fB[Q][N1];
__constant__ float fDg[Q][Q];
__constant__ float fI[2][N1][N1];
__constant__ float fP1[2][Q][N1];
__constant__ double cBd[Q][N1];       // (Dg B)[iq][i]: derivative of GLL Lagrange i at Gauss point iq
__constant__ float fBd[Q][N1];
#if STOKES_K == 2
// pressure basis at the Gauss points, psi_b(qp) [pspace][mode][qp]
__constant__ float fPsi[2][NPRK][Q3];
#endif

template <typename T> struct Tab;
template <> struct Tab<double> {
    static __device__ __forceinline__ double B(int a, int b) { return cB[a][b]; }
    static __device__ __forceinline__ double Dg(int a, int b) { return cDg[a][b]; }
    static __device__ __forceinline__ double I(int h, int a, int b) { return cI[h][a][b]; }
    static __device__ __forceinline__ double P1(int s, int a, int b) { return cP1[s][a][b]; }
    static __device__ __forceinline__ double Bd(int a, int b) { return cBd[a][b]; }
};
template <> struct Tab<float> {
    static __device__ __forceinline__ float B(int a, int b) { return fB[a][b]; }
    static __device__ __forceinline__ float Dg(int a, int b) { return fDg[a][b]; }
    static __device__ __forceinline__ float I(int h, int a, int b) { return fI[h][a][b]; }
    static __device__ __forceinline__ float P1(int s, int a, int b) { return fP1[s][a][b]; }
    static __device__ __forceinline__ float Bd(int a, int b) { return fBd[a][b]; }
};

// Table entries whose index depends on the thread's (i, j): loaded once into
// registers (constant-cache reads with divergent addresses would serialise).
template <typename T> struct Rows {
    T Bi[N1], Bj[N1];      // B[i][m], B[j][m]
    T BTi[Q], BTj[Q];      // B[m][i], B[m][j]
    T Ti[N1], Tj[N1];      // (Dg B)[i][m], (Dg B)[j][m]: derivative of the nodal interpolant
    T DTi[Q], DTj[Q];      // Dg[m][i], Dg[m][j]
    __device__ __forceinline__ void load(int i, int j) {
        #pragma unroll
        for (int m = 0; m < N1; ++m) {
            Bi[m] = Tab<T>::B(i, m); Bj[m] = Tab<T>::B(j, m);
            T si = 0, sj = 0;
            #pragma unroll
            for (int p = 0; p < Q; ++p) { si += Tab<T>::Dg(i, p) * Tab<T>::B(p, m); sj += Tab<T>::Dg(j, p) * Tab<T>::B(p, m); }
            Ti[m] = si; Tj[m] = sj;
        }
        #pragma unroll
        for (int m = 0; m < Q; ++m) {
            BTi[m] = Tab<T>::B(m, i); BTj[m] = Tab<T>::B(m, j);
            DTi[m] = Tab<T>::Dg(m, i); DTj[m] = Tab<T>::Dg(m, j);
        }
    }
};

// Group layout of the FP32 state of conforming k = 2 meshes (read by the
// component-per-lane apply): groups of CPL_E consecutive elements, each a
// header (the 2 element constants of the group's elements, padded) and one
// block per Gauss plane lq holding, field by field, the 9 points of the plane
// of each of the CPL_E elements ([f][element][q9], plane padded to a 16-byte
// multiple: the reads of a warp, three fields at a time, fall on distinct
// shared-memory banks).  A group is one contiguous 16-byte-multiple block.
constexpr int CPL_E = 10;
constexpr int CPL_HDR = 24;
constexpr int CPL_FS = N2 * CPL_E;                                 // values per field and plane
constexpr int CPL_PL = (STATE_FIELDS * CPL_FS + 3) / 4 * 4;       // values per plane
constexpr int CPL_GROUP = CPL_HDR + N1 * CPL_PL;                   // values per group
static_assert(K != 2 || (CPL_E == CPL_GROUP_ELEMS && CPL_GROUP == CPL_GROUP_VALUES), "group layout of k = 2");

// Linearised-state slots of element e, with the layout arithmetic done once:
// the element constants s = 0, 1 and field f at the Gauss point q9 + N2 lq
// (q9 = i + N1 j).  Element-major [E][SSTRIDE] layout (constants, shift
// slot, then field-major q^3 values), or the group layout above (cpl != 0).
struct StateRef {
    int64_t c0, f0;       // slot of constant 0, of field 0 at point 0
    int cstride;          // between the two constants
    int fstride, lstride; // between fields, between Gauss planes
    __device__ __forceinline__ StateRef(int64_t e, int cpl) {
        if (cpl) {
            const int64_t gg = e / CPL_E;
            const int el = int(e - gg * CPL_E);
            c0 = gg * CPL_GROUP + el;
            cstride = CPL_E;
            f0 = gg * CPL_GROUP + CPL_HDR + el * N2;
            fstride = CPL_FS;
            lstride = CPL_PL;
        } else {
            c0 = e * SSTRIDE;
            cstride = 1;
            f0 = e * SSTRIDE + 2 + state_shift(e);
            fstride = Q3;
            lstride = N2;
        }
    }
    __device__ __forceinline__ int64_t c(int s) const { return c0 + s * cstride; }
    __device__ __forceinline__ int64_t f(int field, int lq, int q9) const {
        return f0 + field * fstride + lq * lstride + q9;
    }
};

// --------------------------------------------------------------- helpers
template <typename T> __device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

__device__ __forceinline__ void atomic_add(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add(float* p, float v) { atomicAdd(p, v); }

__device__ __forceinline__ void wsync() { __syncwarp(); }

// Viscosity mu = C (gamma s + delta)^p_n, s = D:D; special-cased for n = 3.
template <typename T>
__device__ __forceinline__ T viscosity(const ElemArgs& a, T DD) {
    T arg = T(a.gamma) * DD + T(a.delta);
    if (a.n_is_3) return T(a.C) * rcbrt_t(arg);
    return T(a.C) * pow(arg, T(a.pexp));
}

// Lane layout of a warp: EPW element slots of N2 lanes; idle lanes form slot EPW.
struct LaneMap {
    int warp, lane, es, ij, i, j;
    __device__ __forceinline__ LaneMap() {
        warp = threadIdx.x >> 5;
        lane = threadIdx.x & 31;
        es = lane / N2;
        if (es > EPW) es = EPW;
        ij = lane - es * N2;
        i = ij % N1;
        j = ij / N1;
    }
};

// slot / qp index within the element tensor: (i, j, l) -> i + N1 (j + N1 l)
__device__ __forceinline__ int sidx(int i, int j, int l) { return i + N1 * (j + N1 * l); }

// ----------------------------------------------------- hanging sweeps
// Forward R_i interpolation on the element tensor held as columns v[c][l]
// (thread (i, j)); sb is the element's shared scratch (N3 values).
template <typename T, int NC>
__device__ void hanging_forward(T (&v)[NC][N1], uint32_t h, bool active, int i, int j, T* sb) {
    for (int c = 0; c < NC; ++c) {
        // x-sweeps: lines parallel to x at (j, l)
        #pragma unroll
        for (int l = 0; l < N1; ++l) sb[sidx(i, j, l)] = v[c][l];
        wsync();
        if (active && h) {
            const int bx = child_bit(h, 0);
            #pragma unroll
            for (int l = 0; l < N1; ++l) {
                if (line_hanging(h, 0, j, l, K)) {
                    T s = 0;
                    #pragma unroll
                    for (int m = 0; m < N1; ++m) s += Tab<T>::I(bx, i, m) * sb[sidx(m, j, l)];
                    v[c][l] = s;
                }
            }
        }
        wsync();
        // y-sweeps: lines parallel to y at (i, l)
        #pragma unroll
        for (int l = 0; l < N1; ++l) sb[sidx(i, j, l)] = v[c][l];
        wsync();
        if (active && h) {
            const int by = child_bit(h, 1);
            #pragma unroll
            for (int l = 0; l < N1; ++l) {
                if (line_hanging(h, 1, i, l, K)) {
                    T s = 0;
                    #pragma unroll
                    for (int m = 0; m < N1; ++m) s += Tab<T>::I(by, j, m) * sb[sidx(i, m, l)];
                    v[c][l] = s;
                }
            }
        }
        wsync();
        // z-sweeps: the thread's own column (registers)
        if (active && h && line_hanging(h, 2, i, j, K)) {
            const int bz = child_bit(h, 2);
            T t[N1];
            #pragma unroll
            for (int l = 0; l < N1; ++l) {
                T s = 0;
                #pragma unroll
                for (int m = 0; m < N1; ++m) s += Tab<T>::I(bz, l, m) * v[c][m];
                t[l] = s;
            }
            #pragma unroll
            for (int l = 0; l < N1; ++l) v[c][l] = t[l];
        }
    }
}

// Transposed R_i interpolation (z^T, then y^T, then x^T).
template <typename T, int NC>
__device__ void hanging_transpose(T (&v)[NC][N1], uint32_t h, bool active, int i, int j, T* sb) {
    for (int c = 0; c < NC; ++c) {
        if (active && h && line_hanging(h, 2, i, j, K)) {
            const int bz = child_bit(h, 2);
            T t[N1];
            #pragma unroll
            for (int m = 0; m < N1; ++m) {
                T s = 0;
                #pragma unroll
                for (int l = 0; l < N1; ++l) s += Tab<T>::I(bz, l, m) * v[c][l];
                t[m] = s;
            }
            #pragma unroll
            for (int l = 0; l < N1; ++l) v[c][l] = t[l];
        }
        #pragma unroll
        for (int l = 0; l < N1; ++l) sb[sidx(i, j, l)] = v[c][l];
        wsync();
        if (active && h) {
            const int by = child_bit(h, 1);
            #pragma unroll
            for (int l = 0; l < N1; ++l) {
                if (line_hanging(h, 1, i, l, K)) {
                    T s = 0;
                    #pragma unroll
                    for (int m = 0; m < N1; ++m) s += Tab<T>::I(by, m, j) * sb[sidx(i, m, l)];
                    v[c][l] = s;
                }
            }
        }
        wsync();
        #pragma unroll
        for (int l = 0; l < N1; ++l) sb[sidx(i, j, l)] = v[c][l];
        wsync();
        if (active && h) {
            const int bx = child_bit(h, 0);
            #pragma unroll
            for (int l = 0; l < N1; ++l) {
                if (line_hanging(h, 0, j, l, K)) {
                    T s = 0;
                    #pragma unroll
                    for (int m = 0; m < N1; ++m) s += Tab<T>::I(bx, m, i) * sb[sidx(m, j, l)];
                    v[c][l] = s;
                }
            }
        }
        wsync();
    }
}

// ----------------------------------------------- sum-factorised gradient
// Exchange buffers hold the element tensor as padded lines; the layout of
// each buffer puts the direction of the next contraction fastest, so that a
// thread reads a whole line with 16-byte vector loads:
//   X layout  xl(i, j, l) = i + LP (j + N1 l)   (xi-lines contiguous)
//   Y layout  yl(i, j, l) = j + LP (i + N1 l)   (eta-lines contiguous)
template <typename T> __device__ __forceinline__ int xl(int i, int j, int l) { return i + LP<T> * (j + N1 * l); }
template <typename T> __device__ __forceinline__ int yl(int i, int j, int l) { return j + LP<T> * (i + N1 * l); }

template <typename T>
__device__ __forceinline__ void load_line(const T* p, T (&o)[N1]) {
    if constexpr (sizeof(T) == 4) {
        #pragma unroll
        for (int k = 0; k < N1; k += 4) {
            const float4 v = *reinterpret_cast<const float4*>(p + k);
            o[k] = v.x;
            if (k + 1 < N1) o[k + 1] = v.y;
            if (k + 2 < N1) o[k + 2] = v.z;
            if (k + 3 < N1) o[k + 3] = v.w;
        }
    } else {
        #pragma unroll
        for (int k = 0; k < N1; k += 2) {
            const double2 v = *reinterpret_cast<const double2*>(p + k);
            o[k] = v.x;
            if (k + 1 < N1) o[k + 1] = v.y;
        }
    }
}

// value v held by the thread of slot (i2, j2) of this thread's element (the
// element's N1^2 threads are consecutive lanes; idle lanes read any lane)
template <typename T>
__device__ __forceinline__ T lane_val(T v, int i2, int j2) {
    const int base = ((threadIdx.x & 31) / N2) * N2;
    return __shfl_sync(0xffffffffu, v, base + i2 + N1 * j2);
}

// Line layouts and loads for a line pitch P (values between consecutive
// lines): the padded pitch LP<T> allows one 16-byte load per line; the packed
// pitch N1 puts the N1^2 lanes of an element on consecutive banks (no store
// conflicts between the elements of a warp) at one scalar load per value.
template <int P> __device__ __forceinline__ int xlp(int i, int j, int l) { return i + P * (j + N1 * l); }
template <int P> __device__ __forceinline__ int ylp(int i, int j, int l) { return j + P * (i + N1 * l); }
template <typename T, int P>
__device__ __forceinline__ void load_line_p(const T* p, T (&o)[N1]) {
    if constexpr (P == LP<T>) {
        load_line<T>(p, o);
    } else {
        #pragma unroll
        for (int k = 0; k < N1; ++k) o[k] = p[k];
    }
}

// Reference gradients at the Gauss points (iq = i, jq = j, lq) of the NC
// fields whose nodal columns the thread holds in vin:
//   zeta: interpolate (registers);  eta: interpolate and differentiate the
//   eta-line through the thread's node column (values from the lanes of that
//   line);  xi: interpolate and differentiate the interpolated xi-line and
//   interpolate the eta-derivative line;  zeta derivative by collocation.
// The lines are exchanged with warp shuffles; buf is not used.
template <typename T, int NC>
__device__ __forceinline__ void ref_gradient(const Rows<T>& R, const T (&vin)[NC][N1], T (&G)[NC][3][Q],
                                             int i, int j, T* /*buf*/) {
    #pragma unroll
    for (int c = 0; c < NC; ++c) {
        T a[Q];
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {
            T s = 0;
            #pragma unroll
            for (int l = 0; l < N1; ++l) s += Tab<T>::B(lq, l) * vin[c][l];
            T si = 0, sd = 0;                         // thread (node i, jq = j)
            #pragma unroll
            for (int m = 0; m < N1; ++m) {
                const T x = lane_val(s, i, m);
                si += R.Bj[m] * x;
                sd += R.Tj[m] * x;
            }
            T sv = 0, sx = 0, sy = 0;                 // thread (iq = i, jq = j)
            #pragma unroll
            for (int m = 0; m < N1; ++m) {
                const T x1 = lane_val(si, m, j);
                const T x2 = lane_val(sd, m, j);
                sv += R.Bi[m] * x1;
                sx += R.Ti[m] * x1;
                sy += R.Bi[m] * x2;
            }
            a[lq] = sv; G[c][0][lq] = sx; G[c][1][lq] = sy;
        }
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {          // zeta derivative, collocated
            T s = 0;
            #pragma unroll
            for (int m = 0; m < Q; ++m) s += Tab<T>::Dg(lq, m) * a[m];
            G[c][2][lq] = s;
        }
    }
}

// Transposed gradients: nodal columns out[c][l] of
//   sum_qp (d phi/d xi) S[c][0] + (d phi/d eta) S[c][1] + (d phi/d zeta) S[c][2] + phi Sv[c]
// (collocated derivative transposes at the Gauss points, then the three
// transposed interpolations); lines exchanged with warp shuffles.
template <typename T, int NC, bool HAS_VAL>
__device__ __forceinline__ void ref_gradient_T(const Rows<T>& R, const T (&S)[NC][3][Q], const T (&Sv)[NC][Q],
                                               T (&out)[NC][N1], int i, int j, T* /*buf*/) {
    #pragma unroll
    for (int c = 0; c < NC; ++c) {
        T t[Q];
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {
            T z = HAS_VAL ? Sv[c][lq] : T(0);
            #pragma unroll
            for (int m = 0; m < Q; ++m) z += Tab<T>::Dg(m, lq) * S[c][2][m];
            T s = z;                                  // thread (iq = i, jq = j)
            #pragma unroll
            for (int m = 0; m < Q; ++m)
                s += R.DTi[m] * lane_val(S[c][0][lq], m, j) + R.DTj[m] * lane_val(S[c][1][lq], i, m);
            T u = 0;                                  // xi^T: thread (node i, jq = j)
            #pragma unroll
            for (int m = 0; m < Q; ++m) u += R.BTi[m] * lane_val(s, m, j);
            T v = 0;                                  // eta^T: thread (node i, node j)
            #pragma unroll
            for (int m = 0; m < Q; ++m) v += R.BTj[m] * lane_val(u, i, m);
            t[lq] = v;
        }
        #pragma unroll
        for (int l = 0; l < N1; ++l) {            // zeta^T
            T s = 0;
            #pragma unroll
            for (int lq = 0; lq < Q; ++lq) s += Tab<T>::B(lq, l) * t[lq];
            out[c][l] = s;
        }
    }
}
// Shared-memory exchange variants of ref_gradient / ref_gradient_T (used by
// the stored-state kernel, where they measured faster than the shuffles;
// the generic element kernel uses the shuffle variants).  The idle lanes of a
// warp (32 mod N1^2) do not store: their slot would share banks with the
// first element's; what they load is never used.
// Reference gradients at the Gauss points (iq = i, jq = j, lq) of the NC
// fields whose nodal columns the thread holds in vin, all fields advancing
// through each stage together (independent chains between warp syncs):
//   zeta: interpolate (registers);  eta: interpolate and differentiate the
//   same line;  xi: interpolate and differentiate the interpolated line, and
//   interpolate the eta-derivative line;  zeta derivative by collocation.
// buf: 3 NC exchange buffers of BUFLEN values.
template <typename T, int NC, int P = LP<T>>
__device__ __forceinline__ void ref_gradient_smem(const Rows<T>& R, const T (&vin)[NC][N1], T (&G)[NC][3][Q],
                                             int i, int j, T* buf) {
    const bool live = (threadIdx.x & 31) < EPW * N2;   // lanes of the warp's elements
    #pragma unroll
    for (int c = 0; c < NC; ++c) {
        T* b0 = buf + (3 * c) * P * N2;
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {
            T s = 0;
            #pragma unroll
            for (int l = 0; l < N1; ++l) s += Tab<T>::B(lq, l) * vin[c][l];
            if (live) b0[ylp<P>(i, j, lq)] = s;
        }
    }
    wsync();
    #pragma unroll
    for (int c = 0; c < NC; ++c) {              // eta: thread (node i, jq = j)
        const T* b0 = buf + (3 * c) * P * N2;
        T* b1 = buf + (3 * c + 1) * P * N2;
        T* b2 = buf + (3 * c + 2) * P * N2;
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {
            T ln[N1];
            load_line_p<T, P>(b0 + ylp<P>(i, 0, lq), ln);
            T si = 0, sd = 0;
            #pragma unroll
            for (int m = 0; m < N1; ++m) { si += R.Bj[m] * ln[m]; sd += R.Tj[m] * ln[m]; }
            if (live) b1[xlp<P>(i, j, lq)] = si;
            if (live) b2[xlp<P>(i, j, lq)] = sd;
        }
    }
    wsync();
    #pragma unroll
    for (int c = 0; c < NC; ++c) {              // xi: thread (iq = i, jq = j)
        const T* b1 = buf + (3 * c + 1) * P * N2;
        const T* b2 = buf + (3 * c + 2) * P * N2;
        T a[Q];
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {
            T l1[N1], l2[N1];
            load_line_p<T, P>(b1 + xlp<P>(0, j, lq), l1);
            load_line_p<T, P>(b2 + xlp<P>(0, j, lq), l2);
            T sv = 0, sx = 0, sy = 0;
            #pragma unroll
            for (int m = 0; m < N1; ++m) { sv += R.Bi[m] * l1[m]; sx += R.Ti[m] * l1[m]; sy += R.Bi[m] * l2[m]; }
            a[lq] = sv; G[c][0][lq] = sx; G[c][1][lq] = sy;
        }
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {        // zeta derivative, collocated
            T s = 0;
            #pragma unroll
            for (int m = 0; m < Q; ++m) s += Tab<T>::Dg(lq, m) * a[m];
            G[c][2][lq] = s;
        }
    }
    wsync();
}

// Transposed gradients: nodal columns out[c][l] of
//   sum_qp (d phi/d xi) S[c][0] + (d phi/d eta) S[c][1] + (d phi/d zeta) S[c][2] + phi Sv[c]
// (collocated derivative transposes at the Gauss points, then the three
// transposed interpolations), NC fields advancing together.
template <typename T, int NC, bool HAS_VAL, int P = LP<T>>
__device__ __forceinline__ void ref_gradient_T_smem(const Rows<T>& R, const T (&S)[NC][3][Q], const T (&Sv)[NC][Q],
                                               T (&out)[NC][N1], int i, int j, T* buf) {
    const bool live = (threadIdx.x & 31) < EPW * N2;   // lanes of the warp's elements
    T t[NC][Q];
    #pragma unroll
    for (int c = 0; c < NC; ++c) {
        T* b0 = buf + (3 * c) * P * N2;
        T* b1 = buf + (3 * c + 1) * P * N2;
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {
            if (live) b0[xlp<P>(i, j, lq)] = S[c][0][lq];
            if (live) b1[ylp<P>(i, j, lq)] = S[c][1][lq];
            T s = HAS_VAL ? Sv[c][lq] : T(0);
            #pragma unroll
            for (int m = 0; m < Q; ++m) s += Tab<T>::Dg(m, lq) * S[c][2][m];
            t[c][lq] = s;
        }
    }
    wsync();
    #pragma unroll
    for (int c = 0; c < NC; ++c) {
        const T* b0 = buf + (3 * c) * P * N2;
        const T* b1 = buf + (3 * c + 1) * P * N2;
        T* b2 = buf + (3 * c + 2) * P * N2;
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {
            T lx[N1], ly[N1];
            load_line_p<T, P>(b0 + xlp<P>(0, j, lq), lx);
            load_line_p<T, P>(b1 + ylp<P>(i, 0, lq), ly);
            T s = t[c][lq];
            #pragma unroll
            for (int m = 0; m < Q; ++m) s += R.DTi[m] * lx[m] + R.DTj[m] * ly[m];
            if (live) b2[xlp<P>(i, j, lq)] = s;
        }
    }
    wsync();
    #pragma unroll
    for (int c = 0; c < NC; ++c) {              // xi^T: thread (node i, jq = j)
        const T* b2 = buf + (3 * c + 2) * P * N2;
        T* b0 = buf + (3 * c) * P * N2;
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {
            T ln[N1];
            load_line_p<T, P>(b2 + xlp<P>(0, j, lq), ln);
            T s = 0;
            #pragma unroll
            for (int m = 0; m < Q; ++m) s += R.BTi[m] * ln[m];
            if (live) b0[ylp<P>(i, j, lq)] = s;
        }
    }
    wsync();
    #pragma unroll
    for (int c = 0; c < NC; ++c) {              // eta^T then zeta^T
        const T* b0 = buf + (3 * c) * P * N2;
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {
            T ln[N1];
            load_line_p<T, P>(b0 + ylp<P>(i, 0, lq), ln);
            T s = 0;
            #pragma unroll
            for (int m = 0; m < Q; ++m) s += R.BTj[m] * ln[m];
            t[c][lq] = s;
        }
        #pragma unroll
        for (int l = 0; l < N1; ++l) {
            T s = 0;
            #pragma unroll
            for (int lq = 0; lq < Q; ++lq) s += Tab<T>::B(lq, l) * t[c][lq];
            out[c][l] = s;
        }
    }
    wsync();
}


// ------------------------------------------------------------ gather
template <typename T>
__device__ __forceinline__ void project3(const double* P, T& x0, T& x1, T& x2) {
    const T p00 = T(P[0]), p11 = T(P[N2]), p22 = T(P[2 * N2]);
    const T p01 = T(P[3 * N2]), p02 = T(P[4 * N2]), p12 = T(P[5 * N2]);
    const T a = x0, b = x1, c = x2;
    x0 = p00 * a + p01 * b + p02 * c;
    x1 = p01 * a + p11 * b + p12 * c;
    x2 = p02 * a + p12 * b + p22 * c;
}

// Global nodes of the thread's column of slots (ij, l = 0..N1-1) of element e:
// read from the element map, or computed from the lattice on conforming
// meshes (node I + NX (J + NY L); no map read).  Filled once per element and
// shared by the gather and the scatter.
struct ColNodes {
    int32_t g[N1];
};

__device__ __forceinline__ void col_nodes(const ElemArgs& a, int64_t e, int ij, bool active, ColNodes& cn) {
    if (!active) {
        #pragma unroll
        for (int l = 0; l < N1; ++l) cn.g[l] = 0;
        return;
    }
    if (a.lat_nx > 0) {
        const int e32 = int(e), nx = int(a.lat_nx), ny = int(a.lat_ny);
        const int ex = e32 % nx, r = e32 / nx;
        const int ey = r % ny, ez = r / ny;
        int I = ex * K + ij % N1, J = ey * K + ij / N1;
        const int NX = int(a.lat_NX), NY = int(a.lat_NY);
        if (I >= NX) I -= NX;
        if (J >= NY) J -= NY;
        const int g0 = I + NX * (J + NY * (ez * K));
        const int step = NX * NY;
        #pragma unroll
        for (int l = 0; l < N1; ++l) cn.g[l] = g0 + l * step;
    } else {
        #pragma unroll
        for (int l = 0; l < N1; ++l) cn.g[l] = a.nodes[e * N3 + ij + N2 * l];
    }
}

// Velocity columns of element e (3 components) from a state vector x,
// with the basal projector applied at bottom-plane slots.
template <typename T, typename TIN>
__device__ __forceinline__ void gather_velocity(const ElemArgs& a, const TIN* x, const ColNodes& cn, int64_t e,
                                                bool active, int ij, T (&v)[3][N1]) {
    #pragma unroll
    for (int l = 0; l < N1; ++l) {
        if (active) {
            const int64_t g = cn.g[l];
            v[0][l] = T(ld(x + 3 * g));
            v[1][l] = T(ld(x + 3 * g + 1));
            v[2][l] = T(ld(x + 3 * g + 2));
        } else {
            v[0][l] = v[1][l] = v[2][l] = T(0);
        }
    }
    if (active) {
        const int pi = a.pidx[e];
        if (pi >= 0) project3<T>(a.pel + int64_t(pi) * 6 * N2 + ij, v[0][0], v[1][0], v[2][0]);
    }
}

template <typename T>
__device__ __forceinline__ void scatter_velocity(const ElemArgs& a, T* y, const ColNodes& cn, int64_t e, bool active,
                                                 int ij, T (&v)[3][N1]) {
    if (!active) return;
    const int pi = a.pidx[e];
    if (pi >= 0) project3<T>(a.pel + int64_t(pi) * 6 * N2 + ij, v[0][0], v[1][0], v[2][0]);
    #pragma unroll
    for (int l = 0; l < N1; ++l) {
        const int64_t g = cn.g[l];
        atomic_add(y + 3 * g, v[0][l]);
        atomic_add(y + 3 * g + 1, v[1][l]);
        atomic_add(y + 3 * g + 2, v[2][l]);
    }
}

// Discontinuous pressure of the element folded per thread: pc[c] =
// sum_{modes b with zeta factor c} p_b f_b(i) g_b(j), so that the pressure at
// Gauss point (i, j, lq) is sum_c P1[lq][c] pc[c] (uniform table reads).
template <typename T, typename TIN>
__device__ __forceinline__ void pressure_fold(const ElemArgs& a, const TIN* x, int64_t e, bool active, int i, int j,
                                              T (&pc)[N1]) {
    const int ps = a.pspace;
    #pragma unroll
    for (int c = 0; c < N1; ++c) pc[c] = T(0);
    if (!active) return;
    const TIN* pe = x + 3 * a.Nv + e * a.npr;
    #pragma unroll
    for (int b = 0; b < NPRK; ++b) {
        if (b < a.npr) {
            const T f = Tab<T>::P1(ps, i, cPm[ps][b][0]) * Tab<T>::P1(ps, j, cPm[ps][b][1]);
            const T pb = T(ld(pe + b)) * f;
            const int cz = cPm[ps][b][2];
            #pragma unroll
            for (int c = 0; c < N1; ++c) if (c == cz) pc[c] += pb;
        }
    }
}

template <typename T>
__device__ __forceinline__ T pressure_at(const T (&pc)[N1], int ps, int lq) {
    T s = 0;
    #pragma unroll
    for (int c = 0; c < N1; ++c) s += Tab<T>::P1(ps, lq, c) * pc[c];
    return s;
}

// Pressure rows: dst[b] = sum_qp psi_b(qp) gq(qp), reduced over the element's
// lanes through the element's shared scratch (3 N3 values) in chunks.
template <typename T>
__device__ void pressure_rows(const T (&gq)[Q], int npr, int ps, int i, int j, int ij, bool active,
                              T* sb, T* dst) {
    constexpr int CH = (3 * N3) / N2;   // rows per chunk
    T h[N1];                            // sum_lq P1[lq][c] gq[lq]
    #pragma unroll
    for (int c = 0; c < N1; ++c) {
        T s = 0;
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) s += Tab<T>::P1(ps, lq, c) * gq[lq];
        h[c] = s;
    }
    for (int b0 = 0; b0 < npr; b0 += CH) {
        #pragma unroll
        for (int cb = 0; cb < CH; ++cb) {
            const int b = b0 + cb;
            T s = 0;
            if (b < npr) {
                const int cz = cPm[ps][b][2];
                T hz = 0;
                #pragma unroll
                for (int c = 0; c < N1; ++c) if (c == cz) hz = h[c];
                s = Tab<T>::P1(ps, i, cPm[ps][b][0]) * Tab<T>::P1(ps, j, cPm[ps][b][1]) * hz;
            }
            if ((threadIdx.x & 31) < EPW * N2) sb[cb * N2 + ij] = s;   // idle lanes do not store
        }
        wsync();
        if (active && ij < CH && b0 + ij < npr) {
            T s = 0;
            for (int t = 0; t < N2; ++t) s += sb[ij * N2 + t];
            dst[b0 + ij] = s;
        }
        wsync();
    }
}

}  // namespace STOKES_NS
}  // namespace dev
}  // namespace stokes
