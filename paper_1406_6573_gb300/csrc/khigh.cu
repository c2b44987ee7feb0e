// Element and basal-face kernels for the velocity degrees k = 5 .. 9 (the
// paper's k = 3, 6, 9 independence study, Section 5; host builder and oracle
// go to k = 9).  One element's (k+1)^2 node columns no longer fit the lanes of
// a warp, so these kernels give one block to one element (or basal face) and
// run the sum factorisation through shared memory with a run-time degree:
//   gather (R_i: element map, basal projector, hanging-node 1-D
//   interpolation) -> reference gradients at the Gauss points (zeta, eta, xi
//   sweeps with B and Bd) -> pointwise physics (Glen viscosity Eq. 2.2, Newton
//   tensor Eq. 2.7, pressure / divergence terms of Eq. 2.5) -> transposed
//   sweeps -> R_i^T -> atomic scatter-add.
// The same modes as the warp-per-element kernels of k = 2, 3, 4: residual,
// linearisation into the stored state, stored-state apply (and its pressure
// block), A-gradient; the fused Jacobian apply is a linearisation into a
// per-mesh FP64 workspace followed by a stored-state apply.  One translation
// unit for all these degrees (run-time sizes keep its compile time short).
#include <cmath>
#include <cstdint>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "common.h"
#include "handles.h"
#include "hanging.h"
#include "khigh.h"
#include "kernels.h"
#include "precond.h"

namespace stokes {

namespace {

constexpr int HT = 256;   // threads per block
constexpr int NM = N1MAX * N1MAX;

// device copy of the 1-D tables of one degree (both pressure spaces)
struct HTab {
    int k, n1, q, npr[2];
    double B[N1MAX][N1MAX];      // [q][i]: GLL Lagrange i at Gauss point q
    double Bd[N1MAX][N1MAX];     // [q][i]: its derivative at Gauss point q
    double I[2][N1MAX][N1MAX];   // hanging interpolation, per half
    double P1[2][N1MAX][N1MAX];  // [pspace][iq][a] pressure 1-D factors at Gauss points
    int pmode[2][NPRMAX][3];
};

// shared copy of the tables used in the sweeps, in the arithmetic type
template <typename T>
struct STab {
    T B[NM], Bd[NM], I[2][NM], P1[NM];
};

template <typename T>
__device__ void load_stab(const HTab* ht, int ps, STab<T>& s) {
    for (int t = threadIdx.x; t < NM; t += blockDim.x) {
        const int a = t / N1MAX, b = t % N1MAX;
        s.B[t] = T(ht->B[a][b]);
        s.Bd[t] = T(ht->Bd[a][b]);
        s.I[0][t] = T(ht->I[0][a][b]);
        s.I[1][t] = T(ht->I[1][a][b]);
        s.P1[t] = T(ht->P1[ps][a][b]);
    }
}

__device__ __forceinline__ int tix(int a, int b) { return a * N1MAX + b; }

template <typename T> __device__ __forceinline__ void atomic_add_t(T* p, T v) { atomicAdd(p, v); }

// Viscosity mu = C (gamma D:D + delta)^p_n (Eq. 2.2, reading 1)
template <typename T>
__device__ __forceinline__ T visc(const ElemArgs& a, T DD) {
    const T arg = T(a.gamma) * DD + T(a.delta);
    if (a.n_is_3) return T(a.C) / cbrt(arg);
    return T(a.C) * pow(arg, T(a.pexp));
}

// node of local slot n = i + n1 (j + n1 l) of element e
__device__ __forceinline__ int64_t node_of(const ElemArgs& a, int64_t e, int n, int k, int n1) {
    if (a.lat_nx > 0) {
        const int64_t nx = a.lat_nx, ny = a.lat_ny, NX = a.lat_NX, NY = a.lat_NY;
        const int64_t ex = e % nx, r = e / nx, ey = r % ny, ez = r / ny;
        const int i = n % n1, j = (n / n1) % n1, l = n / (n1 * n1);
        int64_t I = ex * k + i, J = ey * k + j;
        if (I >= NX) I -= NX;
        if (J >= NY) J -= NY;
        return I + NX * (J + NY * (ez * k + l));
    }
    return a.nodes[e * int64_t(n1) * n1 * n1 + n];
}

// Gather the three velocity components of element e from x into U[c * N3 + n],
// basal projector at bottom-plane slots, hanging-node interpolation (x, y, z
// sweeps of the constrained lines); tmp: N3 * 3 scratch.
template <typename T, typename TIN>
__device__ void gather(const ElemArgs& a, const TIN* x, int64_t e, int k, uint32_t h, const STab<T>& st, T* U, T* tmp) {
    const int n1 = k + 1, N2 = n1 * n1, N3 = N2 * n1;
    const int pi = a.pidx[e];
    for (int n = threadIdx.x; n < N3; n += blockDim.x) {
        const int64_t g = node_of(a, e, n, k, n1);
        T v0 = T(x[3 * g]), v1 = T(x[3 * g + 1]), v2 = T(x[3 * g + 2]);
        if (pi >= 0 && n < N2) {
            const double* P = a.pel + int64_t(pi) * 6 * N2 + n;
            const T p00 = T(P[0]), p11 = T(P[N2]), p22 = T(P[2 * N2]);
            const T p01 = T(P[3 * N2]), p02 = T(P[4 * N2]), p12 = T(P[5 * N2]);
            const T w0 = p00 * v0 + p01 * v1 + p02 * v2;
            const T w1 = p01 * v0 + p11 * v1 + p12 * v2;
            const T w2 = p02 * v0 + p12 * v1 + p22 * v2;
            v0 = w0; v1 = w1; v2 = w2;
        }
        U[n] = v0; U[N3 + n] = v1; U[2 * N3 + n] = v2;
    }
    __syncthreads();
    if ((h & ((1u << HANG_CHILD0) - 1)) == 0) return;
    // forward R_i: x-sweeps, y-sweeps, z-sweeps of the constrained lines
    for (int d = 0; d < 3; ++d) {
        const int b = child_bit(h, d);
        for (int t = threadIdx.x; t < 3 * N3; t += blockDim.x) tmp[t] = U[t];
        __syncthreads();
        for (int t = threadIdx.x; t < 3 * N3; t += blockDim.x) {
            const int c = t / N3, n = t % N3;
            const int i = n % n1, j = (n / n1) % n1, l = n / N2;
            const int pos = d == 0 ? i : (d == 1 ? j : l);
            const int A0 = d == 0 ? j : i, A1 = d == 2 ? j : l;
            if (!line_hanging(h, d, A0, A1, k)) continue;
            T s = 0;
            for (int m = 0; m < n1; ++m) {
                const int nm = d == 0 ? m + n1 * (j + n1 * l) : (d == 1 ? i + n1 * (m + n1 * l) : i + n1 * (j + n1 * m));
                s += st.I[b][tix(pos, m)] * tmp[c * N3 + nm];
            }
            U[t] = s;
        }
        __syncthreads();
    }
}

// Transposed R_i (z^T, y^T, x^T), basal projector, atomic scatter of U into y.
template <typename T>
__device__ void scatter(const ElemArgs& a, T* y, int64_t e, int k, uint32_t h, const STab<T>& st, T* U, T* tmp) {
    const int n1 = k + 1, N2 = n1 * n1, N3 = N2 * n1;
    if ((h & ((1u << HANG_CHILD0) - 1)) != 0) {
        for (int d = 2; d >= 0; --d) {
            const int b = child_bit(h, d);
            for (int t = threadIdx.x; t < 3 * N3; t += blockDim.x) tmp[t] = U[t];
            __syncthreads();
            for (int t = threadIdx.x; t < 3 * N3; t += blockDim.x) {
                const int c = t / N3, n = t % N3;
                const int i = n % n1, j = (n / n1) % n1, l = n / N2;
                const int pos = d == 0 ? i : (d == 1 ? j : l);
                const int A0 = d == 0 ? j : i, A1 = d == 2 ? j : l;
                if (!line_hanging(h, d, A0, A1, k)) continue;
                T s = 0;
                for (int m = 0; m < n1; ++m) {
                    const int nm = d == 0 ? m + n1 * (j + n1 * l) : (d == 1 ? i + n1 * (m + n1 * l) : i + n1 * (j + n1 * m));
                    s += st.I[b][tix(m, pos)] * tmp[c * N3 + nm];
                }
                U[t] = s;
            }
            __syncthreads();
        }
    }
    const int pi = a.pidx[e];
    for (int n = threadIdx.x; n < N3; n += blockDim.x) {
        T v0 = U[n], v1 = U[N3 + n], v2 = U[2 * N3 + n];
        if (pi >= 0 && n < N2) {
            const double* P = a.pel + int64_t(pi) * 6 * N2 + n;
            const T p00 = T(P[0]), p11 = T(P[N2]), p22 = T(P[2 * N2]);
            const T p01 = T(P[3 * N2]), p02 = T(P[4 * N2]), p12 = T(P[5 * N2]);
            const T w0 = p00 * v0 + p01 * v1 + p02 * v2;
            const T w1 = p01 * v0 + p11 * v1 + p12 * v2;
            const T w2 = p02 * v0 + p12 * v1 + p22 * v2;
            v0 = w0; v1 = w1; v2 = w2;
        }
        const int64_t g = node_of(a, e, n, k, n1);
        atomic_add_t(y + 3 * g, v0);
        atomic_add_t(y + 3 * g + 1, v1);
        atomic_add_t(y + 3 * g + 2, v2);
    }
    __syncthreads();
}

// Reference gradients G[(3 c + m) Q3 + qp] of the three components in U:
// m = 0: Bd_x B_y B_z, 1: B_x Bd_y B_z, 2: B_x B_y Bd_z.  Z: 2 N2 q, Y: 3 n1 q^2.
template <typename T>
__device__ void ref_grad(int k, const STab<T>& st, const T* U, T* G, T* Z, T* Y) {
    const int n1 = k + 1, q = n1, N2 = n1 * n1, N3 = N2 * n1, Q3 = q * q * q;
    const int nz = N2 * q, ny = n1 * q * q;
    for (int c = 0; c < 3; ++c) {
        const T* u = U + c * N3;
        for (int t = threadIdx.x; t < nz; t += blockDim.x) {       // [i + n1 j + N2 lq]
            const int ij = t % N2, lq = t / N2;
            T s0 = 0, s1 = 0;
            for (int l = 0; l < n1; ++l) {
                const T v = u[ij + N2 * l];
                s0 += st.B[tix(lq, l)] * v;
                s1 += st.Bd[tix(lq, l)] * v;
            }
            Z[t] = s0;
            Z[nz + t] = s1;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ny; t += blockDim.x) {       // [i + n1 jq + n1 q lq]
            const int i = t % n1, jq = (t / n1) % q, lq = t / (n1 * q);
            T s00 = 0, s10 = 0, s01 = 0;
            for (int j = 0; j < n1; ++j) {
                const int zi = i + n1 * j + N2 * lq;
                s00 += st.B[tix(jq, j)] * Z[zi];
                s10 += st.Bd[tix(jq, j)] * Z[zi];
                s01 += st.B[tix(jq, j)] * Z[nz + zi];
            }
            Y[t] = s00;
            Y[ny + t] = s10;
            Y[2 * ny + t] = s01;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < Q3; t += blockDim.x) {       // [iq + q jq + q^2 lq]
            const int iq = t % q, r = t / q;                      // r = jq + q lq
            T gx = 0, gy = 0, gz = 0;
            for (int i = 0; i < n1; ++i) {
                const int yi = i + n1 * r;
                gx += st.Bd[tix(iq, i)] * Y[yi];
                gy += st.B[tix(iq, i)] * Y[ny + yi];
                gz += st.B[tix(iq, i)] * Y[2 * ny + yi];
            }
            G[(3 * c) * Q3 + t] = gx;
            G[(3 * c + 1) * Q3 + t] = gy;
            G[(3 * c + 2) * Q3 + t] = gz;
        }
        __syncthreads();
    }
}

// Transposed gradients: U[c N3 + n] = sum_qp (Bd_x B_y B_z) G_c0 + (B_x Bd_y B_z) G_c1
// + (B_x B_y Bd_z) G_c2 + (B_x B_y B_z) Sv_c (Sv: NULL or [3 Q3]).
template <typename T>
__device__ void ref_grad_T(int k, const STab<T>& st, const T* G, const T* Sv, T* U, T* Z, T* Y) {
    const int n1 = k + 1, q = n1, N2 = n1 * n1, N3 = N2 * n1;
    const int nz = N2 * q, ny = n1 * q * q;
    for (int c = 0; c < 3; ++c) {
        const T* gx = G + (3 * c) * (q * q * q);
        const T* gy = gx + q * q * q;
        const T* gz = gy + q * q * q;
        for (int t = threadIdx.x; t < ny; t += blockDim.x) {       // xi^T: [i + n1 r], r = jq + q lq
            const int i = t % n1, r = t / n1;
            T a0 = 0, a1 = 0, a2 = 0;
            for (int iq = 0; iq < q; ++iq) {
                const int gi = iq + q * r;
                a0 += st.Bd[tix(iq, i)] * gx[gi] + (Sv ? st.B[tix(iq, i)] * Sv[c * q * q * q + gi] : T(0));
                a1 += st.B[tix(iq, i)] * gy[gi];
                a2 += st.B[tix(iq, i)] * gz[gi];
            }
            Y[t] = a0;
            Y[ny + t] = a1;
            Y[2 * ny + t] = a2;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nz; t += blockDim.x) {       // eta^T: [i + n1 j + N2 lq]
            const int i = t % n1, j = (t / n1) % n1, lq = t / N2;
            T s0 = 0, s1 = 0;
            for (int jq = 0; jq < q; ++jq) {
                const int yi = i + n1 * jq + n1 * q * lq;
                s0 += st.B[tix(jq, j)] * Y[yi] + st.Bd[tix(jq, j)] * Y[ny + yi];
                s1 += st.B[tix(jq, j)] * Y[2 * ny + yi];
            }
            Z[t] = s0;
            Z[nz + t] = s1;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < N3; t += blockDim.x) {       // zeta^T
            const int ij = t % N2, l = t / N2;
            T s = 0;
            for (int lq = 0; lq < q; ++lq)
                s += st.B[tix(lq, l)] * Z[ij + N2 * lq] + st.Bd[tix(lq, l)] * Z[nz + ij + N2 * lq];
            U[c * N3 + t] = s;
        }
        __syncthreads();
    }
}

// pressure modes of the element at the Gauss points: pq[qp] = sum_b psi_b(qp) pe[b]
template <typename T>
__device__ void pressure_at_qp(const HTab* ht, int ps, int k, const STab<T>& st, const T* pe, int npr, T* pq) {
    const int q = k + 1, Q3 = q * q * q;
    for (int t = threadIdx.x; t < Q3; t += blockDim.x) {
        const int iq = t % q, jq = (t / q) % q, lq = t / (q * q);
        T s = 0;
        for (int b = 0; b < npr; ++b) {
            const int* pm = ht->pmode[ps][b];
            s += st.P1[tix(iq, pm[0])] * st.P1[tix(jq, pm[1])] * st.P1[tix(lq, pm[2])] * pe[b];
        }
        pq[t] = s;
    }
    __syncthreads();
}

// pressure rows dst[b] = sum_qp psi_b(qp) gq[qp]
template <typename T>
__device__ void pressure_rows_high(const HTab* ht, int ps, int k, const STab<T>& st, const T* gq, int npr, T* dst) {
    const int q = k + 1, Q3 = q * q * q;
    for (int b = threadIdx.x; b < npr; b += blockDim.x) {
        const int* pm = ht->pmode[ps][b];
        T s = 0;
        for (int t = 0; t < Q3; ++t) {
            const int iq = t % q, jq = (t / q) % q, lq = t / (q * q);
            s += st.P1[tix(iq, pm[0])] * st.P1[tix(jq, pm[1])] * st.P1[tix(lq, pm[2])] * gq[t];
        }
        dst[b] = s;
    }
    __syncthreads();
}

// shared-memory carve-up of the element kernel (in units of T)
struct Carve {
    int64_t U, tmp, Z, Y, G, G2, pq, gq, pe, total;
};
// (the A-gradient keeps mu w detJ D(u), 6 values per Gauss point, in G2 and
// needs no pressure buffers; the other modes need no G2: at k = 9 in FP64
// either carve-up stays within the 227 KB of shared memory of a block)
__host__ __device__ inline Carve carve(int k, int npr, bool grad_a) {
    const int64_t n1 = k + 1, q = n1, N3 = n1 * n1 * n1, Q3 = q * q * q;
    Carve c{};
    int64_t o = 0;
    c.U = o; o += 3 * N3;
    c.tmp = o; o += 3 * N3;
    c.Z = o; o += 2 * n1 * n1 * q;
    c.Y = o; o += 3 * n1 * q * q;
    c.G = o; o += 9 * Q3;
    c.G2 = o; o += grad_a ? 6 * Q3 : 0;
    c.pq = o; o += grad_a ? 0 : Q3;
    c.gq = o; o += grad_a ? 0 : Q3;
    c.pe = o; o += grad_a ? 0 : npr;
    c.total = o;
    return c;
}

enum HMode { H_RESIDUAL = 0, H_LINEARIZE = 1, H_STATE_APPLY = 2, H_STATE_GRADP = 3, H_GRAD_A = 4, H_GRAD_A_PARTIAL = 5 };

// One block per element (grid-stride over elements).
//   T: arithmetic; S: state element type (LINEARIZE output, STATE_* input);
//   TIN: type of the gathered input vector(s)
template <typename T, typename S, typename TIN, int MODE>
__global__ void __launch_bounds__(HT) high_elem_kernel(ElemArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const HTab* ht = static_cast<const HTab*>(a.htab);
    const int k = ht->k, n1 = k + 1, q = n1, Q3 = q * q * q, ps = a.pspace, npr = a.npr;
    __shared__ STab<T> st;
    load_stab<T>(ht, ps, st);
    __syncthreads();
    const Carve cv = carve(k, npr, MODE == H_GRAD_A || MODE == H_GRAD_A_PARTIAL);
    T* sm = reinterpret_cast<T*>(smraw);
    T *U = sm + cv.U, *tmp = sm + cv.tmp, *Z = sm + cv.Z, *Y = sm + cv.Y, *G = sm + cv.G, *G2 = sm + cv.G2;
    T *pq = sm + cv.pq, *gq = sm + cv.gq, *pe = sm + cv.pe;
    const int64_t sstride = a.state_stride;
    double acc = 0.0;      // A-gradient partial of this block
    for (int64_t e = blockIdx.x; e < a.E; e += gridDim.x) {
        const uint32_t h = a.any_hang ? a.hang[e] : 0u;
        if constexpr (MODE == H_GRAD_A || MODE == H_GRAD_A_PARTIAL) {
            // pass 1: D(u) and mu(u) at the Gauss points -> G2 = mu w detJ (D00, D11,
            // D22, 2 D01, 2 D02, 2 D12); pass 2: D(lambda) . G2
            gather<T, double>(a, a.ud, e, k, h, st, U, tmp);
            ref_grad<T>(k, st, U, G, Z, Y);
            for (int t = threadIdx.x; t < Q3; t += blockDim.x) {
                const double* gp = a.geo + e * 10 * Q3 + t;
                T Ji[9];
                for (int f = 0; f < 9; ++f) Ji[f] = T(gp[f * Q3]);
                const T wdj = T(gp[9 * Q3]);
                T g[3][3];
                for (int c = 0; c < 3; ++c)
                    for (int d = 0; d < 3; ++d)
                        g[c][d] = G[(3 * c) * Q3 + t] * Ji[d] + G[(3 * c + 1) * Q3 + t] * Ji[3 + d] +
                                  G[(3 * c + 2) * Q3 + t] * Ji[6 + d];
                const T D00 = g[0][0], D11 = g[1][1], D22 = g[2][2];
                const T D01 = T(0.5) * (g[0][1] + g[1][0]), D02 = T(0.5) * (g[0][2] + g[2][0]), D12 = T(0.5) * (g[1][2] + g[2][1]);
                const T DD = D00 * D00 + D11 * D11 + D22 * D22 + T(2) * (D01 * D01 + D02 * D02 + D12 * D12);
                const T mw = visc<T>(a, DD) * wdj;
                G2[t] = mw * D00; G2[Q3 + t] = mw * D11; G2[2 * Q3 + t] = mw * D22;
                G2[3 * Q3 + t] = T(2) * mw * D01; G2[4 * Q3 + t] = T(2) * mw * D02; G2[5 * Q3 + t] = T(2) * mw * D12;
            }
            __syncthreads();
            gather<T, double>(a, a.lam, e, k, h, st, U, tmp);
            ref_grad<T>(k, st, U, G, Z, Y);
            for (int t = threadIdx.x; t < Q3; t += blockDim.x) {
                const double* gp = a.geo + e * 10 * Q3 + t;
                T Ji[9];
                for (int f = 0; f < 9; ++f) Ji[f] = T(gp[f * Q3]);
                T g[3][3];
                for (int c = 0; c < 3; ++c)
                    for (int d = 0; d < 3; ++d)
                        g[c][d] = G[(3 * c) * Q3 + t] * Ji[d] + G[(3 * c + 1) * Q3 + t] * Ji[3 + d] +
                                  G[(3 * c + 2) * Q3 + t] * Ji[6 + d];
                acc += double(g[0][0] * G2[t] + g[1][1] * G2[Q3 + t] + g[2][2] * G2[2 * Q3 + t] +
                              T(0.5) * (g[0][1] + g[1][0]) * G2[3 * Q3 + t] + T(0.5) * (g[0][2] + g[2][0]) * G2[4 * Q3 + t] +
                              T(0.5) * (g[1][2] + g[2][1]) * G2[5 * Q3 + t]);
            }
            __syncthreads();
            continue;
        }
        // velocity and pressure of the input
        const void* src = MODE == H_LINEARIZE ? (a.u ? a.u : static_cast<const void*>(a.ud)) : a.x;
        const TIN* xin = static_cast<const TIN*>(src);
        if (MODE != H_STATE_GRADP) gather<T, TIN>(a, xin, e, k, h, st, U, tmp);
        if (MODE == H_RESIDUAL || MODE == H_STATE_APPLY || MODE == H_STATE_GRADP) {
            for (int b = threadIdx.x; b < npr; b += blockDim.x) pe[b] = T(xin[3 * a.Nv + e * npr + b]);
            __syncthreads();
            pressure_at_qp<T>(ht, ps, k, st, pe, npr, pq);
        }
        if (MODE != H_STATE_GRADP) ref_grad<T>(k, st, U, G, Z, Y);
        const S* sst = static_cast<const S*>(a.cstate) + e * sstride;
        S* sout = static_cast<S*>(a.state) + e * sstride;
        for (int t = threadIdx.x; t < Q3; t += blockDim.x) {
            T g[3][3];
            T J2[3], wdj, ia, ib;
            if (MODE == H_STATE_APPLY || MODE == H_STATE_GRADP) {
                ia = T(sst[0]); ib = T(sst[1]);
                J2[0] = T(sst[2 + t]); J2[1] = T(sst[2 + Q3 + t]); J2[2] = T(sst[2 + 2 * Q3 + t]);
                wdj = T(sst[2 + 3 * Q3 + t]);
            } else {
                const double* gp = a.geo + e * 10 * Q3 + t;
                ia = T(gp[0]); ib = T(gp[4 * Q3]);
                J2[0] = T(gp[6 * Q3]); J2[1] = T(gp[7 * Q3]); J2[2] = T(gp[8 * Q3]);
                wdj = T(gp[9 * Q3]);
            }
            // physical gradient: Jinv = [[ia, 0, 0], [0, ib, 0], [J2]] on the extruded columns
            for (int c = 0; c < 3; ++c) {
                const T gxr = MODE == H_STATE_GRADP ? T(0) : G[(3 * c) * Q3 + t];
                const T gyr = MODE == H_STATE_GRADP ? T(0) : G[(3 * c + 1) * Q3 + t];
                const T gzr = MODE == H_STATE_GRADP ? T(0) : G[(3 * c + 2) * Q3 + t];
                g[c][0] = gxr * ia + gzr * J2[0];
                g[c][1] = gyr * ib + gzr * J2[1];
                g[c][2] = gzr * J2[2];
            }
            const T E00 = g[0][0], E11 = g[1][1], E22 = g[2][2];
            const T E01 = T(0.5) * (g[0][1] + g[1][0]), E02 = T(0.5) * (g[0][2] + g[2][0]), E12 = T(0.5) * (g[1][2] + g[2][1]);
            const T DD = E00 * E00 + E11 * E11 + E22 * E22 + T(2) * (E01 * E01 + E02 * E02 + E12 * E12);
            T tau[3][3];
            if constexpr (MODE == H_LINEARIZE) {
                const T mu = visc<T>(a, DD);
                const T mk = -T(2) * T(a.gamma) * T(a.pexp) * mu * wdj / (T(a.gamma) * DD + T(a.delta));
                const T sq = (a.picard || !(mk > T(0))) ? T(0) : sqrt(mk);
                if (t == 0) { sout[0] = S(ia); sout[1] = S(ib); }
                sout[2 + t] = S(J2[0]);
                sout[2 + Q3 + t] = S(J2[1]);
                sout[2 + 2 * Q3 + t] = S(J2[2]);
                sout[2 + 3 * Q3 + t] = S(wdj);
                sout[2 + 4 * Q3 + t] = S(mu * wdj);
                sout[2 + 5 * Q3 + t] = S(sq * E00);
                sout[2 + 6 * Q3 + t] = S(sq * E11);
                sout[2 + 7 * Q3 + t] = S(sq * E22);
                sout[2 + 8 * Q3 + t] = S(sq * E01);
                sout[2 + 9 * Q3 + t] = S(sq * E02);
                sout[2 + 10 * Q3 + t] = S(sq * E12);
                continue;
            } else if constexpr (MODE == H_RESIDUAL) {
                const T muw = visc<T>(a, DD) * wdj;
                const T pw = pq[t] * wdj;
                tau[0][0] = muw * E00 - pw; tau[1][1] = muw * E11 - pw; tau[2][2] = muw * E22 - pw;
                tau[0][1] = tau[1][0] = muw * E01;
                tau[0][2] = tau[2][0] = muw * E02;
                tau[1][2] = tau[2][1] = muw * E12;
                // body force as the value term (tmp holds Sv [3][Q3])
                for (int c = 0; c < 3; ++c) tmp[c * Q3 + t] = -wdj * T(a.body[c]);
            } else {
                // stored state: w detJ mu' E = muw E - (Dhat:E) Dhat (Eq. 2.7)
                const T pw = pq[t] * wdj;
                if (MODE == H_STATE_GRADP) {
                    for (int c = 0; c < 3; ++c)
                        for (int d = 0; d < 3; ++d) tau[c][d] = c == d ? -pw : T(0);
                } else {
                    const T muw = T(sst[2 + 4 * Q3 + t]);
                    const T D00 = T(sst[2 + 5 * Q3 + t]), D11 = T(sst[2 + 6 * Q3 + t]), D22 = T(sst[2 + 7 * Q3 + t]);
                    const T D01 = T(sst[2 + 8 * Q3 + t]), D02 = T(sst[2 + 9 * Q3 + t]), D12 = T(sst[2 + 10 * Q3 + t]);
                    const T s = D00 * E00 + D11 * E11 + D22 * E22 + T(2) * (D01 * E01 + D02 * E02 + D12 * E12);
                    tau[0][0] = muw * E00 - s * D00 - pw;
                    tau[1][1] = muw * E11 - s * D11 - pw;
                    tau[2][2] = muw * E22 - s * D22 - pw;
                    tau[0][1] = tau[1][0] = muw * E01 - s * D01;
                    tau[0][2] = tau[2][0] = muw * E02 - s * D02;
                    tau[1][2] = tau[2][1] = muw * E12 - s * D12;
                }
            }
            gq[t] = -wdj * (g[0][0] + g[1][1] + g[2][2]);
            // reference stress S[c][m] = sum_d Jinv[m][d] tau[c][d]
            for (int c = 0; c < 3; ++c) {
                G[(3 * c) * Q3 + t] = ia * tau[c][0];
                G[(3 * c + 1) * Q3 + t] = ib * tau[c][1];
                G[(3 * c + 2) * Q3 + t] = J2[0] * tau[c][0] + J2[1] * tau[c][1] + J2[2] * tau[c][2];
            }
        }
        __syncthreads();
        if constexpr (MODE == H_LINEARIZE) continue;
        else {
            T* y = static_cast<T*>(a.y);
            if (MODE != H_STATE_GRADP) pressure_rows_high<T>(ht, ps, k, st, gq, npr, y + 3 * a.Nv + e * npr);
            ref_grad_T<T>(k, st, G, MODE == H_RESIDUAL ? tmp : nullptr, U, Z, Y);
            scatter<T>(a, y, e, k, h, st, U, tmp);
        }
    }
    if constexpr (MODE == H_GRAD_A || MODE == H_GRAD_A_PARTIAL) {
        __shared__ double red[HT];
        red[threadIdx.x] = acc;
        __syncthreads();
        for (int s2 = HT / 2; s2 > 0; s2 >>= 1) {
            if (int(threadIdx.x) < s2) red[threadIdx.x] += red[threadIdx.x + s2];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if constexpr (MODE == H_GRAD_A) atomicAdd(a.gA, red[0] * a.gA_scale);
            else a.gA_part[blockIdx.x] = red[0];
        }
    }
}

// ------------------------------------------------------------ basal faces
// One block per basal face: bottom-plane gather (projector, hanging lines of
// the plane), 2-D interpolation to the face Gauss points, Robin traction
// (Eqs. 2.4-2.5, the sliding law of the stored or recomputed state), and the
// transposed path; or the log(beta) gradient; or the stored basal state.
template <typename T, int MODE>
__global__ void __launch_bounds__(128) high_face_kernel(FaceArgs a) {
    const HTab* ht = static_cast<const HTab*>(a.htab);
    const int k = ht->k, n1 = k + 1, q = n1, N2 = n1 * n1, N3 = N2 * n1, Q2 = q * q;
    __shared__ STab<T> st;
    __shared__ T V[4][NM], W[4][NM], U2[4][NM], L[NM];
    load_stab<T>(ht, 0, st);
    __syncthreads();
    // 2-D helpers on [4][NM] buffers: nc components
    auto interp = [&](T (*in)[NM], T (*out)[NM], int nc, bool transpose) {
        // forward: nodes (i, j) -> Gauss (iq, jq): x then y;  transpose: reverse
        for (int t = threadIdx.x; t < nc * N2; t += blockDim.x) {
            const int c = t / N2, r = t % N2, a0 = r % n1, a1 = r / n1;
            T s = 0;
            for (int m = 0; m < n1; ++m)
                s += (transpose ? st.B[tix(m, a0)] : st.B[tix(a0, m)]) * in[c][m + n1 * a1];
            W[c][r] = s;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nc * N2; t += blockDim.x) {
            const int c = t / N2, r = t % N2, a0 = r % n1, a1 = r / n1;
            T s = 0;
            for (int m = 0; m < n1; ++m)
                s += (transpose ? st.B[tix(m, a1)] : st.B[tix(a1, m)]) * W[c][a0 + n1 * m];
            out[c][r] = s;
        }
        __syncthreads();
    };
    auto plane_hanging = [&](uint32_t h, T (*v)[NM], int nc, bool transpose) {
        if ((h & ((1u << HANG_CHILD0) - 1)) == 0) return;
        for (int pass = 0; pass < 2; ++pass) {
            const int d = transpose ? 1 - pass : pass;
            const int b = child_bit(h, d);
            for (int t = threadIdx.x; t < nc * N2; t += blockDim.x) W[t / N2][t % N2] = v[t / N2][t % N2];
            __syncthreads();
            for (int t = threadIdx.x; t < nc * N2; t += blockDim.x) {
                const int c = t / N2, r = t % N2, i = r % n1, j = r / n1;
                const int pos = d == 0 ? i : j, other = d == 0 ? j : i;
                if (!line_hanging(h, d, other, 0, k)) continue;
                T s = 0;
                for (int m = 0; m < n1; ++m) {
                    const int rm = d == 0 ? m + n1 * j : i + n1 * m;
                    s += (transpose ? st.I[b][tix(m, pos)] : st.I[b][tix(pos, m)]) * W[c][rm];
                }
                v[c][r] = s;
            }
            __syncthreads();
        }
    };
    auto gather3 = [&](const T* x, int64_t e, T (*v)[NM]) {
        for (int r = threadIdx.x; r < N2; r += blockDim.x) {
            const int64_t g = a.nodes[e * N3 + r];
            T v0 = T(x[3 * g]), v1 = T(x[3 * g + 1]), v2 = T(x[3 * g + 2]);
            const int pi = a.pidx[e];
            if (pi >= 0) {
                const double* P = a.pel + int64_t(pi) * 6 * N2 + r;
                const T p00 = T(P[0]), p11 = T(P[N2]), p22 = T(P[2 * N2]);
                const T p01 = T(P[3 * N2]), p02 = T(P[4 * N2]), p12 = T(P[5 * N2]);
                const T w0 = p00 * v0 + p01 * v1 + p02 * v2, w1 = p01 * v0 + p11 * v1 + p12 * v2;
                const T w2 = p02 * v0 + p12 * v1 + p22 * v2;
                v0 = w0; v1 = w1; v2 = w2;
            }
            v[0][r] = v0; v[1][r] = v1; v[2][r] = v2;
        }
        __syncthreads();
    };
    for (int64_t f = blockIdx.x; f < a.nF; f += gridDim.x) {
        const int64_t e = a.face_elem[f];
        const uint32_t h = a.hang[e];
        // log(beta) at the face nodes, then at the Gauss points
        for (int r = threadIdx.x; r < N2; r += blockDim.x) V[3][r] = T(a.logbeta[a.fmap[f * N2 + r]]);
        __syncthreads();
        {
            T (*lv)[NM] = &V[3];
            plane_hanging(h, lv, 1, false);
            T (*lo)[NM] = reinterpret_cast<T (*)[NM]>(L);
            interp(lv, lo, 1, false);
        }
        auto slide_s = [&](T x2, T& ds) -> T {
            const T xe = x2 + T(a.slide_eps);
            const T sv = pow(xe, T(0.5) * (T(a.slide_m) - T(1)));
            ds = a.slide_picard ? T(0) : T(0.5) * (T(a.slide_m) - T(1)) * sv / xe;
            return sv;
        };
        if constexpr (MODE == FACE_GRAD_LOGBETA) {
            gather3(a.u, e, V);
            plane_hanging(h, V, 3, false);
            interp(V, V, 3, false);
            gather3(a.lam, e, U2);
            plane_hanging(h, U2, 3, false);
            interp(U2, U2, 3, false);
            for (int t = threadIdx.x; t < Q2; t += blockDim.x) {
                const double* fg = a.fgeo + f * 4 * Q2 + t;
                const T wa = T(fg[0]), n0 = T(fg[Q2]), n1v = T(fg[2 * Q2]), n2 = T(fg[3 * Q2]);
                const T bw = exp(L[t]) * wa;
                const T nu = n0 * V[0][t] + n1v * V[1][t] + n2 * V[2][t];
                const T nl = n0 * U2[0][t] + n1v * U2[1][t] + n2 * U2[2][t];
                const T tu[3] = {V[0][t] - nu * n0, V[1][t] - nu * n1v, V[2][t] - nu * n2};
                const T tl[3] = {U2[0][t] - nl * n0, U2[1][t] - nl * n1v, U2[2][t] - nl * n2};
                T sl = T(1);
                if (a.slide) { T ds; sl = slide_s(tu[0] * tu[0] + tu[1] * tu[1] + tu[2] * tu[2], ds); }
                U2[3][t] = bw * sl * (tu[0] * tl[0] + tu[1] * tl[1] + tu[2] * tl[2]);
            }
            __syncthreads();
            T (*sv)[NM] = &U2[3];
            interp(sv, sv, 1, true);
            plane_hanging(h, sv, 1, true);
            for (int r = threadIdx.x; r < N2; r += blockDim.x) atomicAdd(a.g + a.fmap[f * N2 + r], double(U2[3][r]));
            __syncthreads();
        } else if constexpr (MODE == FACE_LINEARIZE) {
            gather3(a.u, e, V);
            plane_hanging(h, V, 3, false);
            interp(V, V, 3, false);
            for (int t = threadIdx.x; t < Q2; t += blockDim.x) {
                const double* fg = a.fgeo + f * 4 * Q2 + t;
                const T wa = T(fg[0]), n0 = T(fg[Q2]), n1v = T(fg[2 * Q2]), n2 = T(fg[3 * Q2]);
                const T bw = exp(L[t]) * wa;
                const T nu = n0 * V[0][t] + n1v * V[1][t] + n2 * V[2][t];
                const T tu[3] = {V[0][t] - nu * n0, V[1][t] - nu * n1v, V[2][t] - nu * n2};
                T ds = T(0), sv = T(1);
                if (a.slide) sv = slide_s(tu[0] * tu[0] + tu[1] * tu[1] + tu[2] * tu[2], ds);
                const T vals[SLIDE_FIELDS] = {bw * sv, T(2) * ds * bw * tu[0], T(2) * ds * bw * tu[1],
                                              T(2) * ds * bw * tu[2], tu[0], tu[1], tu[2], n0, n1v, n2};
                const int64_t o0 = f * SLIDE_FIELDS * Q2 + t;
                for (int c = 0; c < SLIDE_FIELDS; ++c) {
                    if (a.fstate_f32) static_cast<float*>(a.fstate_out)[o0 + c * Q2] = float(vals[c]);
                    else static_cast<double*>(a.fstate_out)[o0 + c * Q2] = double(vals[c]);
                }
            }
            __syncthreads();
        } else {
            const T* x = static_cast<const T*>(a.x);
            gather3(x, e, V);
            plane_hanging(h, V, 3, false);
            interp(V, V, 3, false);
            if (a.slide && !a.fstate && a.ulin) {
                gather3(static_cast<const T*>(a.ulin), e, U2);
                plane_hanging(h, U2, 3, false);
                interp(U2, U2, 3, false);
            } else if (a.slide && !a.fstate) {
                for (int t = threadIdx.x; t < 3 * NM; t += blockDim.x) U2[t / NM][t % NM] = V[t / NM][t % NM];
                __syncthreads();
            }
            for (int t = threadIdx.x; t < Q2; t += blockDim.x) {
                const double* fg = a.fgeo + f * 4 * Q2 + t;
                const T wa = T(fg[0]), n0 = T(fg[Q2]), n1v = T(fg[2 * Q2]), n2 = T(fg[3 * Q2]);
                const T bw = exp(L[t]) * wa;
                const T nv = n0 * V[0][t] + n1v * V[1][t] + n2 * V[2][t];
                const T tw[3] = {V[0][t] - nv * n0, V[1][t] - nv * n1v, V[2][t] - nv * n2};
                T tt[3] = {bw * tw[0], bw * tw[1], bw * tw[2]};
                if (a.slide) {
                    if (a.fstate) {
                        const T* sst = static_cast<const T*>(a.fstate) + f * SLIDE_FIELDS * Q2 + t;
                        const T bws = sst[0];
                        const T vw = sst[Q2] * V[0][t] + sst[2 * Q2] * V[1][t] + sst[3 * Q2] * V[2][t];
                        for (int c = 0; c < 3; ++c) tt[c] = bws * tw[c] + vw * sst[(4 + c) * Q2];
                    } else {
                        const T nu = n0 * U2[0][t] + n1v * U2[1][t] + n2 * U2[2][t];
                        const T tu[3] = {U2[0][t] - nu * n0, U2[1][t] - nu * n1v, U2[2][t] - nu * n2};
                        T ds;
                        const T sv = slide_s(tu[0] * tu[0] + tu[1] * tu[1] + tu[2] * tu[2], ds);
                        if (a.ulin) {
                            const T r = T(2) * ds * (tu[0] * tw[0] + tu[1] * tw[1] + tu[2] * tw[2]);
                            for (int c = 0; c < 3; ++c) tt[c] = bw * (sv * tw[c] + r * tu[c]);
                        } else {
                            for (int c = 0; c < 3; ++c) tt[c] = bw * sv * tw[c];
                        }
                    }
                }
                U2[0][t] = tt[0]; U2[1][t] = tt[1]; U2[2][t] = tt[2];
            }
            __syncthreads();
            interp(U2, U2, 3, true);
            plane_hanging(h, U2, 3, true);
            T* y = static_cast<T*>(a.y);
            for (int r = threadIdx.x; r < N2; r += blockDim.x) {
                T o0 = U2[0][r], o1 = U2[1][r], o2 = U2[2][r];
                const int pi = a.pidx[e];
                if (pi >= 0) {
                    const double* P = a.pel + int64_t(pi) * 6 * N2 + r;
                    const T p00 = T(P[0]), p11 = T(P[N2]), p22 = T(P[2 * N2]);
                    const T p01 = T(P[3 * N2]), p02 = T(P[4 * N2]), p12 = T(P[5 * N2]);
                    const T w0 = p00 * o0 + p01 * o1 + p02 * o2, w1 = p01 * o0 + p11 * o1 + p12 * o2;
                    const T w2 = p02 * o0 + p12 * o1 + p22 * o2;
                    o0 = w0; o1 = w1; o2 = w2;
                }
                const int64_t g = a.nodes[e * N3 + r];
                atomicAdd(y + 3 * g, o0);
                atomicAdd(y + 3 * g + 1, o1);
                atomicAdd(y + 3 * g + 2, o2);
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------- preconditioner assembly
// The column blocks of the velocity block and the M(1/mu) element blocks of
// the Schur approximation (as for k = 2, 3, 4, with run-time sizes).
template <typename T>
__global__ void __launch_bounds__(256) high_colblock_kernel(ColArgs a) {
    const HTab* ht = static_cast<const HTab*>(a.htab);
    const int k = ht->k, n1 = k + 1, q = n1, N2 = n1 * n1, N3 = N2 * n1, Q3 = q * q * q;
    __shared__ STab<T> st;
    load_stab<T>(ht, 0, st);
    __syncthreads();
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t e = t / N3;
    if (e >= a.E) return;
    const int sl = int(t - e * N3);
    const int i = sl % n1, j = (sl / n1) % n1, l = sl / N2;
    const int64_t na = a.nodes[e * N3 + sl];
    const int col = a.col_of[na], pa = a.pos_of[na];
    const T* s0 = static_cast<const T*>(a.state) + e * a.state_stride;
    const T ia = s0[0], ib = s0[1];
    const int bw = a.bw, W = 2 * a.bw + 1;
    T* A = static_cast<T*>(a.A);
    for (int l2 = 0; l2 < n1; ++l2) {
        const int64_t nb = a.nodes[e * N3 + i + n1 * (j + n1 * l2)];
        if (a.col_of[nb] != col) continue;
        const int pb = a.pos_of[nb];
        T K[3][3] = {};
        for (int lq = 0; lq < q; ++lq)
            for (int jq = 0; jq < q; ++jq)
                for (int iq = 0; iq < q; ++iq) {
                    const int qp = iq + q * (jq + q * lq);
                    const T g0 = s0[2 + qp], g1 = s0[2 + Q3 + qp], g2 = s0[2 + 2 * Q3 + qp], muw = s0[2 + 4 * Q3 + qp];
                    const T D00 = s0[2 + 5 * Q3 + qp], D11 = s0[2 + 6 * Q3 + qp], D22 = s0[2 + 7 * Q3 + qp];
                    const T D01 = s0[2 + 8 * Q3 + qp], D02 = s0[2 + 9 * Q3 + qp], D12 = s0[2 + 10 * Q3 + qp];
                    const T bi = st.B[tix(iq, i)], bj = st.B[tix(jq, j)];
                    const T dbi = st.Bd[tix(iq, i)], dbj = st.Bd[tix(jq, j)];
                    const T ra[3] = {dbi * bj * st.B[tix(lq, l)], bi * dbj * st.B[tix(lq, l)], bi * bj * st.Bd[tix(lq, l)]};
                    const T rb[3] = {dbi * bj * st.B[tix(lq, l2)], bi * dbj * st.B[tix(lq, l2)], bi * bj * st.Bd[tix(lq, l2)]};
                    const T pa3[3] = {ra[0] * ia + ra[2] * g0, ra[1] * ib + ra[2] * g1, ra[2] * g2};
                    const T pb3[3] = {rb[0] * ia + rb[2] * g0, rb[1] * ib + rb[2] * g1, rb[2] * g2};
                    const T dot = pa3[0] * pb3[0] + pa3[1] * pb3[1] + pa3[2] * pb3[2];
                    const T Da[3] = {D00 * pa3[0] + D01 * pa3[1] + D02 * pa3[2], D01 * pa3[0] + D11 * pa3[1] + D12 * pa3[2],
                                     D02 * pa3[0] + D12 * pa3[1] + D22 * pa3[2]};
                    const T Db[3] = {D00 * pb3[0] + D01 * pb3[1] + D02 * pb3[2], D01 * pb3[0] + D11 * pb3[1] + D12 * pb3[2],
                                     D02 * pb3[0] + D12 * pb3[1] + D22 * pb3[2]};
                    const T hm = T(0.5) * muw;
                    for (int c = 0; c < 3; ++c)
                        for (int c2 = 0; c2 < 3; ++c2)
                            K[c][c2] += hm * ((c == c2 ? dot : T(0)) + pa3[c2] * pb3[c]) - Da[c] * Db[c2];
                }
        if (l == 0 && l2 == 0 && a.robin && a.fidx[e] >= 0) {
            const int64_t fcs = a.fidx[e];
            for (int jq = 0; jq < q; ++jq)
                for (int iq = 0; iq < q; ++iq) {
                    const int fq = iq + q * jq;
                    T lbq = 0;
                    for (int j2 = 0; j2 < n1; ++j2)
                        for (int i2 = 0; i2 < n1; ++i2)
                            lbq += st.B[tix(iq, i2)] * st.B[tix(jq, j2)] * T(a.logbeta[a.fmap[fcs * N2 + i2 + n1 * j2]]);
                    const double* fg = a.fgeo + fcs * 4 * q * q + fq;
                    const T phi = st.B[tix(iq, i)] * st.B[tix(jq, j)];
                    const T* sst = a.fstate ? static_cast<const T*>(a.fstate) + fcs * SLIDE_FIELDS * q * q + fq : nullptr;
                    const T bws = sst ? sst[0] : exp(lbq) * T(fg[0]);
                    const T w = bws * phi * phi;
                    const T n[3] = {T(fg[q * q]), T(fg[2 * q * q]), T(fg[3 * q * q])};
                    for (int c = 0; c < 3; ++c)
                        for (int c2 = 0; c2 < 3; ++c2) {
                            K[c][c2] += w * ((c == c2 ? T(1) : T(0)) - n[c] * n[c2]);
                            if (sst) K[c][c2] += phi * phi * sst[(4 + c) * q * q] * sst[(1 + c2) * q * q];
                        }
                }
        }
        for (int c = 0; c < 3; ++c)
            for (int c2 = 0; c2 < 3; ++c2) {
                const int r = 3 * pa + c, qq = 3 * pb + c2;
                atomicAdd(A + band_at(col, r, qq - r + bw, W, a.rows), K[c][c2]);
            }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) high_schur_kernel(ColArgs a) {
    const HTab* ht = static_cast<const HTab*>(a.htab);
    const int k = ht->k, q = k + 1, Q3 = q * q * q;
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int per_e = a.schur_full ? a.npr * a.npr : a.npr;
    const int64_t e = t / per_e;
    if (e >= a.E) return;
    const int r = int(t - e * per_e);
    const int b1 = a.schur_full ? r / a.npr : r;
    const int b2 = a.schur_full ? r - b1 * a.npr : r;
    const int ps = a.pspace;
    const int* m1 = ht->pmode[ps][b1];
    const int* m2 = ht->pmode[ps][b2];
    const T* s0 = static_cast<const T*>(a.state) + e * a.state_stride;
    double s = 0;
    for (int qp = 0; qp < Q3; ++qp) {
        const int iq = qp % q, jq = (qp / q) % q, lq = qp / (q * q);
        const double f = ht->P1[ps][iq][m1[0]] * ht->P1[ps][jq][m1[1]] * ht->P1[ps][lq][m1[2]] *
                         ht->P1[ps][iq][m2[0]] * ht->P1[ps][jq][m2[1]] * ht->P1[ps][lq][m2[2]];
        const T wdj = s0[2 + 3 * Q3 + qp], muw = s0[2 + 4 * Q3 + qp];
        s += f * double(wdj * (wdj / muw));
    }
    a.mblk[(e * a.npr + b1) * a.npr + b2] = s;
}

// ------------------------------------------------------------- host side
std::mutex g_ht_mu;
std::vector<std::pair<std::pair<int, int>, void*>> g_ht;   // ((device, k), device table)

inline int elem_grid(int64_t E) { return int(std::min<int64_t>(E, 2048)); }

template <typename T, typename S, typename TIN, int MODE>
int launch_high(const ElemArgs& a, cudaStream_t s) {
    if (a.E == 0) return int(cudaSuccess);
    const Carve cv = carve(a.htab_k, a.npr, MODE == H_GRAD_A || MODE == H_GRAD_A_PARTIAL);
    const size_t smem = size_t(cv.total) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(high_elem_kernel<T, S, TIN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(smem));
    if (e != cudaSuccess) return int(e);
    high_elem_kernel<T, S, TIN, MODE><<<unsigned(elem_grid(a.E)), HT, smem, s>>>(a);
    return int(cudaGetLastError());
}

}  // namespace

int high_tables(int dev, int k, const void** out) {
    std::lock_guard<std::mutex> lock(g_ht_mu);
    for (auto& p : g_ht)
        if (p.first.first == dev && p.first.second == k) { *out = p.second; return STOKES_OK; }
    Tables1D t[2];
    build_tables(k, STOKES_PRESSURE_P, t[0]);
    build_tables(k, STOKES_PRESSURE_Q, t[1]);
    HTab h{};
    h.k = k; h.n1 = k + 1; h.q = k + 1; h.npr[0] = t[0].npr; h.npr[1] = t[1].npr;
    for (int a = 0; a < h.q; ++a)
        for (int b = 0; b < h.n1; ++b) {
            h.B[a][b] = t[0].B[a][b];
            double s = 0;
            for (int m = 0; m < h.q; ++m) s += t[0].Dg[a][m] * t[0].B[m][b];
            h.Bd[a][b] = s;
        }
    for (int hh = 0; hh < 2; ++hh)
        for (int a = 0; a < h.n1; ++a)
            for (int b = 0; b < h.n1; ++b) h.I[hh][a][b] = t[0].I[hh][a][b];
    for (int sp = 0; sp < 2; ++sp) {
        for (int a = 0; a < h.q; ++a)
            for (int b = 0; b < h.n1; ++b) h.P1[sp][a][b] = t[sp].P1[a][b];
        for (int m = 0; m < t[sp].npr; ++m)
            for (int c = 0; c < 3; ++c) h.pmode[sp][m][c] = t[sp].pmode[m][c];
    }
    void* d = nullptr;
    if (dev_alloc(&d, sizeof(HTab)) != cudaSuccess) return fail(STOKES_E_NOMEM, "degree tables");
    if (cudaMemcpy(d, &h, sizeof(HTab), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return fail(STOKES_E_CUDA, "uploading degree tables");
    }
    g_ht.push_back({{dev, k}, d});
    *out = d;
    return STOKES_OK;
}

int64_t high_state_stride(int k) {
    const int64_t q3 = int64_t(k + 1) * (k + 1) * (k + 1);
    return (2 + STATE_FIELDS * q3 + 3) / 4 * 4;
}

int64_t high_grad_a_partials(int64_t E) { return elem_grid(E); }

int launch_elem_high(int mode, int prec, int state_prec, const ElemArgs& a, cudaStream_t s) {
    const bool f32 = prec == STOKES_F32;
    switch (mode) {
        case MODE_RESIDUAL:
            return f32 ? launch_high<float, float, float, H_RESIDUAL>(a, s) : launch_high<double, double, double, H_RESIDUAL>(a, s);
        case MODE_LINEARIZE:
            // FP64 arithmetic; the input is the FP64 state (a.ud), or a.u in
            // the precision prec (the fused apply's linearisation point)
            if (a.u) {
                if (f32) return state_prec == STOKES_F32 ? launch_high<double, float, float, H_LINEARIZE>(a, s)
                                                         : launch_high<double, double, float, H_LINEARIZE>(a, s);
                return state_prec == STOKES_F32 ? launch_high<double, float, double, H_LINEARIZE>(a, s)
                                                : launch_high<double, double, double, H_LINEARIZE>(a, s);
            }
            return state_prec == STOKES_F32 ? launch_high<double, float, double, H_LINEARIZE>(a, s)
                                            : launch_high<double, double, double, H_LINEARIZE>(a, s);
        case MODE_STATE_APPLY:
            if (f32) return state_prec == STOKES_F32 ? launch_high<float, float, float, H_STATE_APPLY>(a, s)
                                                     : launch_high<float, double, float, H_STATE_APPLY>(a, s);
            return launch_high<double, double, double, H_STATE_APPLY>(a, s);
        case MODE_STATE_GRADP:
            if (f32) return launch_high<float, float, float, H_STATE_GRADP>(a, s);
            return launch_high<double, double, double, H_STATE_GRADP>(a, s);
        case MODE_GRAD_A:
            return launch_high<double, double, double, H_GRAD_A>(a, s);
        case MODE_GRAD_A_PARTIAL:
            return launch_high<double, double, double, H_GRAD_A_PARTIAL>(a, s);
        default:
            return int(cudaErrorInvalidValue);
    }
}

int launch_face_high(int mode, int prec, const FaceArgs& a, cudaStream_t s) {
    if (a.nF == 0) return int(cudaSuccess);
    const unsigned grid = unsigned(std::min<int64_t>(a.nF, 4096));
    if (mode == FACE_GRAD_LOGBETA) high_face_kernel<double, FACE_GRAD_LOGBETA><<<grid, 128, 0, s>>>(a);
    else if (mode == FACE_LINEARIZE) high_face_kernel<double, FACE_LINEARIZE><<<grid, 128, 0, s>>>(a);
    else if (prec == STOKES_F32) high_face_kernel<float, FACE_APPLY><<<grid, 128, 0, s>>>(a);
    else high_face_kernel<double, FACE_APPLY><<<grid, 128, 0, s>>>(a);
    return int(cudaGetLastError());
}

int launch_precond_assembly_high(int prec, const ColArgs& a, cudaStream_t s) {
    if (a.E == 0) return int(cudaSuccess);
    const int n1 = a.htab_k + 1;
    const int64_t n1t = a.E * int64_t(n1) * n1 * n1;
    if (prec == STOKES_F32) high_colblock_kernel<float><<<unsigned((n1t + 255) / 256), 256, 0, s>>>(a);
    else high_colblock_kernel<double><<<unsigned((n1t + 255) / 256), 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !a.mblk) return int(e);
    const int64_t n2 = a.E * a.npr * (a.schur_full ? a.npr : 1);
    if (prec == STOKES_F32) high_schur_kernel<float><<<unsigned((n2 + 255) / 256), 256, 0, s>>>(a);
    else high_schur_kernel<double><<<unsigned((n2 + 255) / 256), 256, 0, s>>>(a);
    return int(cudaGetLastError());
}

}  // namespace stokes
