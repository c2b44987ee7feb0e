// Lane-per-component state apply (the Krylov-inner Jacobian, degree 2, FP32).
//
// Three consecutive lanes own one element, lane c holding velocity component
// c of all 27 nodes in registers (ten elements per warp).  The sum-factorised
// contractions (Section 3.3) then run entirely in registers with uniform
// table operands; the only exchange is the physical gradient row of each
// component at a quadrature point (6 warp shuffles), needed to form the
// strain rate D(w) for the pointwise Newton map (Eq. 2.7).  The element's
// pressure rows are accumulated by lane 0 without any reduction, and the
// linearised state is read slot-major, so consecutive elements are read with
// consecutive addresses.  Planes of Gauss points are processed one at a time
// to bound the register footprint.
#pragma once

namespace stokes {
namespace dev {
namespace STOKES_NS {

constexpr int CPT_W = 4;                 // warps per block
constexpr int CPT_EPW = 32 / N1;         // elements per warp (N1 lanes each... see below)

// gather one velocity component of all N3 slots (lattice or element map)
template <typename T>
__device__ __forceinline__ int64_t cpt_node(const ElemArgs& a, int64_t e, int ex, int ey, int ez, int s) {
    const int i = s % N1, j = (s / N1) % N1, l = s / N2;
    if (a.lat_nx > 0) {
        int I = ex * K + i, J = ey * K + j;
        const int NX = int(a.lat_NX), NY = int(a.lat_NY);
        if (I >= NX) I -= NX;
        if (J >= NY) J -= NY;
        return int64_t(I) + int64_t(NX) * (int64_t(J) + int64_t(NY) * int64_t(ez * K + l));
    }
    return a.nodes[e * N3 + s];
}

// In-register hanging-node interpolation of one component (forward or transpose),
// sweeps along x, y, z (transpose: z, y, x) of the constrained lines.
template <typename T, bool TRANSPOSE>
__device__ __forceinline__ void cpt_hanging(T (&v)[N3], uint32_t h) {
    #pragma unroll
    for (int pass = 0; pass < 3; ++pass) {
        const int d = TRANSPOSE ? 2 - pass : pass;
        const int bb = child_bit(h, d);
        #pragma unroll
        for (int p = 0; p < N1; ++p)
            #pragma unroll
            for (int q = 0; q < N1; ++q) {
                // line parallel to d through (p, q) on the other two axes (o0 < o1)
                if (!line_hanging(h, d, p, q, K)) continue;
                T line[N1], out[N1];
                #pragma unroll
                for (int m = 0; m < N1; ++m) {
                    const int idx = d == 0 ? sidx(m, p, q) : (d == 1 ? sidx(p, m, q) : sidx(p, q, m));
                    line[m] = v[idx];
                }
                #pragma unroll
                for (int r = 0; r < N1; ++r) {
                    T s = 0;
                    #pragma unroll
                    for (int m = 0; m < N1; ++m)
                        s += (TRANSPOSE ? Tab<T>::I(bb, m, r) : Tab<T>::I(bb, r, m)) * line[m];
                    out[r] = s;
                }
                #pragma unroll
                for (int m = 0; m < N1; ++m) {
                    const int idx = d == 0 ? sidx(m, p, q) : (d == 1 ? sidx(p, m, q) : sidx(p, q, m));
                    v[idx] = out[m];
                }
            }
    }
}

// basal projector on the bottom-plane slots: component c of P x, the other
// components fetched from the element's sibling lanes
template <typename T>
__device__ __forceinline__ void cpt_project(const ElemArgs& a, int64_t e, bool active, int base, int c,
                                            T (&v)[N3], bool any_basal) {
    if (!any_basal) return;
    const int pi = active ? a.pidx[e] : -1;
    #pragma unroll
    for (int s = 0; s < N2; ++s) {
        const T x0 = __shfl_sync(0xffffffffu, v[s], base);
        const T x1 = __shfl_sync(0xffffffffu, v[s], base + 1);
        const T x2 = __shfl_sync(0xffffffffu, v[s], base + 2);
        if (pi >= 0) {
            const double* P = a.pel + int64_t(pi) * 6 * N2 + s;
            // row c of the symmetric P: (00 11 22 01 02 12)
            const int r0 = c == 0 ? 0 : (c == 1 ? 3 : 4);
            const int r1 = c == 0 ? 3 : (c == 1 ? 1 : 5);
            const int r2 = c == 0 ? 4 : (c == 1 ? 5 : 2);
            v[s] = T(P[r0 * N2]) * x0 + T(P[r1 * N2]) * x1 + T(P[r2 * N2]) * x2;
        }
    }
}

template <typename T, bool PONLY>
__global__ void __launch_bounds__(32 * CPT_W) state_apply_cpt_kernel(ElemArgs a) {
    static_assert(N1 == 3, "lane-per-component kernel is written for degree 2");
    constexpr int EW = 10;                              // elements per warp
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int es = lane / 3;
    const int c = lane - 3 * es;
    const bool idle = es >= EW;
    if (idle) es = EW - 1;
    const int base = idle ? 27 : 3 * es;                // first lane of the element's group
    const int64_t e = (int64_t(blockIdx.x) * CPT_W + warp) * EW + es;
    const bool active = !idle && e < a.E;
    const int64_t E = a.E;
    const T* S = static_cast<const T*>(a.cstate);
    const T* x = static_cast<const T*>(a.x);
    T* y = static_cast<T*>(a.y);
    const int ps = a.pspace;
    const int64_t ee = active ? e : 0;

    int ex = 0, ey = 0, ez = 0;
    if (a.lat_nx > 0) {
        const int e32 = int(ee), nx = int(a.lat_nx), ny = int(a.lat_ny);
        ex = e32 % nx;
        const int r = e32 / nx;
        ey = r % ny;
        ez = r / ny;
    }
    const uint32_t h = active ? a.hang[ee] : 0u;
    const bool any_h = a.any_hang ? (__any_sync(0xffffffffu, (h & ((1u << HANG_CHILD0) - 1)) != 0) != 0) : false;
    const bool any_basal = __any_sync(0xffffffffu, active && a.pidx[ee] >= 0) != 0;

    // pressure dofs of the element
    T pd[NPRK];
    #pragma unroll
    for (int b = 0; b < NPRK; ++b)
        pd[b] = (active && b < a.npr) ? ld(x + 3 * a.Nv + ee * a.npr + b) : T(0);

    T v[N3];
    if constexpr (!PONLY) {
        #pragma unroll
        for (int s = 0; s < N3; ++s) v[s] = active ? ld(x + 3 * cpt_node<T>(a, ee, ex, ey, ez, s) + c) : T(0);
        cpt_project<T>(a, ee, active, base, c, v, any_basal);
        if (any_h && h) cpt_hanging<T, false>(v, h);
    }
    T out[N3];
    #pragma unroll
    for (int s = 0; s < N3; ++s) out[s] = T(0);
    T prow[NPRK];
    #pragma unroll
    for (int b = 0; b < NPRK; ++b) prow[b] = T(0);

    const T ia = active ? S[state_index(true, E, ee, 0)] : T(0);
    const T ib = active ? S[state_index(true, E, ee, 1)] : T(0);

    #pragma unroll
    for (int lq = 0; lq < Q; ++lq) {
        // ---- forward: reference gradient of component c on plane lq
        T gx[N2], gy[N2], gz[N2];
        if constexpr (!PONLY) {
            T av[N2], dz[N2];
            #pragma unroll
            for (int j = 0; j < N1; ++j)
                #pragma unroll
                for (int i = 0; i < N1; ++i) {
                    T s0 = 0, s1 = 0;
                    #pragma unroll
                    for (int l = 0; l < N1; ++l) {
                        s0 += Tab<T>::B(lq, l) * v[sidx(i, j, l)];
                        s1 += Tab<T>::Bd(lq, l) * v[sidx(i, j, l)];
                    }
                    av[i + N1 * j] = s0;
                    dz[i + N1 * j] = s1;
                }
            T ea[N2], eda[N2], edz[N2];   // [jq][i]
            #pragma unroll
            for (int jq = 0; jq < Q; ++jq)
                #pragma unroll
                for (int i = 0; i < N1; ++i) {
                    T s0 = 0, s1 = 0, s2 = 0;
                    #pragma unroll
                    for (int j = 0; j < N1; ++j) {
                        s0 += Tab<T>::B(jq, j) * av[i + N1 * j];
                        s1 += Tab<T>::Bd(jq, j) * av[i + N1 * j];
                        s2 += Tab<T>::B(jq, j) * dz[i + N1 * j];
                    }
                    ea[i + N1 * jq] = s0; eda[i + N1 * jq] = s1; edz[i + N1 * jq] = s2;
                }
            #pragma unroll
            for (int jq = 0; jq < Q; ++jq)
                #pragma unroll
                for (int iq = 0; iq < Q; ++iq) {
                    T s0 = 0, s1 = 0, s2 = 0;
                    #pragma unroll
                    for (int i = 0; i < N1; ++i) {
                        s0 += Tab<T>::Bd(iq, i) * ea[i + N1 * jq];
                        s1 += Tab<T>::B(iq, i) * eda[i + N1 * jq];
                        s2 += Tab<T>::B(iq, i) * edz[i + N1 * jq];
                    }
                    gx[iq + Q * jq] = s0; gy[iq + Q * jq] = s1; gz[iq + Q * jq] = s2;
                }
        } else {
            #pragma unroll
            for (int q = 0; q < N2; ++q) gx[q] = gy[q] = gz[q] = T(0);
        }
        // ---- pointwise Newton map at the 9 Gauss points of the plane
        #pragma unroll
        for (int jq = 0; jq < Q; ++jq)
            #pragma unroll
            for (int iq = 0; iq < Q; ++iq) {
                const int q = iq + Q * jq;
                const int qp = q + N2 * lq;
                T f[STATE_FIELDS];
                #pragma unroll
                for (int r = 0; r < STATE_FIELDS; ++r) f[r] = active ? S[state_index(true, E, ee, 2 + r * Q3 + qp)] : T(0);
                const T g0 = f[0], g1 = f[1], g2 = f[2], wdj = f[3], muw = f[4];
                const T D00 = f[5], D11 = f[6], D22 = f[7], D01 = f[8], D02 = f[9], D12 = f[10];
                // physical gradient row c: Jinv = [[ia,0,0],[0,ib,0],[g0,g1,g2]]
                const T r0 = gx[q] * ia + gz[q] * g0;
                const T r1 = gy[q] * ib + gz[q] * g1;
                const T r2 = gz[q] * g2;
                T g[3][3];
                #pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    g[cc][0] = __shfl_sync(0xffffffffu, r0, base + cc);
                    g[cc][1] = __shfl_sync(0xffffffffu, r1, base + cc);
                    g[cc][2] = __shfl_sync(0xffffffffu, r2, base + cc);
                }
                const T E00 = g[0][0], E11 = g[1][1], E22 = g[2][2];
                const T E01 = T(0.5) * (g[0][1] + g[1][0]);
                const T E02 = T(0.5) * (g[0][2] + g[2][0]);
                const T E12 = T(0.5) * (g[1][2] + g[2][1]);
                const T sdot = D00 * E00 + D11 * E11 + D22 * E22 + T(2) * (D01 * E01 + D02 * E02 + D12 * E12);
                T pq = 0;
                #pragma unroll
                for (int b = 0; b < NPRK; ++b)
                    if (b < a.npr)
                        pq += pd[b] * Tab<T>::P1(ps, iq, cPm[ps][b][0]) * Tab<T>::P1(ps, jq, cPm[ps][b][1]) *
                              Tab<T>::P1(ps, lq, cPm[ps][b][2]);
                const T pw = pq * wdj;
                // row c of wdetJ (mu' E - p I) (Eq. 2.7 as a symmetric map)
                T t0, t1, t2;
                if (c == 0) {
                    t0 = muw * E00 - sdot * D00 - pw; t1 = muw * E01 - sdot * D01; t2 = muw * E02 - sdot * D02;
                } else if (c == 1) {
                    t0 = muw * E01 - sdot * D01; t1 = muw * E11 - sdot * D11 - pw; t2 = muw * E12 - sdot * D12;
                } else {
                    t0 = muw * E02 - sdot * D02; t1 = muw * E12 - sdot * D12; t2 = muw * E22 - sdot * D22 - pw;
                }
                // reference stress of component c, stored over the gradient
                gx[q] = ia * t0;
                gy[q] = ib * t1;
                gz[q] = g0 * t0 + g1 * t1 + g2 * t2;
                if constexpr (!PONLY) {
                    // pressure rows (lane 0 of the element): - w detJ psi_b div w
                    if (c == 0) {
                        const T gq = -wdj * (E00 + E11 + E22);
                        #pragma unroll
                        for (int b = 0; b < NPRK; ++b)
                            if (b < a.npr)
                                prow[b] += gq * Tab<T>::P1(ps, iq, cPm[ps][b][0]) * Tab<T>::P1(ps, jq, cPm[ps][b][1]) *
                                           Tab<T>::P1(ps, lq, cPm[ps][b][2]);
                    }
                }
            }
        // ---- backward: transposed contractions of the plane into the nodal rows
        T t1[N2], t2[N2], t3[N2];   // [jq][i]
        #pragma unroll
        for (int jq = 0; jq < Q; ++jq)
            #pragma unroll
            for (int i = 0; i < N1; ++i) {
                T s0 = 0, s1 = 0, s2 = 0;
                #pragma unroll
                for (int iq = 0; iq < Q; ++iq) {
                    s0 += Tab<T>::Bd(iq, i) * gx[iq + Q * jq];
                    s1 += Tab<T>::B(iq, i) * gy[iq + Q * jq];
                    s2 += Tab<T>::B(iq, i) * gz[iq + Q * jq];
                }
                t1[i + N1 * jq] = s0; t2[i + N1 * jq] = s1; t3[i + N1 * jq] = s2;
            }
        #pragma unroll
        for (int j = 0; j < N1; ++j)
            #pragma unroll
            for (int i = 0; i < N1; ++i) {
                T ab = 0, zb = 0;
                #pragma unroll
                for (int jq = 0; jq < Q; ++jq) {
                    ab += Tab<T>::B(jq, j) * t1[i + N1 * jq] + Tab<T>::Bd(jq, j) * t2[i + N1 * jq];
                    zb += Tab<T>::B(jq, j) * t3[i + N1 * jq];
                }
                #pragma unroll
                for (int l = 0; l < N1; ++l) out[sidx(i, j, l)] += Tab<T>::B(lq, l) * ab + Tab<T>::Bd(lq, l) * zb;
            }
    }

    if constexpr (!PONLY) {
        if (active && c == 0) {
            #pragma unroll
            for (int b = 0; b < NPRK; ++b)
                if (b < a.npr) y[3 * a.Nv + ee * a.npr + b] = prow[b];
        }
    }
    if (any_h && h) cpt_hanging<T, true>(out, h);
    cpt_project<T>(a, ee, active, base, c, out, any_basal);
    if (active) {
        #pragma unroll
        for (int s = 0; s < N3; ++s) atomic_add(y + 3 * cpt_node<T>(a, ee, ex, ey, ez, s) + c, out[s]);
    }
}

template <typename T, bool PONLY>
int launch_state_apply_cpt(const ElemArgs& a, cudaStream_t s) {
    constexpr int EPBLK = CPT_W * 10;
    const int64_t blocks = (a.E + EPBLK - 1) / EPBLK;
    if (blocks == 0) return int(cudaSuccess);
    state_apply_cpt_kernel<T, PONLY><<<unsigned(blocks), 32 * CPT_W, 0, s>>>(a);
    return int(cudaGetLastError());
}

}  // namespace STOKES_NS
}  // namespace dev
}  // namespace stokes
