// Degree-dependent parts of the block preconditioner (Section 4.2, Eq. 4.1):
// assembly of the vertical-column blocks of the velocity block F from the
// linearised state, and the diagonal of the 1/mu-weighted pressure mass
// matrix (the Schur approximation -M(1/mu) of Section 6).
// Included by k2.cu, k3.cu, k4.cu after elem_body.cuh.
#pragma once

#include "precond.h"

namespace stokes {
namespace dev {
namespace STOKES_NS {

// derivative of the GLL Lagrange polynomial i at Gauss point iq: (Dg B)[iq][i]
template <typename T>
__device__ __forceinline__ T Bd(int iq, int i) {
    T s = 0;
    #pragma unroll
    for (int m = 0; m < Q; ++m) s += Tab<T>::Dg(iq, m) * Tab<T>::B(m, i);
    return s;
}

// One thread per (element, slot a = (i, j, l)): the three rows of slot a
// against every slot b = (i, j, l2) of the same element column, i.e. the
// in-column couplings of the element velocity matrix
//   K[(a,c),(b,c')] = sum_qp  muw/2 (delta_cc' grad phi_a . grad phi_b
//                     + d_c' phi_a d_c phi_b) - (Dhat grad phi_a)_c (Dhat grad phi_b)_c'
// (the bilinear form of Eq. 2.6 with the tensor of Eq. 2.7), plus the basal
// Robin block of slot a with itself; accumulated into the banded column
// matrices.  A hanging slot contributes through the node its element map
// names, the coarse neighbour's node at the same local GLL position (an
// injective nearest-node stand-in for the interpolation R_i, so every
// element term stays positive semi-definite); the exact interpolation
// weights are used by the operator, not by this preconditioner.
template <typename T>
__global__ void __launch_bounds__(256) colblock_kernel(ColArgs a) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t e = t / N3;
    if (e >= a.E) return;
    const int sl = int(t - e * N3);
    const int i = sl % N1, j = (sl / N1) % N1, l = sl / N2;
    const int64_t na = a.nodes[e * N3 + sl];
    const int col = a.col_of[na], pa = a.pos_of[na];
    const T* st0 = static_cast<const T*>(a.state);
    const StateRef sr(e, a.state_cpl);
    const T ia = st0[sr.c(0)], ib = st0[sr.c(1)];
    const int bw = a.bw, W = 2 * a.bw + 1;
    T* A = static_cast<T*>(a.A);
    for (int l2 = 0; l2 < N1; ++l2) {
        const int64_t nb = a.nodes[e * N3 + sidx(i, j, l2)];
        if (a.col_of[nb] != col) continue;
        const int pb = a.pos_of[nb];
        T Kab[3][3] = {};
        for (int lq = 0; lq < Q; ++lq)
            for (int jq = 0; jq < Q; ++jq)
                for (int iq = 0; iq < Q; ++iq) {
                    const T* F = st0 + sr.f(0, lq, iq + Q * jq);
                    const int fs = sr.fstride;
                    const T g0 = F[0], g1 = F[fs], g2 = F[2 * fs], muw = F[4 * fs];
                    const T D00 = F[5 * fs], D11 = F[6 * fs], D22 = F[7 * fs];
                    const T D01 = F[8 * fs], D02 = F[9 * fs], D12 = F[10 * fs];
                    const T bi = Tab<T>::B(iq, i), bj = Tab<T>::B(jq, j);
                    const T dbi = Bd<T>(iq, i), dbj = Bd<T>(jq, j);
                    const T ra[3] = {dbi * bj * Tab<T>::B(lq, l), bi * dbj * Tab<T>::B(lq, l), bi * bj * Bd<T>(lq, l)};
                    const T rb[3] = {dbi * bj * Tab<T>::B(lq, l2), bi * dbj * Tab<T>::B(lq, l2), bi * bj * Bd<T>(lq, l2)};
                    const T pa3[3] = {ra[0] * ia + ra[2] * g0, ra[1] * ib + ra[2] * g1, ra[2] * g2};
                    const T pb3[3] = {rb[0] * ia + rb[2] * g0, rb[1] * ib + rb[2] * g1, rb[2] * g2};
                    const T dot = pa3[0] * pb3[0] + pa3[1] * pb3[1] + pa3[2] * pb3[2];
                    const T Da[3] = {D00 * pa3[0] + D01 * pa3[1] + D02 * pa3[2],
                                     D01 * pa3[0] + D11 * pa3[1] + D12 * pa3[2],
                                     D02 * pa3[0] + D12 * pa3[1] + D22 * pa3[2]};
                    const T Db[3] = {D00 * pb3[0] + D01 * pb3[1] + D02 * pb3[2],
                                     D01 * pb3[0] + D11 * pb3[1] + D12 * pb3[2],
                                     D02 * pb3[0] + D12 * pb3[1] + D22 * pb3[2]};
                    const T hm = T(0.5) * muw;
                    #pragma unroll
                    for (int c = 0; c < 3; ++c)
                        #pragma unroll
                        for (int c2 = 0; c2 < 3; ++c2)
                            Kab[c][c2] += hm * ((c == c2 ? dot : T(0)) + pa3[c2] * pb3[c]) - Da[c] * Db[c2];
                }
        // basal Robin term of slot a with itself
        if (l == 0 && l2 == 0 && a.robin && a.fidx[e] >= 0) {
            const int64_t fcs = a.fidx[e];
            for (int jq = 0; jq < Q; ++jq)
                for (int iq = 0; iq < Q; ++iq) {
                    const int fq = iq + Q * jq;
                    T lbq = 0;
                    for (int j2 = 0; j2 < N1; ++j2)
                        for (int i2 = 0; i2 < N1; ++i2)
                            lbq += Tab<T>::B(iq, i2) * Tab<T>::B(jq, j2) * T(a.logbeta[a.fmap[fcs * N2 + i2 + N1 * j2]]);
                    const double* fg = a.fgeo + fcs * 4 * Q * Q + fq;
                    const T phi = Tab<T>::B(iq, i) * Tab<T>::B(jq, j);
                    // nonlinear sliding: beta w s and the rank-one term
                    // v (T u)^T of its derivative from the stored sliding state
                    const T* sst = a.fstate ? static_cast<const T*>(a.fstate) + fcs * SLIDE_FIELDS * Q * Q + fq
                                            : nullptr;
                    const T bws = sst ? sst[0] : exp(lbq) * T(fg[0]);
                    const T w = bws * phi * phi;
                    const T n[3] = {T(fg[Q * Q]), T(fg[2 * Q * Q]), T(fg[3 * Q * Q])};
                    #pragma unroll
                    for (int c = 0; c < 3; ++c)
                        #pragma unroll
                        for (int c2 = 0; c2 < 3; ++c2) {
                            Kab[c][c2] += w * ((c == c2 ? T(1) : T(0)) - n[c] * n[c2]);
                            if (sst) Kab[c][c2] += phi * phi * sst[(4 + c) * Q * Q] * sst[(1 + c2) * Q * Q];
                        }
                }
        }
        #pragma unroll
        for (int c = 0; c < 3; ++c)
            #pragma unroll
            for (int c2 = 0; c2 < 3; ++c2) {
                const int r = 3 * pa + c, q = 3 * pb + c2;
                atomic_add(A + band_at(col, r, q - r + bw, W, a.rows), Kab[c][c2]);
            }
    }
}

// mblk[e][b1][b2] = sum_qp psi_b1 psi_b2 w detJ / mu   (element block of
// M(1/mu); w detJ / mu = (w detJ)^2 / (mu w detJ) from the stored state);
// one thread per (element, b1, b2), or per (element, b) for the diagonal
// only; FP64 accumulation
template <typename T>
__global__ void __launch_bounds__(256) schur_block_kernel(ColArgs a) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int per_e = a.schur_full ? a.npr * a.npr : a.npr;
    const int64_t e = t / per_e;
    if (e >= a.E) return;
    const int r = int(t - e * per_e);
    const int b1 = a.schur_full ? r / a.npr : r;
    const int b2 = a.schur_full ? r - b1 * a.npr : r;
    const int ps = a.pspace;
    const T* st0 = static_cast<const T*>(a.state);
    const StateRef sr(e, a.state_cpl);
    const int a0 = cPm[ps][b1][0], a1 = cPm[ps][b1][1], a2 = cPm[ps][b1][2];
    const int c0 = cPm[ps][b2][0], c1 = cPm[ps][b2][1], c2 = cPm[ps][b2][2];
    // arithmetic of the state's type (a preconditioner block), summed per
    // plane and accumulated across planes in FP64
    double s = 0;
    for (int lq = 0; lq < Q; ++lq) {
        const T pz = Tab<T>::P1(ps, lq, a2) * Tab<T>::P1(ps, lq, c2);
        T sp = 0;
        for (int jq = 0; jq < Q; ++jq) {
            const T py = Tab<T>::P1(ps, jq, a1) * Tab<T>::P1(ps, jq, c1);
            for (int iq = 0; iq < Q; ++iq) {
                const T* F = st0 + sr.f(3, lq, iq + Q * jq);
                const T wdj = F[0], muw = F[sr.fstride];
                sp += Tab<T>::P1(ps, iq, a0) * Tab<T>::P1(ps, iq, c0) * py * (wdj * (wdj / muw));
            }
        }
        s += double(pz * sp);
    }
    a.mblk[(e * a.npr + b1) * a.npr + b2] = s;
}

template <typename T>
int launch_precond_assembly_t(const ColArgs& a, cudaStream_t s) {
    if (a.E == 0) return int(cudaSuccess);
    const int64_t n1 = a.E * N3, n2 = a.E * a.npr * (a.schur_full ? a.npr : 1);
    colblock_kernel<T><<<unsigned((n1 + 255) / 256), 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return int(e);
    if (!a.mblk) return int(cudaSuccess);       // column blocks only (multigrid levels)
    schur_block_kernel<T><<<unsigned((n2 + 255) / 256), 256, 0, s>>>(a);
    return int(cudaGetLastError());
}

}  // namespace STOKES_NS
}  // namespace dev
}  // namespace stokes

#define STOKES_DEFINE_PRECOND(KK)                                                              \
    namespace stokes {                                                                         \
    int launch_precond_assembly_k##KK(int prec, const ColArgs& a, cudaStream_t s) {            \
        return prec == 1 ? dev::STOKES_NS::launch_precond_assembly_t<float>(a, s)              \
                         : dev::STOKES_NS::launch_precond_assembly_t<double>(a, s);            \
    }                                                                                          \
    }
