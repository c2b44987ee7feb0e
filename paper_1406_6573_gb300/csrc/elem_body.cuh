// Element kernels (volume terms) and basal-face kernels, one instantiation set
// per degree STOKES_K.  Included by k2.cu, k3.cu, k4.cu.
#pragma once

#include "elem_kernels.cuh"
#include "tma.cuh"

namespace stokes {
namespace dev {
namespace STOKES_NS {

// Physical gradient from the reference gradient at one quadrature point.
template <typename T>
__device__ __forceinline__ void phys_grad(const T (&G)[3][3][Q], int lq, const T (&Ji)[9], T (&g)[3][3]) {
    #pragma unroll
    for (int c = 0; c < 3; ++c)
        #pragma unroll
        for (int d = 0; d < 3; ++d)
            g[c][d] = G[c][0][lq] * Ji[d] + G[c][1][lq] * Ji[3 + d] + G[c][2][lq] * Ji[6 + d];
}

// Reference stress S[c][m] = sum_d Jinv[m][d] tau[c][d] written back into G.
template <typename T>
__device__ __forceinline__ void ref_stress(T (&G)[3][3][Q], int lq, const T (&Ji)[9], const T (&tau)[3][3]) {
    #pragma unroll
    for (int c = 0; c < 3; ++c)
        #pragma unroll
        for (int m = 0; m < 3; ++m)
            G[c][m][lq] = Ji[3 * m] * tau[c][0] + Ji[3 * m + 1] * tau[c][1] + Ji[3 * m + 2] * tau[c][2];
}

template <typename T>
__device__ __forceinline__ void load_geo(const ElemArgs& a, int64_t e, int qp, bool active, T (&Ji)[9], T& wdj) {
    if (active) {
        const double* gp = a.geo + e * 10 * Q3 + qp;
        #pragma unroll
        for (int f = 0; f < 9; ++f) Ji[f] = T(__ldg(gp + f * Q3));
        wdj = T(__ldg(gp + 9 * Q3));
    } else {
        #pragma unroll
        for (int f = 0; f < 9; ++f) Ji[f] = T(0);
        wdj = T(0);
    }
}

template <typename T>
__device__ __forceinline__ void sym6(const T (&g)[3][3], T& E00, T& E11, T& E22, T& E01, T& E02, T& E12) {
    E00 = g[0][0]; E11 = g[1][1]; E22 = g[2][2];
    E01 = T(0.5) * (g[0][1] + g[1][0]);
    E02 = T(0.5) * (g[0][2] + g[2][0]);
    E12 = T(0.5) * (g[1][2] + g[2][1]);
}

// ============================================================ volume kernel
// Generic element kernel (residual, fused Jacobian, linearisation, A-gradient).
// T: arithmetic type.  S: element type of the stored state (linearize).
// exchange scratch of one element slot: 9 buffers (3 per velocity component),
// padded so that consecutive slots start 12 banks apart (fewer shared-memory
// bank conflicts between the elements of a warp); a multiple of 16 bytes
// packed-line slot of the stored-state kernel: 9 buffers of N1^3 values,
// padded so that consecutive slots start N2 banks apart (FP32), which puts
// the N1^2 lanes of the EPW elements of a warp on distinct banks
template <typename T> constexpr int SLOT_PACKED =
    sizeof(T) == 4 ? (9 * N2 * N1 + 31 - N2) / 32 * 32 + N2 : 9 * N2 * N1 + 2;
template <typename T> constexpr int SLOT =
    sizeof(T) == 4 ? (9 * BUFLEN<T> + 31 - 12) / 32 * 32 + 12 : 9 * BUFLEN<T> + 2;

template <typename T, typename S, int MODE, bool TRANS>
__global__ void __launch_bounds__(32 * GW<T>) elem_kernel(ElemArgs a) {
    extern __shared__ __align__(16) unsigned char smem_dyn[];
    const LaneMap L;
    const int i = L.i, j = L.j, ij = L.ij, es = L.es;
    const int64_t e = int64_t(blockIdx.x) * (GW<T> * EPW) + L.warp * EPW + es;
    const bool active = (es < EPW) && (e < a.E);
    T* sb = reinterpret_cast<T*>(smem_dyn) + (L.warp * (EPW + 1) + es) * SLOT<T>;
    const uint32_t h = active ? a.hang[e] : 0u;
    const bool any_h = a.any_hang ? (__any_sync(0xffffffffu, (h & ((1u << HANG_CHILD0) - 1)) != 0) != 0) : false;
    const int ps = a.pspace;
    Rows<T> R;
    R.load(i, j);
    ColNodes cn;
    col_nodes(a, e, ij, active, cn);

    T G[3][3][Q];     // reference gradients, then reference stresses
    T gq[Q];          // pressure-row integrand  -w detJ div(.)

    if constexpr (MODE == MODE_RESIDUAL) {
        T v[3][N1];
        gather_velocity<T, T>(a, static_cast<const T*>(a.x), cn, e, active, ij, v);
        if (any_h) hanging_forward<T, 3>(v, h, active, i, j, sb);
        T pc[N1];
        pressure_fold<T, T>(a, static_cast<const T*>(a.x), e, active, i, j, pc);
        ref_gradient<T, 3>(R, v, G, i, j, sb);
        T Sv[3][Q];
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {
            T Ji[9], wdj;
            load_geo<T>(a, e, sidx(i, j, lq), active, Ji, wdj);
            T g[3][3];
            phys_grad(G, lq, Ji, g);
            T E00, E11, E22, E01, E02, E12;
            sym6(g, E00, E11, E22, E01, E02, E12);
            const T DD = E00 * E00 + E11 * E11 + E22 * E22 + T(2) * (E01 * E01 + E02 * E02 + E12 * E12);
            const T muw = viscosity<T>(a, DD) * wdj;
            const T pw = pressure_at<T>(pc, ps, lq) * wdj;
            T tau[3][3];
            tau[0][0] = muw * E00 - pw;
            tau[1][1] = muw * E11 - pw;
            tau[2][2] = muw * E22 - pw;
            tau[0][1] = tau[1][0] = muw * E01;
            tau[0][2] = tau[2][0] = muw * E02;
            tau[1][2] = tau[2][1] = muw * E12;
            gq[lq] = -wdj * (g[0][0] + g[1][1] + g[2][2]);
            #pragma unroll
            for (int c = 0; c < 3; ++c) Sv[c][lq] = -wdj * T(a.body[c]);
            ref_stress(G, lq, Ji, tau);
        }
        T out[3][N1];
        ref_gradient_T<T, 3, true>(R, G, Sv, out, i, j, sb);
        pressure_rows<T>(gq, a.npr, ps, i, j, ij, active, sb, static_cast<T*>(a.y) + 3 * a.Nv + e * a.npr);
        if (any_h) hanging_transpose<T, 3>(out, h, active, i, j, sb);
        scatter_velocity<T>(a, static_cast<T*>(a.y), cn, e, active, ij, out);
    } else if constexpr (MODE == MODE_APPLY) {
        // linearisation at u, recomputed at every quadrature point
        T lin[8][Q];     // mu w detJ, kappa w detJ, D(u) (6)
        {
            T v[3][N1];
            gather_velocity<T, T>(a, static_cast<const T*>(a.u), cn, e, active, ij, v);
            if (any_h) hanging_forward<T, 3>(v, h, active, i, j, sb);
            ref_gradient<T, 3>(R, v, G, i, j, sb);
            #pragma unroll
            for (int lq = 0; lq < Q; ++lq) {
                T Ji[9], wdj;
                load_geo<T>(a, e, sidx(i, j, lq), active, Ji, wdj);
                T g[3][3];
                phys_grad(G, lq, Ji, g);
                T E00, E11, E22, E01, E02, E12;
                sym6(g, E00, E11, E22, E01, E02, E12);
                const T DD = E00 * E00 + E11 * E11 + E22 * E22 + T(2) * (E01 * E01 + E02 * E02 + E12 * E12);
                const T mu = viscosity<T>(a, DD);
                lin[0][lq] = mu * wdj;
                // Picard: the viscosity is frozen at u, no derivative term
                lin[1][lq] = a.picard ? T(0)
                                      : T(2) * T(a.gamma) * T(a.pexp) * mu * wdj / (T(a.gamma) * DD + T(a.delta));
                lin[2][lq] = E00; lin[3][lq] = E11; lin[4][lq] = E22;
                lin[5][lq] = E01; lin[6][lq] = E02; lin[7][lq] = E12;
            }
        }
        T v[3][N1];
        gather_velocity<T, T>(a, static_cast<const T*>(a.x), cn, e, active, ij, v);
        if (any_h) hanging_forward<T, 3>(v, h, active, i, j, sb);
        T pc[N1];
        pressure_fold<T, T>(a, static_cast<const T*>(a.x), e, active, i, j, pc);
        ref_gradient<T, 3>(R, v, G, i, j, sb);
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {
            T Ji[9], wdj;
            load_geo<T>(a, e, sidx(i, j, lq), active, Ji, wdj);
            T g[3][3];
            phys_grad(G, lq, Ji, g);
            T E00, E11, E22, E01, E02, E12;
            sym6(g, E00, E11, E22, E01, E02, E12);
            const T muw = lin[0][lq], kw = lin[1][lq];
            const T D00 = lin[2][lq], D11 = lin[3][lq], D22 = lin[4][lq];
            const T D01 = lin[5][lq], D02 = lin[6][lq], D12 = lin[7][lq];
            // mu' E = mu E + kappa (D:E) D is a symmetric map on symmetric
            // tensors (Eq. 2.7): the transpose (TRANS) is the same contraction.
            const T s = kw * (D00 * E00 + D11 * E11 + D22 * E22 + T(2) * (D01 * E01 + D02 * E02 + D12 * E12));
            const T pw = pressure_at<T>(pc, ps, lq) * wdj;
            T tau[3][3];
            tau[0][0] = muw * E00 + s * D00 - pw;
            tau[1][1] = muw * E11 + s * D11 - pw;
            tau[2][2] = muw * E22 + s * D22 - pw;
            tau[0][1] = tau[1][0] = muw * E01 + s * D01;
            tau[0][2] = tau[2][0] = muw * E02 + s * D02;
            tau[1][2] = tau[2][1] = muw * E12 + s * D12;
            gq[lq] = -wdj * (g[0][0] + g[1][1] + g[2][2]);
            ref_stress(G, lq, Ji, tau);
        }
        T out[3][N1];
        T dummy[3][Q];
        ref_gradient_T<T, 3, false>(R, G, dummy, out, i, j, sb);
        pressure_rows<T>(gq, a.npr, ps, i, j, ij, active, sb, static_cast<T*>(a.y) + 3 * a.Nv + e * a.npr);
        if (any_h) hanging_transpose<T, 3>(out, h, active, i, j, sb);
        scatter_velocity<T>(a, static_cast<T*>(a.y), cn, e, active, ij, out);
    } else if constexpr (MODE == MODE_LINEARIZE) {
        T v[3][N1];
        gather_velocity<T, double>(a, a.ud, cn, e, active, ij, v);
        if (any_h) hanging_forward<T, 3>(v, h, active, i, j, sb);
        ref_gradient<T, 3>(R, v, G, i, j, sb);
        S* st = static_cast<S*>(a.state);
        const StateRef sr(active ? e : 0, a.state_cpl);
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {
            const int qp = sidx(i, j, lq);
            T Ji[9], wdj;
            load_geo<T>(a, e, qp, active, Ji, wdj);
            T g[3][3];
            phys_grad(G, lq, Ji, g);
            T E00, E11, E22, E01, E02, E12;
            sym6(g, E00, E11, E22, E01, E02, E12);
            const T DD = E00 * E00 + E11 * E11 + E22 * E22 + T(2) * (E01 * E01 + E02 * E02 + E12 * E12);
            const T mu = viscosity<T>(a, DD);
            // -kappa w detJ >= 0 because p_n = (1-n)/(2n) <= 0
            const T mk = -T(2) * T(a.gamma) * T(a.pexp) * mu * wdj / (T(a.gamma) * DD + T(a.delta));
            const T sq = (a.picard || !(mk > T(0))) ? T(0) : sqrt(mk);   // Picard: no rank-one term
            if (active) {
                S* F = st + sr.f(0, lq, i + N1 * j);
                const int fs = sr.fstride;
                if (qp == 0) { st[sr.c(0)] = S(Ji[0]); st[sr.c(1)] = S(Ji[4]); }
                F[0] = S(Ji[6]);
                F[fs] = S(Ji[7]);
                F[2 * fs] = S(Ji[8]);
                F[3 * fs] = S(wdj);
                F[4 * fs] = S(mu * wdj);
                F[5 * fs] = S(sq * E00);
                F[6 * fs] = S(sq * E11);
                F[7 * fs] = S(sq * E22);
                F[8 * fs] = S(sq * E01);
                F[9 * fs] = S(sq * E02);
                F[10 * fs] = S(sq * E12);
                if (a.state2) {
                    // the FP64 state of the same linearisation point
                    double* st2 = a.state2;
                    const StateRef sr2(e, a.state2_cpl);
                    double* F2 = st2 + sr2.f(0, lq, i + N1 * j);
                    const int fs2 = sr2.fstride;
                    if (qp == 0) { st2[sr2.c(0)] = double(Ji[0]); st2[sr2.c(1)] = double(Ji[4]); }
                    F2[0] = double(Ji[6]);
                    F2[fs2] = double(Ji[7]);
                    F2[2 * fs2] = double(Ji[8]);
                    F2[3 * fs2] = double(wdj);
                    F2[4 * fs2] = double(mu * wdj);
                    F2[5 * fs2] = double(sq * E00);
                    F2[6 * fs2] = double(sq * E11);
                    F2[7 * fs2] = double(sq * E22);
                    F2[8 * fs2] = double(sq * E01);
                    F2[9 * fs2] = double(sq * E02);
                    F2[10 * fs2] = double(sq * E12);
                }
            }
        }
    } else if constexpr (MODE == MODE_GRAD_A || MODE == MODE_GRAD_A_PARTIAL) {
        T acc = 0;
        T Gl[3][3][Q];
        {
            T v[3][N1];
            gather_velocity<T, double>(a, a.lam, cn, e, active, ij, v);
            if (any_h) hanging_forward<T, 3>(v, h, active, i, j, sb);
            ref_gradient<T, 3>(R, v, Gl, i, j, sb);
        }
        T v[3][N1];
        gather_velocity<T, double>(a, a.ud, cn, e, active, ij, v);
        if (any_h) hanging_forward<T, 3>(v, h, active, i, j, sb);
        ref_gradient<T, 3>(R, v, G, i, j, sb);
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {
            T Ji[9], wdj;
            load_geo<T>(a, e, sidx(i, j, lq), active, Ji, wdj);
            T g[3][3], gl[3][3];
            phys_grad(G, lq, Ji, g);
            phys_grad(Gl, lq, Ji, gl);
            T DD = 0, DL = 0;
            #pragma unroll
            for (int c = 0; c < 3; ++c)
                #pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const T Du = T(0.5) * (g[c][d] + g[d][c]);
                    const T Dl = T(0.5) * (gl[c][d] + gl[d][c]);
                    DD += Du * Du;
                    DL += Dl * Du;
                }
            if (active) acc += viscosity<T>(a, DD) * wdj * DL;
        }
        double r = double(acc);
        #pragma unroll
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
        if (L.lane == 0) {
            if constexpr (MODE == MODE_GRAD_A) atomicAdd(a.gA, r * a.gA_scale);
            else a.gA_part[int64_t(blockIdx.x) * GW<T> + L.warp] = r;
        }
    }
}

// ============================================================ basal faces
// Robin term int_{Gamma_b} beta T v . T w ds (Eq. 2.4a in weak form, Eq. 2.5)
// and its log(beta) adjoint product.  One lane per bottom-plane node (i, j) of
// a basal element; 2-D sum factorisation through warp-local shared memory.
template <typename T>
__device__ __forceinline__ void face_gather(const FaceArgs& a, const T* x, int64_t e, bool active, int ij,
                                            T (&v)[3]) {
    if (active) {
        const int64_t g = a.nodes[e * N3 + ij];
        v[0] = T(ld(x + 3 * g)); v[1] = T(ld(x + 3 * g + 1)); v[2] = T(ld(x + 3 * g + 2));
        const int pi = a.pidx[e];
        if (pi >= 0) project3<T>(a.pel + int64_t(pi) * 6 * N2 + ij, v[0], v[1], v[2]);
    } else {
        v[0] = v[1] = v[2] = T(0);
    }
}

// Hanging interpolation on the bottom plane: x-sweeps then y-sweeps (forward)
// or y^T then x^T (transpose), for NC values per slot held in v.
template <typename T, int NC, bool TRANSPOSE>
__device__ void face_hanging(T (&v)[NC], uint32_t h, bool active, int i, int j, T* sb) {
    #pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
        const int axis = TRANSPOSE ? 1 - pass : pass;   // forward: x then y
        #pragma unroll
        for (int c = 0; c < NC; ++c) sb[c * N2 + i + N1 * j] = v[c];
        wsync();
        if (active && h) {
            const int bb = child_bit(h, axis);
            const bool on = (axis == 0) ? line_hanging(h, 0, j, 0, K) : line_hanging(h, 1, i, 0, K);
            if (on) {
                #pragma unroll
                for (int c = 0; c < NC; ++c) {
                    T s = 0;
                    #pragma unroll
                    for (int m = 0; m < N1; ++m) {
                        const T val = (axis == 0) ? sb[c * N2 + m + N1 * j] : sb[c * N2 + i + N1 * m];
                        const int me = (axis == 0) ? i : j;
                        s += (TRANSPOSE ? Tab<T>::I(bb, m, me) : Tab<T>::I(bb, me, m)) * val;
                    }
                    v[c] = s;
                }
            }
        }
        wsync();
    }
}

// values at the face Gauss points (iq = i, jq = j) from bottom-plane nodal values
template <typename T, int NC>
__device__ __forceinline__ void face_interp(const Rows<T>& R, const T (&v)[NC], T (&o)[NC], int i, int j, T* sb) {
    #pragma unroll
    for (int c = 0; c < NC; ++c) sb[c * N2 + i + N1 * j] = v[c];
    wsync();
    T t[NC];
    #pragma unroll
    for (int c = 0; c < NC; ++c) {
        T s = 0;
        #pragma unroll
        for (int m = 0; m < N1; ++m) s += R.Bi[m] * sb[c * N2 + m + N1 * j];
        t[c] = s;
    }
    wsync();
    #pragma unroll
    for (int c = 0; c < NC; ++c) sb[c * N2 + i + N1 * j] = t[c];
    wsync();
    #pragma unroll
    for (int c = 0; c < NC; ++c) {
        T s = 0;
        #pragma unroll
        for (int m = 0; m < N1; ++m) s += R.Bj[m] * sb[c * N2 + i + N1 * m];
        o[c] = s;
    }
    wsync();
}

// transposed interpolation: nodal values from values at face Gauss points
template <typename T, int NC>
__device__ __forceinline__ void face_interp_T(const Rows<T>& R, const T (&v)[NC], T (&o)[NC], int i, int j, T* sb) {
    #pragma unroll
    for (int c = 0; c < NC; ++c) sb[c * N2 + i + N1 * j] = v[c];
    wsync();
    T t[NC];
    #pragma unroll
    for (int c = 0; c < NC; ++c) {
        T s = 0;
        #pragma unroll
        for (int m = 0; m < Q; ++m) s += R.BTi[m] * sb[c * N2 + m + N1 * j];
        t[c] = s;
    }
    wsync();
    #pragma unroll
    for (int c = 0; c < NC; ++c) sb[c * N2 + i + N1 * j] = t[c];
    wsync();
    #pragma unroll
    for (int c = 0; c < NC; ++c) {
        T s = 0;
        #pragma unroll
        for (int m = 0; m < Q; ++m) s += R.BTj[m] * sb[c * N2 + i + N1 * m];
        o[c] = s;
    }
    wsync();
}

// One group of EPW basal faces (faces fg * EPW + fs) on one warp; sb: the
// lane's element scratch (4 N2 values).  Called by face_kernel and by the
// stored-state kernel after its element groups.
template <typename T, int MODE>
__device__ __forceinline__ void face_group(const FaceArgs& a, const LaneMap& L, const Rows<T>& R, int64_t fg,
                                           T* sb) {
    constexpr int Q2 = Q * Q;
    const int i = L.i, j = L.j, ij = L.ij, fs = L.es;
    const int64_t f = fg * EPW + fs;
    const bool active = (fs < EPW) && (f < a.nF);
    const int64_t e = active ? a.face_elem[f] : 0;
    const uint32_t h = active ? a.hang[e] : 0u;
    const bool any_h = __any_sync(0xffffffffu, (h & ((1u << HANG_CHILD0) - 1)) != 0) != 0;

    // log(beta) at the face nodes (hanging-interpolated), then at Gauss points
    T lb[1];
    lb[0] = active ? T(a.logbeta[a.fmap[f * N2 + ij]]) : T(0);
    if (any_h) face_hanging<T, 1, false>(lb, h, active, i, j, sb);
    T lbq[1];
    face_interp<T, 1>(R, lb, lbq, i, j, sb);
    const int fq = i + Q * j;
    T wa = 0, n0 = 0, n1 = 0, n2 = 0;
    if (active) {
        const double* fg = a.fgeo + f * 4 * Q2 + fq;
        wa = T(fg[0]); n0 = T(fg[Q2]); n1 = T(fg[2 * Q2]); n2 = T(fg[3 * Q2]);
    }
    const T bw = exp(lbq[0]) * wa;

    // sliding law factor s(x) = (x + eps)^((m - 1)/2) and its derivative
    auto slide_s = [&](T x2, T& ds) -> T {
        const T xe = x2 + T(a.slide_eps);
        const T sv = pow(xe, T(0.5) * (T(a.slide_m) - T(1)));
        ds = a.slide_picard ? T(0) : T(0.5) * (T(a.slide_m) - T(1)) * sv / xe;
        return sv;
    };

    if constexpr (MODE == FACE_APPLY) {
        T v[3];
        face_gather<T>(a, static_cast<const T*>(a.x), e, active, ij, v);
        if (any_h) face_hanging<T, 3, false>(v, h, active, i, j, sb);
        T vq[3];
        face_interp<T, 3>(R, v, vq, i, j, sb);
        const T nv = n0 * vq[0] + n1 * vq[1] + n2 * vq[2];
        const T tw[3] = {vq[0] - nv * n0, vq[1] - nv * n1, vq[2] - nv * n2};
        T t[3] = {bw * tw[0], bw * tw[1], bw * tw[2]};
        if (a.slide) {
            if (a.fstate) {
                // stored linearisation: beta w s T w + (v . w) T u
                if (active) {
                    const T* sst = static_cast<const T*>(a.fstate) + f * SLIDE_FIELDS * Q2 + fq;
                    const T bws = sst[0];
                    const T vw = sst[Q2] * vq[0] + sst[2 * Q2] * vq[1] + sst[3 * Q2] * vq[2];
                    #pragma unroll
                    for (int c = 0; c < 3; ++c) t[c] = bws * tw[c] + vw * sst[(4 + c) * Q2];
                }
            } else if (a.ulin) {
                // Jacobian at u: beta w (s T w + 2 s' (T u . T w) T u)
                T uu[3];
                face_gather<T>(a, static_cast<const T*>(a.ulin), e, active, ij, uu);
                if (any_h) face_hanging<T, 3, false>(uu, h, active, i, j, sb);
                T uq[3];
                face_interp<T, 3>(R, uu, uq, i, j, sb);
                const T nu = n0 * uq[0] + n1 * uq[1] + n2 * uq[2];
                const T tu[3] = {uq[0] - nu * n0, uq[1] - nu * n1, uq[2] - nu * n2};
                T ds;
                const T sv = slide_s(tu[0] * tu[0] + tu[1] * tu[1] + tu[2] * tu[2], ds);
                const T r = T(2) * ds * (tu[0] * tw[0] + tu[1] * tw[1] + tu[2] * tw[2]);
                #pragma unroll
                for (int c = 0; c < 3; ++c) t[c] = bw * (sv * tw[c] + r * tu[c]);
            } else {
                // residual (u = x): beta w s T u
                T ds;
                const T sv = slide_s(tw[0] * tw[0] + tw[1] * tw[1] + tw[2] * tw[2], ds);
                #pragma unroll
                for (int c = 0; c < 3; ++c) t[c] = bw * sv * tw[c];
            }
        }
        T o[3];
        face_interp_T<T, 3>(R, t, o, i, j, sb);
        if (any_h) face_hanging<T, 3, true>(o, h, active, i, j, sb);
        if (active) {
            const int pi = a.pidx[e];
            if (pi >= 0) project3<T>(a.pel + int64_t(pi) * 6 * N2 + ij, o[0], o[1], o[2]);
            const int64_t g = a.nodes[e * N3 + ij];
            T* y = static_cast<T*>(a.y);
            atomic_add(y + 3 * g, o[0]);
            atomic_add(y + 3 * g + 1, o[1]);
            atomic_add(y + 3 * g + 2, o[2]);
        }
    } else if constexpr (MODE == FACE_LINEARIZE) {
        // stored sliding state at the linearisation point a.u (FP64 arithmetic)
        T v[3];
        face_gather<T>(a, a.u, e, active, ij, v);
        if (any_h) face_hanging<T, 3, false>(v, h, active, i, j, sb);
        T uq[3];
        face_interp<T, 3>(R, v, uq, i, j, sb);
        const T nu = n0 * uq[0] + n1 * uq[1] + n2 * uq[2];
        const T tu[3] = {uq[0] - nu * n0, uq[1] - nu * n1, uq[2] - nu * n2};
        T ds = T(0), sv = T(1);       // linear law: s = 1, s' = 0
        if (a.slide) sv = slide_s(tu[0] * tu[0] + tu[1] * tu[1] + tu[2] * tu[2], ds);
        const T vals[SLIDE_FIELDS] = {bw * sv, T(2) * ds * bw * tu[0], T(2) * ds * bw * tu[1],
                                      T(2) * ds * bw * tu[2], tu[0], tu[1], tu[2], n0, n1, n2};
        if (active) {
            const int64_t o0 = f * SLIDE_FIELDS * Q2 + fq;
            #pragma unroll
            for (int c = 0; c < SLIDE_FIELDS; ++c) {
                if (a.fstate_f32) static_cast<float*>(a.fstate_out)[o0 + c * Q2] = float(vals[c]);
                else static_cast<double*>(a.fstate_out)[o0 + c * Q2] = double(vals[c]);
            }
        }
    } else {
        // g_j += int beta s(|T u|^2) phi_j (T lambda) . (T u) ds
        T v[3], w[3];
        face_gather<T>(a, a.u, e, active, ij, v);
        face_gather<T>(a, a.lam, e, active, ij, w);
        if (any_h) {
            face_hanging<T, 3, false>(v, h, active, i, j, sb);
            face_hanging<T, 3, false>(w, h, active, i, j, sb);
        }
        T vq[3], wq[3];
        face_interp<T, 3>(R, v, vq, i, j, sb);
        face_interp<T, 3>(R, w, wq, i, j, sb);
        const T nu = n0 * vq[0] + n1 * vq[1] + n2 * vq[2];
        const T nl = n0 * wq[0] + n1 * wq[1] + n2 * wq[2];
        const T tu[3] = {vq[0] - nu * n0, vq[1] - nu * n1, vq[2] - nu * n2};
        T sl = T(1);
        if (a.slide) {
            T ds;
            sl = slide_s(tu[0] * tu[0] + tu[1] * tu[1] + tu[2] * tu[2], ds);
        }
        const T s = bw * sl * (tu[0] * (wq[0] - nl * n0) + tu[1] * (wq[1] - nl * n1) + tu[2] * (wq[2] - nl * n2));
        T sv[1] = {s}, o[1];
        face_interp_T<T, 1>(R, sv, o, i, j, sb);
        if (any_h) face_hanging<T, 1, true>(o, h, active, i, j, sb);
        if (active) atomic_add(a.g + a.fmap[f * N2 + ij], double(o[0]));
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(THREADS) face_kernel(FaceArgs a) {
    __shared__ T sbuf[WARPS][EPW + 1][4 * N2];
    const LaneMap L;
    Rows<T> R;
    R.load(L.i, L.j);
    face_group<T, MODE>(a, L, R, int64_t(blockIdx.x) * WARPS + L.warp, sbuf[L.warp][L.es]);
}

// constraint rows y += s (I - P) x at basal nodes b = b0 + t * bstride (atomic:
// run alongside other contributions to y)
template <typename T>
__device__ __forceinline__ void constraint_rows(const ElemArgs& a, int64_t b0, int64_t bstride) {
    const T* x = static_cast<const T*>(a.face.x);
    T* y = static_cast<T*>(a.face.y);
    const T sc = T(a.cscale);
    for (int64_t b = b0; b < a.Nb; b += bstride) {
        const int64_t g = a.basal_nodes[b];
        const double* p = a.basal_P + 6 * b;
        const T x0 = x[3 * g], x1 = x[3 * g + 1], x2 = x[3 * g + 2];
        const T p00 = T(p[0]), p11 = T(p[1]), p22 = T(p[2]), p01 = T(p[3]), p02 = T(p[4]), p12 = T(p[5]);
        atomic_add(y + 3 * g, sc * (x0 - (p00 * x0 + p01 * x1 + p02 * x2)));
        atomic_add(y + 3 * g + 1, sc * (x1 - (p01 * x0 + p11 * x1 + p12 * x2)));
        atomic_add(y + 3 * g + 2, sc * (x2 - (p02 * x0 + p12 * x1 + p22 * x2)));
    }
}

// ================================================== state apply (hot path)
// Line exchanges of the sum factorisation in the stored-state kernel: warp
// shuffles for degrees >= STOKES_STATE_SHFL_MIN_K, shared memory below
// (measured per degree).
#ifndef STOKES_STATE_SHFL_MIN_K
#define STOKES_STATE_SHFL_MIN_K 3
#endif
constexpr bool STATE_SHFL = K >= STOKES_STATE_SHFL_MIN_K;
// shared-memory exchange of the stored-state kernel with packed lines
// (pitch N1) instead of 16-byte padded lines
#ifndef STOKES_STATE_PACKED
#define STOKES_STATE_PACKED 1
#endif
template <typename T> constexpr int STATE_PITCH = STOKES_STATE_PACKED ? N1 : LP<T>;
// exchange slot of one element (the shuffle variant needs it only for the
// pressure rows, 3 N3 values, the hanging-node sweeps and the basal tail;
// consecutive slots start 16 banks apart)
constexpr int SHFL_SLOT = (3 * N3 + 3) / 4 * 4 + ((((3 * N3 + 3) / 4 * 4) % 32 == 0) ? 16 : 0);
template <typename T> constexpr int STATE_SLOT =
    STATE_SHFL ? SHFL_SLOT : (STOKES_STATE_PACKED ? SLOT_PACKED<T> : SLOT<T>);
// latency of the next group's gather hidden behind the current group:
// 0 none, 1 L1 prefetch of the node lines (conforming lattice meshes)
#ifndef STOKES_STATE_PREFETCH
#define STOKES_STATE_PREFETCH 1
#endif
// the streamed state copied with an L2 evict-first policy (off: on the
// 64x64x4 Q3xQ1 slab 0.0491 ms with it against 0.0472 ms without)
#ifndef STOKES_STATE_EVICT_FIRST
#define STOKES_STATE_EVICT_FIRST 0
#endif
// y = J x from the stored linearised state.  Persistent: each warp walks its
// element groups (EPW consecutive elements); the state block of the next
// group (contiguous, 16-byte multiple) is staged into shared memory by a bulk
// asynchronous copy (TMA, cp.async.bulk) completing on a per-warp mbarrier,
// double-buffered, so the state stream overlaps the gather and the forward
// contractions of the current group.
template <typename T>
struct StateApplyCfg {
    // warps per block and resident blocks per SM asked of the compiler
    // (measured on the 64x64x4 slabs and forest): FP32 k = 2 (hanging-node
    // meshes) 8 x 2 at 128 registers; FP32 k = 3 4 x 4 (128 registers, 16
    // warps per SM: 0.059 -> 0.048 ms on the Q3xQ1 slab, forest 0.381 ->
    // 0.284 ms); FP32 k = 4 4 x 3 (168 registers: 0.196 -> 0.166 ms); FP64 4 x 1
#ifdef STATE_W_F32
    static constexpr int W = sizeof(T) == 8 ? 4 : STATE_W_F32;
#else
    static constexpr int W = sizeof(T) == 8 ? 4 : (K == 2 ? 8 : 4);
#endif
#ifdef STATE_MINB_F32
    static constexpr int MINB = sizeof(T) == 4 ? STATE_MINB_F32 : 1;
#else
    static constexpr int MINB = sizeof(T) == 8 ? 1 : (K == 2 ? 2 : (K == 3 ? 4 : 3));
#endif
    static constexpr int BUF = EPW * SSTRIDE;                // values per stage buffer
    static constexpr int SCR = (EPW + 1) * STATE_SLOT<T>;    // scratch per warp
    static constexpr int PER_WARP = ((2 * BUF + SCR) * int(sizeof(T)) + 127) / 128 * 128;
    static constexpr int SMEM = W * PER_WARP + W * 2 * 8;
};

// bytes of the state prefix PONLY reads per element (2 + shift + 4 q^3 values, 16-byte multiple)
template <typename T> constexpr uint32_t STATE_PREFIX_BYTES = ((3 + 4 * Q3) * sizeof(T) + 15) / 16 * 16;

// PONLY: the velocity part of x is taken as zero (B^T p only, used by the
// block preconditioner): no gather, no forward contractions, no pressure rows.
template <typename T, bool PONLY>
__global__ void __launch_bounds__(32 * StateApplyCfg<T>::W, StateApplyCfg<T>::MINB) state_apply_kernel(ElemArgs a) {
    using C = StateApplyCfg<T>;
    constexpr uint32_t PREFIX_BYTES = STATE_PREFIX_BYTES<T>;
    static_assert(STATE_PREFIX_BYTES<T> <= SSTRIDE * sizeof(T), "prefix inside the element block");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const LaneMap L;
    const int i = L.i, j = L.j, ij = L.ij, es = L.es, lane = L.lane;
    unsigned char* wbase = smem_raw + L.warp * C::PER_WARP;
    // stage buffer b of this warp (computed, not an indexed pointer array,
    // which would live in local memory)
    T* const stage0 = reinterpret_cast<T*>(wbase);
    auto stage = [&](int b) { return stage0 + b * C::BUF; };
    T* scratch = reinterpret_cast<T*>(wbase) + 2 * C::BUF;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + C::W * C::PER_WARP) + 2 * L.warp;
    T* sb = scratch + es * STATE_SLOT<T>;
    const int ps = a.pspace;
    const T* S = static_cast<const T*>(a.cstate);
    const T* x = static_cast<const T*>(a.x);
    T* y = static_cast<T*>(a.y);
    Rows<T> R;
    R.load(i, j);

    const int64_t ngroups = (a.E + EPW - 1) / EPW;
    const int64_t gstride = int64_t(gridDim.x) * C::W;
    int64_t g = int64_t(blockIdx.x) * C::W + L.warp;

    auto group_elems = [&](int64_t gg) -> int {
        return int((a.E - gg * EPW) < EPW ? (a.E - gg * EPW) : EPW);
    };
    // stage the state of group gg into buffer b (lane 0).  PONLY needs only the
    // leading fields of each element block (1/a, 1/b, Jinv row 3, w detJ):
    // one copy per element of that prefix instead of the whole group block.
    auto stage_group = [&](int64_t gg, int b) {
        const int ne = group_elems(gg);
        if constexpr (PONLY) {
            mbar_arrive_expect_tx(&bar[b], uint32_t(ne) * PREFIX_BYTES);
            for (int ee = 0; ee < ne; ++ee)
                bulk_g2s(stage(b) + ee * SSTRIDE, S + (gg * EPW + ee) * SSTRIDE, PREFIX_BYTES, &bar[b]);
        } else {
            const uint32_t nb = uint32_t(ne * SSTRIDE * int64_t(sizeof(T)));
            mbar_arrive_expect_tx(&bar[b], nb);
#if STOKES_STATE_EVICT_FIRST
            bulk_g2s_hint(stage(b), S + gg * EPW * SSTRIDE, nb, &bar[b], l2_evict_first_policy());
#else
            bulk_g2s(stage(b), S + gg * EPW * SSTRIDE, nb, &bar[b]);
#endif
        }
    };
    if (lane == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (g < ngroups && lane == 0) stage_group(g, 0);
    for (int it = 0; g < ngroups; g += gstride, ++it) {
        const int buf = it & 1;
        // prefetch the next group into the other buffer (its readers finished
        // at the end of the previous iteration)
        if (lane == 0 && g + gstride < ngroups) {
            fence_proxy_async();
            stage_group(g + gstride, buf ^ 1);
        }
        const int64_t e = g * EPW + es;
        const bool active = (es < EPW) && (e < a.E);
        ColNodes cn;
        col_nodes(a, e, ij, active, cn);
        const uint32_t h = (active && a.any_hang) ? a.hang[e] : 0u;
        const bool any_h = a.any_hang ? (__any_sync(0xffffffffu, (h & ((1u << HANG_CHILD0) - 1)) != 0) != 0) : false;
#if STOKES_STATE_PREFETCH == 1
        {
            // the next group's node lines, pressure block and projector index
            const int64_t en = (g + gstride) * EPW + es;
            if (es < EPW && en < a.E) {
                if (!PONLY && a.lat_nx > 0) {
                    ColNodes cnn;
                    col_nodes(a, en, ij, true, cnn);
                    #pragma unroll
                    for (int l = 0; l < N1; ++l) prefetch_l1(x + 3 * int64_t(cnn.g[l]));
                }
                if (ij == 0) {
                    prefetch_l1(x + 3 * a.Nv + en * a.npr);
                    prefetch_l1(a.pidx + en);
                }
            }
        }
#endif

        T pc[N1];
        pressure_fold<T, T>(a, x, e, active, i, j, pc);
        T G[3][3][Q];
        if constexpr (!PONLY) {
            T v[3][N1];
            gather_velocity<T, T>(a, x, cn, e, active, ij, v);
            if (any_h) hanging_forward<T, 3>(v, h, active, i, j, sb);
            if constexpr (STATE_SHFL) ref_gradient<T, 3>(R, v, G, i, j, sb);
            else ref_gradient_smem<T, 3, STATE_PITCH<T>>(R, v, G, i, j, sb);
        } else {
            #pragma unroll
            for (int c = 0; c < 3; ++c)
                #pragma unroll
                for (int m = 0; m < 3; ++m)
                    #pragma unroll
                    for (int lq = 0; lq < Q; ++lq) G[c][m][lq] = T(0);
        }

        if (!mbar_wait_polls(&bar[buf], uint32_t((it >> 1) & 1), a.wait_polls)) {
            // the staged state never arrived: report, let this warp's copies
            // drain (this group's, and the next group's issued into the other
            // buffer at the top of this iteration), stop
            if (lane == 0) atomicOr(a.err, 1);
            mbar_wait_bounded(&bar[buf], uint32_t((it >> 1) & 1));
            if (g + gstride < ngroups) mbar_wait_bounded(&bar[buf ^ 1], uint32_t(((it + 1) >> 1) & 1));
            return;
        }
        const T* st = stage(buf) + (es < EPW ? es : 0) * SSTRIDE;
        const T ia = st[0], ib = st[1];
        T gq[Q];
        #pragma unroll
        for (int lq = 0; lq < Q; ++lq) {
            const T* f = st + 2 + state_shift(es) + sidx(i, j, lq);
            const T g0 = f[0], g1 = f[Q3], g2 = f[2 * Q3];
            const T wdj = f[3 * Q3];
            if constexpr (PONLY) {
                // tau = -p w detJ I; reference stress S[c][m] = Jinv[m][c] tau_cc
                const T pw = active ? pressure_at<T>(pc, ps, lq) * wdj : T(0);
                G[0][0][lq] = -ia * pw; G[0][1][lq] = T(0); G[0][2][lq] = -g0 * pw;
                G[1][0][lq] = T(0); G[1][1][lq] = -ib * pw; G[1][2][lq] = -g1 * pw;
                G[2][0][lq] = T(0); G[2][1][lq] = T(0); G[2][2][lq] = -g2 * pw;
                gq[lq] = T(0);
                continue;
            }
            const T muw = f[4 * Q3];
            const T D00 = f[5 * Q3], D11 = f[6 * Q3], D22 = f[7 * Q3];
            const T D01 = f[8 * Q3], D02 = f[9 * Q3], D12 = f[10 * Q3];
            // physical gradient: Jinv = [[ia,0,0],[0,ib,0],[g0,g1,g2]]
            T gr[3][3];
            #pragma unroll
            for (int c = 0; c < 3; ++c) {
                const T gz = G[c][2][lq];
                gr[c][0] = G[c][0][lq] * ia + gz * g0;
                gr[c][1] = G[c][1][lq] * ib + gz * g1;
                gr[c][2] = gz * g2;
            }
            T E00, E11, E22, E01, E02, E12;
            sym6(gr, E00, E11, E22, E01, E02, E12);
            // Eq. 2.7 as a symmetric map: w detJ mu' E = muw E - (Dhat:E) Dhat
            const T s = D00 * E00 + D11 * E11 + D22 * E22 + T(2) * (D01 * E01 + D02 * E02 + D12 * E12);
            const T pw = active ? pressure_at<T>(pc, ps, lq) * wdj : T(0);
            T tau[3][3];
            tau[0][0] = muw * E00 - s * D00 - pw;
            tau[1][1] = muw * E11 - s * D11 - pw;
            tau[2][2] = muw * E22 - s * D22 - pw;
            tau[0][1] = tau[1][0] = muw * E01 - s * D01;
            tau[0][2] = tau[2][0] = muw * E02 - s * D02;
            tau[1][2] = tau[2][1] = muw * E12 - s * D12;
            gq[lq] = -wdj * (gr[0][0] + gr[1][1] + gr[2][2]);
            // reference stress S[c][m] = sum_d Jinv[m][d] tau[c][d]
            #pragma unroll
            for (int c = 0; c < 3; ++c) {
                G[c][0][lq] = ia * tau[c][0];
                G[c][1][lq] = ib * tau[c][1];
                G[c][2][lq] = g0 * tau[c][0] + g1 * tau[c][1] + g2 * tau[c][2];
            }
        }
        __syncwarp();
        T out[3][N1];
        T dummy[3][Q];
        if constexpr (STATE_SHFL) ref_gradient_T<T, 3, false>(R, G, dummy, out, i, j, sb);
        else ref_gradient_T_smem<T, 3, false, STATE_PITCH<T>>(R, G, dummy, out, i, j, sb);
        if constexpr (!PONLY) pressure_rows<T>(gq, a.npr, ps, i, j, ij, active, sb, y + 3 * a.Nv + e * a.npr);
        if (any_h) hanging_transpose<T, 3>(out, h, active, i, j, sb);
        scatter_velocity<T>(a, y, cn, e, active, ij, out);
        __syncwarp();
    }
    if constexpr (!PONLY) {
        // basal terms of the same apply, after this warp's element groups
        const int64_t w0 = int64_t(blockIdx.x) * C::W + L.warp;
        if (a.fuse_robin) {
            const int64_t nfg = (a.face.nF + EPW - 1) / EPW;
            for (int64_t fg = w0; fg < nfg; fg += gstride) face_group<T, FACE_APPLY>(a.face, L, R, fg, sb);
        }
        if (a.fuse_constraint) constraint_rows<T>(a, w0 * 32 + lane, gstride * 32);
    }
}


// ---------------------------------------------------------------- launchers
// warps launched by the FP64 element kernel over E elements (whole blocks):
// the number of per-warp partials written in MODE_GRAD_A_PARTIAL
inline int64_t grad_a_partials(int64_t E) {
    const int64_t epb = GW<double> * EPW;
    return (E + epb - 1) / epb * GW<double>;
}

template <typename T, typename S, int MODE, bool TRANS>
int launch_elem_t(const ElemArgs& a, cudaStream_t s) {
    const int64_t epb = GW<T> * EPW;
    const int64_t blocks = (a.E + epb - 1) / epb;
    if (blocks == 0) return int(cudaSuccess);
    const int smem = GW<T> * (EPW + 1) * SLOT<T> * int(sizeof(T));
    static int configured_device = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_device != dev) {
        cudaError_t e = cudaFuncSetAttribute(elem_kernel<T, S, MODE, TRANS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return int(e);
        configured_device = dev;
    }
    elem_kernel<T, S, MODE, TRANS><<<unsigned(blocks), 32 * GW<T>, smem, s>>>(a);
    return int(cudaGetLastError());
}

template <typename T, bool PONLY>
int launch_state_apply_t(const ElemArgs& a, cudaStream_t s) {
    using C = StateApplyCfg<T>;
    if (a.E == 0) return int(cudaSuccess);
    static int configured_device = -1;
    static int max_blocks = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_device != dev) {
        cudaError_t e = cudaFuncSetAttribute(state_apply_kernel<T, PONLY>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return int(e);
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, state_apply_kernel<T, PONLY>, 32 * C::W, C::SMEM);
        if (e != cudaSuccess) return int(e);
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return int(e);
        max_blocks = (per_sm > 0 ? per_sm : 1) * sms;
        configured_device = dev;
    }
    const int64_t blocks = persistent_blocks((a.E + EPW - 1) / EPW, C::W, max_blocks);
    state_apply_kernel<T, PONLY><<<unsigned(blocks), 32 * C::W, C::SMEM, s>>>(a);
    return int(cudaGetLastError());
}

template <typename T, int MODE>
int launch_face_t(const FaceArgs& a, cudaStream_t s) {
    const int64_t blocks = (a.nF + EPB - 1) / EPB;
    if (blocks == 0) return int(cudaSuccess);
    face_kernel<T, MODE><<<unsigned(blocks), THREADS, 0, s>>>(a);
    return int(cudaGetLastError());
}

}  // namespace STOKES_NS
}  // namespace dev
}  // namespace stokes

#include "cpl_apply.cuh"

namespace stokes {
namespace dev {
namespace STOKES_NS {

inline int launch_elem_any(int mode, int prec, int state_prec, bool trans, const ElemArgs& a, cudaStream_t s) {
    const bool f32 = prec == 1;
    switch (mode) {
        case MODE_RESIDUAL:
            return f32 ? launch_elem_t<float, float, MODE_RESIDUAL, false>(a, s)
                       : launch_elem_t<double, double, MODE_RESIDUAL, false>(a, s);
        case MODE_APPLY:
            if (trans) return f32 ? launch_elem_t<float, float, MODE_APPLY, true>(a, s)
                                  : launch_elem_t<double, double, MODE_APPLY, true>(a, s);
            return f32 ? launch_elem_t<float, float, MODE_APPLY, false>(a, s)
                       : launch_elem_t<double, double, MODE_APPLY, false>(a, s);
        case MODE_LINEARIZE:
            return state_prec == 1 ? launch_elem_t<double, float, MODE_LINEARIZE, false>(a, s)
                                   : launch_elem_t<double, double, MODE_LINEARIZE, false>(a, s);
        case MODE_STATE_APPLY:
        case MODE_STATE_GRADP:
            // the pointwise map of Eq. 2.7 is symmetric: the transposed apply
            // runs the same kernel
            if (a.state_cpl) {
#if STOKES_K == 2
                if (!f32) return int(cudaErrorInvalidValue);
                return launch_cpl(a, mode == MODE_STATE_GRADP, s);
#else
                return int(cudaErrorInvalidValue);
#endif
            }
            if (mode == MODE_STATE_GRADP)
                return f32 ? launch_state_apply_t<float, true>(a, s) : launch_state_apply_t<double, true>(a, s);
            return f32 ? launch_state_apply_t<float, false>(a, s) : launch_state_apply_t<double, false>(a, s);
        case MODE_GRAD_A:
            return launch_elem_t<double, double, MODE_GRAD_A, false>(a, s);
        case MODE_GRAD_A_PARTIAL:
            return launch_elem_t<double, double, MODE_GRAD_A_PARTIAL, false>(a, s);
        default:
            return int(cudaErrorInvalidValue);
    }
}

inline int launch_face_any(int mode, int prec, const FaceArgs& a, cudaStream_t s) {
    if (mode == FACE_GRAD_LOGBETA) return launch_face_t<double, FACE_GRAD_LOGBETA>(a, s);
    if (mode == FACE_LINEARIZE) return launch_face_t<double, FACE_LINEARIZE>(a, s);
    return prec == 1 ? launch_face_t<float, FACE_APPLY>(a, s) : launch_face_t<double, FACE_APPLY>(a, s);
}

// Upload the degree-K tables (host struct Tables1D for each pressure space).
inline int upload_tables_any(const void* p) {
    const Tables1D* t = static_cast<const Tables1D*>(p);   // t[0]: P space, t[1]: Q space
    double B[Q][N1], Dg[Q][Q], I[2][N1][N1], P1[2][Q][N1], Bdv[Q][N1];
    float fb[Q][N1], fd[Q][Q], fi[2][N1][N1], fp[2][Q][N1], fbd[Q][N1];
    int pm[2][NPRK > 0 ? NPRK : 1][3] = {};
    int np[2];
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < N1; ++b) { B[a][b] = t[0].B[a][b]; fb[a][b] = float(B[a][b]); }
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b) { Dg[a][b] = t[0].Dg[a][b]; fd[a][b] = float(Dg[a][b]); }
    for (int hh = 0; hh < 2; ++hh)
        for (int a = 0; a < N1; ++a)
            for (int b = 0; b < N1; ++b) { I[hh][a][b] = t[0].I[hh][a][b]; fi[hh][a][b] = float(I[hh][a][b]); }
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < N1; ++b) {
            double sum = 0;
            for (int m = 0; m < Q; ++m) sum += Dg[a][m] * B[m][b];
            Bdv[a][b] = sum;
            fbd[a][b] = float(sum);
        }
    for (int sp = 0; sp < 2; ++sp) {
        np[sp] = t[sp].npr;
        for (int a = 0; a < Q; ++a)
            for (int b = 0; b < N1; ++b) { P1[sp][a][b] = t[sp].P1[a][b]; fp[sp][a][b] = float(P1[sp][a][b]); }
        for (int m = 0; m < t[sp].npr && m < NPRK; ++m)
            for (int c = 0; c < 3; ++c) pm[sp][m][c] = t[sp].pmode[m][c];
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cB, B, sizeof(B));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cDg, Dg, sizeof(Dg));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cI, I, sizeof(I));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cP1, P1, sizeof(P1));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cPm, pm, sizeof(pm));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cNpr, np, sizeof(np));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(fB, fb, sizeof(fb));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(fDg, fd, sizeof(fd));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(fI, fi, sizeof(fi));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(fP1, fp, sizeof(fp));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(cBd, Bdv, sizeof(Bdv));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(fBd, fbd, sizeof(fbd));
#if STOKES_K == 2
    {
        float psi[2][NPRK][Q3] = {};
        for (int sp = 0; sp < 2; ++sp)
            for (int m = 0; m < t[sp].npr && m < NPRK; ++m)
                for (int l = 0; l < Q; ++l)
                    for (int jj = 0; jj < Q; ++jj)
                        for (int ii = 0; ii < Q; ++ii)
                            psi[sp][m][ii + Q * (jj + Q * l)] =
                                float(P1[sp][ii][pm[sp][m][0]] * P1[sp][jj][pm[sp][m][1]] * P1[sp][l][pm[sp][m][2]]);
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(fPsi, psi, sizeof(psi));
        // the component-per-lane apply uses these tables as compile-time
        // constants (q2c): refuse to run if the computed ones differ
        const double S = std::sqrt(0.6);
        const double Bx[3][3] = {{0.3 + 0.5 * S, 0.4, 0.3 - 0.5 * S}, {0, 1, 0}, {0.3 - 0.5 * S, 0.4, 0.3 + 0.5 * S}};
        const double Dx[3][3] = {{-S - 0.5, 2 * S, 0.5 - S}, {-0.5, 0, 0.5}, {S - 0.5, -2 * S, S + 0.5}};
        const double G[3] = {-S, 0.0, S};
        bool same = t[0].npr == 4 && t[1].npr == 1;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                same = same && std::fabs(B[a][b] - Bx[a][b]) < 1e-13 && std::fabs(Bdv[a][b] - Dx[a][b]) < 1e-13;
        for (int qp = 0; qp < Q3 && same; ++qp) {
            const double ex[4] = {1.0, G[qp % 3], G[(qp / 3) % 3], G[qp / 9]};
            for (int m = 0; m < 4; ++m) same = same && std::fabs(psi[0][m][qp] - ex[m]) < 1e-6;
            same = same && std::fabs(psi[1][0][qp] - 1.0) < 1e-6;
        }
        if (e == cudaSuccess && !same) e = cudaErrorInvalidValue;
    }
#endif
    return int(e);
}

}  // namespace STOKES_NS
}  // namespace dev
}  // namespace stokes

#define STOKES_DEFINE_DEGREE(KK)                                                                   \
    namespace stokes {                                                                             \
    int launch_elem_k##KK(int mode, int prec, int state_prec, bool trans, const ElemArgs& a,        \
                          cudaStream_t s) {                                                        \
        return dev::STOKES_NS::launch_elem_any(mode, prec, state_prec, trans, a, s);               \
    }                                                                                              \
    int launch_face_k##KK(int mode, int prec, const FaceArgs& a, cudaStream_t s) {                 \
        return dev::STOKES_NS::launch_face_any(mode, prec, a, s);                                 \
    }                                                                                              \
    int upload_tables_k##KK(const void* t) { return dev::STOKES_NS::upload_tables_any(t); }       \
    int64_t state_stride_k##KK() { return dev::STOKES_NS::SSTRIDE; }                             \
    int64_t grad_a_partials_k##KK(int64_t E) { return dev::STOKES_NS::grad_a_partials(E); }       \
    }
