// Component-per-lane stored-state apply for k = 2 and an FP32 state in the
// group layout (conforming meshes): y = J x with J the Newton Jacobian of
// Eqs. 2.6-2.7 (or its Picard form), both of the element terms of Eq. 2.5 and
// of the basal terms.  Included by elem_body.cuh for STOKES_K == 2.
//
// Lane 3 el + c of a warp owns velocity component c of element el of the
// warp's group of CPL_E = 10 consecutive elements (lanes 30 and 31 idle) and
// runs the whole sum factorisation of that scalar field in registers
// (Section 3.3: 1-D kernels along xi, eta, zeta): 27 nodal values -> the 3
// reference derivatives at the 27 Gauss points -> pointwise stress -> 27
// nodal values.  Nothing goes through shared memory but the state.
//
// The pointwise Newton stress couples the components of an element.  Lane c
// works with the physical directions rotated by c (its direction d' is
// (c + d') mod 3), so that each exchanged value has an index known at compile
// time: per Gauss point, two shuffles sum the contraction Dhat : grad w over
// the lane triplet and two bring the transposed gradient entries d_c w_{c+1}
// and d_c w_{c+2} needed for the symmetric part D(w).
//
// The state of a group (12000 bytes) is staged in shared memory by one bulk
// asynchronous copy (TMA, cp.async.bulk) on a per-warp mbarrier; the copy for
// the warp's next group is issued as soon as the pointwise phase has read the
// buffer, so it overlaps the transposed sweeps, the scatter, the next gather
// and the forward sweeps.
#pragma once

#if STOKES_K == 2

namespace stokes {
namespace dev {
namespace STOKES_NS {

#ifndef CPL_WARPS
#define CPL_WARPS 4
#endif
#ifndef CPL_MINB
#define CPL_MINB 3
#endif
// the next group's velocity, pressure and projector index loaded into
// registers before the current group's transposed sweeps and scatter
#ifndef CPL_PREFETCH
#define CPL_PREFETCH 1
#endif
struct CplCfg {
    static constexpr int W = CPL_WARPS;                  // warps per block
    static constexpr int TAIL = (EPW + 1) * 4 * N2;      // basal face scratch per warp (values)
    static constexpr int PER_WARP = (CPL_GROUP + TAIL) * 4;   // bytes
    static constexpr int SMEM = W * PER_WARP + W * 8;
    static_assert(PER_WARP % 16 == 0, "stage buffers 16-byte aligned");
};

// d_xi, d_eta, d_zeta of the Q2 interpolant of the nodal values w at the 27
// Gauss points (index qi + 3 qj + 9 lq; nodes a + 3 b + 9 l)
__device__ __forceinline__ void cpl_forward(const float (&w)[27], float (&Gx)[27], float (&Gy)[27],
                                            float (&Gz)[27]) {
    float Bw[27], Dw[27];   // [a + 3 b + 9 lq]: zeta interpolated / differentiated
    #pragma unroll
    for (int ab = 0; ab < 9; ++ab)
        #pragma unroll
        for (int lq = 0; lq < 3; ++lq) {
            float sb = 0.f, sd = 0.f;
            #pragma unroll
            for (int l = 0; l < 3; ++l) {
                sb += fB[lq][l] * w[ab + 9 * l];
                sd += fBd[lq][l] * w[ab + 9 * l];
            }
            Bw[ab + 9 * lq] = sb;
            Dw[ab + 9 * lq] = sd;
        }
    float BB[27], BD[27], DB[27];   // [a + 3 qj + 9 lq]
    #pragma unroll
    for (int a = 0; a < 3; ++a)
        #pragma unroll
        for (int lq = 0; lq < 3; ++lq)
            #pragma unroll
            for (int qj = 0; qj < 3; ++qj) {
                float s1 = 0.f, s2 = 0.f, s3 = 0.f;
                #pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const float bw = Bw[a + 3 * b + 9 * lq];
                    s1 += fB[qj][b] * bw;
                    s2 += fBd[qj][b] * bw;
                    s3 += fB[qj][b] * Dw[a + 3 * b + 9 * lq];
                }
                BB[a + 3 * qj + 9 * lq] = s1;
                BD[a + 3 * qj + 9 * lq] = s2;
                DB[a + 3 * qj + 9 * lq] = s3;
            }
    #pragma unroll
    for (int r = 0; r < 9; ++r)          // r = qj + 3 lq
        #pragma unroll
        for (int qi = 0; qi < 3; ++qi) {
            float gx = 0.f, gy = 0.f, gz = 0.f;
            #pragma unroll
            for (int a = 0; a < 3; ++a) {
                gx += fBd[qi][a] * BB[a + 3 * r];
                gy += fB[qi][a] * BD[a + 3 * r];
                gz += fB[qi][a] * DB[a + 3 * r];
            }
            Gx[qi + 3 * r] = gx;
            Gy[qi + 3 * r] = gy;
            Gz[qi + 3 * r] = gz;
        }
}

// transpose of cpl_forward: nodal values from the reference stresses
__device__ __forceinline__ void cpl_transpose(const float (&Sx)[27], const float (&Sy)[27], const float (&Sz)[27],
                                              float (&out)[27]) {
    float Ux[27], Uy[27], Uz[27];   // [a + 3 qj + 9 lq]
    #pragma unroll
    for (int r = 0; r < 9; ++r)
        #pragma unroll
        for (int a = 0; a < 3; ++a) {
            float ux = 0.f, uy = 0.f, uz = 0.f;
            #pragma unroll
            for (int qi = 0; qi < 3; ++qi) {
                ux += fBd[qi][a] * Sx[qi + 3 * r];
                uy += fB[qi][a] * Sy[qi + 3 * r];
                uz += fB[qi][a] * Sz[qi + 3 * r];
            }
            Ux[a + 3 * r] = ux;
            Uy[a + 3 * r] = uy;
            Uz[a + 3 * r] = uz;
        }
    float VB[27], VD[27];   // [a + 3 b + 9 lq]
    #pragma unroll
    for (int a = 0; a < 3; ++a)
        #pragma unroll
        for (int lq = 0; lq < 3; ++lq)
            #pragma unroll
            for (int b = 0; b < 3; ++b) {
                float vb = 0.f, vd = 0.f;
                #pragma unroll
                for (int qj = 0; qj < 3; ++qj) {
                    const int r = a + 3 * qj + 9 * lq;
                    vb += fB[qj][b] * Ux[r] + fBd[qj][b] * Uy[r];
                    vd += fB[qj][b] * Uz[r];
                }
                VB[a + 3 * b + 9 * lq] = vb;
                VD[a + 3 * b + 9 * lq] = vd;
            }
    #pragma unroll
    for (int ab = 0; ab < 9; ++ab)
        #pragma unroll
        for (int l = 0; l < 3; ++l) {
            float s = 0.f;
            #pragma unroll
            for (int lq = 0; lq < 3; ++lq) s += fB[lq][l] * VB[ab + 9 * lq] + fBd[lq][l] * VD[ab + 9 * lq];
            out[ab + 9 * l] = s;
        }
}

// Basal projector P on the bottom-plane nodes (l = 0) of the lane's element,
// component c: v_c <- sum_k P[c][k] v_k (P symmetric, so also its transpose).
// Executed by the whole warp when any of its elements is basal.
__device__ __forceinline__ void cpl_project(const ElemArgs& a, float (&v)[27], int pi, int c, int l1, int l2) {
    const int po1 = c == 0 ? 3 : (c == 1 ? 5 : 4);   // P[c][c+1]: 01, 12, 20
    const int po2 = c == 0 ? 4 : (c == 1 ? 3 : 5);   // P[c][c+2]: 02, 10, 21
    const float* P = a.pel_f + int64_t(pi < 0 ? 0 : pi) * 6 * N2;
    #pragma unroll
    for (int ab = 0; ab < 9; ++ab) {
        const float v1 = __shfl_sync(0xffffffffu, v[ab], l1);
        const float v2 = __shfl_sync(0xffffffffu, v[ab], l2);
        if (pi >= 0) v[ab] = P[c * N2 + ab] * v[ab] + P[po1 * N2 + ab] * v1 + P[po2 * N2 + ab] * v2;
    }
}

// f(n, global node) for the 27 local nodes n = a + 3 b + 9 l of element e:
// from the lattice (conforming structured meshes) or the element map
template <typename F>
__device__ __forceinline__ void cpl_nodes(const ElemArgs& a, int64_t e, bool active, F&& f) {
    if (a.lat_nx > 0) {
        const int e32 = active ? int(e) : 0, nx = int(a.lat_nx), ny = int(a.lat_ny);
        const int ex = e32 % nx, r = e32 / nx;
        const int ey = r % ny, ez = r / ny;
        const int NX = int(a.lat_NX), NY = int(a.lat_NY);
        const int gL = NX * NY;
        int gI[3], gJ[3];
        #pragma unroll
        for (int m = 0; m < 3; ++m) {
            int I = ex * K + m, J = ey * K + m;
            if (I >= NX) I -= NX;
            if (J >= NY) J -= NY;
            gI[m] = I + gL * (ez * K);
            gJ[m] = NX * J;
        }
        #pragma unroll
        for (int n = 0; n < 27; ++n) f(n, int64_t(gI[n % 3] + gJ[(n / 3) % 3] + (n / 9) * gL));
    } else {
        const int32_t* nd = a.nodes + (active ? e : 0) * N3;
        #pragma unroll
        for (int n = 0; n < 27; ++n) f(n, int64_t(nd[n]));
    }
}

template <int PS, bool PONLY>
__global__ void __launch_bounds__(32 * CplCfg::W, CPL_MINB) cpl_state_apply_kernel(ElemArgs a) {
    using C = CplCfg;
    constexpr int NPR = PS == 0 ? K * (K + 1) * (K + 2) / 6 : (K - 1) * (K - 1) * (K - 1);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int el = lane / 3;                     // CPL_E for the idle lanes 30, 31
    const int c = lane - 3 * el;
    const int els = el < CPL_E ? el : 0;         // state column read by the lane
    const int l1 = 3 * el + (c == 2 ? 0 : c + 1);   // lane of component c + 1 (mod 3)
    const int l2 = 3 * el + (c == 0 ? 2 : c - 1);   // lane of component c + 2 (mod 3)
    float* buf = reinterpret_cast<float*>(smem_raw + warp * C::PER_WARP);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + C::W * C::PER_WARP) + warp;
    const float* S = static_cast<const float*>(a.cstate);
    const float* x = static_cast<const float*>(a.x);
    float* y = static_cast<float*>(a.y);

    // lane-dependent state fields: Jinv[2][(c + d') mod 3] (fields 0..2) and
    // row c of Dhat in rotated order (fields 5..10 = 00 11 22 01 02 12)
    const int fz1 = c == 2 ? 0 : c + 1, fz2 = c == 0 ? 2 : c - 1;
    const int fd0 = 5 + c;
    const int fd1 = c == 0 ? 8 : (c == 1 ? 10 : 9);
    const int fd2 = c == 0 ? 9 : (c == 1 ? 8 : 10);

    const int64_t ngroups = (a.E + CPL_E - 1) / CPL_E;
    const int64_t gstride = int64_t(gridDim.x) * C::W;
    int64_t g = int64_t(blockIdx.x) * C::W + warp;

    auto stage = [&](int64_t gg) {   // lane 0 only
        const float* src = S + gg * CPL_GROUP;
        if constexpr (PONLY) {
            // header and, per plane, the leading fields Jinv[2][0..2], w detJ
            mbar_arrive_expect_tx(bar, uint32_t(CPL_HDR + 3 * 4 * CPL_FS) * 4u);
            bulk_g2s(buf, src, CPL_HDR * 4, bar);
            #pragma unroll
            for (int lq = 0; lq < 3; ++lq)
                bulk_g2s(buf + CPL_HDR + lq * CPL_PL, src + CPL_HDR + lq * CPL_PL, 4 * CPL_FS * 4, bar);
        } else {
            mbar_arrive_expect_tx(bar, uint32_t(CPL_GROUP) * 4u);
            bulk_g2s(buf, src, CPL_GROUP * 4, bar);
        }
    };
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    if (g < ngroups && lane == 0) stage(g);

    // inputs of a group: velocity component c at the 27 nodes, pressure
    // coefficients, basal projector index
    float wn[27], pvn[NPR];
    int pin = -1;
    auto load_inputs = [&](int64_t gg) {
        const int64_t en = gg * CPL_E + el;
        const bool an = (el < CPL_E) && (gg < ngroups) && (en < a.E);
        pin = an ? a.pidx[en] : -1;
        #pragma unroll
        for (int b = 0; b < NPR; ++b) pvn[b] = an ? ld(x + 3 * a.Nv + en * NPR + b) : 0.f;
        if constexpr (!PONLY)
            cpl_nodes(a, en, an, [&](int n, int64_t gn) { wn[n] = an ? ld(x + 3 * gn + c) : 0.f; });
    };
#if CPL_PREFETCH
    load_inputs(g);
#endif

    for (int it = 0; g < ngroups; g += gstride, ++it) {
        const int64_t e = g * CPL_E + el;
        const bool active = (el < CPL_E) && (e < a.E);
#if !CPL_PREFETCH
        load_inputs(g);
#endif
        const int pi = pin;
        const bool any_basal = __any_sync(0xffffffffu, pi >= 0) != 0;
        float pv[NPR];
        #pragma unroll
        for (int b = 0; b < NPR; ++b) pv[b] = pvn[b];

        float Gx[27], Gy[27], Gz[27];
        if constexpr (!PONLY) {
            float w[27];
            #pragma unroll
            for (int n = 0; n < 27; ++n) w[n] = wn[n];
            if (any_basal) cpl_project(a, w, pi, c, l1, l2);
            cpl_forward(w, Gx, Gy, Gz);
        }

        if (!mbar_wait_polls(bar, uint32_t(it & 1), a.wait_polls)) {
            // the staged state never arrived: report, let the copy (the only
            // one this warp has in flight) drain, stop
            if (lane == 0) atomicOr(a.err, 1);
            mbar_wait_bounded(bar, uint32_t(it & 1));
            return;
        }
        // rotated rows of Jinv: lane direction d' is the physical direction (c + d') mod 3
        const float ia = buf[els], ib = buf[CPL_E + els];
        const float A0 = c == 0 ? ia : 0.f, A1 = c == 2 ? ia : 0.f, A2 = c == 1 ? ia : 0.f;
        const float B0 = c == 1 ? ib : 0.f, B1 = c == 0 ? ib : 0.f, B2 = c == 2 ? ib : 0.f;
        float rows[NPR];
        #pragma unroll
        for (int b = 0; b < NPR; ++b) rows[b] = 0.f;
        #pragma unroll
        for (int lq = 0; lq < 3; ++lq)
            #pragma unroll
            for (int q9 = 0; q9 < 9; ++q9) {
                const int qp = q9 + 9 * lq;
                const float* F = buf + CPL_HDR + lq * CPL_PL + els * N2 + q9;
                const float wdj = F[3 * CPL_FS];
                const float z0 = F[c * CPL_FS], z1 = F[fz1 * CPL_FS], z2 = F[fz2 * CPL_FS];
                float p = 0.f;
                #pragma unroll
                for (int b = 0; b < NPR; ++b) p += fPsi[PS][b][qp] * pv[b];
                const float pw = p * wdj;
                if constexpr (PONLY) {
                    // tau = -p w detJ I: reference stress of component c is -pw Jinv[m][c]
                    Gx[qp] = -pw * A0;
                    Gy[qp] = -pw * B0;
                    Gz[qp] = -pw * z0;
                } else {
                    const float muw = F[4 * CPL_FS];
                    const float D0 = F[fd0 * CPL_FS], D1 = F[fd1 * CPL_FS], D2 = F[fd2 * CPL_FS];
                    const float gx = Gx[qp], gy = Gy[qp], gz = Gz[qp];
                    // d_{c+d'} w_c
                    const float dv0 = A0 * gx + B0 * gy + z0 * gz;
                    const float dv1 = A1 * gx + B1 * gy + z1 * gz;
                    const float dv2 = A2 * gx + B2 * gy + z2 * gz;
                    // Dhat : D(w) = sum_c sum_d Dhat_cd d_d w_c (Dhat symmetric)
                    const float sc = D0 * dv0 + D1 * dv1 + D2 * dv2;
                    const float s = sc + __shfl_sync(0xffffffffu, sc, l1) + __shfl_sync(0xffffffffu, sc, l2);
                    // d_c w_{c+1} and d_c w_{c+2} from the other two lanes
                    const float t1 = __shfl_sync(0xffffffffu, dv2, l1);
                    const float t2 = __shfl_sync(0xffffffffu, dv1, l2);
                    // Eq. 2.7 as a symmetric map: w detJ mu' E = muw E - (Dhat:E) Dhat
                    const float tau0 = muw * dv0 - s * D0 - pw;
                    const float tau1 = 0.5f * muw * (dv1 + t1) - s * D1;
                    const float tau2 = 0.5f * muw * (dv2 + t2) - s * D2;
                    // reference stress of component c: sum_d Jinv[m][d] tau[c][d]
                    Gx[qp] = A0 * tau0 + A1 * tau1 + A2 * tau2;
                    Gy[qp] = B0 * tau0 + B1 * tau1 + B2 * tau2;
                    Gz[qp] = z0 * tau0 + z1 * tau1 + z2 * tau2;
                    // pressure rows -(psi_b, div w): this lane's share d_c w_c
                    const float gq = -wdj * dv0;
                    #pragma unroll
                    for (int b = 0; b < NPR; ++b) rows[b] += fPsi[PS][b][qp] * gq;
                }
            }
        // the buffer has been read: refill it with the warp's next group
        __syncwarp();
        if (lane == 0 && g + gstride < ngroups) {
            fence_proxy_async();
            stage(g + gstride);
        }
        if constexpr (!PONLY) {
            #pragma unroll
            for (int b = 0; b < NPR; ++b) {
                const float r = rows[b] + __shfl_sync(0xffffffffu, rows[b], l1) +
                                __shfl_sync(0xffffffffu, rows[b], l2);
                if (active && b % 3 == c) y[3 * a.Nv + e * NPR + b] = r;
            }
        }

#if CPL_PREFETCH
        load_inputs(g + gstride);
#endif
        float out[27];
        cpl_transpose(Gx, Gy, Gz, out);
        if (any_basal) cpl_project(a, out, pi, c, l1, l2);
        if (active) cpl_nodes(a, e, true, [&](int n, int64_t gn) { atomic_add(y + 3 * gn + c, out[n]); });
    }
    if constexpr (!PONLY) {
        // basal terms of the same apply, after this warp's element groups
        const LaneMap L;
        const int64_t w0 = int64_t(blockIdx.x) * C::W + warp;
        if (a.fuse_robin) {
            Rows<float> R;
            R.load(L.i, L.j);
            float* sb = reinterpret_cast<float*>(smem_raw + warp * C::PER_WARP) + CPL_GROUP + L.es * 4 * N2;
            const int64_t nfg = (a.face.nF + EPW - 1) / EPW;
            for (int64_t fg = w0; fg < nfg; fg += gstride) face_group<float, FACE_APPLY>(a.face, L, R, fg, sb);
        }
        if (a.fuse_constraint) constraint_rows<float>(a, w0 * 32 + lane, gstride * 32);
    }
}

template <int PS, bool PONLY>
int launch_cpl_t(const ElemArgs& a, cudaStream_t s) {
    using C = CplCfg;
    if (a.E == 0) return int(cudaSuccess);
    static int configured_device = -1;
    static int max_blocks = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_device != dev) {
        cudaError_t e = cudaFuncSetAttribute(cpl_state_apply_kernel<PS, PONLY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
        if (e != cudaSuccess) return int(e);
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cpl_state_apply_kernel<PS, PONLY>, 32 * C::W,
                                                          C::SMEM);
        if (e != cudaSuccess) return int(e);
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return int(e);
        max_blocks = (per_sm > 0 ? per_sm : 1) * sms;
        configured_device = dev;
    }
    const int64_t ngroups = (a.E + CPL_E - 1) / CPL_E;
    int64_t blocks = (ngroups + C::W - 1) / C::W;
    if (blocks > max_blocks) blocks = max_blocks;
    cpl_state_apply_kernel<PS, PONLY><<<unsigned(blocks), 32 * C::W, C::SMEM, s>>>(a);
    return int(cudaGetLastError());
}

inline int launch_cpl(const ElemArgs& a, bool ponly, cudaStream_t s) {
    if (a.pspace == 0) return ponly ? launch_cpl_t<0, true>(a, s) : launch_cpl_t<0, false>(a, s);
    return ponly ? launch_cpl_t<1, true>(a, s) : launch_cpl_t<1, false>(a, s);
}

}  // namespace STOKES_NS
}  // namespace dev
}  // namespace stokes

#endif  // STOKES_K == 2
