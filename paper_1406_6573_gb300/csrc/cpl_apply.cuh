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
// the streamed state is copied with an L2 evict-first policy, so that x and
// y stay in L2 (128x128x8 Q2xP1 slab: 0.0685 -> 0.0649 ms)
#ifndef CPL_STATE_EVICT_FIRST
#define CPL_STATE_EVICT_FIRST 1
#endif
struct CplCfg {
    static constexpr int W = CPL_WARPS;                  // warps per block
    // basal face scratch per warp (values): the face tail's element slots,
    // or 9 bottom-plane values per lane for the face term in the element pass
    static constexpr int TAIL = (EPW + 1) * 4 * N2 > 9 * 32 ? (EPW + 1) * 4 * N2 : 9 * 32;
    static constexpr int PER_WARP = (CPL_GROUP + TAIL) * 4;   // bytes
    static constexpr int SMEM = W * PER_WARP + W * 8;
    static_assert(PER_WARP % 16 == 0, "stage buffers 16-byte aligned");
};

// Q2 1-D tables as compile-time constants: GLL nodes (-1, 0, 1), Gauss
// points (-s, 0, s) with s = sqrt(3/5).  B[q][i] = l_i(g_q) and
// Bd[q][i] = l_i'(g_q) are centro-symmetric (B[2-q][2-i] = B[q][i]) and
// centro-antisymmetric (Bd[2-q][2-i] = -Bd[q][i]), so each 3-point line is
// applied through its even part w0 + w2 and odd part w0 - w2 (the even-odd
// decomposition of symmetric collocation matrices; Solomonoff, "A fast
// algorithm for spectral differentiation", J. Comput. Phys. 98, 1992), and
// the zero and unit entries of the middle row fold away:
//   B  = [[0.3 + s/2, 0.4, 0.3 - s/2], [0, 1, 0], [0.3 - s/2, 0.4, 0.3 + s/2]]
//   Bd = [[-s - 1/2, 2 s, 1/2 - s], [-1/2, 0, 1/2], [s - 1/2, -2 s, s + 1/2]]
// The library checks, when it uploads its tables, that its own (computed)
// tables equal these.
namespace q2c {
constexpr float S = 0.774596669241483377f;   // sqrt(3/5)
constexpr float HS = 0.5f * S;
// pressure basis at the Gauss points: P_{k-1} = span{1, xi, eta, zeta}
// (Legendre P_1 = x, modes in the order of the host tables) or Q_0 = {1}
__device__ __forceinline__ constexpr float gq(int i) { return i == 0 ? -S : (i == 1 ? 0.f : S); }
template <int PS>
__device__ __forceinline__ constexpr float psi(int b, int qp) {
    return PS == 1 ? 1.f : (b == 0 ? 1.f : (b == 1 ? gq(qp % 3) : (b == 2 ? gq((qp / 3) % 3) : gq(qp / 9))));
}
}  // namespace q2c

// q = B w (values at the Gauss points of a line)
__device__ __forceinline__ void q2_b(float w0, float w1, float w2, float& q0, float& q1, float& q2) {
    const float e = w0 + w2, o = w0 - w2;
    const float t = fmaf(0.3f, e, 0.4f * w1);
    q0 = fmaf(q2c::HS, o, t);
    q2 = fmaf(-q2c::HS, o, t);
    q1 = w1;
}
// d = Bd w (derivatives at the Gauss points of a line)
__device__ __forceinline__ void q2_d(float w0, float w1, float w2, float& d0, float& d1, float& d2) {
    const float e = w0 + w2, o = w0 - w2;
    const float u = q2c::S * fmaf(-2.f, w1, e);
    const float v = -0.5f * o;
    d0 = v - u;
    d1 = v;
    d2 = v + u;
}
// n = B^T s
__device__ __forceinline__ void q2_bt(float s0, float s1, float s2, float& n0, float& n1, float& n2) {
    const float E = s0 + s2, O = s0 - s2;
    const float a = 0.3f * E;
    n0 = fmaf(q2c::HS, O, a);
    n2 = fmaf(-q2c::HS, O, a);
    n1 = fmaf(0.4f, E, s1);
}
// n = Bd^T t
__device__ __forceinline__ void q2_dt(float t0, float t1, float t2, float& n0, float& n1, float& n2) {
    const float m = q2c::S * (t0 - t2);
    const float h = 0.5f * (t0 + t1 + t2);
    n0 = -m - h;
    n1 = m + m;
    n2 = h - m;
}

// zeta and eta stages of the forward sweeps of the nodal values w (nodes
// a + 3 b + 9 l): BB = (B x B) w, BD = (Bd x B) w, DB = (B x Bd) w along
// (eta, zeta), indexed a + 3 qj + 9 lq; the xi stage (Bd, B, B along xi)
// then gives d_xi, d_eta, d_zeta of the Q2 interpolant at the Gauss point
// qi + 3 qj + 9 lq, one line of three points at a time
__device__ __forceinline__ void cpl_forward_ze(const float (&w)[27], float (&BB)[27], float (&BD)[27],
                                               float (&DB)[27]) {
    float Bw[27], Dw[27];   // [a + 3 b + 9 lq]: zeta interpolated / differentiated
    #pragma unroll
    for (int ab = 0; ab < 9; ++ab) {
        q2_b(w[ab], w[ab + 9], w[ab + 18], Bw[ab], Bw[ab + 9], Bw[ab + 18]);
        q2_d(w[ab], w[ab + 9], w[ab + 18], Dw[ab], Dw[ab + 9], Dw[ab + 18]);
    }
    #pragma unroll
    for (int a = 0; a < 3; ++a)
        #pragma unroll
        for (int lq = 0; lq < 3; ++lq) {
            const int o = a + 9 * lq;
            q2_b(Bw[o], Bw[o + 3], Bw[o + 6], BB[o], BB[o + 3], BB[o + 6]);
            q2_d(Bw[o], Bw[o + 3], Bw[o + 6], BD[o], BD[o + 3], BD[o + 6]);
            q2_b(Dw[o], Dw[o + 3], Dw[o + 6], DB[o], DB[o + 3], DB[o + 6]);
        }
}

// eta and zeta stages of the transposed sweeps: nodal values from the xi-
// transposed reference stresses U (indexed a + 3 qj + 9 lq)
__device__ __forceinline__ void cpl_transpose_ez(const float (&Ux)[27], const float (&Uy)[27],
                                                 const float (&Uz)[27], float (&out)[27]) {
    float VB[27], VD[27];   // [a + 3 b + 9 lq]
    #pragma unroll
    for (int a = 0; a < 3; ++a)
        #pragma unroll
        for (int lq = 0; lq < 3; ++lq) {
            const int o = a + 9 * lq;
            float b0, b1, b2, d0, d1, d2;
            q2_bt(Ux[o], Ux[o + 3], Ux[o + 6], b0, b1, b2);
            q2_dt(Uy[o], Uy[o + 3], Uy[o + 6], d0, d1, d2);
            VB[o] = b0 + d0; VB[o + 3] = b1 + d1; VB[o + 6] = b2 + d2;
            q2_bt(Uz[o], Uz[o + 3], Uz[o + 6], VD[o], VD[o + 3], VD[o + 6]);
        }
    #pragma unroll
    for (int ab = 0; ab < 9; ++ab) {
        float b0, b1, b2, d0, d1, d2;
        q2_bt(VB[ab], VB[ab + 9], VB[ab + 18], b0, b1, b2);
        q2_dt(VD[ab], VD[ab + 9], VD[ab + 18], d0, d1, d2);
        out[ab] = b0 + d0; out[ab + 9] = b1 + d1; out[ab + 18] = b2 + d2;
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

// Basal Robin term (Eqs. 2.4-2.5) of the lane's element, component c, from
// the projected nodal values w (bottom plane l = 0 of a basal element): the
// values at the 3 x 3 face Gauss points (B x B), the traction
// t_c = bws (v_c - (n . v) n_c) + (vv . v) Tu_c with the stored basal state
// (bws = beta w |J_s| s, vv = 2 beta w |J_s| s' T u and T u of the nonlinear
// sliding law, n the unit normal), and the transposed interpolation back to
// the 9 bottom-plane nodes, written to the lane's scratch scr[n * 32].  The
// whole warp executes it (the n . v and vv . v sums are lane-triplet
// shuffles); lanes of elements without a basal face write zeros.
__device__ __forceinline__ void cpl_face(const ElemArgs& a, const float (&w)[27], int64_t e, bool active, int c,
                                         int l1, int l2, float* scr) {
    const int f = active ? a.fidx[e] : -1;
    const bool has = f >= 0;
    float T[9], vq[9];
    #pragma unroll
    for (int a3 = 0; a3 < 3; ++a3) q2_b(w[a3], w[a3 + 3], w[a3 + 6], T[a3], T[a3 + 3], T[a3 + 6]);
    #pragma unroll
    for (int qj = 0; qj < 3; ++qj)
        q2_b(T[3 * qj], T[3 * qj + 1], T[3 * qj + 2], vq[3 * qj], vq[3 * qj + 1], vq[3 * qj + 2]);
    const float* F = static_cast<const float*>(a.face.fstate) + int64_t(has ? f : 0) * SLIDE_FIELDS * 9;
    float t[9];
    #pragma unroll
    for (int q = 0; q < 9; ++q) {
        const float bws = has ? ld(F + q) : 0.f;
        const float nc = has ? ld(F + (7 + c) * 9 + q) : 0.f;
        const float nv0 = nc * vq[q];
        const float nv = nv0 + __shfl_sync(0xffffffffu, nv0, l1) + __shfl_sync(0xffffffffu, nv0, l2);
        float tq = bws * fmaf(-nv, nc, vq[q]);
        if (a.face.slide) {
            const float vvc = has ? ld(F + (1 + c) * 9 + q) : 0.f;
            const float tuc = has ? ld(F + (4 + c) * 9 + q) : 0.f;
            const float vw0 = vvc * vq[q];
            const float vw = vw0 + __shfl_sync(0xffffffffu, vw0, l1) + __shfl_sync(0xffffffffu, vw0, l2);
            tq = fmaf(vw, tuc, tq);
        }
        t[q] = tq;
    }
    #pragma unroll
    for (int qj = 0; qj < 3; ++qj) q2_bt(t[3 * qj], t[3 * qj + 1], t[3 * qj + 2], T[3 * qj], T[3 * qj + 1], T[3 * qj + 2]);
    #pragma unroll
    for (int a3 = 0; a3 < 3; ++a3) {
        float o0, o1, o2;
        q2_bt(T[a3], T[a3 + 3], T[a3 + 6], o0, o1, o2);
        scr[a3 * 32] = o0;
        scr[(a3 + 3) * 32] = o1;
        scr[(a3 + 6) * 32] = o2;
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
#if CPL_STATE_EVICT_FIRST
            bulk_g2s_hint(buf, src, CPL_GROUP * 4, bar, l2_evict_first_policy());
#else
            bulk_g2s(buf, src, CPL_GROUP * 4, bar);
#endif
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

        // zeta and eta stages of the forward sweeps (before the wait: they
        // overlap the arrival of the staged state)
        float BB[27], BD[27], DB[27];
        // basal Robin term in the element pass (face scratch of the lane)
        const bool face_here = !PONLY && a.face_in_elements && any_basal;
        float* fscr = reinterpret_cast<float*>(smem_raw + warp * C::PER_WARP) + CPL_GROUP + lane;
        if constexpr (!PONLY) {
            float w[27];
            #pragma unroll
            for (int n = 0; n < 27; ++n) w[n] = wn[n];
            if (any_basal) cpl_project(a, w, pi, c, l1, l2);
            if (face_here) cpl_face(a, w, e, active, c, l1, l2, fscr);
            cpl_forward_ze(w, BB, BD, DB);
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
        // per line r = qj + 3 lq of three Gauss points along xi: xi stage of
        // the forward sweeps, pointwise stress, xi stage of the transposed
        // sweeps (U indexed a + 3 qj + 9 lq)
        float Ux[27], Uy[27], Uz[27];
        #pragma unroll
        for (int r = 0; r < 9; ++r) {
            const int lq = r / 3, o = 3 * r;
            float gx[3], gy[3], gz[3];
            if constexpr (!PONLY) {
                q2_d(BB[o], BB[o + 1], BB[o + 2], gx[0], gx[1], gx[2]);
                q2_b(BD[o], BD[o + 1], BD[o + 2], gy[0], gy[1], gy[2]);
                q2_b(DB[o], DB[o + 1], DB[o + 2], gz[0], gz[1], gz[2]);
            }
            float sx[3], sy[3], sz[3];
            #pragma unroll
            for (int qi = 0; qi < 3; ++qi) {
                const int qp = qi + o, q9 = qi + 3 * (r % 3);
                const float* F = buf + CPL_HDR + lq * CPL_PL + els * N2 + q9;
                const float wdj = F[3 * CPL_FS];
                const float z0 = F[c * CPL_FS], z1 = F[fz1 * CPL_FS], z2 = F[fz2 * CPL_FS];
                float p = 0.f;
                #pragma unroll
                for (int b = 0; b < NPR; ++b) p += q2c::psi<PS>(b, qp) * pv[b];
                const float pw = p * wdj;
                if constexpr (PONLY) {
                    // tau = -p w detJ I: reference stress of component c is -pw Jinv[m][c]
                    sx[qi] = -pw * A0;
                    sy[qi] = -pw * B0;
                    sz[qi] = -pw * z0;
                } else {
                    const float muw = F[4 * CPL_FS];
                    const float D0 = F[fd0 * CPL_FS], D1 = F[fd1 * CPL_FS], D2 = F[fd2 * CPL_FS];
                    // d_{c+d'} w_c
                    const float dv0 = A0 * gx[qi] + B0 * gy[qi] + z0 * gz[qi];
                    const float dv1 = A1 * gx[qi] + B1 * gy[qi] + z1 * gz[qi];
                    const float dv2 = A2 * gx[qi] + B2 * gy[qi] + z2 * gz[qi];
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
                    sx[qi] = A0 * tau0 + A1 * tau1 + A2 * tau2;
                    sy[qi] = B0 * tau0 + B1 * tau1 + B2 * tau2;
                    sz[qi] = z0 * tau0 + z1 * tau1 + z2 * tau2;
                    // pressure rows -(psi_b, div w): this lane's share d_c w_c
                    const float gq = -wdj * dv0;
                    #pragma unroll
                    for (int b = 0; b < NPR; ++b) rows[b] += q2c::psi<PS>(b, qp) * gq;
                }
            }
            q2_dt(sx[0], sx[1], sx[2], Ux[o], Ux[o + 1], Ux[o + 2]);
            q2_bt(sy[0], sy[1], sy[2], Uy[o], Uy[o + 1], Uy[o + 2]);
            q2_bt(sz[0], sz[1], sz[2], Uz[o], Uz[o + 1], Uz[o + 2]);
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
        cpl_transpose_ez(Ux, Uy, Uz, out);
        if (face_here) {
            #pragma unroll
            for (int n = 0; n < 9; ++n) out[n] += fscr[n * 32];
        }
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
    const int64_t blocks = persistent_blocks((a.E + CPL_E - 1) / CPL_E, C::W, max_blocks);
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
