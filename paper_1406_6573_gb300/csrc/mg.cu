// Geometric multigrid for the velocity block (see mg.h).
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_runtime.h>

#include "mg.h"
#include "precond.h"
#include "vec.h"

namespace stokes {
namespace {

constexpr int TPB = 256;

inline unsigned blocks_for(int64_t n) { return unsigned((n + TPB - 1) / TPB); }

// coarse FP64 velocity at node (Xc, Yc, Z) <- fine velocity at (2 Xc, 2 Yc, Z)
__global__ void inject_u_kernel(int64_t NXc, int64_t NYc, int64_t NZ, int64_t NX, int64_t NY, const double* __restrict__ uf,
                                double* __restrict__ uc) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= NXc * NYc * NZ) return;
    const int64_t Xc = t % NXc, r = t / NXc, Yc = r % NYc, Z = r / NYc;
    const int64_t gf = 2 * Xc + NX * (2 * Yc + NY * Z);
    uc[3 * t] = uf[3 * gf];
    uc[3 * t + 1] = uf[3 * gf + 1];
    uc[3 * t + 2] = uf[3 * gf + 2];
}

// coarse log(beta) at basal node (Xc, Yc) <- fine at (2 Xc, 2 Yc)
__global__ void inject_lb_kernel(int64_t NXc, int64_t NYc, int64_t NX, const double* __restrict__ lf, double* __restrict__ lc) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= NXc * NYc) return;
    const int64_t Xc = t % NXc, Yc = t / NXc;
    lc[t] = lf[2 * Xc + NX * 2 * Yc];
}

// 1-D Q2 interpolation weights: fine lattice index X from the coarse nodes
// (coarse element cx = X div 4 spans fine X = 4 cx .. 4 cx + 4 and coarse
// nodes 2 cx, 2 cx + 1, 2 cx + 2; local coordinate (X mod 4) / 2 - 1)
__device__ __forceinline__ int interp_1d(int64_t X, int64_t NXc, bool periodic, int64_t (&ic)[3], float (&w)[3]) {
    if ((X & 1) == 0) {
        ic[0] = X / 2;
        w[0] = 1.f;
        return 1;
    }
    const int64_t cx = X / 4;
    const bool r1 = (X % 4) == 1;    // xi = -1/2 (r1) or +1/2
    w[0] = r1 ? 0.375f : -0.125f;
    w[1] = 0.75f;
    w[2] = r1 ? -0.125f : 0.375f;
    for (int m = 0; m < 3; ++m) {
        int64_t c = 2 * cx + m;
        if (periodic && c >= NXc) c -= NXc;
        ic[m] = c;
    }
    return 3;
}

// out_f = P x_c (velocity part): Q2 interpolation in x and y, identity in z
template <typename T>
__global__ void prolong_kernel(int64_t NX, int64_t NY, int64_t NZ, int64_t NXc, int64_t NYc, int periodic,
                               const T* __restrict__ xc, T* __restrict__ out) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= NX * NY * NZ) return;
    const int64_t X = t % NX, r = t / NX, Y = r % NY, Z = r / NY;
    int64_t ix[3], iy[3];
    float wx[3], wy[3];
    const int nxp = interp_1d(X, NXc, periodic != 0, ix, wx);
    const int nyp = interp_1d(Y, NYc, periodic != 0, iy, wy);
    T s0 = 0, s1 = 0, s2 = 0;
    for (int b = 0; b < nyp; ++b)
        for (int a = 0; a < nxp; ++a) {
            const int64_t gc = ix[a] + NXc * (iy[b] + NYc * Z);
            const T w = T(wx[a] * wy[b]);
            s0 += w * xc[3 * gc];
            s1 += w * xc[3 * gc + 1];
            s2 += w * xc[3 * gc + 2];
        }
    out[3 * t] = s0;
    out[3 * t + 1] = s1;
    out[3 * t + 2] = s2;
}

// fine lattice offsets d and weights of the coarse node Xc in P^T (the
// transpose of interp_1d): vertex nodes (Xc even) reach X = 2 Xc + {0, +-1,
// +-3}, midpoint nodes (Xc odd) X = 2 Xc + {0, +-1}
__device__ __forceinline__ int restrict_1d(int64_t Xc, int64_t NX, bool periodic, int64_t (&ix)[5], float (&w)[5]) {
    const int64_t X0 = 2 * Xc;
    int n = 0;
    auto add = [&](int d, float wt) {
        int64_t X = X0 + d;
        if (periodic) {
            if (X < 0) X += NX;
            if (X >= NX) X -= NX;
        } else if (X < 0 || X >= NX) {
            return;
        }
        ix[n] = X;
        w[n] = wt;
        ++n;
    };
    if ((Xc & 1) == 0) {
        add(-3, -0.125f); add(-1, 0.375f); add(0, 1.f); add(1, 0.375f); add(3, -0.125f);
    } else {
        add(-1, 0.75f); add(0, 1.f); add(1, 0.75f);
    }
    return n;
}

// b_c = P^T r_f (velocity part)
template <typename T>
__global__ void restrict_kernel(int64_t NX, int64_t NY, int64_t NZ, int64_t NXc, int64_t NYc, int periodic,
                                const T* __restrict__ rf, T* __restrict__ bc) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= NXc * NYc * NZ) return;
    const int64_t Xc = t % NXc, r = t / NXc, Yc = r % NYc, Z = r / NYc;
    int64_t ix[5], iy[5];
    float wx[5], wy[5];
    const int nx = restrict_1d(Xc, NX, periodic != 0, ix, wx);
    const int ny = restrict_1d(Yc, NY, periodic != 0, iy, wy);
    T s0 = 0, s1 = 0, s2 = 0;
    for (int b = 0; b < ny; ++b)
        for (int a = 0; a < nx; ++a) {
            const int64_t gf = ix[a] + NX * (iy[b] + NY * Z);
            const T w = T(wx[a] * wy[b]);
            s0 += w * rf[3 * gf];
            s1 += w * rf[3 * gf + 1];
            s2 += w * rf[3 * gf + 2];
        }
    bc[3 * t] = s0;
    bc[3 * t + 1] = s1;
    bc[3 * t + 2] = s2;
}

// v_g <- P_b v_g at the basal nodes (the slip projector; zero for no-slip)
template <typename T>
__global__ void project_kernel(int64_t Nb, const int32_t* __restrict__ nodes, const double* __restrict__ P,
                               T* __restrict__ v) {
    const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (b >= Nb) return;
    const int64_t g = nodes[b];
    const double* p = P + 6 * b;
    const T x0 = v[3 * g], x1 = v[3 * g + 1], x2 = v[3 * g + 2];
    const T p00 = T(p[0]), p11 = T(p[1]), p22 = T(p[2]), p01 = T(p[3]), p02 = T(p[4]), p12 = T(p[5]);
    v[3 * g] = p00 * x0 + p01 * x1 + p02 * x2;
    v[3 * g + 1] = p01 * x0 + p11 * x1 + p12 * x2;
    v[3 * g + 2] = p02 * x0 + p12 * x1 + p22 * x2;
}

int dalloc(void** p, size_t bytes) {
    if (dev_alloc(p, bytes) != cudaSuccess) {
        *p = nullptr;
        return fail(STOKES_E_NOMEM, "multigrid workspace");
    }
    if (cudaMemset(*p, 0, bytes) != cudaSuccess) return fail(STOKES_E_CUDA, "clearing the multigrid workspace");
    return STOKES_OK;
}

ColSolveArgs level_cs(const MgLevel& Lv, double scale) {
    const stokes_mesh* m = Lv.mesh;
    ColSolveArgs c{};
    c.ncol = m->h.ncol; c.Nv = m->h.Nv; c.colmax = m->h.colmax; c.bw = Lv.bw;
    c.col_nodes = m->d_col_nodes; c.col_len = m->d_col_len; c.col_basal = m->d_col_basal;
    c.basal_P = m->d_basal_P; c.scale = scale; c.A = Lv.A;
    return c;
}

#define MG_CK(call)                     \
    do {                                \
        int rc_ = (call);               \
        if (rc_) return rc_;            \
    } while (0)
#define MG_CU(call, what)                                       \
    do {                                                        \
        cudaError_t e_ = cudaError_t(call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);      \
    } while (0)

int project(const MgLevel& Lv, int prec, void* v, cudaStream_t s) {
    const stokes_mesh* m = Lv.mesh;
    if (m->h.Nb == 0) return STOKES_OK;
    if (prec == STOKES_F32)
        project_kernel<float><<<blocks_for(m->h.Nb), TPB, 0, s>>>(m->h.Nb, m->d_basal_nodes, m->d_basal_P,
                                                                  static_cast<float*>(v));
    else
        project_kernel<double><<<blocks_for(m->h.Nb), TPB, 0, s>>>(m->h.Nb, m->d_basal_nodes, m->d_basal_P,
                                                                   static_cast<double*>(v));
    MG_CU(cudaGetLastError(), "basal projection");
    return STOKES_OK;
}

int transfer(const MgLevel& F, const MgLevel& Cl, int prec, bool periodic, bool up, const void* in, void* out,
             cudaStream_t s) {
    if (up) {
        const int64_t n = F.NX * F.NY * F.NZ;
        if (prec == STOKES_F32)
            prolong_kernel<float><<<blocks_for(n), TPB, 0, s>>>(F.NX, F.NY, F.NZ, Cl.NX, Cl.NY, periodic,
                                                                static_cast<const float*>(in), static_cast<float*>(out));
        else
            prolong_kernel<double><<<blocks_for(n), TPB, 0, s>>>(F.NX, F.NY, F.NZ, Cl.NX, Cl.NY, periodic,
                                                                 static_cast<const double*>(in), static_cast<double*>(out));
    } else {
        const int64_t n = Cl.NX * Cl.NY * Cl.NZ;
        if (prec == STOKES_F32)
            restrict_kernel<float><<<blocks_for(n), TPB, 0, s>>>(F.NX, F.NY, F.NZ, Cl.NX, Cl.NY, periodic,
                                                                 static_cast<const float*>(in), static_cast<float*>(out));
        else
            restrict_kernel<double><<<blocks_for(n), TPB, 0, s>>>(F.NX, F.NY, F.NZ, Cl.NX, Cl.NY, periodic,
                                                                  static_cast<const double*>(in), static_cast<double*>(out));
    }
    MG_CU(cudaGetLastError(), "multigrid transfer");
    return STOKES_OK;
}

// x = omega C^-1 b  (first smoothing step from x = 0)
int smooth_first(Multigrid& mg, MgLevel& Lv, cudaStream_t s) {
    MG_CU(launch_col_solve(mg.prec, level_cs(Lv, Lv.scale), Lv.b, Lv.t, s), "column solve");
    MG_CU(vec_axpby(Lv.nu, mg.omega, nullptr, mg.prec, Lv.t, 0.0, mg.prec, Lv.x, s), "smoothing");
    return STOKES_OK;
}

// r = b - A x (velocity part)
int residual(Multigrid& mg, MgLevel& Lv, cudaStream_t s) {
    MG_CK(stokes_state_apply(Lv.st, Lv.x, Lv.r, s));
    MG_CU(vec_axpby(Lv.nu, 1.0, nullptr, mg.prec, Lv.b, -1.0, mg.prec, Lv.r, s), "residual");
    return STOKES_OK;
}

// x += omega C^-1 (b - A x)
int smooth(Multigrid& mg, MgLevel& Lv, cudaStream_t s) {
    MG_CK(residual(mg, Lv, s));
    MG_CU(launch_col_solve(mg.prec, level_cs(Lv, Lv.scale), Lv.r, Lv.t, s), "column solve");
    MG_CU(vec_axpby(Lv.nu, mg.omega, nullptr, mg.prec, Lv.t, 1.0, mg.prec, Lv.x, s), "smoothing");
    return STOKES_OK;
}

int vcycle(Multigrid& mg, size_t l, cudaStream_t s) {
    MgLevel& Lv = mg.L[l];
    MG_CK(smooth_first(mg, Lv, s));
    if (l + 1 == mg.L.size()) {
        for (int it = 1; it < mg.coarse_sweeps; ++it) MG_CK(smooth(mg, Lv, s));
        return STOKES_OK;
    }
    MgLevel& C = mg.L[l + 1];
    MG_CK(residual(mg, Lv, s));
    MG_CK(project(Lv, mg.prec, Lv.r, s));
    MG_CK(transfer(Lv, C, mg.prec, mg.periodic, false, Lv.r, C.b, s));
    MG_CK(project(C, mg.prec, C.b, s));
    MG_CK(vcycle(mg, l + 1, s));
    MG_CK(transfer(Lv, C, mg.prec, mg.periodic, true, C.x, Lv.t, s));
    MG_CK(project(Lv, mg.prec, Lv.t, s));
    MG_CU(vec_axpby(Lv.nu, 1.0, nullptr, mg.prec, Lv.t, 1.0, mg.prec, Lv.x, s), "coarse correction");
    MG_CK(smooth(mg, Lv, s));
    return STOKES_OK;
}

}  // namespace

bool mg_eligible(const stokes_mesh* m) {
    return m && m->on_device && m->h.lattice && m->h.k == 2 && m->h.n_hang == 0 && m->h.nx % 2 == 0 &&
           m->h.ny % 2 == 0 && m->h.nx >= 4 && m->h.ny >= 4;
}

int mg_create(Multigrid& mg, const stokes_mesh* fine, stokes_state* st_fine, void* A_fine, int bw_fine, int prec) {
    mg_destroy(mg);
    if (!mg_eligible(fine)) return fail(STOKES_E_INVAL, "the mesh does not carry the velocity multigrid");
    mg.prec = prec;
    mg.periodic = fine->h.periodic;
    const size_t isz = prec == STOKES_F32 ? 4 : 8;
    MgLevel L0;
    L0.mesh = const_cast<stokes_mesh*>(fine);
    L0.st = st_fine;
    L0.A = A_fine;
    L0.bw = bw_fine;
    L0.n = 3 * fine->h.Nv + fine->h.Np;
    L0.nu = 3 * fine->h.Nv;
    L0.NX = fine->h.latNX; L0.NY = fine->h.latNY; L0.NZ = int64_t(fine->h.nz) * fine->h.k + 1;
    mg.L.push_back(L0);
    MgLevel& F0 = mg.L[0];
    MG_CK(dalloc(&F0.b, size_t(F0.n) * isz));
    MG_CK(dalloc(&F0.x, size_t(F0.n) * isz));
    MG_CK(dalloc(&F0.r, size_t(F0.n) * isz));
    MG_CK(dalloc(&F0.t, size_t(F0.n) * isz));
    MG_CK(dalloc(reinterpret_cast<void**>(&mg.dsc), sizeof(double)));
    while (true) {
        const MgLevel& P = mg.L.back();
        const HostMesh& h = P.mesh->h;
        if (h.nx % 2 || h.ny % 2 || h.nx / 2 < 2 || h.ny / 2 < 2) break;
        // coarse mesh: the fine lattice heights at the coarse GLL points
        // (the fine element vertices, lattice points 2 Xc, 2 Yc)
        stokes_mesh_desc d{};
        d.nx = h.nx / 2; d.ny = h.ny / 2; d.nz = h.nz; d.k = 2;
        d.pressure_space = h.pspace; d.periodic_xy = h.periodic ? 1 : 0;
        d.Lx = h.Lx; d.Ly = h.Ly; d.basal_bc = h.basal_bc; d.device = fine->device;
        const int64_t NXc = h.periodic ? int64_t(d.nx) * 2 : int64_t(d.nx) * 2 + 1;
        const int64_t NYc = h.periodic ? int64_t(d.ny) * 2 : int64_t(d.ny) * 2 + 1;
        std::vector<double> bed(size_t(NXc * NYc)), surf(size_t(NXc * NYc));
        for (int64_t Yc = 0; Yc < NYc; ++Yc)
            for (int64_t Xc = 0; Xc < NXc; ++Xc) {
                const int64_t g0 = 2 * Xc + P.NX * (2 * Yc);
                const int64_t g1 = g0 + P.NX * P.NY * (P.NZ - 1);
                bed[size_t(Xc + NXc * Yc)] = h.node_xyz[size_t(3 * g0 + 2)];
                surf[size_t(Xc + NXc * Yc)] = h.node_xyz[size_t(3 * g1 + 2)];
            }
        d.bed_nodes = bed.data();
        d.surface_nodes = surf.data();
        MgLevel C;
        C.owned = true;
        MG_CK(stokes_mesh_create(&d, &C.mesh));
        const HostMesh& hc = C.mesh->h;
        C.n = 3 * hc.Nv + hc.Np;
        C.nu = 3 * hc.Nv;
        C.NX = hc.latNX; C.NY = hc.latNY; C.NZ = int64_t(hc.nz) * hc.k + 1;
        C.bw = 3 * hc.bnode + 2;
        C.band_elems = size_t(3) * hc.colmax * size_t(2 * C.bw + 1) * size_t(band_cols(hc.ncol));
        mg.L.push_back(C);
        MgLevel& Cl = mg.L.back();
        MG_CK(stokes_state_create(Cl.mesh, prec, &Cl.st));
        MG_CK(dalloc(&Cl.A, Cl.band_elems * isz));
        MG_CK(dalloc(&Cl.b, size_t(Cl.n) * isz));
        MG_CK(dalloc(&Cl.x, size_t(Cl.n) * isz));
        MG_CK(dalloc(&Cl.r, size_t(Cl.n) * isz));
        MG_CK(dalloc(&Cl.t, size_t(Cl.n) * isz));
        MG_CK(dalloc(reinterpret_cast<void**>(&Cl.u64), size_t(Cl.n) * 8));
        MG_CK(dalloc(reinterpret_cast<void**>(&Cl.logbeta), size_t(std::max<int64_t>(hc.Nb, 1)) * 8));
    }
    if (mg.L.size() < 2) {
        mg_destroy(mg);
        return fail(STOKES_E_INVAL, "the mesh is too small for the velocity multigrid");
    }
    return STOKES_OK;
}

int mg_setup(Multigrid& mg, const stokes_params* p, const double* up_fine, double fine_scale, cudaStream_t s) {
    mg.L[0].scale = fine_scale;
    for (size_t l = 1; l < mg.L.size(); ++l) {
        MgLevel& F = mg.L[l - 1];
        MgLevel& C = mg.L[l];
        const double* uf = l == 1 ? up_fine : F.u64;
        inject_u_kernel<<<blocks_for(C.NX * C.NY * C.NZ), TPB, 0, s>>>(C.NX, C.NY, C.NZ, F.NX, F.NY, uf, C.u64);
        MG_CU(cudaGetLastError(), "multigrid injection");
        stokes_params pc = *p;
        if (p->robin && p->logbeta) {
            const double* lf = l == 1 ? p->logbeta : F.logbeta;
            inject_lb_kernel<<<blocks_for(C.NX * C.NY), TPB, 0, s>>>(C.NX, C.NY, F.NX, lf, C.logbeta);
            MG_CU(cudaGetLastError(), "multigrid injection");
            pc.logbeta = C.logbeta;
        }
        pc.constraint_scale = C.scale > 0 ? C.scale : 1.0;
        MG_CK(stokes_linearize(C.st, &pc, C.u64, s));
        // column blocks of the coarse velocity block (no Schur blocks)
        const stokes_mesh* m = C.mesh;
        MG_CU(cudaMemsetAsync(C.A, 0, C.band_elems * (mg.prec == STOKES_F32 ? 4 : 8), s), "clearing column blocks");
        ColArgs a{};
        a.E = m->h.E; a.ncol = m->h.ncol; a.npr = m->h.npr; a.pspace = m->h.pspace; a.bw = C.bw;
        a.rows = 3 * m->h.colmax;
        a.fstate = C.st->slide ? C.st->d_fstate : nullptr;
        a.robin = pc.robin && m->h.nF > 0;
        a.nodes = m->d_nodes; a.hang = m->d_hang; a.col_of = m->d_col_of; a.pos_of = m->d_pos_of;
        a.fidx = m->d_fidx; a.fmap = m->d_fmap; a.fgeo = m->d_fgeo; a.logbeta = pc.logbeta;
        a.state = C.st->d_state; a.state_cpl = C.st->cpl; a.A = C.A; a.mblk = nullptr; a.schur_full = 0;
        MG_CU(launch_precond_assembly(m->h.k, mg.prec, a, s), "coarse column assembly");
        if (!(C.scale > 0)) {
            // constraint rows scaled to the mean diagonal of this level's velocity block
            MG_CU(launch_col_diag_sum(mg.prec, level_cs(C, 1.0), mg.dsc, s), "diagonal scale");
            double sum = 0;
            MG_CU(cudaMemcpyAsync(&sum, mg.dsc, sizeof(double), cudaMemcpyDeviceToHost, s), "readback");
            MG_CU(cudaStreamSynchronize(s), "sync");
            C.scale = sum / double(3 * m->h.Nv);
            if (!(C.scale > 0)) C.scale = 1.0;
        }
        C.st->params.constraint_scale = C.scale;
        MG_CU(launch_col_factor(mg.prec, level_cs(C, C.scale), s), "coarse column factorisation");
    }
    return STOKES_OK;
}

int mg_apply(Multigrid& mg, const void* r, void* z, cudaStream_t s) {
    MgLevel& L0 = mg.L[0];
    MG_CU(vec_axpby(L0.nu, 1.0, nullptr, mg.prec, r, 0.0, mg.prec, L0.b, s), "multigrid input");
    MG_CK(vcycle(mg, 0, s));
    MG_CU(vec_axpby(L0.nu, 1.0, nullptr, mg.prec, L0.x, 0.0, mg.prec, z, s), "multigrid output");
    return STOKES_OK;
}

void mg_destroy(Multigrid& mg) {
    for (MgLevel& Lv : mg.L) {
        for (void* p : {Lv.b, Lv.x, Lv.r, Lv.t}) if (p) cudaFree(p);
        if (Lv.owned) {
            if (Lv.A) cudaFree(Lv.A);
            if (Lv.u64) cudaFree(Lv.u64);
            if (Lv.logbeta) cudaFree(Lv.logbeta);
            if (Lv.st) stokes_state_destroy(Lv.st);
            if (Lv.mesh) stokes_mesh_destroy(Lv.mesh);
        }
    }
    mg.L.clear();
    if (mg.dsc) cudaFree(mg.dsc);
    mg.dsc = nullptr;
}

}  // namespace stokes
