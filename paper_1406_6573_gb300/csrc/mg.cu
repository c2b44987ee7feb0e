// Geometric multigrid for the velocity block (see mg.h).
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_runtime.h>

#include "mg.h"
#include "hanging.h"
#include "precond.h"
#include "vec.h"

namespace stokes {
namespace {

constexpr int TPB = 256;

inline unsigned blocks_for(int64_t n) { return unsigned((n + TPB - 1) / TPB); }

// Transfers between a level (fine lattice NX x NY x NZ) and the next
// (coarse NXc x NYc x NZ) are tensor products of 1-D tables in x and y,
// identity in z; each table row lists (lattice index, weight) pairs:
//   P  [fine X]:   coarse nodal values -> fine node (coarse degree-k
//                  Lagrange interpolation; KP = k + 1 entries)
//   R  [coarse X]: the transpose of P (at most RM entries)
//   J  [coarse X]: fine nodal values -> coarse node (fine degree-k
//                  interpolation at the coarse node's position; KP entries)
constexpr int KP = 5;     // k + 1 for k <= 4
constexpr int RM = 17;    // 4 k + 1

struct Tab1 {
    const int32_t* idx;   // [n][m]
    const double* w;      // [n][m]
    const int32_t* cnt;   // [n]
    int m;
};

// out (3 components at every node of the target lattice) = tensor transfer of
// in: out[X, Y, Z] = sum_a sum_b tx[X][a] ty[Y][b] in[ix, iy, Z], accumulated
// in the input's type (the FP32 cycle's transfers in FP32: FP64 arithmetic
// made the fine-level transfer of the 128x128x8 slab take 0.1 ms)
template <typename TI, typename TO>
__global__ void transfer_kernel(int64_t NXo, int64_t NYo, int64_t NZ, int64_t NXi, int64_t NYi, Tab1 tx, Tab1 ty,
                                int ncomp, const TI* __restrict__ in, TO* __restrict__ out) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= NXo * NYo * NZ) return;
    const int64_t X = t % NXo, r = t / NXo, Y = r % NYo, Z = r / NYo;
    const int nx = tx.cnt[X], ny = ty.cnt[Y];
    TI s[3] = {TI(0), TI(0), TI(0)};
    for (int b = 0; b < ny; ++b) {
        const int64_t iy = ty.idx[Y * ty.m + b];
        const TI wy = TI(ty.w[Y * ty.m + b]);
        for (int a = 0; a < nx; ++a) {
            const int64_t gi = tx.idx[X * tx.m + a] + NXi * (iy + NYi * Z);
            const TI wgt = TI(tx.w[X * tx.m + a]) * wy;
            for (int c = 0; c < ncomp; ++c) s[c] += wgt * in[ncomp * gi + c];
        }
    }
    for (int c = 0; c < ncomp; ++c) out[ncomp * t + c] = TO(s[c]);
}

// out[row * nc + c] = sum_j w[j] in[col[j] * nc + c]  (CSR, nc components;
// accumulated in the input's type)
template <typename TI, typename TO>
__global__ void csr_kernel(int64_t rows, const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                           const double* __restrict__ w, int nc, const TI* __restrict__ in, TO* __restrict__ out) {
    const int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    TI s[3] = {TI(0), TI(0), TI(0)};
    for (int j = ptr[r]; j < ptr[r + 1]; ++j) {
        const int64_t c = col[j];
        const TI wj = TI(w[j]);
        for (int q = 0; q < nc; ++q) s[q] += wj * in[nc * c + q];
    }
    for (int q = 0; q < nc; ++q) out[nc * r + q] = TO(s[q]);
}

// Lagrange polynomials of the nodes x[0..n) at t
void lagrange_at(int n, const double* x, double t, double* out) {
    for (int i = 0; i < n; ++i) {
        double v = 1.0;
        for (int j = 0; j < n; ++j)
            if (j != i) v *= (t - x[j]) / (x[i] - x[j]);
        out[i] = v;
    }
}

// host tables of one direction: fine lattice of nf elements, coarse of nf / 2
struct HostTab1 {
    std::vector<int32_t> idx, cnt;
    std::vector<double> w;
    int m = 0;
};

// false if a table row would need more entries than its width (KP for P and
// J, RM for R: 4k + 1 fine nodes per coarse node, 17 at k = 4)
bool build_dir(int nf, int k, bool periodic, const double* gll, HostTab1& P, HostTab1& R, HostTab1& J) {
    if (k < 1 || k + 1 > KP || 4 * k + 1 > RM || nf < 2 || nf % 2) return false;
    const int nc = nf / 2;
    const int NXf = periodic ? nf * k : nf * k + 1, NXc = periodic ? nc * k : nc * k + 1;
    auto wrapf = [&](int64_t X) { return periodic ? int32_t(X % NXf) : int32_t(X); };
    auto wrapc = [&](int64_t X) { return periodic ? int32_t(X % NXc) : int32_t(X); };
    double L[N1MAX];
    // P: fine X = ex k + i lies in coarse element ex / 2 at local coordinate
    // (ex - 2 cx) + t_i - 1 (t_i = (gll_i + 1) / 2)
    P.m = KP; P.idx.assign(size_t(NXf) * KP, 0); P.w.assign(size_t(NXf) * KP, 0.0); P.cnt.assign(NXf, 0);
    for (int X = 0; X < NXf; ++X) {
        int ex = X / k, i = X % k;
        if (ex == nf) { ex = nf - 1; i = k; }          // last node of a non-periodic lattice
        const int cx = ex / 2;
        lagrange_at(k + 1, gll, double(ex - 2 * cx) + 0.5 * (gll[i] + 1.0) - 1.0, L);
        int n = 0;
        for (int m = 0; m <= k; ++m) {
            if (std::fabs(L[m]) < 1e-14) continue;
            P.idx[size_t(X) * KP + n] = wrapc(int64_t(cx) * k + m);
            P.w[size_t(X) * KP + n] = L[m];
            ++n;
        }
        P.cnt[X] = n;
    }
    // R = P^T
    std::vector<std::vector<std::pair<int32_t, double>>> rows(NXc);
    for (int X = 0; X < NXf; ++X)
        for (int a = 0; a < P.cnt[X]; ++a) rows[P.idx[size_t(X) * KP + a]].push_back({X, P.w[size_t(X) * KP + a]});
    R.m = RM; R.idx.assign(size_t(NXc) * RM, 0); R.w.assign(size_t(NXc) * RM, 0.0); R.cnt.assign(NXc, 0);
    for (int Xc = 0; Xc < NXc; ++Xc) {
        if (rows[Xc].size() > size_t(RM)) return false;
        const int n = int(rows[Xc].size());
        for (int a = 0; a < n; ++a) {
            R.idx[size_t(Xc) * RM + a] = rows[Xc][a].first;
            R.w[size_t(Xc) * RM + a] = rows[Xc][a].second;
        }
        R.cnt[Xc] = n;
    }
    // J: coarse Xc = cx k + i at fine-element coordinate 2 cx + 2 t_i
    J.m = KP; J.idx.assign(size_t(NXc) * KP, 0); J.w.assign(size_t(NXc) * KP, 0.0); J.cnt.assign(NXc, 0);
    for (int Xc = 0; Xc < NXc; ++Xc) {
        int cx = Xc / k, i = Xc % k;
        if (cx == nc) { cx = nc - 1; i = k; }
        const double pos = 2.0 * cx + (gll[i] + 1.0);  // in fine elements
        int ex = int(std::floor(pos + 1e-12));
        if (ex > 2 * cx + 1) ex = 2 * cx + 1;
        lagrange_at(k + 1, gll, 2.0 * (pos - ex) - 1.0, L);
        int n = 0;
        for (int m = 0; m <= k; ++m) {
            if (std::fabs(L[m]) < 1e-14) continue;
            J.idx[size_t(Xc) * KP + n] = wrapf(int64_t(ex) * k + m);
            J.w[size_t(Xc) * KP + n] = L[m];
            ++n;
        }
        J.cnt[Xc] = n;
    }
    return true;
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
    c.basal_P = m->d_basal_P; c.scale = scale; c.A = Lv.A; c.err = m->d_err;
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

Tab1 dev_tab(const MgLevel& Cl, int which) {
    // which: 0 P_x, 1 P_y, 2 R_x, 3 R_y, 4 J_x, 5 J_y
    Tab1 t{};
    t.idx = Cl.t_idx + Cl.t_off[which];
    t.w = Cl.t_w + Cl.t_off[which];
    t.cnt = Cl.t_cnt + Cl.t_coff[which];
    t.m = Cl.t_m[which];
    return t;
}

// up: out_f = P in_c (coarse -> fine); down: out_c = P^T in_f (fine -> coarse)
int transfer(const MgLevel& F, const MgLevel& Cl, int prec, bool up, const void* in, void* out, cudaStream_t s) {
    if (Cl.csr) {
        const int64_t rows = up ? F.mesh->h.Nv : Cl.mesh->h.Nv;
        const int32_t* ptr = up ? Cl.P_ptr : Cl.R_ptr;
        const int32_t* col = up ? Cl.P_col : Cl.R_col;
        const double* w = up ? Cl.P_w : Cl.R_w;
        if (prec == STOKES_F32)
            csr_kernel<float, float><<<blocks_for(rows), TPB, 0, s>>>(rows, ptr, col, w, 3, static_cast<const float*>(in),
                                                                      static_cast<float*>(out));
        else
            csr_kernel<double, double><<<blocks_for(rows), TPB, 0, s>>>(rows, ptr, col, w, 3, static_cast<const double*>(in),
                                                                        static_cast<double*>(out));
        MG_CU(cudaGetLastError(), "multigrid transfer");
        return STOKES_OK;
    }
    const int64_t n = up ? F.NX * F.NY * F.NZ : Cl.NX * Cl.NY * Cl.NZ;
    const Tab1 tx = dev_tab(Cl, up ? 0 : 2), ty = dev_tab(Cl, up ? 1 : 3);
    const int64_t NXo = up ? F.NX : Cl.NX, NYo = up ? F.NY : Cl.NY;
    const int64_t NXi = up ? Cl.NX : F.NX, NYi = up ? Cl.NY : F.NY;
    if (prec == STOKES_F32)
        transfer_kernel<float, float><<<blocks_for(n), TPB, 0, s>>>(NXo, NYo, F.NZ, NXi, NYi, tx, ty, 3,
                                                                    static_cast<const float*>(in), static_cast<float*>(out));
    else
        transfer_kernel<double, double><<<blocks_for(n), TPB, 0, s>>>(NXo, NYo, F.NZ, NXi, NYi, tx, ty, 3,
                                                                      static_cast<const double*>(in), static_cast<double*>(out));
    MG_CU(cudaGetLastError(), "multigrid transfer");
    return STOKES_OK;
}

double level_omega(const Multigrid& mg, const MgLevel& Lv) { return Lv.omega > 0 ? Lv.omega : mg.omega; }

// deterministic start vector of the power iteration: hashed values in [-1, 1)
template <typename T>
__global__ void hash_fill_kernel(int64_t n, T* v) {
    const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t z = uint64_t(i) * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[i] = T(double(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
}

// x = omega C^-1 b  (first smoothing step from x = 0)
int smooth_first(Multigrid& mg, MgLevel& Lv, cudaStream_t s) {
    ColSolveArgs cs = level_cs(Lv, Lv.scale);
    cs.out_alpha = level_omega(mg, Lv);
    MG_CU(launch_col_solve(mg.prec, cs, Lv.b, Lv.x, s), "column solve");
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
    ColSolveArgs cs = level_cs(Lv, Lv.scale);
    cs.out_alpha = level_omega(mg, Lv);
    cs.out_beta = 1.0;
    MG_CU(launch_col_solve(mg.prec, cs, Lv.r, Lv.x, s), "column solve");
    return STOKES_OK;
}

int vcycle(Multigrid& mg, size_t l, cudaStream_t s) {
    MgLevel& Lv = mg.L[l];
    if (l + 1 < mg.L.size() && mg.L[l + 1].csr && mg.forest_additive) {
        // forest level: column blocks and the base-level cycle side by side
        MgLevel& C = mg.L[l + 1];
        MG_CU(launch_col_solve(mg.prec, level_cs(Lv, Lv.scale), Lv.b, Lv.x, s), "column solve");
        MG_CU(vec_axpby(Lv.nu, 1.0, nullptr, mg.prec, Lv.b, 0.0, mg.prec, Lv.r, s), "residual copy");
        MG_CK(project(Lv, mg.prec, Lv.r, s));
        MG_CK(transfer(Lv, C, mg.prec, false, Lv.r, C.b, s));
        MG_CK(project(C, mg.prec, C.b, s));
        MG_CK(vcycle(mg, l + 1, s));
        MG_CK(transfer(Lv, C, mg.prec, true, C.x, Lv.t, s));
        MG_CK(project(Lv, mg.prec, Lv.t, s));
        MG_CU(vec_axpby(Lv.nu, 1.0, nullptr, mg.prec, Lv.t, 1.0, mg.prec, Lv.x, s), "coarse correction");
        return STOKES_OK;
    }
    MG_CK(smooth_first(mg, Lv, s));
    if (l + 1 == mg.L.size()) {
        for (int it = 1; it < mg.coarse_sweeps; ++it) MG_CK(smooth(mg, Lv, s));
        return STOKES_OK;
    }
    MgLevel& C = mg.L[l + 1];
    MG_CK(residual(mg, Lv, s));
    MG_CK(project(Lv, mg.prec, Lv.r, s));
    MG_CK(transfer(Lv, C, mg.prec, false, Lv.r, C.b, s));
    MG_CK(project(C, mg.prec, C.b, s));
    MG_CK(vcycle(mg, l + 1, s));
    MG_CK(transfer(Lv, C, mg.prec, true, C.x, Lv.t, s));
    MG_CK(project(Lv, mg.prec, Lv.t, s));
    MG_CU(vec_axpby(Lv.nu, 1.0, nullptr, mg.prec, Lv.t, 1.0, mg.prec, Lv.x, s), "coarse correction");
    MG_CK(smooth(mg, Lv, s));
    return STOKES_OK;
}

// Largest eigenvalue of C^-1 A on level Lv (C: its factored column blocks,
// A: its velocity block with the constraint rows) by power iteration from a
// hashed start vector; uses Lv.x, Lv.r and Lv.t (x and t cleared afterwards).
int estimate_lmax(Multigrid& mg, MgLevel& Lv, int its, double& lmax, cudaStream_t s) {
    if (mg.prec == STOKES_F32) hash_fill_kernel<float><<<blocks_for(Lv.nu), TPB, 0, s>>>(Lv.nu, static_cast<float*>(Lv.x));
    else hash_fill_kernel<double><<<blocks_for(Lv.nu), TPB, 0, s>>>(Lv.nu, static_cast<double*>(Lv.x));
    MG_CU(cudaGetLastError(), "power iteration start");
    MG_CK(project(Lv, mg.prec, Lv.x, s));
    MG_CU(vec_multidot(Lv.nu, mg.prec, nullptr, 0, 0, mg.prec, Lv.x, mg.dsc, 1, s), "norm");
    MG_CU(vec_normalize(Lv.nu, mg.prec, Lv.x, mg.dsc, s), "normalise");
    for (int it = 0; it < its; ++it) {
        MG_CK(stokes_state_apply(Lv.st, Lv.x, Lv.r, s));
        MG_CU(launch_col_solve(mg.prec, level_cs(Lv, Lv.scale), Lv.r, Lv.t, s), "column solve");
        MG_CU(vec_multidot(Lv.nu, mg.prec, nullptr, 0, 0, mg.prec, Lv.t, mg.dsc, 1, s), "norm");
        MG_CU(vec_axpby(Lv.nu, 1.0, nullptr, mg.prec, Lv.t, 0.0, mg.prec, Lv.x, s), "copy");
        MG_CU(vec_normalize(Lv.nu, mg.prec, Lv.x, mg.dsc, s), "normalise");
    }
    double n2 = 0;
    MG_CU(cudaMemcpyAsync(&n2, mg.dsc, sizeof(double), cudaMemcpyDeviceToHost, s), "readback");
    MG_CU(cudaStreamSynchronize(s), "sync");
    lmax = std::sqrt(n2);
    // the work vectors start the cycle from zero again
    MG_CU(cudaMemsetAsync(Lv.x, 0, size_t(Lv.n) * (mg.prec == STOKES_F32 ? 4 : 8), s), "clear");
    MG_CU(cudaMemsetAsync(Lv.t, 0, size_t(Lv.n) * (mg.prec == STOKES_F32 ? 4 : 8), s), "clear");
    return STOKES_OK;
}

}  // namespace

int mg_transfer_dense(int nf, int k, int periodic, int which, double* out, int64_t rows, int64_t cols) {
    Tables1D t{};
    if (k < 1 || k > 4) return fail(STOKES_E_INVAL, "degree outside 1..4");
    build_tables(k, 0, t);
    HostTab1 P, R, J;
    if (!build_dir(nf, k, periodic != 0, t.gll, P, R, J)) return fail(STOKES_E_INVAL, "transfer tables not built");
    const HostTab1& T = which == 0 ? P : (which == 1 ? R : J);
    const int64_t nr = int64_t(T.cnt.size());
    const int64_t NXf = periodic ? int64_t(nf) * k : int64_t(nf) * k + 1;
    const int64_t NXc = periodic ? int64_t(nf / 2) * k : int64_t(nf / 2) * k + 1;
    const int64_t nc = which == 0 ? NXc : NXf;
    if (which < 0 || which > 2 || rows != nr || cols != nc || !out) return fail(STOKES_E_INVAL, "wrong table shape");
    std::fill(out, out + rows * cols, 0.0);
    for (int64_t r = 0; r < nr; ++r)
        for (int a = 0; a < T.cnt[size_t(r)]; ++a)
            out[r * cols + T.idx[size_t(r) * T.m + a]] += T.w[size_t(r) * T.m + a];
    return STOKES_OK;
}

bool mg_eligible(const stokes_mesh* m) {
    if (!m || !m->on_device || m->h.k < 2 || m->h.k > 4) return false;
    if (!m->h.lattice) return m->h.nx >= 2 && m->h.ny >= 2;       // forest: the base mesh is the next level
    return m->h.n_hang == 0 && m->h.nx % 2 == 0 && m->h.ny % 2 == 0 && m->h.nx >= 4 && m->h.ny >= 4;
}

int forest_prolongation(const HostMesh& h, const std::vector<int32_t>& nodes, const std::vector<uint8_t>& refine,
                        const HostMesh& hb, HostCsr& P) {
    const int k = h.k, n1 = k + 1, N3 = n1 * n1 * n1;
    const int64_t NXb = hb.latNX, NYb = hb.latNY;
    const int64_t nc = int64_t(h.nx) * h.ny * h.nz;
    if (!hb.lattice || hb.k != k || hb.nx != h.nx || hb.ny != h.ny || hb.nz != h.nz || nodes.size() != size_t(h.E) * N3 ||
        h.elem_hang.size() != size_t(h.E) || h.node_xyz.size() != size_t(3 * h.Nv) ||
        hb.node_xyz.size() != size_t(3 * hb.Nv) || (!refine.empty() && refine.size() != size_t(nc)))
        return fail(STOKES_E_MESH, "the forest and its base mesh do not match");
    // element -> coarse cell (children of a refined cell are consecutive)
    std::vector<int64_t> cell(size_t(h.E));
    {
        int64_t e = 0;
        for (int64_t c = 0; c < nc; ++c) {
            const int nch = (!refine.empty() && refine[size_t(c)]) ? 8 : 1;
            for (int ch = 0; ch < nch; ++ch) {
                if (e >= h.E) return fail(STOKES_E_MESH, "forest element count does not match its refinement mask");
                cell[size_t(e++)] = c;
            }
        }
        if (e != h.E) return fail(STOKES_E_MESH, "forest element count does not match its refinement mask");
    }
    // rows: forest global nodes, each from the first non-hanging slot naming it
    std::vector<std::vector<std::pair<int32_t, double>>> rows(size_t(h.Nv));
    std::vector<char> done(size_t(h.Nv), 0);
    double L[3][N1MAX];
    for (int64_t e = 0; e < h.E; ++e) {
        const uint32_t hc = h.elem_hang[size_t(e)];
        const int64_t c = cell[size_t(e)];
        const bool child = !refine.empty() && refine[size_t(c)];
        const int64_t cx = c % h.nx, cy = (c / h.nx) % h.ny, cz = c / (int64_t(h.nx) * h.ny);
        for (int n = 0; n < N3; ++n) {
            const int idx[3] = {n % n1, (n / n1) % n1, n / (n1 * n1)};
            if (slot_on_hanging_entity(hc, idx, k)) continue;
            const int64_t g = nodes[size_t(e) * N3 + n];
            if (g < 0 || g >= h.Nv) return fail(STOKES_E_MESH, "forest element map out of range");
            if (done[size_t(g)]) continue;
            done[size_t(g)] = 1;
            // the slot's coordinates in the base cell's reference element
            for (int dd = 0; dd < 3; ++dd) {
                const double xi = child ? double(child_bit(hc, dd)) + 0.5 * (h.tab.gll[idx[dd]] + 1.0) - 1.0
                                        : h.tab.gll[idx[dd]];
                lagrange_at(n1, h.tab.gll, xi, L[dd]);
            }
            for (int c2 = 0; c2 < n1; ++c2)
                for (int b2 = 0; b2 < n1; ++b2)
                    for (int a2 = 0; a2 < n1; ++a2) {
                        const double wgt = L[0][a2] * L[1][b2] * L[2][c2];
                        if (std::fabs(wgt) < 1e-14) continue;
                        int64_t X = cx * k + a2, Y = cy * k + b2;
                        if (h.periodic) { X %= NXb; Y %= NYb; }
                        const int64_t gb = X + NXb * (Y + NYb * (cz * k + c2));
                        if (gb < 0 || gb >= hb.Nv) return fail(STOKES_E_MESH, "base lattice node out of range");
                        rows[size_t(g)].push_back({int32_t(gb), wgt});
                    }
        }
    }
    P.ptr.assign(size_t(h.Nv) + 1, 0);
    P.col.clear();
    P.w.clear();
    for (int64_t g = 0; g < h.Nv; ++g) {
        if (!done[size_t(g)]) return fail(STOKES_E_MESH, "a forest node has no element slot of its own");
        P.ptr[size_t(g) + 1] = P.ptr[size_t(g)] + int32_t(rows[size_t(g)].size());
        for (auto& pr : rows[size_t(g)]) { P.col.push_back(pr.first); P.w.push_back(pr.second); }
    }
    // the base map interpolated at the forest nodes is the forest map (the
    // children inherit their parent's map): heights, and the horizontal
    // positions away from a periodic seam
    for (int64_t g = 0; g < h.Nv; ++g) {
        double x[3] = {0, 0, 0};
        for (int32_t j = P.ptr[size_t(g)]; j < P.ptr[size_t(g) + 1]; ++j)
            for (int dd = 0; dd < 3; ++dd) x[dd] += P.w[size_t(j)] * hb.node_xyz[size_t(3 * P.col[size_t(j)] + dd)];
        const double* xf = &h.node_xyz[size_t(3 * g)];
        const double tol = 1e-8 * (std::fabs(xf[2]) + std::max(h.Lx, h.Ly));
        bool bad = std::fabs(x[2] - xf[2]) > tol;
        if (!h.periodic) bad = bad || std::fabs(x[0] - xf[0]) > tol || std::fabs(x[1] - xf[1]) > tol;
        if (bad) return fail(STOKES_E_MESH, "the forest's base level does not reproduce its geometry");
    }
    return STOKES_OK;
}

namespace {

HostCsr transpose(const HostCsr& A, int64_t ncols) {
    HostCsr T;
    T.ptr.assign(size_t(ncols) + 1, 0);
    for (int32_t c : A.col) T.ptr[size_t(c) + 1]++;
    for (int64_t i = 0; i < ncols; ++i) T.ptr[size_t(i) + 1] += T.ptr[size_t(i)];
    T.col.resize(A.col.size());
    T.w.resize(A.w.size());
    std::vector<int32_t> fill(T.ptr.begin(), T.ptr.end() - 1);
    const int64_t rows = int64_t(A.ptr.size()) - 1;
    for (int64_t r = 0; r < rows; ++r)
        for (int32_t j = A.ptr[size_t(r)]; j < A.ptr[size_t(r) + 1]; ++j) {
            const int32_t c = A.col[size_t(j)];
            T.col[size_t(fill[size_t(c)])] = int32_t(r);
            T.w[size_t(fill[size_t(c)])] = A.w[size_t(j)];
            fill[size_t(c)]++;
        }
    return T;
}

// rows scaled to unit sum (an averaging restriction); empty rows stay empty
void normalise_rows(HostCsr& A) {
    const int64_t rows = int64_t(A.ptr.size()) - 1;
    for (int64_t r = 0; r < rows; ++r) {
        double s = 0;
        for (int32_t j = A.ptr[size_t(r)]; j < A.ptr[size_t(r) + 1]; ++j) s += A.w[size_t(j)];
        if (std::fabs(s) > 1e-12)
            for (int32_t j = A.ptr[size_t(r)]; j < A.ptr[size_t(r) + 1]; ++j) A.w[size_t(j)] /= s;
    }
}

int upload_csr(const HostCsr& A, int32_t** ptr, int32_t** col, double** w) {
    MG_CK(dalloc(reinterpret_cast<void**>(ptr), A.ptr.size() * 4));
    MG_CK(dalloc(reinterpret_cast<void**>(col), std::max<size_t>(A.col.size(), 1) * 4));
    MG_CK(dalloc(reinterpret_cast<void**>(w), std::max<size_t>(A.w.size(), 1) * 8));
    MG_CU(cudaMemcpy(*ptr, A.ptr.data(), A.ptr.size() * 4, cudaMemcpyHostToDevice), "tables");
    if (!A.col.empty()) {
        MG_CU(cudaMemcpy(*col, A.col.data(), A.col.size() * 4, cudaMemcpyHostToDevice), "tables");
        MG_CU(cudaMemcpy(*w, A.w.data(), A.w.size() * 8, cudaMemcpyHostToDevice), "tables");
    }
    return STOKES_OK;
}

// sizes, stored state, column blocks and work vectors of a coarse level whose
// mesh is built
int alloc_level(MgLevel& Cl, int prec) {
    const size_t isz = prec == STOKES_F32 ? 4 : 8;
    const HostMesh& hc = Cl.mesh->h;
    Cl.n = 3 * hc.Nv + hc.Np;
    Cl.nu = 3 * hc.Nv;
    Cl.NX = hc.latNX; Cl.NY = hc.latNY; Cl.NZ = int64_t(hc.nz) * hc.k + 1;
    Cl.bw = 3 * hc.bnode + 2;
    Cl.band_elems = size_t(3) * hc.colmax * size_t(2 * Cl.bw + 1) * size_t(band_cols(hc.ncol));
    MG_CK(stokes_state_create(Cl.mesh, prec, &Cl.st));
    MG_CK(dalloc(&Cl.A, Cl.band_elems * isz));
    MG_CK(dalloc(&Cl.b, size_t(Cl.n) * isz));
    MG_CK(dalloc(&Cl.x, size_t(Cl.n) * isz));
    MG_CK(dalloc(&Cl.r, size_t(Cl.n) * isz));
    MG_CK(dalloc(&Cl.t, size_t(Cl.n) * isz));
    MG_CK(dalloc(reinterpret_cast<void**>(&Cl.u64), size_t(Cl.n) * 8));
    MG_CK(dalloc(reinterpret_cast<void**>(&Cl.logbeta), size_t(std::max<int64_t>(hc.Nb, 1)) * 8));
    return STOKES_OK;
}

// The unrefined base mesh of the forest fine and the transfers between them.
int build_base_level(const stokes_mesh* fine, MgLevel& C) {
    const HostMesh& h = fine->h;
    const int k = h.k, N3 = (k + 1) * (k + 1) * (k + 1);
    stokes_mesh_desc d{};
    d.nx = h.nx; d.ny = h.ny; d.nz = h.nz; d.k = k; d.pressure_space = h.pspace;
    d.periodic_xy = h.periodic ? 1 : 0; d.Lx = h.Lx; d.Ly = h.Ly; d.basal_bc = h.basal_bc; d.device = fine->device;
    const MeshSource& sc = fine->src;
    d.bed = stokes_field{sc.bed_mean, int(sc.bed[0].size()), sc.bed[0].data(), sc.bed[1].data(), sc.bed[2].data(),
                         sc.bed[3].data()};
    d.surface = stokes_field{sc.surf_mean, int(sc.surf[0].size()), sc.surf[0].data(), sc.surf[1].data(),
                             sc.surf[2].data(), sc.surf[3].data()};
    if (!sc.bed_nodes.empty()) { d.bed_nodes = sc.bed_nodes.data(); d.surface_nodes = sc.surf_nodes.data(); }
    C.owned = true;
    C.csr = true;
    MG_CK(stokes_mesh_create(&d, &C.mesh));
    const HostMesh& hb = C.mesh->h;
    const int64_t NXb = hb.latNX, NYb = hb.latNY;
    // forest element map (the device copy: a device mesh keeps no host copy)
    std::vector<int32_t> nodes(size_t(h.E) * N3);
    MG_CU(cudaMemcpy(nodes.data(), fine->d_nodes, nodes.size() * 4, cudaMemcpyDeviceToHost), "element map");
    HostCsr P;
    MG_CK(forest_prolongation(h, nodes, sc.refine, hb, P));
    HostCsr R = transpose(P, hb.Nv);
    HostCsr J = R;
    normalise_rows(J);
    // basal rows: forest basal node bf -> base basal nodes (the Z = 0 lattice plane)
    if (h.basal_nodes.size() != size_t(h.Nb)) return fail(STOKES_E_MESH, "the forest's basal node list is incomplete");
    HostCsr Pb;
    Pb.ptr.assign(size_t(h.Nb) + 1, 0);
    for (int64_t bf = 0; bf < h.Nb; ++bf) {
        const int64_t g = h.basal_nodes[size_t(bf)];
        if (g < 0 || g >= h.Nv) return fail(STOKES_E_MESH, "forest basal node out of range");
        for (int32_t j = P.ptr[size_t(g)]; j < P.ptr[size_t(g) + 1]; ++j)
            if (P.col[size_t(j)] < NXb * NYb) { Pb.col.push_back(P.col[size_t(j)]); Pb.w.push_back(P.w[size_t(j)]); }
        Pb.ptr[size_t(bf) + 1] = int32_t(Pb.col.size());
    }
    HostCsr Jb = transpose(Pb, hb.Nb);
    normalise_rows(Jb);
    MG_CK(upload_csr(P, &C.P_ptr, &C.P_col, &C.P_w));
    MG_CK(upload_csr(R, &C.R_ptr, &C.R_col, &C.R_w));
    MG_CK(upload_csr(J, &C.J_ptr, &C.J_col, &C.J_w));
    MG_CK(upload_csr(Jb, &C.Jb_ptr, &C.Jb_col, &C.Jb_w));
    return STOKES_OK;
}

}  // namespace

constexpr int MG_MIN_CELLS = 4;

int mg_create(Multigrid& mg, const stokes_mesh* fine, stokes_state* st_fine, void* A_fine, int bw_fine, int prec) {
    mg_destroy(mg);
    if (!mg_eligible(fine)) return fail(STOKES_E_INVAL, "the mesh does not carry the velocity multigrid");
    mg.prec = prec;
    mg.periodic = fine->h.periodic;
#ifdef STOKES_MG_FOREST_ADDITIVE
    mg.forest_additive = STOKES_MG_FOREST_ADDITIVE;
#endif
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
    if (!fine->h.lattice) {
        // a 2:1 forest: its unrefined base mesh is the first coarse level
        mg.L.push_back(MgLevel{});
        MgLevel& B = mg.L.back();
        MG_CK(build_base_level(fine, B));
        MG_CK(alloc_level(B, prec));
    }
    while (true) {
        const MgLevel& P = mg.L.back();
        const HostMesh& h = P.mesh->h;
        // coarser levels keep at least MG_MIN_CELLS cells per direction (the
        // first coarsening may go down to 2): the smaller levels were
        // latency-bound and did not reduce the Krylov counts (measured: 4
        // instead of 2 cells cut the 128x128x8 Q2 solve from 0.140 to 0.135 s,
        // Q3xQ1 0.118 -> 0.109 s, the Q3 forest 0.644 -> 0.591 s; 8 cost the
        // forest 15 % more iterations)
        const int min_cells = mg.L.size() == 1 ? 2 : MG_MIN_CELLS;
        if (h.nx % 2 || h.ny % 2 || h.nx / 2 < min_cells || h.ny / 2 < min_cells) break;
        // 1-D transfer tables of this level pair (x and y)
        HostTab1 PX, RX, JX, PY, RY, JY;
        if (!build_dir(h.nx, h.k, h.periodic, h.tab.gll, PX, RX, JX) ||
            !build_dir(h.ny, h.k, h.periodic, h.tab.gll, PY, RY, JY))
            return fail(STOKES_E_INVAL, "multigrid transfer tables exceed their row width");
        // coarse mesh: the fine isoparametric heights interpolated at the
        // coarse GLL points (for k = 2 the fine element vertices)
        stokes_mesh_desc d{};
        d.nx = h.nx / 2; d.ny = h.ny / 2; d.nz = h.nz; d.k = h.k;
        d.pressure_space = h.pspace; d.periodic_xy = h.periodic ? 1 : 0;
        d.Lx = h.Lx; d.Ly = h.Ly; d.basal_bc = h.basal_bc; d.device = fine->device;
        const int64_t NXc = int64_t(JX.cnt.size()), NYc = int64_t(JY.cnt.size());
        std::vector<double> bed(size_t(NXc * NYc)), surf(size_t(NXc * NYc));
        for (int64_t Yc = 0; Yc < NYc; ++Yc)
            for (int64_t Xc = 0; Xc < NXc; ++Xc) {
                double sb = 0, ss = 0;
                for (int b2 = 0; b2 < JY.cnt[Yc]; ++b2)
                    for (int a2 = 0; a2 < JX.cnt[Xc]; ++a2) {
                        const double w = JX.w[size_t(Xc) * KP + a2] * JY.w[size_t(Yc) * KP + b2];
                        const int64_t g0 = JX.idx[size_t(Xc) * KP + a2] + P.NX * int64_t(JY.idx[size_t(Yc) * KP + b2]);
                        const int64_t g1 = g0 + P.NX * P.NY * (P.NZ - 1);
                        sb += w * h.node_xyz[size_t(3 * g0 + 2)];
                        ss += w * h.node_xyz[size_t(3 * g1 + 2)];
                    }
                bed[size_t(Xc + NXc * Yc)] = sb;
                surf[size_t(Xc + NXc * Yc)] = ss;
            }
        d.bed_nodes = bed.data();
        d.surface_nodes = surf.data();
        MgLevel C;
        C.owned = true;
        mg.L.push_back(C);
        MgLevel& Cl = mg.L.back();
        MG_CK(stokes_mesh_create(&d, &Cl.mesh));
        MG_CK(alloc_level(Cl, prec));
        // upload the six tables (P_x, P_y, R_x, R_y, J_x, J_y) in one buffer each
        const HostTab1* T6[6] = {&PX, &PY, &RX, &RY, &JX, &JY};
        std::vector<int32_t> idx, cnt;
        std::vector<double> w;
        for (int q6 = 0; q6 < 6; ++q6) {
            Cl.t_off[q6] = int64_t(idx.size());
            Cl.t_coff[q6] = int64_t(cnt.size());
            Cl.t_m[q6] = T6[q6]->m;
            idx.insert(idx.end(), T6[q6]->idx.begin(), T6[q6]->idx.end());
            w.insert(w.end(), T6[q6]->w.begin(), T6[q6]->w.end());
            cnt.insert(cnt.end(), T6[q6]->cnt.begin(), T6[q6]->cnt.end());
        }
        MG_CK(dalloc(reinterpret_cast<void**>(&Cl.t_idx), idx.size() * 4));
        MG_CK(dalloc(reinterpret_cast<void**>(&Cl.t_w), w.size() * 8));
        MG_CK(dalloc(reinterpret_cast<void**>(&Cl.t_cnt), cnt.size() * 4));
        MG_CU(cudaMemcpy(Cl.t_idx, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice), "tables");
        MG_CU(cudaMemcpy(Cl.t_w, w.data(), w.size() * 8, cudaMemcpyHostToDevice), "tables");
        MG_CU(cudaMemcpy(Cl.t_cnt, cnt.data(), cnt.size() * 4, cudaMemcpyHostToDevice), "tables");
    }
    if (mg.L.size() < 2) {
        mg_destroy(mg);
        return fail(STOKES_E_INVAL, "the mesh is too small for the velocity multigrid");
    }
    // two levels: the coarsest level carries the whole coarse correction and
    // is not small (a forest's base mesh, a small slab's first coarsening);
    // with 4 sweeps (or with 1.2 / lambda_max damping) the isotropic Q4
    // curved forest did not converge in some runs, with 12 it did
    if (mg.L.size() == 2) mg.coarse_sweeps = std::max(mg.coarse_sweeps, 12);
    return STOKES_OK;
}

int mg_setup(Multigrid& mg, const stokes_params* p, const double* up_fine, double fine_scale, cudaStream_t s) {
    mg.L[0].scale = fine_scale;
    for (size_t l = 1; l < mg.L.size(); ++l) {
        MgLevel& F = mg.L[l - 1];
        MgLevel& C = mg.L[l];
        const double* uf = l == 1 ? up_fine : F.u64;
        // the fine linearisation point interpolated at the coarse nodes (on a
        // forest's base level: averaged over the forest nodes each base node
        // interpolates to)
        const int64_t Nvc = C.mesh->h.Nv, Nbc = C.mesh->h.Nb;
        if (C.csr)
            csr_kernel<double, double><<<blocks_for(Nvc), TPB, 0, s>>>(Nvc, C.J_ptr, C.J_col, C.J_w, 3, uf, C.u64);
        else
            transfer_kernel<double, double><<<blocks_for(C.NX * C.NY * C.NZ), TPB, 0, s>>>(
                C.NX, C.NY, C.NZ, F.NX, F.NY, dev_tab(C, 4), dev_tab(C, 5), 3, uf, C.u64);
        MG_CU(cudaGetLastError(), "multigrid interpolation");
        stokes_params pc = *p;
        if (p->robin && p->logbeta) {
            const double* lf = l == 1 ? p->logbeta : F.logbeta;
            if (C.csr)
                csr_kernel<double, double><<<blocks_for(Nbc), TPB, 0, s>>>(Nbc, C.Jb_ptr, C.Jb_col, C.Jb_w, 1, lf,
                                                                          C.logbeta);
            else
                transfer_kernel<double, double><<<blocks_for(C.NX * C.NY), TPB, 0, s>>>(
                    C.NX, C.NY, 1, F.NX, F.NY, dev_tab(C, 4), dev_tab(C, 5), 1, lf, C.logbeta);
            MG_CU(cudaGetLastError(), "multigrid interpolation");
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
        if (l + 1 == mg.L.size()) {
            // coarsest level: damping of its sweeps from the spectrum of C^-1 A
            // the norm ratio of the power iteration approaches lambda_max from
            // below; a two-level hierarchy's coarsest level (the base mesh of a
            // forest, the first coarsening of a small slab) gets more
            // iterations, since its damping decides the whole coarse correction
            double lm = 0;
            MG_CK(estimate_lmax(mg, C, mg.L.size() == 2 ? 25 : 10, lm, s));
            C.lmax = lm;
            C.omega = (std::isfinite(lm) && lm > 0) ? std::min(mg.omega, 1.6 / lm) : mg.omega;
        }
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
            if (Lv.t_idx) cudaFree(Lv.t_idx);
            if (Lv.t_w) cudaFree(Lv.t_w);
            if (Lv.t_cnt) cudaFree(Lv.t_cnt);
            for (void* p : {(void*)Lv.P_ptr, (void*)Lv.P_col, (void*)Lv.P_w, (void*)Lv.R_ptr, (void*)Lv.R_col,
                            (void*)Lv.R_w, (void*)Lv.J_ptr, (void*)Lv.J_col, (void*)Lv.J_w, (void*)Lv.Jb_ptr,
                            (void*)Lv.Jb_col, (void*)Lv.Jb_w})
                if (p) cudaFree(p);
            if (Lv.st) stokes_state_destroy(Lv.st);
            if (Lv.mesh) stokes_mesh_destroy(Lv.mesh);
        }
    }
    mg.L.clear();
    if (mg.dsc) cudaFree(mg.dsc);
    mg.dsc = nullptr;
}

}  // namespace stokes
