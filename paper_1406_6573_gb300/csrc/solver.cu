// Inexact Newton-Krylov driver on device vectors (Section 4).
//
//  * Newton (Section 4.1): the FP64 residual of Eq. 2.5, the Jacobian of
//    Eqs. 2.6-2.7 from the linearised state, backtracking on ||r||_2 so that
//    the residual decreases, Eisenstat-Walker forcing (choice 2) for the
//    inexact linear solves.
//  * Krylov (Section 4.2): right-preconditioned flexible GMRES(m) with the
//    block upper-triangular preconditioner of Eq. 4.1, F~ = vertical-column
//    blocks of F, S~ = -M(1/mu) (Section 6).  Classical Gram-Schmidt with
//    FP64 accumulation, one reorthogonalisation pass when the first removes
//    more than (1 - STOKES_REORTH_THETA) of ||w||^2.
//  * Mixed precision: with inner precision FP32 the Krylov vectors, the
//    operator applies and the preconditioner run in FP32; every restart
//    recomputes the linear residual in FP64 with the FP64 state (iterative
//    refinement), so the FP64 Newton update can be resolved below FP32
//    round-off.  With inner precision FP64 the same loop is plain FP64.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "handles.h"
#include "mg.h"
#include "vec.h"

using namespace stokes;

struct stokes_solver {
    const stokes_mesh* mesh = nullptr;
    stokes_solver_opts o{};
    int inner = STOKES_F32;
    stokes_state* st_in = nullptr;
    stokes_state* st64 = nullptr;
    int64_t n = 0, nu = 0;
    int64_t ld = 0;                    // column stride of the Krylov bases V, Z (n rounded up to 64)
    size_t isz = 4;
    double *r = nullptr, *dl = nullptr, *rl = nullptr, *trial = nullptr, *rt = nullptr, *tmp64 = nullptr;
    void *V = nullptr, *Z = nullptr, *tin = nullptr, *tz = nullptr;
    void *A = nullptr, *md = nullptr;        // md: inverse element blocks of M(1/mu) (inner precision)
    double* mblk = nullptr;                  // element blocks of M(1/mu) before inversion (FP64)
    double* dsc = nullptr;             // device scalars
    size_t band_elems = 0;
    int bw = 0;
    Multigrid mg;                      // velocity-block multigrid (velocity_mg on an eligible mesh)
    bool use_mg = false;
};

namespace {

template <typename T>
void dfree(T*& p) {
    if (p) cudaFree(reinterpret_cast<void*>(p));
    p = nullptr;
}

void free_solver(stokes_solver* s) {
    mg_destroy(s->mg);
    dfree(s->r); dfree(s->dl); dfree(s->rl); dfree(s->trial); dfree(s->rt); dfree(s->tmp64);
    dfree(s->V); dfree(s->Z); dfree(s->tin); dfree(s->tz); dfree(s->A); dfree(s->md); dfree(s->mblk); dfree(s->dsc);
    if (s->st_in) stokes_state_destroy(s->st_in);
    if (s->st64 && s->st64 != s->st_in) stokes_state_destroy(s->st64);
    s->st_in = s->st64 = nullptr;
}

#define CK(call)                                                    \
    do {                                                            \
        int rc_ = (call);                                           \
        if (rc_) return rc_;                                        \
    } while (0)
#define CU(call, what)                                              \
    do {                                                            \
        int e_ = int(call);                                         \
        if (e_) return cuda_fail(cudaError_t(e_), what);            \
    } while (0)
// CU with the work recorded under a profiler class when tracing is on
#define TU(cls, call, what) CU(timed(S->mesh, cls, st, [&] { return int(call); }), what)

// ||x||_2 of an FP64 device vector (synchronises)
int norm64(stokes_solver* S, const double* x, int64_t n, double& out, cudaStream_t st) {
    TU(PROF_VECTOR, vec_multidot(n, STOKES_F64, x, 0, 0, STOKES_F64, x, S->dsc, 1, st), "norm");
    double h = 0;
    TU(PROF_TRANSFER, cudaMemcpyAsync(&h, S->dsc, sizeof(double), cudaMemcpyDeviceToHost, st), "norm readback");
    CU(cudaStreamSynchronize(st), "norm sync");
    out = std::sqrt(h);
    return STOKES_OK;
}

// The mesh's device status word, set by a kernel whose bounded wait for a
// staged copy expired (its contribution to the output is then missing).
// Read after every restart cycle and every Newton step; if set it is cleared
// and the solve returns STOKES_E_CUDA rather than a result built on a wrong
// operator product.
int device_status(stokes_solver* S, cudaStream_t st) {
    int flag = 0;
    TU(PROF_TRANSFER, cudaMemcpyAsync(&flag, S->mesh->d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "status readback");
    CU(cudaStreamSynchronize(st), "status sync");
    if (flag) {
        CU(cudaMemsetAsync(S->mesh->d_err, 0, sizeof(int), st), "clearing the status word");
        CU(cudaStreamSynchronize(st), "status sync");
        return fail(STOKES_E_CUDA, "a kernel gave up waiting for a staged copy during the solve (status word set)");
    }
    return STOKES_OK;
}

int op_inner(stokes_solver* S, const void* x, void* y, bool trans, cudaStream_t st) {
    return trans ? stokes_state_apply_transpose(S->st_in, x, y, st) : stokes_state_apply(S->st_in, x, y, st);
}

int op64(stokes_solver* S, const double* x, double* y, bool trans, cudaStream_t st) {
    return trans ? stokes_state_apply_transpose(S->st64, x, y, st) : stokes_state_apply(S->st64, x, y, st);
}

// exact element blocks of the Schur approximation for small pressure spaces
int schur_full(const stokes_mesh* m) { return m->h.npr <= 4 ? 1 : 0; }

ColSolveArgs colsolve_args(stokes_solver* S, double scale) {
    const stokes_mesh* m = S->mesh;
    ColSolveArgs c{};
    c.ncol = m->h.ncol; c.Nv = m->h.Nv; c.colmax = m->h.colmax; c.bw = S->bw;
    c.col_nodes = m->d_col_nodes; c.col_len = m->d_col_len; c.col_basal = m->d_col_basal;
    c.basal_P = m->d_basal_P; c.scale = scale; c.A = S->A; c.err = m->d_err;
    return c;
}

// preconditioner set-up from the inner state: column blocks of F, their
// factorisation, and the Schur diagonal.  With scale_out, the mean
// |diagonal| of the velocity block is returned before factorisation.
int precond_setup(stokes_solver* S, const stokes_params* p, const double* up, cudaStream_t st,
                  double* scale_out = nullptr) {
    const stokes_mesh* m = S->mesh;
    TU(PROF_SETUP, cudaMemsetAsync(S->A, 0, S->band_elems * S->isz, st), "clearing column blocks");
    ColArgs a{};
    a.E = m->h.E; a.ncol = m->h.ncol; a.npr = m->h.npr; a.pspace = m->h.pspace; a.bw = S->bw;
    a.rows = 3 * m->h.colmax;
    a.fstate = S->st_in->slide ? S->st_in->d_fstate : nullptr;
    a.robin = p->robin && m->h.nF > 0;
    a.nodes = m->d_nodes; a.hang = m->d_hang; a.col_of = m->d_col_of; a.pos_of = m->d_pos_of;
    a.fidx = m->d_fidx; a.fmap = m->d_fmap; a.fgeo = m->d_fgeo; a.logbeta = p->logbeta;
    a.state = S->st_in->d_state; a.state_cpl = S->st_in->cpl; a.A = S->A; a.mblk = S->mblk; a.schur_full = schur_full(m);
    a.htab = m->htab; a.htab_k = m->h.k; a.state_stride = state_stride(m->h.k);
    TU(PROF_SETUP, launch_precond_assembly(m->h.k, S->inner, a, st), "preconditioner assembly");
    TU(PROF_SETUP, launch_schur_invert(S->inner, m->h.E, m->h.npr, schur_full(m), S->mblk, S->md, st), "Schur inversion");
    double scale = p->constraint_scale;
    if (scale_out) {
        TU(PROF_SETUP, launch_col_diag_sum(S->inner, colsolve_args(S, scale), S->dsc, st), "diagonal scale");
        double sum = 0;
        TU(PROF_TRANSFER, cudaMemcpyAsync(&sum, S->dsc, sizeof(double), cudaMemcpyDeviceToHost, st), "readback");
        CU(cudaStreamSynchronize(st), "sync");
        scale = sum / double(3 * m->h.Nv);
        if (!(scale > 0)) scale = 1.0;
        *scale_out = scale;
    }
    TU(PROF_SETUP, launch_col_factor(S->inner, colsolve_args(S, scale), st), "column factorisation");
    if (S->use_mg) CK(timed(S->mesh, PROF_SETUP, st, [&] { return mg_setup(S->mg, p, up, scale, st); }));
    return STOKES_OK;
}

// z = M^{-1} v  (inner precision):  z_p = -M(1/mu)^{-1} v_p (element blocks),
// z_u = F~^{-1}(v_u - B^T z_p)
int precond_apply(stokes_solver* S, const void* v, void* z, cudaStream_t st) {
    const stokes_mesh* m = S->mesh;
    TU(PROF_PRECOND, launch_schur_apply(S->inner, m->h.Nv, m->h.E, m->h.npr, schur_full(m), S->md, v, z, st), "Schur apply");
    CK(state_gradp(S->st_in, z, S->tz, st));
    TU(PROF_PRECOND, vec_axpby(S->nu, 1.0, nullptr, S->inner, v, -1.0, S->inner, S->tz, st), "preconditioner update");
    if (S->use_mg)
        CK(timed(S->mesh, PROF_PRECOND, st, [&] { return mg_apply(S->mg, S->tz, z, st); }));
    else
        TU(PROF_PRECOND, launch_col_solve(S->inner, colsolve_args(S, 1.0), S->tz, z, st), "column solve");
    return STOKES_OK;
}

// One FGMRES(m) cycle on A x = b with b = tin (inner precision), x0 = 0.
// Adds Z y to the FP64 vector dl.  Returns the number of iterations in its.
// Second Gram-Schmidt pass when the first removes more than (1 - theta) of
// ||w||^2; above that the Pythagorean norm is accurate to about eps / theta.
#ifndef STOKES_REORTH_THETA
#define STOKES_REORTH_THETA 0.1
#endif

int fgmres_cycle(stokes_solver* S, bool trans, double tol_rel, int max_its, int& its, cudaStream_t st) {
    const int64_t n = S->n;
    const int m = std::min(S->o.restart, max_its);
    const int ip = S->inner;
    const size_t isz = S->isz;
    auto Vj = [&](int j) { return static_cast<char*>(S->V) + size_t(j) * S->ld * isz; };
    auto Zj = [&](int j) { return static_cast<char*>(S->Z) + size_t(j) * S->ld * isz; };
    std::vector<double> H(size_t(m + 1) * m, 0.0), cs(m, 0.0), sn(m, 0.0), g(m + 1, 0.0), h(m + 2, 0.0);
    // V_0 = b / ||b||
    TU(PROF_VECTOR, vec_axpby(n, 1.0, nullptr, ip, S->tin, 0.0, ip, Vj(0), st), "copy");
    TU(PROF_ORTHOG, vec_multidot(n, ip, Vj(0), 0, 0, ip, Vj(0), S->dsc, 1, st), "dot");
    TU(PROF_TRANSFER, cudaMemcpyAsync(h.data(), S->dsc, sizeof(double), cudaMemcpyDeviceToHost, st), "readback");
    CU(cudaStreamSynchronize(st), "sync");
    const double beta = std::sqrt(h[0]);
    its = 0;
    if (!(beta > 0)) return STOKES_OK;
    TU(PROF_ORTHOG, vec_normalize(n, ip, Vj(0), S->dsc, st), "normalize");
    g[0] = beta;
    int k = 0;
    for (; k < m; ++k) {
        CK(precond_apply(S, Vj(k), Zj(k), st));
        CK(op_inner(S, Zj(k), Vj(k + 1), trans, st));
        // Classical Gram-Schmidt with FP64-accurate sums.  Pass 1 gives
        // h = V^T w and ||w||^2 together; when the projection leaves more
        // than theta of ||w||^2 the new norm follows from Pythagoras,
        // ||w - V h||^2 = ||w||^2 - ||h||^2, and pass 2 subtracts and
        // normalises at once.  Otherwise (cancellation) w' = w - V h is
        // formed, V^T w' and ||w'||^2 are taken in one pass, and a last pass
        // subtracts the correction and normalises.
        TU(PROF_ORTHOG, vec_multidot(n, ip, S->V, S->ld, k + 1, ip, Vj(k + 1), S->dsc, 1, st), "orthogonalisation dots");
        TU(PROF_TRANSFER, cudaMemcpyAsync(h.data(), S->dsc, sizeof(double) * (k + 2), cudaMemcpyDeviceToHost, st), "readback");
        CU(cudaStreamSynchronize(st), "sync");
        const double w2 = h[k + 1];
        if (!std::isfinite(w2)) return fail(STOKES_E_NONFINITE, "non-finite Krylov vector");
        double hh = 0;
        for (int i = 0; i <= k; ++i) { H[size_t(i) * m + k] = h[i]; hh += h[i] * h[i]; }
        double hn2 = w2 - hh;
        const double* hdev = S->dsc;
        if (hn2 < STOKES_REORTH_THETA * w2) {
            TU(PROF_ORTHOG, vec_multiaxpy(n, ip, Vj(k + 1), S->V, S->ld, k + 1, S->dsc, 1.0, S->dsc + (m + 1), st),
               "orthogonalisation");
            TU(PROF_TRANSFER, cudaMemcpyAsync(h.data(), S->dsc + (m + 1), sizeof(double) * (k + 2), cudaMemcpyDeviceToHost, st),
               "readback");
            CU(cudaStreamSynchronize(st), "sync");
            hh = 0;
            for (int i = 0; i <= k; ++i) { H[size_t(i) * m + k] += h[i]; hh += h[i] * h[i]; }
            hn2 = std::max(h[k + 1] - hh, 0.0);
            hdev = S->dsc + (m + 1);
        }
        // breakdown (the new direction lies in the Krylov space up to
        // rounding): no new basis vector; the cycle ends after this column
        double hk1 = std::sqrt(std::max(hn2, 0.0));
        if (!(hk1 > 1e-14 * std::sqrt(w2))) hk1 = 0.0;
        if (hk1 > 0)
            TU(PROF_ORTHOG, vec_multiaxpy(n, ip, Vj(k + 1), S->V, S->ld, k + 1, hdev, 1.0 / hk1, nullptr, st),
               "orthogonalisation");
        // Givens rotations on column k
        for (int i = 0; i < k; ++i) {
            const double a = H[size_t(i) * m + k], b = H[size_t(i + 1) * m + k];
            H[size_t(i) * m + k] = cs[i] * a + sn[i] * b;
            H[size_t(i + 1) * m + k] = -sn[i] * a + cs[i] * b;
        }
        const double a = H[size_t(k) * m + k];
        const double rr = std::hypot(a, hk1);
        if (!(rr > 0)) break;          // A z_k = 0 here: column k adds nothing (and would not be invertible)
        cs[k] = rr > 0 ? a / rr : 1.0;
        sn[k] = rr > 0 ? hk1 / rr : 0.0;
        H[size_t(k) * m + k] = rr;
        g[k + 1] = -sn[k] * g[k];
        g[k] = cs[k] * g[k];
        ++its;
        if (std::fabs(g[k + 1]) <= tol_rel * beta || hk1 == 0) { ++k; break; }
    }
    // y = H^{-1} g (upper triangular k x k), dl += Z y
    std::vector<double> y(k, 0.0);
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int j = i + 1; j < k; ++j) s -= H[size_t(i) * m + j] * y[j];
        y[i] = s / H[size_t(i) * m + i];
    }
    TU(PROF_TRANSFER, cudaMemcpyAsync(S->dsc, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st), "coefficients");
    TU(PROF_VECTOR, vec_combine(n, ip, S->Z, S->ld, k, S->dsc, STOKES_F64, S->dl, st), "update");
    CU(cudaStreamSynchronize(st), "sync");
    return STOKES_OK;
}

// Solve J dl = rhs (FP64 device rhs) to ||rhs - J dl|| <= eta ||rhs||; dl and rl
// (final linear residual) are FP64.  Operators/preconditioner from the
// current states.
int linear_solve(stokes_solver* S, const double* rhs, double nrhs, double eta, bool trans, int& its_total,
                 cudaStream_t st) {
    const int64_t n = S->n;
    TU(PROF_VECTOR, cudaMemsetAsync(S->dl, 0, sizeof(double) * n, st), "clear");
    TU(PROF_VECTOR, vec_axpby(n, 1.0, nullptr, STOKES_F64, rhs, 0.0, STOKES_F64, S->rl, st), "copy");
    double nrl = nrhs;
    its_total = 0;
    const double floor_rel = S->inner == STOKES_F32 ? 1e-5 : 1e-13;
    while (its_total < S->o.max_krylov && nrl > eta * nrhs) {
        TU(PROF_VECTOR, vec_axpby(n, 1.0, nullptr, STOKES_F64, S->rl, 0.0, S->inner, S->tin, st), "to inner precision");
        const double tol = std::max(eta * nrhs / nrl, floor_rel);
        int its = 0;
        CK(fgmres_cycle(S, trans, tol, S->o.max_krylov - its_total, its, st));
        its_total += its;
        // FP64 residual of the accumulated update (iterative refinement)
        CK(op64(S, S->dl, S->tmp64, trans, st));
        TU(PROF_VECTOR, vec_axpby(n, 1.0, nullptr, STOKES_F64, rhs, 0.0, STOKES_F64, S->rl, st), "residual");
        TU(PROF_VECTOR, vec_axpby(n, -1.0, nullptr, STOKES_F64, S->tmp64, 1.0, STOKES_F64, S->rl, st), "residual");
        CK(norm64(S, S->rl, n, nrl, st));
        CK(device_status(S, st));
        if (its == 0) break;
    }
    return STOKES_OK;
}

}  // namespace

extern "C" {

int stokes_solver_create(const stokes_mesh* mesh, const stokes_solver_opts* opts, stokes_solver** out) {
    int rc = check_common(mesh, STOKES_F64);
    if (rc) return rc;
    if (!out) return fail(STOKES_E_INVAL, "out is NULL");
    *out = nullptr;
    stokes_solver* S = new (std::nothrow) stokes_solver();
    if (!S) return fail(STOKES_E_NOMEM, "host allocation failed");
    S->mesh = mesh;
    stokes_solver_opts o{STOKES_F32, 30, 1000, 50, 1e-10, 0.1, 1};
    if (opts) o = *opts;
    if (o.restart < 1) o.restart = 30;
    if (o.restart > 31) o.restart = 31;   // multi-dot / multi-axpy handle at most 32 vectors
    if (o.max_krylov < 1) o.max_krylov = 1000;
    if (o.max_newton < 1) o.max_newton = 50;
    if (!(o.rtol > 0)) o.rtol = 1e-10;
    if (!(o.eta_max > 0)) o.eta_max = 0.1;
    if (o.inner_prec != STOKES_F32 && o.inner_prec != STOKES_F64) { delete S; return fail(STOKES_E_INVAL, "inner_prec"); }
    S->o = o;
    S->inner = o.inner_prec;
    S->isz = S->inner == STOKES_F32 ? 4 : 8;
    S->n = 3 * mesh->h.Nv + mesh->h.Np;
    S->ld = (S->n + 63) / 64 * 64;
    S->nu = 3 * mesh->h.Nv;
    S->bw = 3 * mesh->h.bnode + 2;
    DeviceGuard g(mesh->device);
    if (g.err != cudaSuccess) { delete S; return cuda_fail(g.err, "selecting the device"); }
    rc = stokes_state_create(mesh, S->inner, &S->st_in);
    if (rc == STOKES_OK) {
        if (S->inner == STOKES_F64) S->st64 = S->st_in;
        else rc = stokes_state_create(mesh, STOKES_F64, &S->st64);
    }
    const size_t n = size_t(S->n);
    S->band_elems = size_t(3) * mesh->h.colmax * size_t(2 * S->bw + 1) * size_t(band_cols(mesh->h.ncol));
    auto alloc = [&](void** p, size_t bytes) {
        if (rc) return;
        if (dev_alloc(p, bytes) != cudaSuccess) { *p = nullptr; rc = fail(STOKES_E_NOMEM, "solver workspace"); }
    };
    alloc(reinterpret_cast<void**>(&S->r), n * 8);
    alloc(reinterpret_cast<void**>(&S->dl), n * 8);
    alloc(reinterpret_cast<void**>(&S->rl), n * 8);
    alloc(reinterpret_cast<void**>(&S->trial), n * 8);
    alloc(reinterpret_cast<void**>(&S->rt), n * 8);
    alloc(reinterpret_cast<void**>(&S->tmp64), n * 8);
    alloc(&S->V, size_t(S->ld) * S->isz * size_t(o.restart + 1));
    alloc(&S->Z, size_t(S->ld) * S->isz * size_t(o.restart));
    alloc(&S->tin, n * S->isz);
    alloc(&S->tz, n * S->isz);
    alloc(&S->A, S->band_elems * S->isz);
    alloc(&S->md, std::max<size_t>(1, size_t(mesh->h.Np) * size_t(mesh->h.npr)) * S->isz);
    alloc(reinterpret_cast<void**>(&S->mblk), std::max<size_t>(1, size_t(mesh->h.Np) * size_t(mesh->h.npr)) * 8);
    alloc(reinterpret_cast<void**>(&S->dsc), sizeof(double) * size_t(2 * o.restart + 8));
    if (!rc && o.velocity_mg && mg_eligible(mesh)) {
        rc = mg_create(S->mg, mesh, S->st_in, S->A, S->bw, S->inner);
        S->use_mg = rc == STOKES_OK;
    }
    if (rc) { free_solver(S); delete S; return rc; }
    *out = S;
    return STOKES_OK;
}

int stokes_solver_destroy(stokes_solver* solver) {
    if (!solver) return STOKES_OK;
    DeviceGuard g(solver->mesh->device);
    free_solver(solver);
    delete solver;
    return STOKES_OK;
}

int stokes_newton_solve(stokes_solver* S, const stokes_params* params, double* up, stokes_solve_report* rep,
                        void* stream) {
    if (!S) return fail(STOKES_E_INVAL, "solver is NULL");
    const stokes_mesh* mesh = S->mesh;
    int rc = check_params(mesh, params);
    if (rc) return rc;
    if (!up) return fail(STOKES_E_INVAL, "up is NULL");
    DeviceGuard g(mesh->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "selecting the device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = S->n;
    stokes_solve_report R{};
    auto t0 = std::chrono::steady_clock::now();
    // The constraint rows s (I - P) are scaled to the mean diagonal of the
    // velocity block at the first linearisation, so that FP32 arithmetic
    // resolves them next to rows of very different magnitude (SI units);
    // the solution does not depend on s.
    stokes_params P = *params;
    CK(stokes_linearize(S->st_in, &P, up, st));
    CK(precond_setup(S, &P, up, st, &P.constraint_scale));
    R.constraint_scale = P.constraint_scale;
    params = &P;
    CK(stokes_residual(mesh, params, up, S->r, STOKES_F64, st));
    double nr = 0;
    CK(norm64(S, S->r, n, nr, st));
    const double nr0 = nr;
    R.res0 = nr0;
    if (!std::isfinite(nr0)) {
        if (rep) *rep = R;
        return fail(STOKES_E_NONFINITE, "the residual at the initial guess is not finite");
    }
    R.history[0] = nr0;
    double eta = S->o.eta_max, nr_prev = nr;
    int k = 0;
    for (; k < S->o.max_newton; ++k) {
        if (nr <= S->o.rtol * nr0) { R.converged = 1; break; }
        if (k > 0) {   // Eisenstat-Walker choice 2 with safeguards
            const double ratio = nr / nr_prev;
            double e2 = 0.9 * ratio * ratio;
            const double safe = 0.9 * eta * eta;
            if (safe > 0.1) e2 = std::max(e2, safe);
            eta = std::min(e2, S->o.eta_max);
            eta = std::max(eta, 0.5 * S->o.rtol * nr0 / nr);
        }
        if (S->st64 != S->st_in) CK(linearize_pair(S->st_in, S->st64, params, up, st));
        else CK(stokes_linearize(S->st_in, params, up, st));
        CK(precond_setup(S, params, up, st));
        // rhs = -r
        TU(PROF_VECTOR, vec_axpby(n, -1.0, nullptr, STOKES_F64, S->r, 0.0, STOKES_F64, S->trial, st), "rhs");
        int its = 0;
        CK(linear_solve(S, S->trial, nr, eta, false, its, st));
        R.krylov_its += its;
        if (k < 64) R.krylov_per_newton[k] = its;
        // backtracking line search on ||r||
        double alpha = 1.0, nrt = 0;
        for (int cut = 0;; ++cut) {
            TU(PROF_VECTOR, vec_axpby(n, 1.0, nullptr, STOKES_F64, up, 0.0, STOKES_F64, S->trial, st), "trial");
            TU(PROF_VECTOR, vec_axpby(n, alpha, nullptr, STOKES_F64, S->dl, 1.0, STOKES_F64, S->trial, st), "trial");
            CK(stokes_residual(mesh, params, S->trial, S->rt, STOKES_F64, st));
            CK(norm64(S, S->rt, n, nrt, st));
            if (nrt <= (1.0 - 1e-4 * alpha) * nr || cut >= 12) break;
            alpha *= 0.5;
            R.line_search_cuts++;
        }
        CK(device_status(S, st));
        if (!std::isfinite(nrt)) {
            R.newton_its = k + 1;
            R.res_final = nrt;
            if (rep) *rep = R;
            return fail(STOKES_E_NONFINITE, "non-finite residual after the Newton update (up left at the last iterate)");
        }
        if (!(nrt < nr)) {
            // twelve halvings without any decrease: the step is rejected, up
            // keeps the last iterate and the solve stops (E_NOCONV)
            R.line_search_failed = 1;
            break;
        }
        TU(PROF_VECTOR, cudaMemcpyAsync(up, S->trial, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "update");
        TU(PROF_VECTOR, cudaMemcpyAsync(S->r, S->rt, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "update");
        nr_prev = nr;
        nr = nrt;
        if (k + 1 < 64) R.history[k + 1] = nr;
    }
    if (nr <= S->o.rtol * nr0) R.converged = 1;
    CU(cudaStreamSynchronize(st), "sync");
    R.newton_its = k;
    R.res_final = nr;
    R.mg_levels = S->use_mg ? int(S->mg.L.size()) : 0;
    R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = R;
    return R.converged ? STOKES_OK : fail(STOKES_E_NOCONV, "Newton did not reach rtol");
}

int stokes_linear_solve(stokes_solver* S, const stokes_params* params, const double* up_lin, const double* b,
                        double* x, int transpose, double rtol, stokes_solve_report* rep, void* stream) {
    if (!S) return fail(STOKES_E_INVAL, "solver is NULL");
    const stokes_mesh* mesh = S->mesh;
    int rc = check_params(mesh, params);
    if (rc) return rc;
    if (!up_lin || !b || !x) return fail(STOKES_E_INVAL, "up_lin, b and x must be non-NULL");
    DeviceGuard g(mesh->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "selecting the device");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = S->n;
    stokes_solve_report R{};
    auto t0 = std::chrono::steady_clock::now();
    if (S->st64 != S->st_in) CK(linearize_pair(S->st_in, S->st64, params, up_lin, st));
    else CK(stokes_linearize(S->st_in, params, up_lin, st));
    CK(precond_setup(S, params, up_lin, st));
    double nb = 0;
    CK(norm64(S, b, n, nb, st));
    if (!std::isfinite(nb)) return fail(STOKES_E_NONFINITE, "the right-hand side is not finite");
    int its = 0;
    CK(linear_solve(S, b, nb, rtol, transpose != 0, its, st));
    TU(PROF_VECTOR, cudaMemcpyAsync(x, S->dl, sizeof(double) * n, cudaMemcpyDeviceToDevice, st), "solution");
    double nrl = 0;
    CK(norm64(S, S->rl, n, nrl, st));
    R.krylov_its = its;
    R.res0 = nb;
    R.mg_levels = S->use_mg ? int(S->mg.L.size()) : 0;
    R.res_final = nrl;
    R.converged = nrl <= rtol * nb;
    if (!std::isfinite(nrl)) {
        if (rep) *rep = R;
        return fail(STOKES_E_NONFINITE, "non-finite linear residual");
    }
    R.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (rep) *rep = R;
    return R.converged ? STOKES_OK : fail(STOKES_E_NOCONV, "Krylov solve did not reach rtol");
}

}  // extern "C"
