// C-ABI entry points (include/stokes.h): argument checking, device memory of
// the mesh handle, and the launch sequence of each operator.
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include <cuda_runtime.h>

#include "handles.h"
#include "mg.h"
#include "khigh.h"

using namespace stokes;

namespace {

thread_local std::string g_err;

constexpr int MAX_DEVICES = 64;
std::mutex g_tables_mu;
bool g_tables_done[MAX_DEVICES][KMAX + 1];

int ensure_tables(int dev, int k) {
    std::lock_guard<std::mutex> lk(g_tables_mu);
    if (dev < 0 || dev >= MAX_DEVICES) return fail(STOKES_E_INVAL, "device ordinal out of range");
    if (g_tables_done[dev][k]) return STOKES_OK;
    Tables1D t[2];
    build_tables(k, STOKES_PRESSURE_P, t[0]);
    if (k >= 2) build_tables(k, STOKES_PRESSURE_Q, t[1]); else t[1] = t[0];
    int e = 0;
    switch (k) {
        case 2: e = upload_tables_k2(t); break;
        case 3: e = upload_tables_k3(t); break;
        case 4: e = upload_tables_k4(t); break;
        default:
            if (k < 5 || k > KMAX) return fail(STOKES_E_INVAL, "the GPU kernels are built for degrees k = 2 .. 9");
            g_tables_done[dev][k] = true;     // k >= 5: tables in device memory (high_tables)
            return STOKES_OK;
    }
    if (e != 0) return cuda_fail(cudaError_t(e), "uploading basis tables");
    g_tables_done[dev][k] = true;
    return STOKES_OK;
}

template <typename T>
int upload(T** dst, const std::vector<T>& src) {
    *dst = nullptr;
    if (src.empty()) return STOKES_OK;
    cudaError_t e = dev_alloc(reinterpret_cast<void**>(dst), src.size() * sizeof(T));
    if (e != cudaSuccess) { *dst = nullptr; return fail(STOKES_E_NOMEM, "cudaMalloc of mesh data failed"); }
    e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "uploading mesh data");
    return STOKES_OK;
}


void free_mesh_device(stokes_mesh* m) {
    for (cudaEvent_t ev : m->prof.pool) cudaEventDestroy(ev);
    m->prof.pool.clear();
    void* ptrs[] = {m->d_nodes, m->d_hang, m->d_geo, m->d_pidx, m->d_pel, m->d_pel_f, m->d_face_elem, m->d_fidx,
                    m->d_fgeo, m->d_fmap, m->d_basal_nodes, m->d_basal_P, m->d_err, m->d_col_of,
                    m->d_pos_of, m->d_col_nodes, m->d_col_len, m->d_col_basal, m->d_hwork};
    for (void* p : ptrs) if (p) cudaFree(p);
}

}  // namespace

namespace stokes {

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* where) {
    return fail(STOKES_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

static_assert(STOKES_WAIT_POLLS_DEFAULT == WAIT_POLLS_DEFAULT, "header and kernels agree on the poll limit");

// allocation-failure test hook: number of device allocations still allowed
// before the next one fails (-1: never fail)
std::atomic<int64_t> g_alloc_budget{-1};

cudaError_t dev_alloc(void** p, size_t bytes) {
    int64_t b = g_alloc_budget.load();
    while (b >= 0) {
        if (b == 0) { *p = nullptr; return cudaErrorMemoryAllocation; }
        if (g_alloc_budget.compare_exchange_weak(b, b - 1)) break;
    }
    return cudaMalloc(p, bytes);
}

int launch_elem(int k, int mode, int prec, int state_prec, bool trans, const ElemArgs& a, cudaStream_t s) {
    switch (k) {
        case 2: return launch_elem_k2(mode, prec, state_prec, trans, a, s);
        case 3: return launch_elem_k3(mode, prec, state_prec, trans, a, s);
        case 4: return launch_elem_k4(mode, prec, state_prec, trans, a, s);
    }
    if (k >= 5 && k <= KMAX) return launch_elem_high(mode, prec, state_prec, a, s);
    return int(cudaErrorInvalidValue);
}

int64_t state_stride(int k) {
    switch (k) {
        case 2: return state_stride_k2();
        case 3: return state_stride_k3();
        case 4: return state_stride_k4();
    }
    if (k >= 5 && k <= KMAX) return high_state_stride(k);
    return 0;
}

int64_t grad_a_partials(int k, int64_t E) {
    switch (k) {
        case 2: return grad_a_partials_k2(E);
        case 3: return grad_a_partials_k3(E);
        case 4: return grad_a_partials_k4(E);
    }
    if (k >= 5 && k <= KMAX) return high_grad_a_partials(E);
    return 0;
}

int launch_face(int k, int mode, int prec, const FaceArgs& a, cudaStream_t s) {
    switch (k) {
        case 2: return launch_face_k2(mode, prec, a, s);
        case 3: return launch_face_k3(mode, prec, a, s);
        case 4: return launch_face_k4(mode, prec, a, s);
    }
    if (k >= 5 && k <= KMAX) return launch_face_high(mode, prec, a, s);
    return int(cudaErrorInvalidValue);
}

int launch_precond_assembly(int k, int prec, const ColArgs& a, cudaStream_t s) {
    switch (k) {
        case 2: return launch_precond_assembly_k2(prec, a, s);
        case 3: return launch_precond_assembly_k3(prec, a, s);
        case 4: return launch_precond_assembly_k4(prec, a, s);
    }
    if (k >= 5 && k <= KMAX) return launch_precond_assembly_high(prec, a, s);
    return int(cudaErrorInvalidValue);
}

// Linearised states of degree 2 in FP32 are stored slot-major for the
// lane-per-component apply; all others element-major.
int check_common(const stokes_mesh* m, int prec) {
    if (!m) return fail(STOKES_E_INVAL, "mesh is NULL");
    if (!m->on_device) return fail(STOKES_E_INVAL, "mesh was built for the host only (device = -1)");
    if (prec != STOKES_F64 && prec != STOKES_F32) return fail(STOKES_E_INVAL, "prec must be STOKES_F64 or STOKES_F32");
    return STOKES_OK;
}

int check_params(const stokes_mesh* m, const stokes_params* p) {
    if (!p) return fail(STOKES_E_INVAL, "params is NULL");
    if (!(p->n >= 1.0) || !(p->A > 0) || !(p->C0 > 0) || !(p->gamma > 0) || !(p->delta > 0))
        return fail(STOKES_E_INVAL, "params: need n >= 1, A > 0, C0 > 0, gamma > 0, delta > 0");
    if (p->robin && !p->logbeta && m->h.Nb > 0) return fail(STOKES_E_INVAL, "params: robin = 1 needs logbeta");
    if (!(p->constraint_scale > 0)) return fail(STOKES_E_INVAL, "params: constraint_scale must be > 0");
    if (sliding_nonlinear(p) && !(p->sliding_m > 0 && p->sliding_eps > 0))
        return fail(STOKES_E_INVAL, "params: the sliding law needs sliding_m > 0 and sliding_eps > 0");
    return STOKES_OK;
}

ElemArgs elem_args(const stokes_mesh* m, const stokes_params* p) {
    ElemArgs a{};
    a.E = m->h.E; a.Nv = m->h.Nv; a.npr = m->h.npr; a.pspace = m->h.pspace;
    a.any_hang = m->h.n_hang > 0;
    a.nodes = m->d_nodes; a.hang = m->d_hang; a.geo = m->d_geo; a.pidx = m->d_pidx; a.pel = m->d_pel;
    a.pel_f = m->d_pel_f;
    a.err = m->d_err;
    a.wait_polls = m->wait_polls;
    a.htab = m->htab;
    a.htab_k = m->h.k;
    a.state_stride = state_stride(m->h.k);
    if (m->h.lattice) {
        a.lat_nx = m->h.nx; a.lat_ny = m->h.ny; a.lat_NX = m->h.latNX; a.lat_NY = m->h.latNY;
    }
    if (p) {
        a.C = p->C0 * std::pow(p->A, -1.0 / p->n);
        a.gamma = p->gamma; a.delta = p->delta;
        a.pexp = (1.0 - p->n) / (2.0 * p->n);
        a.n_is_3 = (p->n == 3.0);
        a.picard = p->linearization == STOKES_LIN_PICARD;
        for (int c = 0; c < 3; ++c) a.body[c] = p->body[c];
    }
    return a;
}

FaceArgs face_args(const stokes_mesh* m, const stokes_params* p) {
    FaceArgs f{};
    f.nF = m->h.nF; f.Nv = m->h.Nv;
    f.face_elem = m->d_face_elem; f.nodes = m->d_nodes; f.hang = m->d_hang;
    f.pidx = m->d_pidx; f.pel = m->d_pel; f.fgeo = m->d_fgeo; f.fmap = m->d_fmap;
    f.logbeta = p ? p->logbeta : nullptr;
    f.htab = m->htab;
    if (sliding_nonlinear(p)) {
        f.slide = 1;
        f.slide_m = p->sliding_m;
        f.slide_eps = p->sliding_eps;
        f.slide_picard = p->linearization == STOKES_LIN_PICARD;
    }
    return f;
}

size_t vec_bytes(const stokes_mesh* m, int prec) {
    return size_t(3 * m->h.Nv + m->h.Np) * (prec == STOKES_F32 ? 4 : 8);
}

int operator_sequence(const stokes_mesh* m, const stokes_params* p, int mode, int prec, int state_prec,
                      bool trans, const void* x, const void* u, const void* cstate, void* y, cudaStream_t s,
                      int state_cpl, const void* fstate, const void* fstate_elements) {
    int e = timed(m, 0, s, [&] { return int(cudaMemsetAsync(y, 0, vec_bytes(m, prec), s)); });
    if (e) return cuda_fail(cudaError_t(e), "clearing the output");
    ElemArgs a = elem_args(m, p);
    a.x = x; a.y = y; a.u = u; a.cstate = cstate;
    a.state_cpl = state_cpl;
    const bool robin = p->robin && m->h.nF > 0;
    const bool high = m->h.k >= 5;
    if (high && mode == MODE_APPLY) {
        // k >= 5: fused Jacobian = linearisation at u into the mesh's FP64
        // workspace, then the stored-state element apply; the basal face term
        // below recomputes its sliding linearisation from u
        ElemArgs al = a;
        al.u = u;
        al.state = m->d_hwork;
        al.state_cpl = 0;
        e = timed(m, 1, s, [&] { return launch_elem(m->h.k, MODE_LINEARIZE, prec, STOKES_F64, false, al, s); });
        if (e) return cuda_fail(cudaError_t(e), "linearisation kernel launch");
        a.cstate = m->d_hwork;
        e = timed(m, 1, s, [&] { return launch_elem(m->h.k, MODE_STATE_APPLY, prec, STOKES_F64, trans, a, s); });
        if (e) return cuda_fail(cudaError_t(e), "element kernel launch");
    } else if (mode == MODE_STATE_APPLY && !high) {
        // the stored-state kernel also does the basal Robin term and the
        // constraint rows (one launch per apply)
        a.face = face_args(m, p);
        a.face.x = x; a.face.y = y;
        a.face.fstate = fstate;   // the sliding law linearised with the state
        a.fuse_robin = robin;
        if (robin && fstate_elements) {
            // the component-per-lane kernel adds the face term of its basal
            // elements in the element pass, from the stored basal state
            a.face.fstate = fstate_elements;
            a.face_in_elements = 1;
            a.fuse_robin = 0;
            a.fidx = m->d_fidx;
        }
        a.fuse_constraint = 1;
        a.Nb = m->h.Nb; a.basal_nodes = m->d_basal_nodes; a.basal_P = m->d_basal_P;
        a.cscale = p->constraint_scale;
    }
    if (!(high && mode == MODE_APPLY)) {
        e = timed(m, 1, s, [&] { return launch_elem(m->h.k, mode, prec, state_prec, trans, a, s); });
        if (e) return cuda_fail(cudaError_t(e), "element kernel launch");
    }
    if (mode == MODE_STATE_GRADP) return STOKES_OK;   // zero velocity input: no Robin or (I - P) term
    if (mode == MODE_STATE_APPLY && !high) return STOKES_OK;
    if (robin) {
        FaceArgs f = face_args(m, p);
        f.x = x; f.y = y;
        f.ulin = u;               // fused Jacobian: the linearisation point; residual: NULL (u = x)
        if (mode == MODE_STATE_APPLY) f.fstate = fstate;   // k >= 5 stored state: its sliding state
        e = timed(m, 2, s, [&] { return launch_face(m->h.k, FACE_APPLY, prec, f, s); });
        if (e) return cuda_fail(cudaError_t(e), "basal face kernel launch");
    }
    e = timed(m, 3, s, [&] {
        return launch_constraint(prec, m->h.Nb, m->d_basal_nodes, m->d_basal_P, p->constraint_scale, x, y, s);
    });
    if (e) return cuda_fail(cudaError_t(e), "constraint kernel launch");
    return STOKES_OK;
}

int state_gradp(const stokes_state* st, const void* x, void* y, cudaStream_t s) {
    return operator_sequence(st->mesh, &st->params, MODE_STATE_GRADP, st->prec, st->prec, false, x, nullptr,
                             st->d_state, y, s, st->cpl);
}

}  // namespace stokes

extern "C" {

const char* stokes_last_error(void) { return g_err.c_str(); }

int stokes_mesh_create(const stokes_mesh_desc* desc, stokes_mesh** out) {
    if (!desc || !out) return fail(STOKES_E_INVAL, "desc and out must be non-NULL");
    *out = nullptr;
    stokes_mesh* m = new (std::nothrow) stokes_mesh();
    if (!m) return fail(STOKES_E_NOMEM, "host allocation failed");
    std::string err;
    int rc;
    try {
        rc = build_host_mesh(*desc, m->h, err);
    } catch (const std::bad_alloc&) {
        rc = STOKES_E_NOMEM; err = "host allocation failed while building the mesh";
    }
    if (rc != STOKES_OK) { delete m; return fail(rc, err); }
    {
        // keep the mesh's sources for related meshes (multigrid levels)
        const int64_t nc = int64_t(desc->nx) * desc->ny * desc->nz;
        if (desc->refine) m->src.refine.assign(desc->refine, desc->refine + nc);
        auto keep = [](const stokes_field& f, std::vector<double>* v, double& mean) {
            mean = f.mean;
            const double* arr[4] = {f.amp, f.kx, f.ky, f.phase};
            for (int q4 = 0; q4 < 4; ++q4) v[q4].assign(arr[q4], arr[q4] + (f.n_modes > 0 ? f.n_modes : 0));
        };
        keep(desc->bed, m->src.bed, m->src.bed_mean);
        keep(desc->surface, m->src.surf, m->src.surf_mean);
        if (desc->bed_nodes) {
            const int64_t NXg = int64_t(desc->nx) * desc->k + (desc->periodic_xy ? 0 : 1);
            const int64_t NYg = int64_t(desc->ny) * desc->k + (desc->periodic_xy ? 0 : 1);
            m->src.bed_nodes.assign(desc->bed_nodes, desc->bed_nodes + NXg * NYg);
            m->src.surf_nodes.assign(desc->surface_nodes, desc->surface_nodes + NXg * NYg);
        }
    }
    m->device = desc->device;
    if (desc->device >= 0) {
        if (m->h.k < 2 || m->h.k > KMAX) {
            delete m;
            return fail(STOKES_E_INVAL, "the GPU kernels are built for degrees k = 2 .. 9");
        }
        DeviceGuard g(desc->device);
        if (g.err != cudaSuccess) { delete m; return cuda_fail(g.err, "selecting the device"); }
        rc = ensure_tables(desc->device, m->h.k);
        if (rc == STOKES_OK) rc = upload(&m->d_nodes, m->h.elem_nodes);
        if (rc == STOKES_OK) rc = upload(&m->d_hang, m->h.elem_hang);
        if (rc == STOKES_OK) rc = upload(&m->d_geo, m->h.geo);
        if (rc == STOKES_OK) rc = upload(&m->d_pidx, m->h.elem_pidx);
        if (rc == STOKES_OK) rc = upload(&m->d_pel, m->h.pel);
        if (rc == STOKES_OK) rc = upload(&m->d_pel_f, std::vector<float>(m->h.pel.begin(), m->h.pel.end()));
        if (rc == STOKES_OK) rc = upload(&m->d_face_elem, m->h.face_elem);
        if (rc == STOKES_OK) rc = upload(&m->d_fgeo, m->h.fgeo);
        if (rc == STOKES_OK) rc = upload(&m->d_fmap, m->h.fmap);
        if (rc == STOKES_OK) rc = upload(&m->d_basal_nodes, m->h.basal_nodes);
        if (rc == STOKES_OK) rc = upload(&m->d_basal_P, m->h.basal_P);
        if (rc == STOKES_OK) rc = upload(&m->d_err, std::vector<int>(1, 0));
        if (rc == STOKES_OK) rc = upload(&m->d_fidx, m->h.elem_fidx);
        if (rc == STOKES_OK) rc = upload(&m->d_col_of, m->h.col_of);
        if (rc == STOKES_OK) rc = upload(&m->d_pos_of, m->h.pos_of);
        if (rc == STOKES_OK) rc = upload(&m->d_col_nodes, m->h.col_nodes);
        if (rc == STOKES_OK) rc = upload(&m->d_col_len, m->h.col_len);
        if (rc == STOKES_OK) {
            std::vector<int32_t> cb(size_t(m->h.ncol), -1);
            for (int64_t b = 0; b < m->h.Nb; ++b) {
                const int32_t g = m->h.basal_nodes[b];
                if (m->h.pos_of[g] == 0) cb[m->h.col_of[g]] = int32_t(b);
            }
            rc = upload(&m->d_col_basal, cb);
        }
        if (rc == STOKES_OK && m->h.k >= 5) {
            // degree tables of the block-per-element kernels, and the FP64
            // linearisation workspace of their fused Jacobian apply
            rc = high_tables(desc->device, m->h.k, &m->htab);
            if (rc == STOKES_OK &&
                dev_alloc(reinterpret_cast<void**>(&m->d_hwork), size_t(m->h.E) * size_t(high_state_stride(m->h.k)) * 8) !=
                    cudaSuccess) {
                m->d_hwork = nullptr;
                rc = fail(STOKES_E_NOMEM, "cudaMalloc of the linearisation workspace failed");
            }
        }
        if (rc != STOKES_OK) { free_mesh_device(m); delete m; return rc; }
        m->on_device = true;
        // the large per-qp arrays live on the device only
        std::vector<double>().swap(m->h.geo);
        std::vector<int32_t>().swap(m->h.elem_nodes);
    }
    *out = m;
    return STOKES_OK;
}

int stokes_profile_begin(const stokes_mesh* mesh) {
    if (!mesh || !mesh->on_device) return fail(STOKES_E_INVAL, "profiling needs a device mesh");
    mesh->prof.active = true;
    mesh->prof.recs.clear();
    mesh->prof.used = 0;
    return STOKES_OK;
}

int stokes_profile_end(const stokes_mesh* mesh, stokes_profile* out) {
    if (!mesh || !out) return fail(STOKES_E_INVAL, "mesh and out must be non-NULL");
    std::memset(out, 0, sizeof(*out));
    if (!mesh->prof.active) return fail(STOKES_E_INVAL, "profiling was not started");
    mesh->prof.active = false;
    DeviceGuard g(mesh->device);
    stokes_kernel_time* slot[PROF_CLASSES] = {&out->clear, &out->element, &out->face, &out->constraint,
                                              &out->precond, &out->orthog, &out->vector, &out->setup,
                                              &out->transfer};
    for (auto& r : mesh->prof.recs) {
        cudaEvent_t a = mesh->prof.pool[r.second], b = mesh->prof.pool[r.second + 1];
        cudaError_t ce = cudaEventSynchronize(b);
        if (ce != cudaSuccess) return cuda_fail(ce, "profiling event");
        float ms = 0.f;
        ce = cudaEventElapsedTime(&ms, a, b);
        if (ce != cudaSuccess) return cuda_fail(ce, "profiling event");
        slot[r.first]->launches += 1;
        slot[r.first]->ms += ms;
    }
    mesh->prof.recs.clear();
    mesh->prof.used = 0;
    return STOKES_OK;
}

int stokes_mesh_status(const stokes_mesh* mesh) {
    if (!mesh || !mesh->on_device) return fail(STOKES_E_INVAL, "status needs a device mesh");
    DeviceGuard g(mesh->device);
    cudaError_t ce = cudaDeviceSynchronize();
    if (ce != cudaSuccess) return cuda_fail(ce, "device synchronisation");
    int flag = 0;
    ce = cudaMemcpy(&flag, mesh->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (ce != cudaSuccess) return cuda_fail(ce, "reading the status word");
    if (flag) {
        cudaMemset(mesh->d_err, 0, sizeof(int));
        return fail(STOKES_E_CUDA, "a kernel gave up waiting for a staged copy (status word set)");
    }
    return STOKES_OK;
}

int stokes_debug_wait_limit(stokes_mesh* mesh, uint32_t polls) {
    if (!mesh || !mesh->on_device) return fail(STOKES_E_INVAL, "the wait-limit hook needs a device mesh");
    mesh->wait_polls = polls;
    return STOKES_OK;
}

int64_t stokes_debug_fail_alloc_after(int64_t n) {
    return g_alloc_budget.exchange(n < 0 ? -1 : n);
}

int stokes_debug_forest_prolongation(const stokes_mesh* forest, const stokes_mesh* base, int64_t* nnz,
                                     double* rowsum_err) {
    using namespace stokes;
    if (!forest || !base || !nnz || !rowsum_err) return fail(STOKES_E_INVAL, "null argument");
    if (forest->on_device || base->on_device) return fail(STOKES_E_INVAL, "host-only meshes expected");
    HostCsr P;
    const int rc = forest_prolongation(forest->h, forest->h.elem_nodes, forest->src.refine, base->h, P);
    if (rc != STOKES_OK) return rc;
    double worst = 0;
    for (size_t g = 0; g + 1 < P.ptr.size(); ++g) {
        double sum = 0;
        for (int32_t j = P.ptr[g]; j < P.ptr[g + 1]; ++j) sum += P.w[size_t(j)];
        worst = std::max(worst, std::fabs(sum - 1.0));
    }
    *nnz = int64_t(P.col.size());
    *rowsum_err = worst;
    return STOKES_OK;
}

int stokes_debug_mg_transfer(int nf, int k, int periodic, int which, double* out, int64_t rows, int64_t cols) {
    return stokes::mg_transfer_dense(nf, k, periodic, which, out, rows, cols);
}

int stokes_mesh_destroy(stokes_mesh* mesh) {
    if (!mesh) return STOKES_OK;
    if (mesh->on_device) {
        DeviceGuard g(mesh->device);
        free_mesh_device(mesh);
    }
    delete mesh;
    return STOKES_OK;
}

int stokes_mesh_sizes(const stokes_mesh* mesh, stokes_sizes* out) {
    if (!mesh || !out) return fail(STOKES_E_INVAL, "mesh and out must be non-NULL");
    out->E = mesh->h.E; out->Nv = mesh->h.Nv; out->Np = mesh->h.Np; out->Nb = mesh->h.Nb;
    out->k = mesh->h.k; out->npr = mesh->h.npr; out->n_hanging_elems = mesh->h.n_hang;
    return STOKES_OK;
}

int stokes_mesh_node_coords(const stokes_mesh* mesh, double* xyz) {
    if (!mesh || !xyz) return fail(STOKES_E_INVAL, "mesh and xyz must be non-NULL");
    std::memcpy(xyz, mesh->h.node_xyz.data(), mesh->h.node_xyz.size() * sizeof(double));
    return STOKES_OK;
}

int stokes_mesh_basal_nodes(const stokes_mesh* mesh, int64_t* nodes) {
    if (!mesh || !nodes) return fail(STOKES_E_INVAL, "mesh and nodes must be non-NULL");
    for (int64_t b = 0; b < mesh->h.Nb; ++b) nodes[b] = mesh->h.basal_nodes[b];
    return STOKES_OK;
}

int stokes_residual(const stokes_mesh* mesh, const stokes_params* params, const void* up, void* r,
                    int prec, void* stream) {
    int rc = check_common(mesh, prec);
    if (rc) return rc;
    if ((rc = check_params(mesh, params))) return rc;
    if (!up || !r) return fail(STOKES_E_INVAL, "up and r must be non-NULL device pointers");
    DeviceGuard g(mesh->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "selecting the device");
    return operator_sequence(mesh, params, MODE_RESIDUAL, prec, prec, false, up, nullptr, nullptr, r,
                             static_cast<cudaStream_t>(stream));
}

static int jacobian_common(const stokes_mesh* mesh, const stokes_params* params, const void* up_lin,
                           const void* x, void* y, int prec, void* stream, bool trans) {
    int rc = check_common(mesh, prec);
    if (rc) return rc;
    if ((rc = check_params(mesh, params))) return rc;
    if (!up_lin || !x || !y) return fail(STOKES_E_INVAL, "up_lin, x and y must be non-NULL device pointers");
    if (x == y) return fail(STOKES_E_INVAL, "x and y must not alias");
    DeviceGuard g(mesh->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "selecting the device");
    return operator_sequence(mesh, params, MODE_APPLY, prec, prec, trans, x, up_lin, nullptr, y,
                             static_cast<cudaStream_t>(stream));
}

int stokes_jacobian_apply(const stokes_mesh* mesh, const stokes_params* params, const void* up_lin,
                          const void* x, void* y, int prec, void* stream) {
    return jacobian_common(mesh, params, up_lin, x, y, prec, stream, false);
}

int stokes_jacobian_apply_transpose(const stokes_mesh* mesh, const stokes_params* params, const void* up_lin,
                                    const void* x, void* y, int prec, void* stream) {
    return jacobian_common(mesh, params, up_lin, x, y, prec, stream, true);
}

int stokes_param_grad(const stokes_mesh* mesh, const stokes_params* params, const double* up,
                      const double* lambda, double* g_logbeta, double* g_A, void* stream) {
    int rc = check_common(mesh, STOKES_F64);
    if (rc) return rc;
    if ((rc = check_params(mesh, params))) return rc;
    if (!up || !lambda) return fail(STOKES_E_INVAL, "up and lambda must be non-NULL device pointers");
    DeviceGuard g(mesh->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "selecting the device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (g_logbeta) {
        cudaError_t ce = cudaMemsetAsync(g_logbeta, 0, size_t(mesh->h.Nb) * sizeof(double), s);
        if (ce != cudaSuccess) return cuda_fail(ce, "clearing g_logbeta");
        if (params->robin && mesh->h.nF > 0) {
            FaceArgs f = face_args(mesh, params);
            f.u = up; f.lam = lambda; f.g = g_logbeta;
            int e = launch_face(mesh->h.k, FACE_GRAD_LOGBETA, STOKES_F64, f, s);
            if (e) return cuda_fail(cudaError_t(e), "log(beta) gradient kernel launch");
        }
    }
    if (g_A) {
        cudaError_t ce = cudaMemsetAsync(g_A, 0, sizeof(double), s);
        if (ce != cudaSuccess) return cuda_fail(ce, "clearing g_A");
        ElemArgs a = elem_args(mesh, params);
        a.ud = up; a.lam = lambda; a.gA = g_A;
        a.gA_scale = -1.0 / (params->n * params->A);
        int e = launch_elem(mesh->h.k, MODE_GRAD_A, STOKES_F64, STOKES_F64, false, a, s);
        if (e) return cuda_fail(cudaError_t(e), "A gradient kernel launch");
    }
    return STOKES_OK;
}

int stokes_state_create(const stokes_mesh* mesh, int prec, stokes_state** out) {
    int rc = check_common(mesh, prec);
    if (rc) return rc;
    if (!out) return fail(STOKES_E_INVAL, "out is NULL");
    *out = nullptr;
    stokes_state* st = new (std::nothrow) stokes_state();
    if (!st) return fail(STOKES_E_NOMEM, "host allocation failed");
    st->mesh = mesh;
    st->prec = prec;
    DeviceGuard g(mesh->device);
    if (g.err != cudaSuccess) { delete st; return cuda_fail(g.err, "selecting the device"); }
    // FP32 states of conforming k = 2 meshes use the group layout of the
    // component-per-lane apply kernel
    st->cpl = (STOKES_CPL && prec == STOKES_F32 && mesh->h.k == 2 && mesh->h.n_hang == 0) ? 1 : 0;
    const size_t values = st->cpl ? size_t((mesh->h.E + CPL_GROUP_ELEMS - 1) / CPL_GROUP_ELEMS) * CPL_GROUP_VALUES
                                  : size_t(mesh->h.E) * size_t(state_stride(mesh->h.k));
    const size_t bytes = values * (prec == STOKES_F32 ? 4 : 8);
    if (dev_alloc(&st->d_state, bytes) != cudaSuccess) {
        delete st;
        return fail(STOKES_E_NOMEM, "cudaMalloc of the linearised state failed");
    }
    // padding slots of the last group are read (never used) by the apply
    if (cudaMemset(st->d_state, 0, bytes) != cudaSuccess) {
        cudaFree(st->d_state);
        delete st;
        return fail(STOKES_E_CUDA, "clearing the linearised state failed");
    }
    if (mesh->h.nF > 0) {
        const int q = mesh->h.k + 1;
        const size_t fbytes = size_t(mesh->h.nF) * SLIDE_FIELDS * q * q * (prec == STOKES_F32 ? 4 : 8);
        if (dev_alloc(&st->d_fstate, fbytes) != cudaSuccess) {
            cudaFree(st->d_state);
            delete st;
            return fail(STOKES_E_NOMEM, "cudaMalloc of the sliding state failed");
        }
    }
    *out = st;
    return STOKES_OK;
}

int stokes_state_destroy(stokes_state* state) {
    if (!state) return STOKES_OK;
    DeviceGuard g(state->mesh->device);
    if (state->d_state) cudaFree(state->d_state);
    if (state->d_fstate) cudaFree(state->d_fstate);
    delete state;
    return STOKES_OK;
}

int stokes_linearize(stokes_state* state, const stokes_params* params, const double* up_lin, void* stream) {
    if (!state) return fail(STOKES_E_INVAL, "state is NULL");
    const stokes_mesh* mesh = state->mesh;
    int rc = check_common(mesh, state->prec);
    if (rc) return rc;
    if ((rc = check_params(mesh, params))) return rc;
    if (!up_lin) return fail(STOKES_E_INVAL, "up_lin is NULL");
    DeviceGuard g(mesh->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "selecting the device");
    ElemArgs a = elem_args(mesh, params);
    a.ud = up_lin;
    a.state = state->d_state;
    a.state_cpl = state->cpl;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int e = timed(mesh, PROF_ELEMENT, s, [&] {
        return launch_elem(mesh->h.k, MODE_LINEARIZE, STOKES_F64, state->prec, false, a, s);
    });
    if (e) return cuda_fail(cudaError_t(e), "linearize kernel launch");
    state->slide = sliding_nonlinear(params) && mesh->h.nF > 0;
    state->face_lin = params->robin && mesh->h.nF > 0;
    if (state->face_lin) {
        FaceArgs f = face_args(mesh, params);
        f.u = up_lin;
        f.fstate_out = state->d_fstate;
        f.fstate_f32 = state->prec == STOKES_F32;
        e = timed(mesh, PROF_FACE, s, [&] { return launch_face(mesh->h.k, FACE_LINEARIZE, STOKES_F64, f, s); });
        if (e) return cuda_fail(cudaError_t(e), "basal linearisation kernel launch");
    }
    state->params = *params;
    state->linearized = true;
    return STOKES_OK;
}

static int state_apply_common(const stokes_state* state, const void* x, void* y, void* stream, bool trans,
                              int mode = MODE_STATE_APPLY) {
    if (!state) return fail(STOKES_E_INVAL, "state is NULL");
    if (!state->linearized) return fail(STOKES_E_INVAL, "state has not been linearized");
    const stokes_mesh* mesh = state->mesh;
    int rc = check_common(mesh, state->prec);
    if (rc) return rc;
    if (!x || !y) return fail(STOKES_E_INVAL, "x and y must be non-NULL device pointers");
    if (x == y) return fail(STOKES_E_INVAL, "x and y must not alias");
    DeviceGuard g(mesh->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "selecting the device");
    return operator_sequence(mesh, &state->params, mode, state->prec, state->prec, trans, x,
                             nullptr, state->d_state, y, static_cast<cudaStream_t>(stream), state->cpl,
                             state->slide ? state->d_fstate : nullptr,
                             state->cpl && state->face_lin ? state->d_fstate : nullptr);
}

int stokes_state_apply(const stokes_state* state, const void* x, void* y, void* stream) {
    return state_apply_common(state, x, y, stream, false);
}

int stokes_state_apply_transpose(const stokes_state* state, const void* x, void* y, void* stream) {
    return state_apply_common(state, x, y, stream, true);
}

int stokes_state_apply_pressure_block(const stokes_state* state, const void* x, void* y, void* stream) {
    return state_apply_common(state, x, y, stream, false, MODE_STATE_GRADP);
}

}  // extern "C"

namespace stokes {
// Both states of the mixed-precision solver (FP32 inner, FP64 outer) at one
// linearisation point: one FP64 pass of the element kernel writes both
// (k <= 4), the basal states one launch each; otherwise two linearisations.
int linearize_pair(stokes_state* s32, stokes_state* s64, const stokes_params* params, const double* up_lin,
                   void* stream) {
    if (!s32 || !s64 || s32->mesh != s64->mesh || s32->prec != STOKES_F32 || s64->prec != STOKES_F64 ||
        s32->mesh->h.k > 4) {
        int rc = stokes_linearize(s32, params, up_lin, stream);
        if (rc) return rc;
        return s64 && s64 != s32 ? stokes_linearize(s64, params, up_lin, stream) : STOKES_OK;
    }
    const stokes_mesh* mesh = s32->mesh;
    int rc = check_common(mesh, STOKES_F32);
    if (rc) return rc;
    if ((rc = check_params(mesh, params))) return rc;
    if (!up_lin) return fail(STOKES_E_INVAL, "up_lin is NULL");
    DeviceGuard g(mesh->device);
    if (g.err != cudaSuccess) return cuda_fail(g.err, "selecting the device");
    ElemArgs a = elem_args(mesh, params);
    a.ud = up_lin;
    a.state = s32->d_state;
    a.state_cpl = s32->cpl;
    a.state2 = static_cast<double*>(s64->d_state);
    a.state2_cpl = s64->cpl;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int e = timed(mesh, PROF_ELEMENT, s, [&] {
        return launch_elem(mesh->h.k, MODE_LINEARIZE, STOKES_F64, STOKES_F32, false, a, s);
    });
    if (e) return cuda_fail(cudaError_t(e), "linearize kernel launch");
    for (stokes_state* st : {s32, s64}) {
        st->slide = sliding_nonlinear(params) && mesh->h.nF > 0;
        st->face_lin = params->robin && mesh->h.nF > 0;
        if (st->face_lin) {
            FaceArgs f = face_args(mesh, params);
            f.u = up_lin;
            f.fstate_out = st->d_fstate;
            f.fstate_f32 = st->prec == STOKES_F32;
            e = timed(mesh, PROF_FACE, s, [&] { return launch_face(mesh->h.k, FACE_LINEARIZE, STOKES_F64, f, s); });
            if (e) return cuda_fail(cudaError_t(e), "basal linearisation kernel launch");
        }
        st->params = *params;
        st->linearized = true;
    }
    return STOKES_OK;
}
}  // namespace stokes
