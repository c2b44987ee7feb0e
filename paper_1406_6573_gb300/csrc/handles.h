// Internal handle definitions and helpers shared by the C-ABI layer (capi.cu)
// and the Newton-Krylov driver (solver.cu).
#pragma once

#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "common.h"
#include "kernels.h"
#include "precond.h"

namespace stokes {

// Event pairs recorded around launches while profiling is active.
struct Profiler {
    bool active = false;
    std::vector<cudaEvent_t> pool;            // reusable events
    std::vector<std::pair<int, size_t>> recs; // (kernel class, index of the start event)
    size_t used = 0;
    cudaEvent_t next() {
        if (used == pool.size()) {
            cudaEvent_t ev;
            if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
            pool.push_back(ev);
        }
        return pool[used++];
    }
};

int fail(int code, const std::string& msg);
// cudaMalloc through the allocation-failure test hook (stokes_debug_fail_alloc_after)
cudaError_t dev_alloc(void** p, size_t bytes);
// stokes_linearize of an FP32 and an FP64 state of one mesh at one point
// (one element pass writes both where the kernels allow)
int linearize_pair(stokes_state* s32, stokes_state* s64, const stokes_params* params, const double* up_lin,
                   void* stream);
int cuda_fail(cudaError_t e, const char* where);

// Make `dev` current for the duration of a call, restoring the caller's device.
// Profiler classes (the fields of stokes_profile, in order)
enum ProfClass : int {
    PROF_CLEAR = 0, PROF_ELEMENT, PROF_FACE, PROF_CONSTRAINT,
    PROF_PRECOND, PROF_ORTHOG, PROF_VECTOR, PROF_SETUP, PROF_TRANSFER, PROF_CLASSES
};

struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev) {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) err = cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int launch_elem(int k, int mode, int prec, int state_prec, bool trans, const ElemArgs& a, cudaStream_t s);
int64_t grad_a_partials(int k, int64_t E);
int launch_face(int k, int mode, int prec, const FaceArgs& a, cudaStream_t s);
int launch_precond_assembly(int k, int prec, const ColArgs& a, cudaStream_t s);
int64_t state_stride(int k);

}  // namespace stokes

// Host copy of what a mesh was built from (geometry and refinement), so that
// related meshes (the multigrid's base and coarse levels) can be built.
struct MeshSource {
    std::vector<uint8_t> refine;                      // [ncoarse] or empty
    std::vector<double> bed[4], surf[4];              // modal fields: amp, kx, ky, phase
    double bed_mean = 0, surf_mean = 0;
    std::vector<double> bed_nodes, surf_nodes;        // gridded heights, or empty
};

struct stokes_mesh {
    mutable stokes::Profiler prof;
    stokes::HostMesh h;
    MeshSource src;
    int device = -1;
    bool on_device = false;
    int32_t* d_nodes = nullptr;
    uint32_t* d_hang = nullptr;
    double* d_geo = nullptr;
    int32_t* d_pidx = nullptr;
    double* d_pel = nullptr;
    float* d_pel_f = nullptr;      // the same projector entries in FP32 (FP32 kernels)
    int32_t* d_face_elem = nullptr;
    int32_t* d_fidx = nullptr;
    double* d_fgeo = nullptr;
    int32_t* d_fmap = nullptr;
    int32_t* d_basal_nodes = nullptr;
    double* d_basal_P = nullptr;
    int* d_err = nullptr;          // status word written by kernels (bounded waits)
    uint32_t wait_polls = stokes::WAIT_POLLS_DEFAULT;   // first-wait poll limit (test hook)
    // vertical node columns (preconditioner)
    int32_t* d_col_of = nullptr;
    int32_t* d_pos_of = nullptr;
    int32_t* d_col_nodes = nullptr;
    int32_t* d_col_len = nullptr;
    int32_t* d_col_basal = nullptr;
    // k >= 5: degree tables (device, shared per device and degree) and the
    // FP64 linearisation workspace [E][state stride] of the fused apply
    const void* htab = nullptr;
    double* d_hwork = nullptr;
};

namespace stokes {
// Run `launch` between two recorded events when profiling (class c).
template <typename F>
int timed(const stokes_mesh* m, int c, cudaStream_t s, F&& launch) {
    if (!m->prof.active) return launch();
    cudaEvent_t a = m->prof.next(), b = m->prof.next();
    if (!a || !b) return launch();
    size_t ia = m->prof.used - 2;
    cudaEventRecord(a, s);
    int rc = launch();
    cudaEventRecord(b, s);
    m->prof.recs.push_back({c, ia});
    return rc;
}
}  // namespace stokes

struct stokes_state {
    const stokes_mesh* mesh = nullptr;
    int prec = 0;
    void* d_state = nullptr;
    int cpl = 0;               // group layout, applied by the component-per-lane kernel
    void* d_fstate = nullptr;  // stored sliding state [nF][SLIDE_FIELDS][q^2] (nonlinear sliding law)
    int slide = 0;             // the last linearisation used the nonlinear sliding law
    int face_lin = 0;          // d_fstate holds the basal state of the last linearisation
                               // (Robin term on; both sliding laws)
    stokes_params params{};
    bool linearized = false;
};

namespace stokes {

int check_common(const stokes_mesh* m, int prec);
int check_params(const stokes_mesh* m, const stokes_params* p);
ElemArgs elem_args(const stokes_mesh* m, const stokes_params* p);
FaceArgs face_args(const stokes_mesh* m, const stokes_params* p);
size_t vec_bytes(const stokes_mesh* m, int prec);
// y = (element terms of x) + Robin(x) + (I - P) x ; mode selects the element term
int operator_sequence(const stokes_mesh* m, const stokes_params* p, int mode, int prec, int state_prec,
                      bool trans, const void* x, const void* u, const void* cstate, void* y, cudaStream_t s,
                      int state_cpl = 0, const void* fstate = nullptr,
                      const void* fstate_elements = nullptr);
// the nonlinear sliding law is in use (robin term, sliding_m not 0 or 1)
inline bool sliding_nonlinear(const stokes_params* p) {
    return p && p->robin && p->sliding_m != 0.0 && p->sliding_m != 1.0;
}
// velocity part of y = B^T p  for the pressure part of x (from the stored state)
int state_gradp(const stokes_state* st, const void* x, void* y, cudaStream_t s);

}  // namespace stokes
