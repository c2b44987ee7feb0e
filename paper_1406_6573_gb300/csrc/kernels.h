// Kernel argument blocks and launcher declarations (host + device).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace stokes {

// polls of an mbarrier before a kernel gives up waiting for a staged copy
// (each poll may suspend the thread for a hardware-chosen interval)
constexpr uint32_t WAIT_POLLS_DEFAULT = 1u << 22;

// Blocks of a persistent kernel whose warps walk `groups` work items with a
// grid stride: one warp per item up to the resident blocks `max_blocks`.
// (Fewer blocks with the same number of rounds, so that every warp takes
// part in the last one, measured slower: 0.0692 against 0.0654 ms for the
// Q2 apply on the 128x128x8 slab, no gain at k = 3, 4.)
inline int64_t persistent_blocks(int64_t groups, int warps_per_block, int64_t max_blocks) {
    const int64_t blocks = (groups + warps_per_block - 1) / warps_per_block;
    return blocks < max_blocks ? blocks : max_blocks;
}

enum ElemMode : int {
    MODE_RESIDUAL = 0,     // r  = R^T(int sigma(u, p) : grad v - b . v) , -(q, div u)
    MODE_APPLY = 1,        // y  = J(u) x, linearisation recomputed per quadrature point
    MODE_LINEARIZE = 2,    // state <- per-qp Newton coefficients at u (FP64 arithmetic)
    MODE_STATE_APPLY = 3,  // y  = J x from the stored state
    MODE_GRAD_A = 4,       // g_A = -(1/(n A)) int mu D(lambda) : D(u)
    MODE_STATE_GRADP = 5,  // velocity rows of B^T p for the pressure part of x (stored state)
    MODE_GRAD_A_PARTIAL = 6,  // per-warp partial sums of the A-gradient integral (fixed-order variant)
};

// Linearised state, per element: two element constants (Jinv[0][0] = 1/a,
// Jinv[1][1] = 1/b: x and y are affine in xi and eta on the extruded slab
// meshes, so the first two rows of Jinv are diagonal and constant), then
// STATE_FIELDS values per quadrature point: Jinv[2][0..2], w detJ, mu w detJ,
// Dhat (6: 00 11 22 01 02 12).
constexpr int STATE_FIELDS = 11;

// FP32 states of conforming k = 2 meshes are stored in groups of 10 elements
// (3000 values per group, 12000 bytes) and applied by the component-per-lane
// kernel; STOKES_CPL = 0 keeps them in the element-major layout of the
// warp-per-element-group kernel.
#ifndef STOKES_CPL
#define STOKES_CPL 1
#endif
constexpr int CPL_GROUP_ELEMS = 10;
constexpr int CPL_GROUP_VALUES = 3000;

struct FaceArgs {
    int64_t nF, Nv;
    const int32_t* face_elem;  // [nF]
    const int32_t* nodes;
    const uint32_t* hang;
    const int32_t* pidx;
    const double* pel;
    const double* fgeo;        // [nF][4][q^2]
    const int32_t* fmap;       // [nF][n1^2]
    const double* logbeta;     // [Nb]
    const void* x;             // vector whose basal trace enters beta T x
    void* y;                   // output (accumulated)
    const double* u;           // gradient, linearisation: state (FP64)
    const double* lam;         // gradient: adjoint
    double* g;                 // gradient output [Nb] (accumulated)
    // nonlinear sliding law (slide = 1): traction beta s(|T u|^2) T u,
    // s(x) = (x + slide_eps)^((slide_m - 1)/2)
    int slide, slide_picard;
    double slide_m, slide_eps;
    const void* ulin;          // apply: linearisation point u (type of x); NULL: the residual (u = x)
    const void* fstate;        // apply: stored sliding state [nF][7][q^2] (type of x), used when set
    void* fstate_out;          // linearisation output (fstate_f32: float, else double)
    int fstate_f32;
    const void* htab;          // degree tables of the k >= 5 kernels (device)
};
// stored basal state per basal Gauss point: beta w s, then
// v = 2 beta w s' T u (3) and T u (3): the Jacobian's face term on w is
// beta w s T w + (v . w) T u; then the unit normal n (3) of the face at the
// point (read by the component-per-lane apply, which adds the face term of
// its basal elements in the element pass).  Linear law: s = 1, v = 0.
constexpr int SLIDE_FIELDS = 10;

struct ElemArgs {
    int64_t E, Nv;
    int npr, pspace, any_hang;
    const int32_t* nodes;      // [E][n1^3]
    const uint32_t* hang;      // [E]
    const double* geo;         // [E][10][q^3]
    const int32_t* pidx;       // [E]
    const double* pel;         // [nP][6][n1^2]
    const float* pel_f;        // the same in FP32
    const void* x;             // input state vector (residual: up; apply: direction)
    void* y;                   // output state vector (accumulated; zeroed by the caller)
    const void* u;             // linearisation point (fused apply), same type as x
    const double* ud;          // FP64 state (linearize, gradient)
    const double* lam;         // FP64 adjoint (gradient)
    void* state;               // [E][state stride] (linearize output)
    const void* cstate;        // same (state apply input)
    int state_cpl;             // state in the group layout (k = 2, FP32, conforming mesh)
    double* state2;            // linearize, k <= 4: a second (FP64) state written by the same
    int state2_cpl;            // pass (NULL: none), and its layout flag
    double C, gamma, delta, pexp;
    int n_is_3;
    int picard;                // linearisation: 0 Newton (Eq. 2.7), 1 Picard (viscosity frozen)
    double body[3];
    double* gA;                // gradient output (accumulated)
    double* gA_part;           // per-warp partials, indexed blockIdx.x * warps_per_block + warp
    double gA_scale;
    int64_t lat_nx, lat_ny, lat_NX, lat_NY;   // conforming lattice (lat_nx > 0): node index
                               // computed as I + NX (J + NY L) instead of read from nodes
    int* err;                  // device status word (bounded waits that expired)
    uint32_t wait_polls;       // poll limit of the first wait for a group's staged state
                               // (WAIT_POLLS_DEFAULT; smaller only through the test hook);
                               // the drain after a give-up always uses WAIT_POLLS_DEFAULT
    int persistent_blocks;     // grid size of the persistent state-apply kernel
    // basal terms done by the stored-state kernel after its element groups
    // (one launch per apply): the Robin term (face, fuse_robin) and the
    // constraint rows s (I - P) x at the Nb basal nodes (fuse_constraint)
    int fuse_robin, fuse_constraint;
    // component-per-lane apply: basal Robin term of the basal elements added
    // in the element pass from the stored basal state (face.fstate), instead
    // of the face tail; fidx: basal face of each element (-1 if none)
    int face_in_elements;
    const int32_t* fidx;
    // k >= 5 kernels: degree tables (device), the degree, the state stride
    const void* htab;
    int htab_k;
    int64_t state_stride;
    FaceArgs face;
    int64_t Nb;
    const int32_t* basal_nodes;
    const double* basal_P;     // [Nb][6]
    double cscale;
};


enum FaceMode : int { FACE_APPLY = 0, FACE_GRAD_LOGBETA = 1, FACE_LINEARIZE = 2 };

// Per-degree launchers (one translation unit per degree).  prec: 0 f64, 1 f32.
// Return a cudaError_t value.
#define STOKES_DECLARE_DEGREE(KK)                                                            \
    int launch_elem_k##KK(int mode, int prec, int state_prec, bool trans, const ElemArgs& a,  \
                          cudaStream_t s);                                                    \
    int launch_face_k##KK(int mode, int prec, const FaceArgs& a, cudaStream_t s);             \
    int upload_tables_k##KK(const void* tables_k);                                            \
    int64_t state_stride_k##KK();                                                             \
    int64_t grad_a_partials_k##KK(int64_t E);
STOKES_DECLARE_DEGREE(2)
STOKES_DECLARE_DEGREE(3)
STOKES_DECLARE_DEGREE(4)
#undef STOKES_DECLARE_DEGREE

// Degree-independent kernels (misc.cu).
int launch_constraint(int prec, int64_t Nb, const int32_t* basal_nodes, const double* basal_P, double scale,
                      const void* x, void* y, cudaStream_t s);

}  // namespace stokes

#ifdef __CUDACC__
__device__ __forceinline__ double rcbrt_t(double x) { return rcbrt(x); }
__device__ __forceinline__ float rcbrt_t(float x) { return rcbrtf(x); }
#endif
