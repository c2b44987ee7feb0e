/*
 * stokes.h -- C-ABI of the GB300 matrix-free high-order nonlinear Stokes operator.
 *
 * The library evaluates, on one GPU, the discrete operator of the paper
 * "Solution of nonlinear Stokes equations discretized by high-order finite
 * elements on nonconforming and anisotropic meshes, with application to ice
 * sheet dynamics" (Isaac, Stadler, Ghattas):
 *
 *   residual  r(u, p)    of the weak form, Eq. 2.5 (Section 2.2), Glen flow
 *                        law Eq. 2.2 with basal Robin sliding and no
 *                        penetration, Eq. 2.4;
 *   Jacobian  J(u)[w, q] Newton linearisation, Eqs. 2.6-2.7 (Section 2.3);
 *   J^T                  transpose action (Section 4.1: A(u) is symmetric);
 *   gradients            adjoint products with d r / d log(beta) and d r / d A
 *                        (the "adjoint equations" of Section 2.3 and 8.3).
 *
 * Discretisation (Section 3.2): isoparametric Q_k velocity on GLL nodes, tensor
 * Gauss quadrature with k+1 points per direction, discontinuous P_{k-1} or
 * Q_{k-2} pressure, hexahedral meshes with one level of 2:1 refinement and
 * hanging-node restriction R_i (hanging-node figure of Section 3.2.1).  The
 * operator is applied matrix-free with sum-factorised tensor contractions
 * (Section 3.3).
 *
 * Conventions shared by every entry point
 *   - All vector arguments are CALLER-OWNED DEVICE pointers on the mesh's
 *     device, contiguous, of the element type given by `prec`
 *     (STOKES_F64: double, STOKES_F32: float) unless stated otherwise.
 *   - A state vector "up" has length 3*Nv + Np: the velocity node-major and
 *     interleaved (u_x, u_y, u_z of node 0, then node 1, ...), followed by the
 *     discontinuous pressure, element-major ([E][npr]).
 *   - Global nodes are ordered by reference position (Z, then Y, then X,
 *     X and Y wrapped on periodic meshes); elements by coarse cell (x fastest,
 *     then y, then z) with a refined cell replaced by its 8 children in the
 *     order bx + 2 by + 4 bz.
 *   - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = legacy default stream).  Nothing is allocated per call: the mesh
 *     handle owns its device metadata and workspaces, which is why calls that
 *     share a mesh must not run concurrently on different streams.
 *   - Return value: STOKES_OK or a negative error code; stokes_last_error()
 *     returns a message for the calling thread's last failure.  No exception
 *     crosses the ABI.
 *   - Constraints: basal nodes carry the nodal projector P (P = 0 for no-slip;
 *     P = I - n n^T for u . n = 0, n the normalised area-weighted nodal normal).
 *     The residual evaluated is r_c(u) = P r(P u) + s (I - P) u and the
 *     Jacobian P J(P u) P + s (I - P), its exact derivative
 *     (s = params->constraint_scale).
 */
#ifndef STOKES_GB300_H
#define STOKES_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define STOKES_OK            0
#define STOKES_E_INVAL      -1   /* bad argument: NULL pointer, size, enum     */
#define STOKES_E_MESH       -2   /* invalid mesh: inverted element, bad mask   */
#define STOKES_E_NOMEM      -3   /* device or host allocation failed           */
#define STOKES_E_CUDA       -4   /* a CUDA runtime call or launch failed       */
#define STOKES_E_NONFINITE  -5   /* a non-finite value was produced            */
#define STOKES_E_NOCONV     -6   /* solver did not reach its tolerance         */

/* ---- enums ---------------------------------------------------------------- */
#define STOKES_F64 0
#define STOKES_F32 1

#define STOKES_PRESSURE_P 0      /* P_{k-1}^disc: Legendre products, degree <= k-1 */
#define STOKES_PRESSURE_Q 1      /* Q_{k-2}^disc: Lagrange on (k-1)^3 Gauss points */

#define STOKES_BASE_NOSLIP 0     /* u = 0 on the base                           */
#define STOKES_BASE_SLIP   1     /* u . n = 0 on the base (plus Robin if enabled) */

/* A smooth periodic field f(x,y) = mean + sum_m amp[m] cos(kx[m] x + ky[m] y
 * + phase[m]).  Host pointers, read during stokes_mesh_create only. */
typedef struct {
    double mean;
    int n_modes;
    const double* amp;
    const double* kx;
    const double* ky;
    const double* phase;
} stokes_field;

/* Mesh description (all host memory, read during stokes_mesh_create only).
 * Geometry: x = Lx X / nx, y = Ly Y / ny, z = bed + (Z / nz)(surface - bed),
 * evaluated at the GLL nodes of each coarse cell (isoparametric map); refined
 * children inherit the parent map (Section 3.1).
 * Meshes are extruded columns: x and y are affine in each cell and only z
 * follows the bed and surface, so the inverse Jacobian has the rows
 * (1/a, 0, 0), (0, 1/b, 0) and one general third row; the stored linearised
 * state and its applies rely on this (p6est-type meshes of thin ice).
 * Bed and surface come from the modal fields, or, when bed_nodes and
 * surface_nodes are non-NULL, from heights given on the horizontal GLL
 * lattice of the coarse grid: point (X, Y), X = k cx + i, Y = k cy + j, at
 * x = Lx (cx + (xi_i + 1)/2) / nx, y = Ly (cy + (xi_j + 1)/2) / ny (xi_i the
 * GLL nodes of degree k), stored [Y][X] with X fastest; NX = k nx + 1,
 * NY = k ny + 1 points, or k nx and k ny on periodic meshes (X = k nx is
 * X = 0).  A gridded bed is interpolated by the degree-k map like any
 * other. */
typedef struct {
    int nx, ny, nz;               /* coarse hexahedral grid                     */
    int k;                        /* velocity degree: 1 <= k <= 9 for host-only
                                     meshes (device = -1), 2 <= k <= 4 on a
                                     device (the kernels' degrees)              */
    int pressure_space;           /* STOKES_PRESSURE_P or STOKES_PRESSURE_Q      */
    int periodic_xy;              /* 1: periodic in x and y                      */
    double Lx, Ly;                /* horizontal extent                           */
    stokes_field bed, surface;
    const uint8_t* refine;        /* [nx*ny*nz] 1 = split once into 8, or NULL   */
    int basal_bc;                 /* STOKES_BASE_NOSLIP or STOKES_BASE_SLIP      */
    int device;                   /* CUDA device ordinal, or -1: host-only mesh  */
    const double* bed_nodes;      /* optional gridded bed [NY][NX], or NULL      */
    const double* surface_nodes;  /* optional gridded surface [NY][NX], or NULL  */
} stokes_mesh_desc;

/* Physical parameters.  mu = C0 A^(-1/n) (gamma D:D + delta)^((1-n)/(2n));
 * the paper's Glen law (Eq. 2.2) is C0 = 1, gamma = 1/2, delta = eps. */
typedef struct {
    double n, A, C0, gamma, delta;
    double body[3];               /* body force b                               */
    int robin;                    /* 1: add int_{Gamma_b} beta T v . T u ds      */
    const double* logbeta;        /* DEVICE, [Nb] FP64 nodal log(beta) at the
                                     basal nodes (ascending global node order);
                                     required when robin = 1                   */
    double constraint_scale;      /* s > 0 of the constraint rows: the operator
                                     is P J P + s (I - P) and the residual
                                     P r(P u) + s (I - P) u; the solution does
                                     not depend on s.  1 = plain projector;
                                     the solver picks s ~ the diagonal of J so
                                     that FP32 arithmetic resolves these rows. */
    int linearization;            /* STOKES_LIN_NEWTON: the Newton Jacobian of
                                     Eqs. 2.6-2.7 (default, 0); STOKES_LIN_PICARD:
                                     the fixed-viscosity (Picard) operator
                                     A(u) w = int mu(u) D(v):D(w) - ..., i.e. no
                                     derivative of mu.  Affects the Jacobian
                                     applies, stokes_linearize and the solver
                                     (a Picard iteration); not the residual. */
    double sliding_m;             /* basal sliding law: the Robin traction is
                                     beta s(|T u|^2) T u with
                                     s(x) = (x + sliding_eps)^((m-1)/2), a
                                     Weertman-type power law (Eq. 2.3 leaves
                                     the dependence on |T u| open); 0 or 1:
                                     the linear law beta T u of Eq. 2.4a.
                                     Otherwise m > 0 and sliding_eps > 0.  The
                                     Newton Jacobian adds
                                     2 beta s'(|T u|^2) (T u . T w) T u (the
                                     Picard form keeps s and drops it). */
    double sliding_eps;           /* regularisation of |T u|^2 (velocity^2)   */
} stokes_params;

#define STOKES_LIN_NEWTON 0
#define STOKES_LIN_PICARD 1

typedef struct {
    int64_t E;        /* elements                                               */
    int64_t Nv;       /* independent velocity nodes (3 Nv velocity dofs)        */
    int64_t Np;       /* pressure dofs = E * npr                                */
    int64_t Nb;       /* basal nodes                                            */
    int32_t k, npr;   /* velocity degree, pressure dofs per element             */
    int64_t n_hanging_elems;  /* elements with at least one hanging face/edge   */
} stokes_sizes;

typedef struct stokes_mesh stokes_mesh;
typedef struct stokes_state stokes_state;

/* Build the mesh on the host (node numbering, hanging-node codes, geometry at
 * quadrature points in FP64) and upload it to `desc->device`.
 * Errors: E_INVAL (bad sizes/enums), E_MESH (detJ <= 0), E_NOMEM, E_CUDA.
 * On success *out owns all device memory; release with stokes_mesh_destroy. */
int stokes_mesh_create(const stokes_mesh_desc* desc, stokes_mesh** out);
int stokes_mesh_destroy(stokes_mesh* mesh);
int stokes_mesh_sizes(const stokes_mesh* mesh, stokes_sizes* out);

/* Synchronise the mesh's device and report STOKES_E_CUDA if a kernel gave up
 * on a bounded wait since the last call (the status word is then cleared).
 * Kernels never spin without a limit; this is how such an event is seen. */
int stokes_mesh_status(const stokes_mesh* mesh);

/* Host copies of mesh data for verification: physical coordinates of the
 * global nodes [Nv][3] (x, y wrapped into [0, L) on periodic meshes) and the
 * global node index of each basal node [Nb].  Caller-owned host buffers. */
int stokes_mesh_node_coords(const stokes_mesh* mesh, double* xyz);
int stokes_mesh_basal_nodes(const stokes_mesh* mesh, int64_t* nodes);

/* Residual r_c(up) (Eq. 2.5 with the constraints above).  up, r: [3Nv+Np].
 * prec selects the arithmetic and the element type of up and r. */
int stokes_residual(const stokes_mesh* mesh, const stokes_params* params,
                    const void* up, void* r, int prec, void* stream);

/* y = J_c(up_lin) x, the Newton Jacobian of Eqs. 2.6-2.7 at up_lin, fused:
 * the linearisation is recomputed at every quadrature point.  On meshes of
 * degree k >= 5 (block-per-element kernels) the call linearises into a
 * per-mesh FP64 workspace and applies from it: two such calls on one mesh
 * must not overlap on the GPU (they race on the workspace). */
int stokes_jacobian_apply(const stokes_mesh* mesh, const stokes_params* params,
                          const void* up_lin, const void* x, void* y,
                          int prec, void* stream);

/* y = J_c(up_lin)^T x (transposed pointwise map and coupling blocks). */
int stokes_jacobian_apply_transpose(const stokes_mesh* mesh, const stokes_params* params,
                                    const void* up_lin, const void* x, void* y,
                                    int prec, void* stream);

/* Adjoint products with the parameter Jacobians at the state up (FP64):
 *   g_logbeta[j] = lambda^T d r_c / d log(beta_j)   (device, [Nb], overwritten)
 *   *g_A         = lambda^T d r_c / d A             (device, 1 double, overwritten)
 * Either output may be NULL.  up, lambda: device FP64 [3Nv+Np]. */
int stokes_param_grad(const stokes_mesh* mesh, const stokes_params* params,
                      const double* up, const double* lambda,
                      double* g_logbeta, double* g_A, void* stream);

/* ---- Fixed-order A-gradient that allocates nothing ------------------------
 * The paper has no counterpart of this call; it is a library utility.
 * *g_A = lambda^T d r_c / d A, the quantity stokes_param_grad returns in g_A,
 * but the per-warp partial sums are written to a library-owned device scratch
 * (a file-scope static array of STOKES_GRAD_A_MAX_PARTIALS doubles, 1 MiB on
 * each device) and then added by one block in a fixed order, so repeated
 * calls on the same inputs give bitwise identical results (stokes_param_grad
 * adds them with atomics, in an order that varies).
 * Allocation: none.  The call makes no cudaMalloc or cudaFree and calls no
 * library that allocates.  It serves callers that cannot allocate device
 * memory at this point: a caller whose device memory is fully reserved by its
 * own pool (a solver holding its Krylov bases at scale), or a loop that shares
 * its stream with other work and cannot take the device-wide synchronisation
 * that cudaFree implies.
 * Size limit: the element kernel writes one partial per launched warp,
 * ceil(E / (4 e_w)) * 4 of them with e_w = 32 / (k+1)^2 elements per warp
 * (3, 2, 1 for k = 2, 3, 4); a mesh that needs more than
 * STOKES_GRAD_A_MAX_PARTIALS (E > 393,216 for k = 2, 262,144 for k = 3,
 * 131,072 for k = 4) returns STOKES_E_INVAL before any launch.
 * Zero state: nothing in the scratch has to start at zero; every partial that
 * is read is written earlier in the same call.
 * Concurrency: the scratch is shared by every call on a device.  Two calls
 * whose executions overlap (different streams or host threads, same device)
 * race on it and both results are undefined; callers serialise them.
 * Set-up: the first call on each device resolves the scratch address with
 * cudaGetSymbolAddress and caches it; make that first call before beginning
 * any stream capture on that device.  The cached address lives as long as
 * the process and belongs to the device's primary context at the time of
 * that first call: after cudaDeviceReset (or anything else that destroys
 * and recreates the primary context) the address is stale, so do not call
 * this entry point again in that process after a device reset.
 * up, lambda: device FP64 [3Nv+Np]; g_A: device, 1 double, overwritten. */
#define STOKES_GRAD_A_MAX_PARTIALS 131072
int stokes_param_grad_A_fixed_order(const stokes_mesh* mesh, const stokes_params* params,
                                    const double* up, const double* lambda, double* g_A,
                                    void* stream);

/* Linearised state: the per-quadrature-point Newton coefficients at up_lin
 * (geometry, mu, and the rank-one term of Eq. 2.7), evaluated in FP64 and
 * stored in `prec`, so that repeated Jacobian applies (Krylov iterations)
 * stream them instead of recomputing the viscosity.  With a nonlinear
 * sliding law (params->sliding_m not 0 or 1) the linearisation also stores,
 * per basal Gauss point, beta w s, 2 beta w s' T u and T u, which the basal
 * term of the applies uses.  The state owns its device arrays (about
 * 1200 bytes per Q2 element in FP32, plus 7 values per basal Gauss point);
 * the FP32 state of a conforming k = 2 mesh is stored in groups of 10
 * elements for the component-per-lane apply kernel, every other state
 * element by element (the layout is internal to the library). */
int stokes_state_create(const stokes_mesh* mesh, int prec, stokes_state** out);
int stokes_state_destroy(stokes_state* state);
/* up_lin: device FP64 [3Nv+Np]. params is copied into the state; the device
 * array params->logbeta points to must stay valid while the state is applied
 * (the copy keeps the pointer, not the values). */
int stokes_linearize(stokes_state* state, const stokes_params* params,
                     const double* up_lin, void* stream);
/* y = J_c x from the stored state; x, y of the state's precision. */
int stokes_state_apply(const stokes_state* state, const void* x, void* y, void* stream);
int stokes_state_apply_transpose(const stokes_state* state, const void* x, void* y,
                                 void* stream);
/* y = J_c (0, x_p): the velocity rows are P B^T x_p, the pressure-to-velocity
 * block of the Newton system (the off-diagonal block of the block
 * preconditioner, Eq. 4.1), the pressure rows are zero; the velocity part of
 * x is ignored.  Reads only the geometric part of the stored state. */
int stokes_state_apply_pressure_block(const stokes_state* state, const void* x, void* y,
                                      void* stream);

/* ---- Newton-Krylov solver (Section 4) -------------------------------------
 * Inexact Newton with backtracking on ||r||_2 and Eisenstat-Walker forcing;
 * right-preconditioned FGMRES(m) with the block upper-triangular
 * preconditioner of Eq. 4.1 (velocity block: exact vertical-column blocks of
 * F; Schur complement: -diag of the 1/mu-weighted pressure mass, Section 6).
 * inner_prec = STOKES_F32: Krylov vectors, operator applies and
 * preconditioner in FP32, the linear residual recomputed in FP64 at every
 * restart (iterative refinement), residual and Newton update in FP64.
 * inner_prec = STOKES_F64: the same loop entirely in FP64.
 * The solver handle owns its workspaces (allocated by stokes_solver_create:
 * about (2m+3) inner-precision and 6 FP64 state vectors, two linearised
 * states and the banded column blocks). */
typedef struct stokes_solver stokes_solver;

typedef struct {
    int inner_prec;      /* STOKES_F32 (mixed precision) or STOKES_F64               */
    int restart;         /* FGMRES restart length m (default 30, at most 31)          */
    int max_krylov;      /* Krylov iterations per linear solve (default 1000)         */
    int max_newton;      /* Newton steps (default 50)                                 */
    double rtol;         /* Newton stop: ||r|| <= rtol ||r_0|| (default 1e-10)        */
    double eta_max;      /* cap of the forcing term (default 0.1)                     */
    int velocity_mg;     /* 1: the velocity block of the preconditioner is a geometric
                            multigrid V-cycle (horizontal semi-coarsening that keeps the
                            node columns, as the paper's column-preserving aggregation
                            of Section 5; column-block smoother) on meshes of degree
                            2, 3, 4: conforming meshes with nx, ny even and >= 4, and
                            2:1 forests with nx, ny >= 2, whose unrefined base mesh is
                            the first coarse level (the default when opts is NULL);
                            other meshes, and 0, use the column blocks alone       */
} stokes_solver_opts;

typedef struct {
    int converged, newton_its, krylov_its, line_search_cuts;
    double res0, res_final, seconds;
    double constraint_scale;     /* s used by stokes_newton_solve (see stokes_params) */
    double history[64];          /* ||r_j||, j = 0 .. newton_its (first 64)          */
    int krylov_per_newton[64];
    int line_search_failed;      /* 1: twelve step halvings gave no decrease of ||r||;
                                    the step was rejected, up holds the last accepted
                                    iterate and the solve returned STOKES_E_NOCONV */
    int mg_levels;               /* levels of the velocity multigrid (0: column blocks) */
} stokes_solve_report;

int stokes_solver_create(const stokes_mesh* mesh, const stokes_solver_opts* opts, stokes_solver** out);
int stokes_solver_destroy(stokes_solver* solver);
/* Both solvers read the mesh's device status word (stokes_mesh_status) after
 * every restart cycle and every Newton step: if a kernel gave up waiting for
 * a staged copy the word is cleared and the solve returns STOKES_E_CUDA.
 *
 * Solve r_c(up) = 0 starting from the device FP64 state up (overwritten).
 * The solver replaces params->constraint_scale by the mean diagonal of the
 * velocity block at the first linearisation (reported in the report); the
 * residual norms it reports use that scale.
 * Returns STOKES_E_NOCONV (report filled) if rtol is not reached, and
 * STOKES_E_NONFINITE if the residual at the initial guess or after an update
 * is not finite (up then holds the last finite iterate). */
int stokes_newton_solve(stokes_solver* solver, const stokes_params* params, double* up,
                        stokes_solve_report* report, void* stream);
/* Solve J_c(up_lin) x = b (transpose = 0) or J_c(up_lin)^T x = b (transpose = 1)
 * to ||b - J x|| <= rtol ||b||; up_lin, b, x: device FP64 [3Nv+Np].
 * Returns STOKES_E_NOCONV if rtol is not reached and STOKES_E_NONFINITE if b
 * or the final linear residual is not finite. */
int stokes_linear_solve(stokes_solver* solver, const stokes_params* params, const double* up_lin,
                        const double* b, double* x, int transpose, double rtol,
                        stokes_solve_report* report, void* stream);

/* Test hooks (failure injection on the host side; no kernel is made to
 * fault or hang).
 *
 * stokes_debug_wait_limit: poll limit of the first wait of the stored-state
 * applies (stokes_state_apply*, stokes_state_apply_pressure_block) for the
 * staged state of each element group; default STOKES_WAIT_POLLS_DEFAULT.
 * With a small limit (0: give up at once) the warps that run out set the
 * mesh's status word, wait for their own copies in flight with the default
 * limit and return, so the apply's output is incomplete and
 * stokes_mesh_status (and the solvers) report STOKES_E_CUDA.  Restore the
 * default after the test.  Returns STOKES_E_INVAL for a host-only mesh.
 *
 * stokes_debug_fail_alloc_after: the library's next n device allocations
 * succeed and the one after fails as if the device were out of memory (the
 * entry point making it returns STOKES_E_NOMEM and frees what it had
 * allocated); n < 0 switches the hook off (the default).  Process-wide;
 * returns the previous setting.
 *
 * stokes_debug_forest_prolongation: builds, on the host, the prolongation of
 * the velocity multigrid from base (the unrefined mesh of forest: same grid,
 * degree, geometry and periodicity, no refinement) to forest, and checks that
 * it reproduces the forest's node coordinates from the base's (heights, and
 * x, y away from a periodic seam).  Both meshes host-only (device = -1).
 * *nnz receives the prolongation's entries, *rowsum_err the largest
 * |row sum - 1|.  STOKES_E_MESH if the meshes do not match or the check
 * fails; STOKES_E_INVAL for device meshes.
 *
 * stokes_debug_mg_transfer: a dense host copy of one 1-D transfer table of
 * the velocity multigrid between a lattice of nf elements of degree k
 * (1 <= k <= 4, nf even) and its semi-coarsening of nf / 2 elements, with
 * NXf = k nf (+ 1 unless periodic) and NXc = k nf / 2 (+ 1 unless periodic)
 * nodes: which = 0 the prolongation P [NXf][NXc] (degree-k interpolation of
 * coarse nodal values at the fine nodes), 1 the restriction R = P^T
 * [NXc][NXf], 2 the interpolation J [NXc][NXf] of fine nodal values at the
 * coarse nodes.  out: host, rows x cols row-major.  STOKES_E_INVAL on a wrong
 * shape or degree. */
#define STOKES_WAIT_POLLS_DEFAULT 4194304u
int stokes_debug_wait_limit(stokes_mesh* mesh, uint32_t polls);
int64_t stokes_debug_fail_alloc_after(int64_t n);
int stokes_debug_forest_prolongation(const stokes_mesh* forest, const stokes_mesh* base, int64_t* nnz,
                                     double* rowsum_err);
int stokes_debug_mg_transfer(int nf, int k, int periodic, int which, double* out, int64_t rows, int64_t cols);

/* Per-kernel timing (tracing).  Between stokes_profile_begin and
 * stokes_profile_end every operator call on this mesh, and every launch and
 * transfer of a solver built on it, records a CUDA event pair around the
 * work on the caller's stream; end synchronises on the recorded events and
 * returns launch counts and summed device times per class.  Recording costs
 * a few microseconds of host time per launch and no device work. */
typedef struct {
    int64_t launches;
    double ms;
} stokes_kernel_time;

typedef struct {
    stokes_kernel_time clear;       /* output zeroing (cudaMemsetAsync)          */
    stokes_kernel_time element;     /* volume element kernel                     */
    stokes_kernel_time face;        /* basal Robin face kernel                   */
    stokes_kernel_time constraint;  /* (I - P) constraint kernel                 */
    stokes_kernel_time precond;     /* solver: preconditioner apply (Schur
                                       block, update, column solves)           */
    stokes_kernel_time orthog;      /* solver: Gram-Schmidt passes, norms      */
    stokes_kernel_time vector;      /* solver: vector updates and copies       */
    stokes_kernel_time setup;       /* solver: preconditioner set-up per
                                       linearisation (assembly, factorisation) */
    stokes_kernel_time transfer;    /* solver: host <-> device scalar copies   */
} stokes_profile;

int stokes_profile_begin(const stokes_mesh* mesh);
int stokes_profile_end(const stokes_mesh* mesh, stokes_profile* out);

/* Message describing the calling thread's last error ("" if none). */
const char* stokes_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* STOKES_GB300_H */
