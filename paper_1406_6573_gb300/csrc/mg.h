// Geometric multigrid for the velocity block of the block preconditioner
// (Eq. 4.1).  The paper approximates F^{-1} by smoothed-aggregation AMG whose
// aggregates keep the vertical node columns together (Section 5): thin ice
// couples nodes far more strongly along a column than across columns, so the
// coarse spaces coarsen only horizontally.  Here the same idea is built
// geometrically on conforming slab meshes of degree 2, 3, 4:
//  * levels: the mesh semi-coarsened by 2 in x and y (columns and the vertical
//    node lattice kept) down to 4 cells per direction (2 for the first
//    coarse level of a small mesh), each level a mesh of its own (the fine isoparametric
//    heights at the coarse GLL points), with its own stored FP32 (or FP64)
//    state linearised at the fine velocity interpolated to its nodes (the
//    coarse operator is the rediscretised Newton Jacobian) and log(beta)
//    interpolated to its basal nodes;
//  * smoother: the exact vertical-column block solves of each level (damped
//    block Jacobi), i.e. line relaxation in the strongly coupled direction;
//  * transfers: degree-k interpolation of the coarse nodal values to the fine
//    nodes in x and y (tensor products of 1-D tables), identity in z;
//    restriction its transpose; the basal slip projector applied around
//    both, so that corrections stay in the constrained space;
//  * V(1,1) cycle; on the coarsest level four damped
//    column-Jacobi sweeps (twelve when there are only two levels), the
//    damping capped at 1.6 / lambda_max(C^-1 A)
//    (power iteration per linearisation): on isotropic high-order coarse
//    meshes the column blocks miss strong horizontal couplings and the
//    cycle's damping alone would amplify some error components.
// On a 2:1 forest (one refinement level, hanging faces and edges) the first
// coarse level is the unrefined base mesh: the base Q_k functions are exact
// on the forest (children inherit the parent map and the hanging nodes
// interpolate the coarse trace), so the prolongation evaluates them at the
// forest's independent nodes; restriction is its transpose, and the base
// level's linearisation point and log(beta) are averaging restrictions of
// the forest's fields.  The forest level adds its column-block solve and the
// prolongated base-level cycle (additive two-level form); the base mesh then
// coarsens as above.
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "handles.h"

namespace stokes {

struct MgLevel {
    stokes_mesh* mesh = nullptr;          // coarse levels: owned; level 0: the solver's mesh
    stokes_state* st = nullptr;           // coarse levels: owned; level 0: the solver's inner state
    bool owned = false;
    void* A = nullptr;                    // column blocks (coarse levels; level 0 uses the solver's)
    size_t band_elems = 0;
    int bw = 0;
    double scale = 0.0;                   // constraint-row scale of this level (0: not chosen yet)
    double omega = 0.0;                   // smoother damping of this level (0: the cycle's omega)
    double lmax = 0.0;                    // coarsest level: estimate of the largest eigenvalue of C^-1 A
    int64_t n = 0, nu = 0;                // full state length, velocity length
    int64_t NX = 0, NY = 0, NZ = 0;       // node lattice (NX, NY: columns per direction)
    void *b = nullptr, *x = nullptr, *r = nullptr, *t = nullptr;   // work vectors (pressure parts zero)
    double* u64 = nullptr;                // coarse linearisation point (FP64)
    double* logbeta = nullptr;            // coarse log(beta) at the basal nodes
    // 1-D transfer tables between the previous (finer) level and this one:
    // P_x, P_y, R_x, R_y, J_x, J_y at offsets t_off (entries) and t_coff (rows)
    int32_t* t_idx = nullptr;
    double* t_w = nullptr;
    int32_t* t_cnt = nullptr;
    int64_t t_off[6] = {}, t_coff[6] = {};
    int t_m[6] = {};
    // a base level under a 2:1 forest: sparse transfers instead of the tables
    // (rows of P: the forest's nodes; of R = P^T and of the averaging
    // restriction J = D^-1 P^T: this level's nodes; Jb: J on the basal nodes)
    bool csr = false;
    int32_t *P_ptr = nullptr, *P_col = nullptr, *R_ptr = nullptr, *R_col = nullptr;
    int32_t *J_ptr = nullptr, *J_col = nullptr, *Jb_ptr = nullptr, *Jb_col = nullptr;
    double *P_w = nullptr, *R_w = nullptr, *J_w = nullptr, *Jb_w = nullptr;
};

// compressed sparse rows (host)
struct HostCsr {
    std::vector<int32_t> ptr, col;
    std::vector<double> w;
};

// P: the base mesh hb's nodal values -> the nodes of the 2:1 forest h whose
// unrefined mesh it is (element map nodes [E][n1^3], refinement mask of the
// coarse cells, empty for none); checks that P reproduces the forest's node
// coordinates from the base mesh's.  Host only.
int forest_prolongation(const HostMesh& h, const std::vector<int32_t>& nodes, const std::vector<uint8_t>& refine,
                        const HostMesh& hb, HostCsr& P);

// dense copy of a 1-D transfer table between a lattice of nf elements and
// its semi-coarsening (nf / 2 elements), degree k: which 0 = P (coarse ->
// fine, [NXf][NXc]), 1 = R = P^T ([NXc][NXf]), 2 = J (fine -> coarse
// interpolation, [NXc][NXf]).  Host only.
int mg_transfer_dense(int nf, int k, int periodic, int which, double* out, int64_t rows, int64_t cols);

struct Multigrid {
    std::vector<MgLevel> L;
    int prec = 1;
    bool periodic = false;
    double omega = 0.8;                   // damping of the column-Jacobi smoother
    // sweeps on the coarsest level of hierarchies of three or more levels:
    // the Krylov counts did not change between 12 and 4 (128x128x8 Q2,
    // 64x64x4 Q3 and Q4 slabs, Q3 forest), and 4 saved 8-12 % of the solve
    // time (2 sweeps: the forest needed 10 % more iterations); two-level
    // hierarchies use 12 (mg_create)
    int coarse_sweeps = 4;
    // a forest level (next level on sparse transfers): additive correction
    // x = C^-1 b + P V(P^T b) instead of the smoothed cycle.  The forest's
    // column blocks stand in for the hanging slots by single nodes, so they
    // are not the exact diagonal blocks, and damped block Jacobi with them
    // can amplify error components: measured, the smoothed cycle diverged on
    // a Q2 forest (FGMRES stagnated) and saved 10-15 % of the iterations on
    // the Q3 forests; the additive form converged on all of them.
    bool forest_additive = true;
    double* dsc = nullptr;                // device scalar (diagonal sums)
};

// the mesh can carry the multigrid: degree 2, 3 or 4, and either a
// conforming lattice mesh with nx and ny even and >= 4, or a 2:1 forest (its
// unrefined base mesh is the first coarse level)
bool mg_eligible(const stokes_mesh* m);
// levels and work vectors; level 0 uses the given state and column blocks
int mg_create(Multigrid& mg, const stokes_mesh* fine, stokes_state* st_fine, void* A_fine, int bw_fine,
              int prec);
// per linearisation: coarse states at the injected up_fine, their column blocks
int mg_setup(Multigrid& mg, const stokes_params* p, const double* up_fine, double fine_scale, cudaStream_t s);
// z_u = V-cycle(r_u) on the velocity parts (z's pressure part is not touched)
int mg_apply(Multigrid& mg, const void* r, void* z, cudaStream_t s);
void mg_destroy(Multigrid& mg);

}  // namespace stokes
