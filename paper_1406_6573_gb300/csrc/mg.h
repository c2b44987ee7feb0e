// Geometric multigrid for the velocity block of the block preconditioner
// (Eq. 4.1).  The paper approximates F^{-1} by smoothed-aggregation AMG whose
// aggregates keep the vertical node columns together (Section 5): thin ice
// couples nodes far more strongly along a column than across columns, so the
// coarse spaces coarsen only horizontally.  Here the same idea is built
// geometrically on conforming slab meshes of degree 2, 3, 4:
//  * levels: the mesh semi-coarsened by 2 in x and y (columns and the vertical
//    node lattice kept), each level a mesh of its own (the fine isoparametric
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
//  * V(1,1) cycle; on the coarsest level (a few columns) several damped
//    column-Jacobi sweeps.
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
};

struct Multigrid {
    std::vector<MgLevel> L;
    int prec = 1;
    bool periodic = false;
    double omega = 0.8;                   // damping of the column-Jacobi smoother
    int coarse_sweeps = 12;
    double* dsc = nullptr;                // device scalar (diagonal sums)
};

// the mesh can carry the multigrid: conforming lattice mesh of degree 2, 3 or
// 4, nx and ny even and >= 4
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
