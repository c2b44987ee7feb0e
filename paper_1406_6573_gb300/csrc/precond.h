// Block upper-triangular preconditioner of the linearised Stokes system
// (Section 4.2, Eq. 4.1):  A~ = [F~ B^T; 0 S~]  with
//   F~ = the vertical-column blocks of F (banded, factored per column), and
//   S~ = -diag M(1/mu), the inverse-viscosity weighted pressure mass (Section 6).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace stokes {

struct ColArgs {
    int64_t E, ncol;
    int npr, pspace, bw, robin;
    const int32_t* nodes;      // [E][n1^3]
    const uint32_t* hang;      // [E]
    const int32_t* col_of;     // [Nv]
    const int32_t* pos_of;     // [Nv]
    const int32_t* fidx;       // [E]
    const int32_t* fmap;       // [nF][n1^2]
    const double* fgeo;        // [nF][4][q^2]
    const double* logbeta;     // [Nb]
    const void* state;         // linearised state (element type = prec)
    void* A;                   // [3 colmax][2 bw + 1][ncol] banded column matrices
    void* md;                  // [E npr] diagonal of M(1/mu)
};

int launch_precond_assembly_k2(int prec, const ColArgs& a, cudaStream_t s);
int launch_precond_assembly_k3(int prec, const ColArgs& a, cudaStream_t s);
int launch_precond_assembly_k4(int prec, const ColArgs& a, cudaStream_t s);

struct ColSolveArgs {
    int64_t ncol, Nv;
    int colmax, bw;
    const int32_t* col_nodes;  // [colmax][ncol]
    const int32_t* col_len;    // [ncol]
    const int32_t* col_basal;  // [ncol] basal index of the column's lowest node, or -1
    const double* basal_P;     // [Nb][6]
    double scale;              // constraint-row scale s of P F P + s (I - P)
    void* A;                   // banded matrices (factored in place)
};

// constraints (P F P + I - P on the basal node block) + banded LU per column
int launch_col_factor(int prec, const ColSolveArgs& a, cudaStream_t s);
// out[0] = sum over all columns of |diag| of the assembled blocks
int launch_col_diag_sum(int prec, const ColSolveArgs& a, double* out, cudaStream_t s);
// z_u = F~^{-1} r_u on the velocity part (z, r: state vectors of type prec)
int launch_col_solve(int prec, const ColSolveArgs& a, const void* r, void* z, cudaStream_t s);
// z_p = -r_p / md (pressure part)
int launch_schur_apply(int prec, int64_t Nv, int64_t Np, const void* md, const void* r, void* z, cudaStream_t s);

}  // namespace stokes
