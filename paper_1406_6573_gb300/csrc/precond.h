// Block upper-triangular preconditioner of the linearised Stokes system
// (Section 4.2, Eq. 4.1):  A~ = [F~ B^T; 0 S~]  with
//   F~ = the vertical-column blocks of F (banded, factored per column), and
//   S~ = -M(1/mu), the inverse-viscosity weighted pressure mass (Section 6),
//        block diagonal for the discontinuous pressure: its element blocks
//        inverted exactly for npr <= 4 (k = 2 with P_1), its diagonal for the
//        larger pressure spaces (measured: the full blocks cut the FGMRES
//        iterations on the Q2 x P1 slab by 13 %, but not for Q3 x Q1 or
//        Q4 x P3, where they only add work).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace stokes {

// Banded column matrices: entry (row r, band slot s) of column c, with the
// columns in blocks of BAND_CB; a block holds its rows and slots contiguously
// ([ncol / BAND_CB][rows][W][BAND_CB], ncol rounded up to BAND_CB), so that
// one warp's columns read one contiguous run of W BAND_CB values per row.
constexpr int BAND_CB = 32;
__host__ __device__ inline int64_t band_at(int64_t c, int r, int s, int W, int rows) {
    return ((c / BAND_CB) * (int64_t(rows) * W) + int64_t(r) * W + s) * BAND_CB + (c % BAND_CB);
}
__host__ __device__ inline int64_t band_cols(int64_t ncol) { return (ncol + BAND_CB - 1) / BAND_CB * BAND_CB; }

struct ColArgs {
    int64_t E, ncol;
    int npr, pspace, bw, robin;
    int schur_full;            // assemble the whole element blocks of M(1/mu) (else their diagonal)
    const int32_t* nodes;      // [E][n1^3]
    const uint32_t* hang;      // [E]
    const int32_t* col_of;     // [Nv]
    const int32_t* pos_of;     // [Nv]
    const int32_t* fidx;       // [E]
    const int32_t* fmap;       // [nF][n1^2]
    const double* fgeo;        // [nF][4][q^2]
    const double* logbeta;     // [Nb]
    int rows;                  // rows of the band matrices (3 colmax)
    const void* fstate;        // stored sliding state of the state (NULL: linear sliding law)
    const void* state;         // linearised state (element type = prec)
    int state_cpl;             // the state is in the group layout of k = 2 FP32 states
    void* A;                   // [3 colmax][2 bw + 1][ncol] banded column matrices
    double* mblk;              // [E][npr][npr] M(1/mu) element blocks (FP64, assembly output)
    const void* htab;          // k >= 5: degree tables (device), degree, state stride
    int htab_k;
    int64_t state_stride;
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
    int* err;                  // status word for bounded waits that expired (may be NULL)
    double out_alpha = 1.0;    // the solve stores z = out_beta z + out_alpha C^-1 r
    double out_beta = 0.0;     // (velocity part; out_beta 0 does not read z)
};

// constraints (P F P + I - P on the basal node block) + banded LU per column
int launch_col_factor(int prec, const ColSolveArgs& a, cudaStream_t s);
// out[0] = sum over all columns of |diag| of the assembled blocks
int launch_col_diag_sum(int prec, const ColSolveArgs& a, double* out, cudaStream_t s);
// z_u = out_beta z_u + out_alpha F~^{-1} r_u on the velocity part (z, r: state
// vectors of type prec; z_u = F~^{-1} r_u with the defaults)
int launch_col_solve(int prec, const ColSolveArgs& a, const void* r, void* z, cudaStream_t s);
// full: minv[e] = inverse of the element block mblk[e] (npr x npr, SPD);
// otherwise minv[e npr + b] = 1 / mblk[e][b][b] (inverse diagonal); in prec
int launch_schur_invert(int prec, int64_t E, int npr, int full, const double* mblk, void* minv, cudaStream_t s);
// z_p = -minv r_p (pressure part; element blocks or diagonal, as inverted)
int launch_schur_apply(int prec, int64_t Nv, int64_t E, int npr, int full, const void* minv, const void* r,
                       void* z, cudaStream_t s);

}  // namespace stokes
