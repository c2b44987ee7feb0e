// Internal declarations shared by the host mesh builder, the CUDA kernels and
// the C-ABI layer of the GB300 nonlinear Stokes operator library.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/stokes.h"

namespace stokes {

constexpr int KMAX = 9;           // highest velocity degree of the host mesh builder and tables
                                  // (the GPU kernels are built for k = 2, 3, 4)
constexpr int N1MAX = KMAX + 1;   // nodes (and Gauss points) per direction
constexpr int NPRMAX = (KMAX - 1) * (KMAX - 1) * (KMAX - 1);   // largest pressure space: Q_{k-2} at
                                  // k = 9, (k - 1)^3 = 512 modes (P_{k-1} has 165)
static_assert(NPRMAX >= KMAX * (KMAX + 1) * (KMAX + 2) / 6, "P_{k-1} fits");

// Hanging-node code of an element (one 32-bit word).
//   bits 0..5   face f = 2 d + s hanging (d axis, s = 0 minus side, 1 plus side)
//   bits 6..17  edge parallel to axis d at sides (s0, s1) of the two other
//               axes o0 < o1 hanging: bit 6 + 4 d + s0 + 2 s1
//   bits 18..20 child position b_d within the parent cell (fine elements)
constexpr int HANG_FACE0 = 0;
constexpr int HANG_EDGE0 = 6;
constexpr int HANG_CHILD0 = 18;

// 1-D tables of one degree k (host copy; mirrored in device constant memory).
struct Tables1D {
    int k = 0, n1 = 0, q = 0, npr = 0;
    double gll[N1MAX], gllw[N1MAX];
    double gauss[N1MAX], gaussw[N1MAX];
    double B[N1MAX][N1MAX];      // B[iq][i]  = ell_i(g_iq), GLL Lagrange at Gauss points
    double Dg[N1MAX][N1MAX];     // Dg[iq][m] = derivative of the Gauss-point Lagrange
                                 //             polynomial m at g_iq (collocation)
    double I[2][N1MAX][N1MAX];   // I[b][i][m] = ell_m((xi_i + 2 b - 1) / 2): coarse GLL
                                 //              values -> half-interval b fine nodes
    double P1[N1MAX][N1MAX];     // pressure 1-D factors at Gauss points, P1[iq][a]
    int pmode[NPRMAX][3];        // pressure mode exponents / indices (a, b, c)
};

void build_tables(int k, int pspace, Tables1D& t);

// Host-side mesh data (what the kernels read, before upload).
struct HostMesh {
    int nx = 0, ny = 0, nz = 0, k = 0, n1 = 0, q = 0, npr = 0, pspace = 0;
    bool periodic = false;
    double Lx = 1, Ly = 1;
    int basal_bc = 0;
    int64_t E = 0, Nv = 0, Np = 0, Nb = 0, n_hang = 0;
    bool lattice = false;              // conforming lattice numbering (no refinement input)
    int64_t latNX = 0, latNY = 0;      // node lattice extents in x, y
    Tables1D tab;
    std::vector<int32_t> elem_nodes;   // [E][n1^3] node gathered into each local slot
    std::vector<uint32_t> elem_hang;   // [E] hanging code
    std::vector<double> geo;           // [E][10][q^3]: Jinv[m][d] (3m+d), w detJ
    std::vector<int32_t> elem_pidx;    // [E] -1 or row of pel
    std::vector<double> pel;           // [nP][6][n1^2] P at local slots (i, j, 0)
    int64_t nP = 0;
    std::vector<int32_t> elem_fidx;    // [E] -1 or basal face index
    std::vector<int32_t> face_elem;    // [nF]
    std::vector<double> fgeo;          // [nF][4][q^2]: w |J_s|, n_x, n_y, n_z
    std::vector<int32_t> fmap;         // [nF][n1^2] basal node index of slot (i, j, 0)
    int64_t nF = 0;
    std::vector<int32_t> basal_nodes;  // [Nb] global node of each basal node
    std::vector<double> basal_P;       // [Nb][6] P00 P11 P22 P01 P02 P12
    std::vector<double> node_xyz;      // [Nv][3]
    // vertical node columns (nodes sharing the reference (X, Y) position),
    // used by the column-block preconditioner of the velocity block
    int64_t ncol = 0;
    int colmax = 0;                    // most nodes in one column
    int bnode = 0;                     // largest in-element distance of two column positions
    std::vector<int32_t> col_of;       // [Nv] column of each node
    std::vector<int32_t> pos_of;       // [Nv] position (Z rank) within its column
    std::vector<int32_t> col_nodes;    // [colmax][ncol] node at (pos, column), -1 padding
    std::vector<int32_t> col_len;      // [ncol]
};

// Returns STOKES_OK or an error code; `err` receives a message on failure.
int build_host_mesh(const stokes_mesh_desc& d, HostMesh& m, std::string& err);

// Evaluate a modal field at (x, y).
double eval_field(const stokes_field& f, double x, double y);

}  // namespace stokes
