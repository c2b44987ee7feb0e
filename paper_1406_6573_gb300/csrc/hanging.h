// Hanging-node predicates of the factored restriction R_i (host and device).
//
// R_i of an element with hanging faces or edges (hanging-node figure of
// Section 3.2.1) is applied as: gather every local slot from the global node
// it names, then, for each axis d, replace every constrained line of slots
// parallel to d by its 1-D interpolation from the coarse GLL nodes to the
// element's half of the coarse interval (I_{b_d}).  A line is constrained
// when it lies in a hanging face whose normal is not d, or is a hanging edge
// parallel to d.  Every line is interpolated at most once per axis, and the
// product of the per-axis sweeps is the tensor-product interpolation of the
// coarse trace.
#pragma once

#include <cstdint>

#include "common.h"

#ifdef __CUDACC__
#define STOKES_HD __host__ __device__ __forceinline__
#else
#define STOKES_HD inline
#endif

namespace stokes {

// Is the line of slots parallel to axis d, through coordinate a on the first
// other axis (o0) and b on the second (o1), constrained by the code h?
STOKES_HD bool line_hanging(uint32_t h, int d, int a, int b, int k) {
    const int o0 = (d == 0) ? 1 : 0;
    const int o1 = (d == 2) ? 1 : 2;
    if (a == 0 && ((h >> (HANG_FACE0 + 2 * o0)) & 1u)) return true;
    if (a == k && ((h >> (HANG_FACE0 + 2 * o0 + 1)) & 1u)) return true;
    if (b == 0 && ((h >> (HANG_FACE0 + 2 * o1)) & 1u)) return true;
    if (b == k && ((h >> (HANG_FACE0 + 2 * o1 + 1)) & 1u)) return true;
    if ((a == 0 || a == k) && (b == 0 || b == k)) {
        const int s0 = (a == k), s1 = (b == k);
        if ((h >> (HANG_EDGE0 + 4 * d + s0 + 2 * s1)) & 1u) return true;
    }
    return false;
}

// Does the slot idx[3] lie on a hanging face or edge (its value is then
// interpolated from the coarse neighbour)?
STOKES_HD bool slot_on_hanging_entity(uint32_t h, const int idx[3], int k) {
    for (int d = 0; d < 3; ++d) {
        if (idx[d] == 0 && ((h >> (HANG_FACE0 + 2 * d)) & 1u)) return true;
        if (idx[d] == k && ((h >> (HANG_FACE0 + 2 * d + 1)) & 1u)) return true;
    }
    for (int d = 0; d < 3; ++d) {
        const int o0 = (d == 0) ? 1 : 0, o1 = (d == 2) ? 1 : 2;
        const int a = idx[o0], b = idx[o1];
        if ((a == 0 || a == k) && (b == 0 || b == k)) {
            const int s0 = (a == k), s1 = (b == k);
            if ((h >> (HANG_EDGE0 + 4 * d + s0 + 2 * s1)) & 1u) return true;
        }
    }
    return false;
}

STOKES_HD int child_bit(uint32_t h, int d) { return int((h >> (HANG_CHILD0 + d)) & 1u); }

// Transposed hanging interpolation restricted to the bottom plane (zeta = -1)
// of an element, in place on v[i + n1 j] (host helper for the mesh builder).
// Forward order on the plane is x-sweeps then y-sweeps, so the transpose
// applies y^T then x^T.
inline void face_hanging_transpose_host(uint32_t h, const Tables1D& T, double* v) {
    const int k = T.k, n1 = T.n1;
    if ((h & ((1u << HANG_CHILD0) - 1)) == 0) return;
    double tmp[N1MAX];
    const int by = child_bit(h, 1), bx = child_bit(h, 0);
    for (int i = 0; i < n1; ++i) {             // lines parallel to y at (i, l = 0)
        if (!line_hanging(h, 1, i, 0, k)) continue;
        for (int m = 0; m < n1; ++m) {
            double s = 0;
            for (int j = 0; j < n1; ++j) s += T.I[by][j][m] * v[i + n1 * j];
            tmp[m] = s;
        }
        for (int m = 0; m < n1; ++m) v[i + n1 * m] = tmp[m];
    }
    for (int j = 0; j < n1; ++j) {             // lines parallel to x at (j, l = 0)
        if (!line_hanging(h, 0, j, 0, k)) continue;
        for (int m = 0; m < n1; ++m) {
            double s = 0;
            for (int i = 0; i < n1; ++i) s += T.I[bx][i][m] * v[i + n1 * j];
            tmp[m] = s;
        }
        for (int m = 0; m < n1; ++m) v[m + n1 * j] = tmp[m];
    }
}

}  // namespace stokes
