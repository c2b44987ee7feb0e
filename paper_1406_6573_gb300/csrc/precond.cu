// Column-block factorisation and solves of the velocity-block preconditioner
// (degree independent: the band width is a run-time value).
//
// Thin ice couples nodes far more strongly along a vertical column than across
// columns (element aspect ratios 6 to 100 in the paper's meshes, Sections 4.3
// and 7), so the velocity block is approximated by its vertical-column blocks,
// each a banded SPD matrix factored exactly (LU without pivoting).  One thread
// owns one column; band entries are stored column-interleaved so that the
// threads of a warp touch consecutive addresses (band_at).
#include <type_traits>

#include <cuda_runtime.h>

#include "kernels.h"
#include "precond.h"
#include "tma.cuh"

namespace stokes {
namespace {

template <typename T>
__device__ __forceinline__ T& band(T* A, int rows, int W, int bw, int r, int q, int64_t c) {
    return A[band_at(c, r, q - r + bw, W, rows)];
}

template <typename T>
__global__ void col_factor_kernel(ColSolveArgs a) {
    const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (c >= a.ncol) return;
    T* A = static_cast<T*>(a.A);
    const int bw = a.bw, W = 2 * bw + 1;
    const int n = 3 * a.col_len[c];
    const int b = a.col_basal[c];
    if (b >= 0) {
        // the lowest node of the column carries the nodal projector P:
        // K <- P K P + s (I - P) on its rows and columns
        const double* p6 = a.basal_P + 6 * int64_t(b);
        const T P[3][3] = {{T(p6[0]), T(p6[3]), T(p6[4])}, {T(p6[3]), T(p6[1]), T(p6[5])}, {T(p6[4]), T(p6[5]), T(p6[2])}};
        const int qmax = min(n - 1, 2 + bw);
        for (int q = 0; q <= qmax; ++q) {          // rows 0..2: P K
            T v[3];
            for (int r = 0; r < 3; ++r) v[r] = (q - r <= bw) ? band(A, 3 * a.colmax, W, bw, r, q, c) : T(0);
            for (int r = 0; r < 3; ++r)
                if (q - r <= bw) band(A, 3 * a.colmax, W, bw, r, q, c) = P[r][0] * v[0] + P[r][1] * v[1] + P[r][2] * v[2];
        }
        for (int r = 0; r <= qmax; ++r) {          // columns 0..2: K P
            T v[3];
            for (int q = 0; q < 3; ++q) v[q] = (r - q <= bw) ? band(A, 3 * a.colmax, W, bw, r, q, c) : T(0);
            for (int q = 0; q < 3; ++q)
                if (r - q <= bw) band(A, 3 * a.colmax, W, bw, r, q, c) = v[0] * P[0][q] + v[1] * P[1][q] + v[2] * P[2][q];
        }
        const T sc = T(a.scale);
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) band(A, 3 * a.colmax, W, bw, r, q, c) += sc * ((r == q ? T(1) : T(0)) - P[r][q]);
    }
    for (int p = 0; p < n; ++p) {
        const T piv = band(A, 3 * a.colmax, W, bw, p, p, c);
        const T ipiv = T(1) / piv;
        const int rmax = min(n - 1, p + bw);
        for (int r = p + 1; r <= rmax; ++r) {
            T& lrp = band(A, 3 * a.colmax, W, bw, r, p, c);
            const T l = lrp * ipiv;
            lrp = l;
            if (l != T(0))
                for (int q = p + 1; q <= rmax; ++q) band(A, 3 * a.colmax, W, bw, r, q, c) -= l * band(A, 3 * a.colmax, W, bw, p, q, c);
        }
        band(A, 3 * a.colmax, W, bw, p, p, c) = ipiv;   // the solves multiply by 1 / U[p][p]
    }
}

template <typename T>
__global__ void col_solve_kernel(ColSolveArgs a, const T* __restrict__ rhs, T* __restrict__ z) {
    extern __shared__ unsigned char smraw[];
    T* zc = reinterpret_cast<T*>(smraw);       // [3 colmax][blockDim.x]
    const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int nt = blockDim.x, t = threadIdx.x;
    if (c >= a.ncol) return;
    const T* A = static_cast<const T*>(a.A);
    const int bw = a.bw, W = 2 * bw + 1;
    const int len = a.col_len[c], n = 3 * len;
    for (int p = 0; p < len; ++p) {
        const int64_t g = a.col_nodes[int64_t(p) * a.ncol + c];
        for (int k = 0; k < 3; ++k) zc[(3 * p + k) * nt + t] = rhs[3 * g + k];
    }
    for (int r = 1; r < n; ++r) {                // L y = r (unit lower)
        T s = zc[r * nt + t];
        for (int q = max(0, r - bw); q < r; ++q) s -= A[band_at(c, r, q - r + bw, W, 3 * a.colmax)] * zc[q * nt + t];
        zc[r * nt + t] = s;
    }
    for (int r = n - 1; r >= 0; --r) {           // U x = y
        T s = zc[r * nt + t];
        const int qmax = min(n - 1, r + bw);
        for (int q = r + 1; q <= qmax; ++q) s -= A[band_at(c, r, q - r + bw, W, 3 * a.colmax)] * zc[q * nt + t];
        zc[r * nt + t] = s * A[band_at(c, r, bw, W, 3 * a.colmax)];
    }
    const T oa = T(a.out_alpha), ob = T(a.out_beta);
    for (int p = 0; p < len; ++p) {
        const int64_t g = a.col_nodes[int64_t(p) * a.ncol + c];
        for (int k = 0; k < 3; ++k) {
            const T v = oa * zc[(3 * p + k) * nt + t];
            z[3 * g + k] = ob != T(0) ? ob * z[3 * g + k] + v : v;
        }
    }
}

// The same solve with the band width fixed at compile time.  The band entries
// of a row are loaded CS_AHEAD rows before they are used (a ring of
// CS_AHEAD + 1 rows in registers, the row loop unrolled by the ring length so
// that every ring index is known at compile time): one thread per column
// would otherwise keep a single row of loads in flight, too few bytes per SM
// to cover the DRAM latency of the 227 MB band of the 128x128x8 Q2 slab.
// The arithmetic is the same, in the same order, as in col_solve_kernel.
#ifndef CS_AHEAD
#define CS_AHEAD 3
#endif
template <typename T, int BW>
__global__ void col_solve_band_kernel(ColSolveArgs a, const T* __restrict__ rhs, T* __restrict__ z) {
    extern __shared__ unsigned char smraw[];
    T* zc = reinterpret_cast<T*>(smraw);       // [3 colmax][blockDim.x]
    const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int nt = blockDim.x, t = threadIdx.x;
    if (c >= a.ncol) return;
    constexpr int W = 2 * BW + 1;
    constexpr int R = CS_AHEAD + 1;
    const int64_t ncol = a.ncol;
    const T* A = static_cast<const T*>(a.A) + band_at(c, 0, 0, W, 3 * a.colmax);
    const int len = a.col_len[c], n = 3 * len;
    for (int p = 0; p < len; ++p) {
        const int64_t g = a.col_nodes[int64_t(p) * ncol + c];
        for (int k = 0; k < 3; ++k) zc[(3 * p + k) * nt + t] = rhs[3 * g + k];
    }
    if (n == 0) return;
    auto row = [&](int r) { return A + int64_t(r) * W * BAND_CB; };
    // L y = r (unit lower): row r holds L[r][r - d] at band slot BW - d;
    // row r lives in ring slot r mod R
    T L[R][BW];
    auto loadL = [&](int r, T (&dst)[BW]) {
        #pragma unroll
        for (int d = 1; d <= BW; ++d) dst[d - 1] = (r < n && r - d >= 0) ? row(r)[(BW - d) * BAND_CB] : T(0);
    };
    #pragma unroll
    for (int u = 1; u < R; ++u) loadL(u, L[u]);
    for (int r0 = 0; r0 < n; r0 += R) {
        #pragma unroll
        for (int u = 0; u < R; ++u) {
            const int r = r0 + u;
            if (r >= 1 && r < n) {
                loadL(r + R - 1, L[(u + R - 1) % R]);   // into the slot of row r - 1
                T s = zc[r * nt + t];
                #pragma unroll
                for (int d = 1; d <= BW; ++d)
                    if (r - d >= 0) s -= L[u][d - 1] * zc[(r - d) * nt + t];
                zc[r * nt + t] = s;
            }
        }
    }
    // U x = y: row r holds 1 / U[r][r] at slot BW and U[r][r + d] at slot BW + d;
    // row n - 1 - i lives in ring slot i mod R
    T U[R][BW + 1];
    auto loadU = [&](int r, T (&dst)[BW + 1]) {
        #pragma unroll
        for (int d = 0; d <= BW; ++d) dst[d] = (r >= 0 && r + d < n) ? row(r)[(BW + d) * BAND_CB] : T(0);
    };
    #pragma unroll
    for (int u = 0; u < R - 1; ++u) loadU(n - 1 - u, U[u]);
    for (int i0 = 0; i0 < n; i0 += R) {
        #pragma unroll
        for (int u = 0; u < R; ++u) {
            const int r = n - 1 - (i0 + u);
            if (r >= 0) {
                loadU(r - (R - 1), U[(u + R - 1) % R]);   // into the slot of row r + 1
                T s = zc[r * nt + t];
                #pragma unroll
                for (int d = 1; d <= BW; ++d)
                    if (r + d < n) s -= U[u][d] * zc[(r + d) * nt + t];
                zc[r * nt + t] = s * U[u][0];
            }
        }
    }
    const T oa = T(a.out_alpha), ob = T(a.out_beta);
    for (int p = 0; p < len; ++p) {
        const int64_t g = a.col_nodes[int64_t(p) * ncol + c];
        for (int k = 0; k < 3; ++k) {
            const T v = oa * zc[(3 * p + k) * nt + t];
            z[3 * g + k] = ob != T(0) ? ob * z[3 * g + k] + v : v;
        }
    }
}

// Shared-memory variants for one band block (BAND_CB columns, one warp, one
// thread per column): the whole block (rows x W x BAND_CB values, contiguous
// in the band layout) is staged by bulk asynchronous copies (TMA,
// cp.async.bulk) on an mbarrier.  The factorisation then updates shared
// memory instead of global memory (the global version's dependent
// read-modify-writes took about 0.4 ms per launch at every size) and writes
// the block back; the solve has every band entry in shared memory before its
// sequential sweeps (the global version, latency-bound on its band loads,
// took about 52 us per launch on the small levels of the multigrid).  The
// factorisation's arithmetic is that of col_factor_kernel, in the same order;
// the solve sums each row's band terms from the farthest to the nearest row.
constexpr uint32_t STAGE_CHUNK = 32768;

// lane 0 stages nbytes from src into dst; false (status word set, the copies
// drained) if the copy does not arrive within the poll limit
__device__ __forceinline__ bool stage_band_block(void* dst, const void* src, uint32_t nbytes, uint64_t* bar,
                                                 int* err) {
    using namespace dev;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(bar, nbytes);
        for (uint32_t o = 0; o < nbytes; o += STAGE_CHUNK) {
            const uint32_t len = nbytes - o < STAGE_CHUNK ? nbytes - o : STAGE_CHUNK;
            bulk_g2s(static_cast<unsigned char*>(dst) + o, static_cast<const unsigned char*>(src) + o, len, bar);
        }
    }
    __syncwarp();
    if (mbar_wait_polls(bar, 0, WAIT_POLLS_DEFAULT)) return true;
    if (threadIdx.x == 0 && err) atomicOr(err, 1);
    mbar_wait_bounded(bar, 0);
    return false;
}

template <typename T, int BW>
__global__ void __launch_bounds__(BAND_CB) col_factor_smem_kernel(ColSolveArgs a) {
    extern __shared__ __align__(128) unsigned char smraw[];
    constexpr int W = 2 * BW + 1;
    const int rows = 3 * a.colmax, lane = threadIdx.x;
    const int64_t nval = int64_t(rows) * W * BAND_CB;
    T* S = reinterpret_cast<T*>(smraw);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + nval * sizeof(T));
    T* G = static_cast<T*>(a.A) + int64_t(blockIdx.x) * nval;
    if (!stage_band_block(S, G, uint32_t(nval * sizeof(T)), bar, a.err)) return;
    const int64_t c = int64_t(blockIdx.x) * BAND_CB + lane;
    auto at = [&](int r, int q) -> T& { return S[(r * W + (q - r + BW)) * BAND_CB + lane]; };
    if (c < a.ncol) {
        const int n = 3 * a.col_len[c];
        const int b = a.col_basal[c];
        if (b >= 0) {
            const double* p6 = a.basal_P + 6 * int64_t(b);
            const T P[3][3] = {{T(p6[0]), T(p6[3]), T(p6[4])}, {T(p6[3]), T(p6[1]), T(p6[5])}, {T(p6[4]), T(p6[5]), T(p6[2])}};
            const int qmax = min(n - 1, 2 + BW);
            for (int q = 0; q <= qmax; ++q) {          // rows 0..2: P K
                T v[3];
                for (int r = 0; r < 3; ++r) v[r] = (q - r <= BW) ? at(r, q) : T(0);
                for (int r = 0; r < 3; ++r)
                    if (q - r <= BW) at(r, q) = P[r][0] * v[0] + P[r][1] * v[1] + P[r][2] * v[2];
            }
            for (int r = 0; r <= qmax; ++r) {          // columns 0..2: K P
                T v[3];
                for (int q = 0; q < 3; ++q) v[q] = (r - q <= BW) ? at(r, q) : T(0);
                for (int q = 0; q < 3; ++q)
                    if (r - q <= BW) at(r, q) = v[0] * P[0][q] + v[1] * P[1][q] + v[2] * P[2][q];
            }
            const T sc = T(a.scale);
            for (int r = 0; r < 3; ++r)
                for (int q = 0; q < 3; ++q) at(r, q) += sc * ((r == q ? T(1) : T(0)) - P[r][q]);
        }
        for (int p = 0; p < n; ++p) {
            const T ipiv = T(1) / at(p, p);
            T prow[BW];                                 // U[p][p + 1 .. p + BW]
            #pragma unroll
            for (int d = 1; d <= BW; ++d) prow[d - 1] = p + d < n ? at(p, p + d) : T(0);
            #pragma unroll
            for (int dr = 1; dr <= BW; ++dr) {
                const int r = p + dr;
                if (r >= n) break;
                T& lrp = at(r, p);
                const T l = lrp * ipiv;
                lrp = l;
                if (l != T(0)) {
                    #pragma unroll
                    for (int dq = 1; dq <= BW; ++dq)
                        if (p + dq < n) at(r, p + dq) -= l * prow[dq - 1];
                }
            }
            at(p, p) = ipiv;                            // the solves multiply by 1 / U[p][p]
        }
    }
    __syncwarp();
    const int64_t n16 = nval * int64_t(sizeof(T)) / 16;
    const uint4* s16 = reinterpret_cast<const uint4*>(S);
    uint4* g16 = reinterpret_cast<uint4*>(G);
    for (int64_t i = lane; i < n16; i += BAND_CB) g16[i] = s16[i];
}

template <typename T, int BW>
__global__ void __launch_bounds__(BAND_CB) col_solve_smem_kernel(ColSolveArgs a, const T* __restrict__ rhs,
                                                                 T* __restrict__ z) {
    extern __shared__ __align__(128) unsigned char smraw[];
    constexpr int W = 2 * BW + 1;
    const int rows = 3 * a.colmax, lane = threadIdx.x;
    const int64_t nval = int64_t(rows) * W * BAND_CB;
    T* S = reinterpret_cast<T*>(smraw);
    T* zc = S + nval;                                   // [rows][BAND_CB]
    uint64_t* bar = reinterpret_cast<uint64_t*>(zc + int64_t(rows) * BAND_CB);
    const T* G = static_cast<const T*>(a.A) + int64_t(blockIdx.x) * nval;
    const int64_t c = int64_t(blockIdx.x) * BAND_CB + lane;
    const int64_t ncol = a.ncol;
    // the band copy is issued first; the right-hand side is gathered while it lands
    {
        using namespace dev;
        if (lane == 0) {
            mbar_init(bar, 1);
            fence_mbar_init();
            const uint32_t nbytes = uint32_t(nval * sizeof(T));
            mbar_arrive_expect_tx(bar, nbytes);
            for (uint32_t o = 0; o < nbytes; o += STAGE_CHUNK) {
                const uint32_t len = nbytes - o < STAGE_CHUNK ? nbytes - o : STAGE_CHUNK;
                bulk_g2s(reinterpret_cast<unsigned char*>(S) + o, reinterpret_cast<const unsigned char*>(G) + o, len,
                         bar);
            }
        }
    }
    const int len = c < ncol ? a.col_len[c] : 0, n = 3 * len;
    // node indices, then the right-hand side: two rounds of independent loads
    int32_t* gidx = reinterpret_cast<int32_t*>(bar + 2);   // [colmax][BAND_CB]
    #pragma unroll 8
    for (int p = 0; p < len; ++p) gidx[p * BAND_CB + lane] = a.col_nodes[int64_t(p) * ncol + c];
    #pragma unroll 4
    for (int p = 0; p < len; ++p) {
        const int64_t g = gidx[p * BAND_CB + lane];
        #pragma unroll
        for (int k = 0; k < 3; ++k) zc[(3 * p + k) * BAND_CB + lane] = rhs[3 * g + k];
    }
    __syncwarp();
    if (!dev::mbar_wait_polls(bar, 0, WAIT_POLLS_DEFAULT)) {
        if (lane == 0 && a.err) atomicOr(a.err, 1);
        dev::mbar_wait_bounded(bar, 0);
        return;
    }
    auto A = [&](int r, int slot) { return S[(r * W + slot) * BAND_CB + lane]; };
    // the last BW + 1 solution values in a register ring (slot: row mod RING);
    // the term of the previous row is subtracted last, so that one FMA per row
    // waits on it
    constexpr int RING = BW + 1;
    T zr[RING];
    // L y = r (unit lower): L[r][r - d] at band slot BW - d
    for (int r0 = 0; r0 < n; r0 += RING) {
        #pragma unroll
        for (int u = 0; u < RING; ++u) {
            const int r = r0 + u;
            if (r < n) {
                T s = zc[r * BAND_CB + lane];
                #pragma unroll
                for (int d = BW; d >= 1; --d)
                    if (r - d >= 0) s -= A(r, BW - d) * zr[(u - d + RING) % RING];
                zr[u] = s;
                zc[r * BAND_CB + lane] = s;
            }
        }
    }
    // U x = y: 1 / U[r][r] at slot BW, U[r][r + d] at slot BW + d (ring slot:
    // (n - 1 - r) mod RING)
    for (int i0 = 0; i0 < n; i0 += RING) {
        #pragma unroll
        for (int u = 0; u < RING; ++u) {
            const int r = n - 1 - (i0 + u);
            if (r >= 0) {
                T s = zc[r * BAND_CB + lane];
                #pragma unroll
                for (int d = BW; d >= 1; --d)
                    if (r + d < n) s -= A(r, BW + d) * zr[(u - d + RING) % RING];
                s *= A(r, BW);
                zr[u] = s;
                zc[r * BAND_CB + lane] = s;
            }
        }
    }
    const T oa = T(a.out_alpha), ob = T(a.out_beta);
    for (int p = 0; p < len; ++p) {
        const int64_t g = gidx[p * BAND_CB + lane];
        #pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T v = oa * zc[(3 * p + k) * BAND_CB + lane];
            z[3 * g + k] = ob != T(0) ? ob * z[3 * g + k] + v : v;
        }
    }
}

// z_p(e) = -minv(e) r_p(e): one thread per pressure dof (e, b); with full
// blocks minv holds npr x npr per element, otherwise one inverse diagonal
// entry per dof
template <typename T>
__global__ void schur_apply_kernel(int64_t Nv, int64_t E, int npr, int full, const T* __restrict__ minv,
                                   const T* __restrict__ r, T* __restrict__ z) {
    const int64_t np = E * npr;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < np; t += int64_t(gridDim.x) * blockDim.x) {
        if (!full) {
            z[3 * Nv + t] = -minv[t] * r[3 * Nv + t];
            continue;
        }
        const int64_t e = t / npr;
        const int b = int(t - e * npr);
        const T* row = minv + (e * npr + b) * npr;
        const T* re = r + 3 * Nv + e * npr;
        T s = 0;
        for (int c = 0; c < npr; ++c) s += row[c] * re[c];
        z[3 * Nv + t] = -s;
    }
}

// inverse diagonal of each element block: minv[e npr + b] = 1 / m[e][b][b]
template <typename T>
__global__ void schur_invert_diag_kernel(int64_t E, int npr, const double* __restrict__ m, T* __restrict__ minv) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= E * npr) return;
    const int64_t e = t / npr;
    const int b = int(t - e * npr);
    minv[t] = T(1.0 / m[(e * npr + b) * npr + b]);
}

// inverse of each SPD element block (Gauss-Jordan without pivoting, FP64, in
// place on the block), stored in T; one thread per element
template <typename T>
__global__ void schur_invert_kernel(int64_t E, int npr, double* __restrict__ m, T* __restrict__ minv) {
    const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= E) return;
    double* A = m + e * npr * npr;
    for (int p = 0; p < npr; ++p) {
        const double piv = 1.0 / A[p * npr + p];
        for (int c = 0; c < npr; ++c) A[p * npr + c] *= (c == p ? 1.0 : piv);
        A[p * npr + p] = piv;
        for (int r = 0; r < npr; ++r) {
            if (r == p) continue;
            const double f = A[r * npr + p];
            if (f == 0.0) continue;
            for (int c = 0; c < npr; ++c) A[r * npr + c] -= (c == p ? 0.0 : f * A[p * npr + c]);
            A[r * npr + p] = -f * piv;
        }
    }
    T* out = minv + e * npr * npr;
    for (int i = 0; i < npr * npr; ++i) out[i] = T(A[i]);
}

// mean |diagonal| of the assembled (unconstrained) column blocks
template <typename T>
__global__ void col_diag_kernel(ColSolveArgs a, double* out) {
    __shared__ double red[8];
    const int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    double s = 0;
    if (c < a.ncol) {
        const T* A = static_cast<const T*>(a.A);
        const int W = 2 * a.bw + 1, n = 3 * a.col_len[c];
        for (int r = 0; r < n; ++r) s += fabs(double(A[band_at(c, r, a.bw, W, 3 * a.colmax)]));
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(out, t);
    }
}

int solve_threads(int colmax, int bytes) {
    int nt = 128;
    while (nt > 32 && int64_t(3) * colmax * nt * bytes > 96 * 1024) nt /= 2;
    return nt;
}

}  // namespace

namespace {

// largest dynamic shared memory a block may opt in to on the current device
int smem_optin() {
    static int cached_dev = -1, val = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev != cached_dev) {
        if (cudaDeviceGetAttribute(&val, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) val = 0;
        cached_dev = dev;
    }
    return val;
}

// raise a kernel's dynamic shared-memory limit to the opt-in maximum (once per device)
template <typename K>
cudaError_t allow_smem(K kernel) {
    static int done_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev == done_dev) return e;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin());
    if (e == cudaSuccess) done_dev = dev;
    return e;
}

template <typename T>
size_t band_block_bytes(const ColSolveArgs& a) {
    return size_t(3) * a.colmax * size_t(2 * a.bw + 1) * BAND_CB * sizeof(T);
}

// the shared-memory solve runs where the levels are latency-bound (at most one
// wave of band blocks, one 32-thread block per SM at these block sizes);
// above that the register-ring kernel streams the band at a higher rate
// (16384 columns of the Q2 slab: 78 us in 3.4 waves against 55 us)
int64_t smem_solve_max_cols() {
    static int cached_dev = -1, sms = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (dev != cached_dev) {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 0;
        cached_dev = dev;
    }
    return int64_t(sms) * BAND_CB;
}

template <typename T, int BW>
cudaError_t factor_smem(const ColSolveArgs& a, size_t bytes, cudaStream_t s) {
    cudaError_t e = allow_smem(col_factor_smem_kernel<T, BW>);
    if (e != cudaSuccess) return e;
    col_factor_smem_kernel<T, BW><<<unsigned(band_cols(a.ncol) / BAND_CB), BAND_CB, bytes, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int BW>
cudaError_t solve_smem(const ColSolveArgs& a, size_t bytes, const void* r, void* z, cudaStream_t s) {
    cudaError_t e = allow_smem(col_solve_smem_kernel<T, BW>);
    if (e != cudaSuccess) return e;
    col_solve_smem_kernel<T, BW><<<unsigned(band_cols(a.ncol) / BAND_CB), BAND_CB, bytes, s>>>(
        a, static_cast<const T*>(r), static_cast<T*>(z));
    return cudaGetLastError();
}

// a shared-memory launch that the device refuses (its limit, less a margin
// for the block's reserved shared memory, is checked first) falls back to the
// global-memory kernels
constexpr size_t SMEM_MARGIN = 1024;

template <typename T>
int col_factor_t(const ColSolveArgs& a, cudaStream_t s) {
    const size_t bytes = band_block_bytes<T>(a) + 16;
    if (bytes + SMEM_MARGIN <= size_t(smem_optin())) {
        cudaError_t e = cudaErrorInvalidValue;
        switch (a.bw) {
            case 8: e = factor_smem<T, 8>(a, bytes, s); break;
            case 11: e = factor_smem<T, 11>(a, bytes, s); break;
            case 14: e = factor_smem<T, 14>(a, bytes, s); break;
            default: break;
        }
        if (e == cudaSuccess) return 0;
        (void)cudaGetLastError();
    }
    const unsigned blocks = unsigned((a.ncol + 127) / 128);
    col_factor_kernel<T><<<blocks, 128, 0, s>>>(a);
    return int(cudaGetLastError());
}

template <typename T>
int col_solve_smem_t(const ColSolveArgs& a, const void* r, void* z, cudaStream_t s, bool& done) {
    done = false;
    const size_t bytes = band_block_bytes<T>(a) + size_t(3) * a.colmax * BAND_CB * sizeof(T) + 16 +
                         size_t(a.colmax) * BAND_CB * 4;
    if (a.ncol > smem_solve_max_cols() || bytes + SMEM_MARGIN > size_t(smem_optin())) return 0;
    cudaError_t e = cudaSuccess;
    switch (a.bw) {
        case 8: e = solve_smem<T, 8>(a, bytes, r, z, s); break;
        case 11: e = solve_smem<T, 11>(a, bytes, r, z, s); break;
        case 14: e = solve_smem<T, 14>(a, bytes, r, z, s); break;
        default: return 0;
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return 0;
    }
    done = true;
    return 0;
}

}  // namespace

int launch_col_factor(int prec, const ColSolveArgs& a, cudaStream_t s) {
    if (a.ncol == 0) return 0;
    return prec == 1 ? col_factor_t<float>(a, s) : col_factor_t<double>(a, s);
}

int launch_col_diag_sum(int prec, const ColSolveArgs& a, double* out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
    if (e != cudaSuccess) return int(e);
    if (a.ncol == 0) return 0;
    const unsigned blocks = unsigned((a.ncol + 255) / 256);
    if (prec == 1) col_diag_kernel<float><<<blocks, 256, 0, s>>>(a, out);
    else col_diag_kernel<double><<<blocks, 256, 0, s>>>(a, out);
    return int(cudaGetLastError());
}

int launch_col_solve(int prec, const ColSolveArgs& a, const void* r, void* z, cudaStream_t s) {
    if (a.ncol == 0) return 0;
    {
        bool done = false;
        const int rc = prec == 1 ? col_solve_smem_t<float>(a, r, z, s, done) : col_solve_smem_t<double>(a, r, z, s, done);
        if (done || rc) return rc;
    }
    const int bytes = prec == 1 ? 4 : 8;
    const int nt = solve_threads(a.colmax, bytes);
    const size_t sm = size_t(3) * a.colmax * nt * bytes;
    const unsigned blocks = unsigned((a.ncol + nt - 1) / nt);
    auto run = [&](auto kernel, auto* tag) -> cudaError_t {
        using T = std::remove_pointer_t<decltype(tag)>;
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        if (e != cudaSuccess) return e;
        kernel<<<blocks, nt, sm, s>>>(a, static_cast<const T*>(r), static_cast<T*>(z));
        return cudaSuccess;
    };
    cudaError_t e;
    // band widths 3k + 2 of the degrees 2, 3, 4 (bnode = k) run the fixed-band kernel
    if (prec == 1) {
        float* tag = nullptr;
        switch (a.bw) {
            case 8: e = run(col_solve_band_kernel<float, 8>, tag); break;
            case 11: e = run(col_solve_band_kernel<float, 11>, tag); break;
            case 14: e = run(col_solve_band_kernel<float, 14>, tag); break;
            default: e = run(col_solve_kernel<float>, tag);
        }
    } else {
        double* tag = nullptr;
        switch (a.bw) {
            case 8: e = run(col_solve_band_kernel<double, 8>, tag); break;
            case 11: e = run(col_solve_band_kernel<double, 11>, tag); break;
            case 14: e = run(col_solve_band_kernel<double, 14>, tag); break;
            default: e = run(col_solve_kernel<double>, tag);
        }
    }
    if (e != cudaSuccess) return int(e);
    return int(cudaGetLastError());
}

int launch_schur_invert(int prec, int64_t E, int npr, int full, const double* mblk, void* minv, cudaStream_t s) {
    if (E == 0 || npr == 0) return 0;
    double* m = const_cast<double*>(mblk);
    if (full) {
        const unsigned blocks = unsigned((E + 127) / 128);
        if (prec == 1) schur_invert_kernel<float><<<blocks, 128, 0, s>>>(E, npr, m, static_cast<float*>(minv));
        else schur_invert_kernel<double><<<blocks, 128, 0, s>>>(E, npr, m, static_cast<double*>(minv));
    } else {
        const unsigned blocks = unsigned((E * npr + 255) / 256);
        if (prec == 1) schur_invert_diag_kernel<float><<<blocks, 256, 0, s>>>(E, npr, m, static_cast<float*>(minv));
        else schur_invert_diag_kernel<double><<<blocks, 256, 0, s>>>(E, npr, m, static_cast<double*>(minv));
    }
    return int(cudaGetLastError());
}

int launch_schur_apply(int prec, int64_t Nv, int64_t E, int npr, int full, const void* minv, const void* r,
                       void* z, cudaStream_t s) {
    const int64_t np = E * npr;
    if (np == 0) return 0;
    int64_t blocks = (np + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (prec == 1)
        schur_apply_kernel<float><<<unsigned(blocks), 256, 0, s>>>(Nv, E, npr, full, static_cast<const float*>(minv),
                                                                   static_cast<const float*>(r), static_cast<float*>(z));
    else
        schur_apply_kernel<double><<<unsigned(blocks), 256, 0, s>>>(Nv, E, npr, full, static_cast<const double*>(minv),
                                                                    static_cast<const double*>(r), static_cast<double*>(z));
    return int(cudaGetLastError());
}

}  // namespace stokes
