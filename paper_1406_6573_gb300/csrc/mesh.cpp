// Host mesh builder: element list, global node numbering, hanging-node codes,
// isoparametric geometry at the quadrature points, basal faces and nodal
// constraint projectors.
//
// Section 3.1 (meshing): a forest of hexahedra with 2:1 balance; here a
// coarse nx x ny x nz grid (periodic in x and y for the slab workloads) in
// which cells may be split once into 8 children, so 2:1 balance holds by
// construction.  Children inherit the parent's isoparametric map.
// Section 3.2.1: global nodes are the non-hanging element nodes; element
// values at hanging nodes are interpolated from the coarse neighbour by the
// restriction R_i.  R_i is stored in factored form: every local slot of an
// element names one global node (for a slot on a hanging face or edge: the
// node of the parent cell's GLL lattice at the same slot, which lies on the
// coarse neighbour), and a per-element code lists the hanging faces and
// edges, so that R_i = (1-D interpolation along each constrained line) o
// (gather).  The kernels apply it with the same 1-D contractions as the
// operator (Section 3.3).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "common.h"
#include "hanging.h"

namespace stokes {
namespace {

constexpr double KEYSCALE = 67108864.0;  // 2^26: positions are exact binary fractions of it

struct Key {
    int64_t z, y, x;
    bool operator<(const Key& o) const {
        if (z != o.z) return z < o.z;
        if (y != o.y) return y < o.y;
        return x < o.x;
    }
    bool operator==(const Key& o) const { return z == o.z && y == o.y && x == o.x; }
};

struct Builder {
    const stokes_mesh_desc& d;
    HostMesh& m;
    std::vector<uint8_t> refine;
    std::vector<int32_t> cell;     // coarse cell of each element
    std::vector<int8_t> child;     // child index 0..7, or -1
    double t[N1MAX];               // (xi_i + 1) / 2
    int64_t kx_wrap = 0, ky_wrap = 0;

    Builder(const stokes_mesh_desc& d_, HostMesh& m_) : d(d_), m(m_) {}

    int ncoarse() const { return m.nx * m.ny * m.nz; }

    bool coarse_unrefined(int cx, int cy, int cz) const {
        if (cz < 0 || cz >= m.nz) return false;
        if (m.periodic) {
            cx = ((cx % m.nx) + m.nx) % m.nx;
            cy = ((cy % m.ny) + m.ny) % m.ny;
        } else if (cx < 0 || cx >= m.nx || cy < 0 || cy >= m.ny) {
            return false;
        }
        return !refine[cx + m.nx * (cy + m.ny * cz)];
    }

    // reference position of local slot idx along one axis
    double own_pos(int c, int b, int idx) const {
        if (b < 0) return double(c) + t[idx];
        return (double(c) + 0.5 * b) + 0.5 * t[idx];
    }

    Key make_key(double X, double Y, double Z) const {
        Key k;
        k.x = std::llround(X * KEYSCALE);
        k.y = std::llround(Y * KEYSCALE);
        k.z = std::llround(Z * KEYSCALE);
        if (m.periodic) {
            k.x = ((k.x % kx_wrap) + kx_wrap) % kx_wrap;
            k.y = ((k.y % ky_wrap) + ky_wrap) % ky_wrap;
        }
        return k;
    }

    uint32_t hang_code(int e) const {
        int ch = child[e];
        if (ch < 0) return 0;
        int c = cell[e];
        int cc[3] = {c % m.nx, (c / m.nx) % m.ny, c / (m.nx * m.ny)};
        int b[3] = {ch & 1, (ch >> 1) & 1, (ch >> 2) & 1};
        uint32_t h = 0;
        for (int a = 0; a < 3; ++a) h |= uint32_t(b[a]) << (HANG_CHILD0 + a);
        for (int a = 0; a < 3; ++a) {
            for (int s = 0; s < 2; ++s) {
                if (b[a] != s) continue;          // face not on the parent boundary
                int o[3] = {cc[0], cc[1], cc[2]};
                o[a] += s ? 1 : -1;
                if (coarse_unrefined(o[0], o[1], o[2])) h |= 1u << (HANG_FACE0 + 2 * a + s);
            }
        }
        for (int a = 0; a < 3; ++a) {             // edges parallel to axis a
            int o0 = (a == 0) ? 1 : 0, o1 = (a == 2) ? 1 : 2;
            for (int s1 = 0; s1 < 2; ++s1)
                for (int s0 = 0; s0 < 2; ++s0) {
                    if (b[o0] != s0 || b[o1] != s1) continue;  // not on a parent edge
                    int d0 = s0 ? 1 : -1, d1 = s1 ? 1 : -1;
                    bool hang = false;
                    for (int w = 1; w < 4 && !hang; ++w) {
                        int o[3] = {cc[0], cc[1], cc[2]};
                        if (w & 1) o[o0] += d0;
                        if (w & 2) o[o1] += d1;
                        hang = coarse_unrefined(o[0], o[1], o[2]);
                    }
                    if (hang) h |= 1u << (HANG_EDGE0 + 4 * a + s0 + 2 * s1);
                }
        }
        return h;
    }
};

inline int slot(int n1, int i, int j, int l) { return i + n1 * (j + n1 * l); }

}  // namespace

int build_host_mesh(const stokes_mesh_desc& d, HostMesh& m, std::string& err) {
    if (d.nx < 1 || d.ny < 1 || d.nz < 1) { err = "grid sizes must be >= 1"; return STOKES_E_INVAL; }
    if (d.k < 1 || d.k > KMAX) { err = "velocity degree k must be in 1..9"; return STOKES_E_INVAL; }
    if (d.pressure_space != STOKES_PRESSURE_P && d.pressure_space != STOKES_PRESSURE_Q) {
        err = "unknown pressure space"; return STOKES_E_INVAL;
    }
    if (d.pressure_space == STOKES_PRESSURE_Q && d.k < 2) {
        err = "Q_{k-2} pressure needs k >= 2"; return STOKES_E_INVAL;
    }
    if (d.basal_bc != STOKES_BASE_NOSLIP && d.basal_bc != STOKES_BASE_SLIP) {
        err = "unknown basal condition"; return STOKES_E_INVAL;
    }
    if (!(d.Lx > 0) || !(d.Ly > 0)) { err = "Lx and Ly must be positive"; return STOKES_E_INVAL; }
    if ((d.bed.n_modes > 0 && (!d.bed.amp || !d.bed.kx || !d.bed.ky || !d.bed.phase)) ||
        (d.surface.n_modes > 0 && (!d.surface.amp || !d.surface.kx || !d.surface.ky || !d.surface.phase))) {
        err = "field with modes but NULL coefficient arrays"; return STOKES_E_INVAL;
    }
    if ((d.bed_nodes == nullptr) != (d.surface_nodes == nullptr)) {
        err = "bed_nodes and surface_nodes must be given together"; return STOKES_E_INVAL;
    }
    const int64_t ncoarse = int64_t(d.nx) * d.ny * d.nz;
    if (ncoarse > (int64_t(1) << 31) / 8) { err = "grid too large"; return STOKES_E_INVAL; }

    m.nx = d.nx; m.ny = d.ny; m.nz = d.nz; m.k = d.k; m.n1 = d.k + 1; m.q = d.k + 1;
    m.pspace = d.pressure_space; m.periodic = d.periodic_xy != 0;
    m.Lx = d.Lx; m.Ly = d.Ly; m.basal_bc = d.basal_bc;
    build_tables(m.k, m.pspace, m.tab);
    m.npr = m.tab.npr;
    const int k = m.k, n1 = m.n1, q = m.q, A = n1 * n1 * n1, Q3 = q * q * q, Q2 = q * q;

    Builder B(d, m);
    B.kx_wrap = int64_t(std::llround(m.nx * KEYSCALE));
    B.ky_wrap = int64_t(std::llround(m.ny * KEYSCALE));
    for (int i = 0; i < n1; ++i) B.t[i] = 0.5 * (m.tab.gll[i] + 1.0);
    B.refine.assign(ncoarse, 0);
    bool any_refine_input = d.refine != nullptr;
    if (d.refine) for (int64_t c = 0; c < ncoarse; ++c) B.refine[c] = d.refine[c] ? 1 : 0;

    // ---------------------------------------------------------------- cells
    for (int64_t c = 0; c < ncoarse; ++c) {
        if (!B.refine[c]) { B.cell.push_back(int32_t(c)); B.child.push_back(-1); }
        else for (int ch = 0; ch < 8; ++ch) { B.cell.push_back(int32_t(c)); B.child.push_back(int8_t(ch)); }
    }
    const int64_t E = int64_t(B.cell.size());
    m.E = E;
    m.Np = E * m.npr;
    m.elem_hang.resize(E);
    m.n_hang = 0;
    for (int64_t e = 0; e < E; ++e) {
        m.elem_hang[e] = B.hang_code(int(e));
        if (m.elem_hang[e] & ((1u << HANG_CHILD0) - 1)) ++m.n_hang;
    }

    // ------------------------------------------------------- node numbering
    m.elem_nodes.assign(size_t(E) * A, -1);
    auto cell_xyz = [&](int64_t e, int cc[3], int b[3]) {
        int c = B.cell[e];
        cc[0] = c % m.nx; cc[1] = (c / m.nx) % m.ny; cc[2] = c / (m.nx * m.ny);
        int ch = B.child[e];
        for (int a = 0; a < 3; ++a) b[a] = ch < 0 ? -1 : ((ch >> a) & 1);
    };
    if (!any_refine_input) {
        // conforming lattice: node (I, J, L) -> I + NX (J + NY L), which is the
        // (Z, Y, X) order of the reference positions
        const int64_t NX = m.periodic ? int64_t(m.nx) * k : int64_t(m.nx) * k + 1;
        const int64_t NY = m.periodic ? int64_t(m.ny) * k : int64_t(m.ny) * k + 1;
        const int64_t NZ = int64_t(m.nz) * k + 1;
        m.Nv = NX * NY * NZ;
        m.lattice = true;
        m.latNX = NX;
        m.latNY = NY;
        #pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < E; ++e) {
            int cc[3], b[3];
            cell_xyz(e, cc, b);
            for (int l = 0; l < n1; ++l)
                for (int j = 0; j < n1; ++j)
                    for (int i = 0; i < n1; ++i) {
                        int64_t I = int64_t(cc[0]) * k + i, J = int64_t(cc[1]) * k + j;
                        int64_t L = int64_t(cc[2]) * k + l;
                        if (m.periodic) { I %= NX; J %= NY; }
                        m.elem_nodes[size_t(e) * A + slot(n1, i, j, l)] = int32_t(I + NX * (J + NY * L));
                    }
        }
        if (m.Nv >= (int64_t(1) << 31)) { err = "too many nodes"; return STOKES_E_INVAL; }
        m.ncol = NX * NY;
        m.col_of.resize(size_t(m.Nv));
        m.pos_of.resize(size_t(m.Nv));
        for (int64_t g = 0; g < m.Nv; ++g) { m.col_of[g] = int32_t(g % m.ncol); m.pos_of[g] = int32_t(g / m.ncol); }
    } else {
        std::vector<Key> keys;
        keys.reserve(size_t(E) * A);
        std::vector<uint8_t> hanging_slot(size_t(E) * A, 0);
        for (int64_t e = 0; e < E; ++e) {
            int cc[3], b[3];
            cell_xyz(e, cc, b);
            uint32_t h = m.elem_hang[e];
            for (int l = 0; l < n1; ++l)
                for (int j = 0; j < n1; ++j)
                    for (int i = 0; i < n1; ++i) {
                        int idx[3] = {i, j, l};
                        bool hs = slot_on_hanging_entity(h, idx, k);
                        hanging_slot[size_t(e) * A + slot(n1, i, j, l)] = hs;
                        if (!hs)
                            keys.push_back(B.make_key(B.own_pos(cc[0], b[0], i), B.own_pos(cc[1], b[1], j),
                                                      B.own_pos(cc[2], b[2], l)));
                    }
        }
        std::vector<Key> uniq = keys;
        std::sort(uniq.begin(), uniq.end());
        uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
        m.Nv = int64_t(uniq.size());
        if (m.Nv >= (int64_t(1) << 31)) { err = "too many nodes"; return STOKES_E_INVAL; }
        {   // columns: distinct (Y, X) positions; nodes arrive in increasing Z
            std::vector<std::pair<int64_t, int64_t>> yx(size_t(m.Nv));
            for (int64_t g = 0; g < m.Nv; ++g) yx[g] = {uniq[g].y, uniq[g].x};
            std::vector<std::pair<int64_t, int64_t>> cols = yx;
            std::sort(cols.begin(), cols.end());
            cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
            m.ncol = int64_t(cols.size());
            m.col_of.resize(size_t(m.Nv));
            m.pos_of.resize(size_t(m.Nv));
            std::vector<int32_t> cnt(size_t(m.ncol), 0);
            for (int64_t g = 0; g < m.Nv; ++g) {
                int64_t c = int64_t(std::lower_bound(cols.begin(), cols.end(), yx[g]) - cols.begin());
                m.col_of[g] = int32_t(c);
                m.pos_of[g] = cnt[c]++;
            }
        }
        auto find = [&](const Key& kk) -> int64_t {
            auto it = std::lower_bound(uniq.begin(), uniq.end(), kk);
            if (it == uniq.end() || !(*it == kk)) return -1;
            return int64_t(it - uniq.begin());
        };
        bool bad = false;
        #pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < E; ++e) {
            int cc[3], b[3];
            cell_xyz(e, cc, b);
            for (int l = 0; l < n1; ++l)
                for (int j = 0; j < n1; ++j)
                    for (int i = 0; i < n1; ++i) {
                        size_t s = size_t(e) * A + slot(n1, i, j, l);
                        Key kk;
                        if (hanging_slot[s])   // parent lattice slot, on the coarse neighbour
                            kk = B.make_key(double(cc[0]) + B.t[i], double(cc[1]) + B.t[j], double(cc[2]) + B.t[l]);
                        else
                            kk = B.make_key(B.own_pos(cc[0], b[0], i), B.own_pos(cc[1], b[1], j),
                                            B.own_pos(cc[2], b[2], l));
                        int64_t g = find(kk);
                        if (g < 0) bad = true;
                        m.elem_nodes[s] = int32_t(g);
                    }
        }
        if (bad) { err = "internal: hanging slot without a global node"; return STOKES_E_MESH; }
    }

    // ------------------------------------------------------- node columns
    m.col_len.assign(size_t(m.ncol), 0);
    for (int64_t g = 0; g < m.Nv; ++g) m.col_len[m.col_of[g]] = std::max(m.col_len[m.col_of[g]], m.pos_of[g] + 1);
    m.colmax = 0;
    for (int64_t c = 0; c < m.ncol; ++c) m.colmax = std::max(m.colmax, m.col_len[c]);
    m.col_nodes.assign(size_t(m.colmax) * m.ncol, -1);
    for (int64_t g = 0; g < m.Nv; ++g) m.col_nodes[size_t(m.pos_of[g]) * m.ncol + m.col_of[g]] = int32_t(g);
    {
        int bn = 0;
        #pragma omp parallel for schedule(static) reduction(max : bn)
        for (int64_t e = 0; e < E; ++e) {
            for (int j = 0; j < n1; ++j)
                for (int i = 0; i < n1; ++i)
                    for (int l = 0; l < n1; ++l)
                        for (int l2 = 0; l2 < n1; ++l2) {
                            const int64_t a = m.elem_nodes[size_t(e) * A + slot(n1, i, j, l)];
                            const int64_t b = m.elem_nodes[size_t(e) * A + slot(n1, i, j, l2)];
                            if (m.col_of[a] == m.col_of[b]) bn = std::max(bn, std::abs(m.pos_of[a] - m.pos_of[b]));
                        }
        }
        m.bnode = bn;
    }

    // ------------------------------------------------------------- geometry
    // horizontal lattice of bed / surface values at the GLL nodes of coarse cells
    const int64_t HX = int64_t(m.nx) * n1, HY = int64_t(m.ny) * n1;
    std::vector<double> bedH(size_t(HX * HY)), surfH(size_t(HX * HY));
    #pragma omp parallel for schedule(static)
    for (int64_t hy = 0; hy < HY; ++hy) {
        int cy = int(hy / n1), j = int(hy % n1);
        double y = m.Ly * (double(cy) + B.t[j]) / m.ny;
        for (int64_t hx = 0; hx < HX; ++hx) {
            int cx = int(hx / n1), i = int(hx % n1);
            double x = m.Lx * (double(cx) + B.t[i]) / m.nx;
            if (d.bed_nodes) {
                // gridded heights on the horizontal GLL lattice
                const int64_t NXg = int64_t(m.nx) * k + (m.periodic ? 0 : 1);
                int64_t X = int64_t(cx) * k + i, Y = int64_t(cy) * k + j;
                if (m.periodic) { X %= int64_t(m.nx) * k; Y %= int64_t(m.ny) * k; }
                bedH[size_t(hy * HX + hx)] = d.bed_nodes[size_t(Y * NXg + X)];
                surfH[size_t(hy * HX + hx)] = d.surface_nodes[size_t(Y * NXg + X)];
            } else {
                bedH[size_t(hy * HX + hx)] = eval_field(d.bed, x, y);
                surfH[size_t(hy * HX + hx)] = eval_field(d.surface, x, y);
            }
        }
    }
    m.geo.assign(size_t(E) * 10 * Q3, 0.0);
    m.node_xyz.assign(size_t(m.Nv) * 3, 0.0);
    const Tables1D& T = m.tab;
    double wq3[N1MAX * N1MAX * N1MAX];
    for (int lq = 0; lq < q; ++lq)
        for (int jq = 0; jq < q; ++jq)
            for (int iq = 0; iq < q; ++iq)
                wq3[iq + q * (jq + q * lq)] = T.gaussw[iq] * T.gaussw[jq] * T.gaussw[lq];
    // basal faces: elements whose bottom face lies on z = 0
    m.elem_fidx.assign(E, -1);
    for (int64_t e = 0; e < E; ++e) {
        int cc[3], b[3];
        cell_xyz(e, cc, b);
        if (cc[2] == 0 && b[2] <= 0) { m.elem_fidx[e] = int32_t(m.face_elem.size()); m.face_elem.push_back(int32_t(e)); }
    }
    m.nF = int64_t(m.face_elem.size());
    m.fgeo.assign(size_t(m.nF) * 4 * Q2, 0.0);
    std::vector<double> face_nrm(size_t(m.nF) * 3 * A, 0.0);   // int phi_a n ds per slot
    bool inverted = false;

    #pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        int cc[3], b[3];
        cell_xyz(e, cc, b);
        double X[3][N1MAX * N1MAX * N1MAX];      // element geometry nodes, per coordinate
        double Xp[3][N1MAX * N1MAX * N1MAX];
        // parent (coarse cell) geometry nodes
        for (int l = 0; l < n1; ++l)
            for (int j = 0; j < n1; ++j)
                for (int i = 0; i < n1; ++i) {
                    size_t h = size_t((int64_t(cc[1]) * n1 + j) * HX + int64_t(cc[0]) * n1 + i);
                    double zeta = (double(cc[2]) + B.t[l]) / m.nz;
                    int a = slot(n1, i, j, l);
                    Xp[0][a] = m.Lx * (double(cc[0]) + B.t[i]) / m.nx;
                    Xp[1][a] = m.Ly * (double(cc[1]) + B.t[j]) / m.ny;
                    Xp[2][a] = bedH[h] + zeta * (surfH[h] - bedH[h]);
                }
        if (b[0] < 0) {
            std::memcpy(X, Xp, sizeof(X));
        } else {
            // child map = parent map restricted: X = (I_bx x I_by x I_bz) Xp
            for (int c = 0; c < 3; ++c) {
                double t1[N1MAX * N1MAX * N1MAX], t2[N1MAX * N1MAX * N1MAX];
                for (int l = 0; l < n1; ++l) for (int j = 0; j < n1; ++j) for (int i = 0; i < n1; ++i) {
                    double s = 0; for (int mm = 0; mm < n1; ++mm) s += T.I[b[0]][i][mm] * Xp[c][slot(n1, mm, j, l)];
                    t1[slot(n1, i, j, l)] = s;
                }
                for (int l = 0; l < n1; ++l) for (int j = 0; j < n1; ++j) for (int i = 0; i < n1; ++i) {
                    double s = 0; for (int mm = 0; mm < n1; ++mm) s += T.I[b[1]][j][mm] * t1[slot(n1, i, mm, l)];
                    t2[slot(n1, i, j, l)] = s;
                }
                for (int l = 0; l < n1; ++l) for (int j = 0; j < n1; ++j) for (int i = 0; i < n1; ++i) {
                    double s = 0; for (int mm = 0; mm < n1; ++mm) s += T.I[b[2]][l][mm] * t2[slot(n1, i, j, mm)];
                    X[c][slot(n1, i, j, l)] = s;
                }
            }
        }
        // node coordinates of the independent nodes held in own (non-hanging) slots
        uint32_t h = m.elem_hang[e];
        for (int l = 0; l < n1; ++l) for (int j = 0; j < n1; ++j) for (int i = 0; i < n1; ++i) {
            int idx[3] = {i, j, l};
            if (slot_on_hanging_entity(h, idx, k)) continue;
            int a = slot(n1, i, j, l);
            int64_t g = m.elem_nodes[size_t(e) * A + a];
            double x = X[0][a], y = X[1][a];
            if (m.periodic) {
                // canonical representative in [0, L): the seam maps to 0
                x = std::fmod(x, m.Lx); y = std::fmod(y, m.Ly);
                if (x < 0) x += m.Lx;
                if (y < 0) y += m.Ly;
                if (m.Lx - x < 1e-12 * m.Lx) x = 0.0;
                if (m.Ly - y < 1e-12 * m.Ly) y = 0.0;
            }
            m.node_xyz[size_t(g) * 3 + 0] = x;
            m.node_xyz[size_t(g) * 3 + 1] = y;
            m.node_xyz[size_t(g) * 3 + 2] = X[2][a];
        }
        // Jacobian at the volume quadrature points: values at Gauss points by
        // three interpolation sweeps, then collocated derivatives
        double Jm[3][3][N1MAX * N1MAX * N1MAX];   // Jm[d][mref][qp]
        for (int c = 0; c < 3; ++c) {
            double t1[N1MAX * N1MAX * N1MAX], t2[N1MAX * N1MAX * N1MAX], t3[N1MAX * N1MAX * N1MAX];
            for (int l = 0; l < n1; ++l) for (int j = 0; j < n1; ++j) for (int iq = 0; iq < q; ++iq) {
                double s = 0; for (int i = 0; i < n1; ++i) s += T.B[iq][i] * X[c][slot(n1, i, j, l)];
                t1[iq + q * (j + n1 * l)] = s;
            }
            for (int l = 0; l < n1; ++l) for (int jq = 0; jq < q; ++jq) for (int iq = 0; iq < q; ++iq) {
                double s = 0; for (int j = 0; j < n1; ++j) s += T.B[jq][j] * t1[iq + q * (j + n1 * l)];
                t2[iq + q * (jq + q * l)] = s;
            }
            for (int lq = 0; lq < q; ++lq) for (int jq = 0; jq < q; ++jq) for (int iq = 0; iq < q; ++iq) {
                double s = 0; for (int l = 0; l < n1; ++l) s += T.B[lq][l] * t2[iq + q * (jq + q * l)];
                t3[iq + q * (jq + q * lq)] = s;
            }
            for (int lq = 0; lq < q; ++lq) for (int jq = 0; jq < q; ++jq) for (int iq = 0; iq < q; ++iq) {
                double sx = 0, sy = 0, sz = 0;
                for (int mm = 0; mm < q; ++mm) {
                    sx += T.Dg[iq][mm] * t3[mm + q * (jq + q * lq)];
                    sy += T.Dg[jq][mm] * t3[iq + q * (mm + q * lq)];
                    sz += T.Dg[lq][mm] * t3[iq + q * (jq + q * mm)];
                }
                int qp = iq + q * (jq + q * lq);
                Jm[c][0][qp] = sx; Jm[c][1][qp] = sy; Jm[c][2][qp] = sz;
            }
        }
        double* G = &m.geo[size_t(e) * 10 * Q3];
        for (int qp = 0; qp < Q3; ++qp) {
            double a00 = Jm[0][0][qp], a01 = Jm[0][1][qp], a02 = Jm[0][2][qp];
            double a10 = Jm[1][0][qp], a11 = Jm[1][1][qp], a12 = Jm[1][2][qp];
            double a20 = Jm[2][0][qp], a21 = Jm[2][1][qp], a22 = Jm[2][2][qp];
            double c00 = a11 * a22 - a12 * a21, c01 = a12 * a20 - a10 * a22, c02 = a10 * a21 - a11 * a20;
            double det = a00 * c00 + a01 * c01 + a02 * c02;
            if (!(det > 0)) { inverted = true; det = 1.0; }
            double id = 1.0 / det;
            // inverse: Jinv[m][dd] (rows: reference direction, cols: physical)
            double inv[3][3] = {
                {c00 * id, (a02 * a21 - a01 * a22) * id, (a01 * a12 - a02 * a11) * id},
                {c01 * id, (a00 * a22 - a02 * a20) * id, (a02 * a10 - a00 * a12) * id},
                {c02 * id, (a01 * a20 - a00 * a21) * id, (a00 * a11 - a01 * a10) * id}};
            for (int mm = 0; mm < 3; ++mm)
                for (int dd = 0; dd < 3; ++dd) G[size_t(3 * mm + dd) * Q3 + qp] = inv[mm][dd];
            G[size_t(9) * Q3 + qp] = wq3[qp] * det;
        }
        // basal face geometry (zeta = -1): tangents from the bottom-plane nodes
        int32_t f = m.elem_fidx[e];
        if (f >= 0) {
            double tx[3][N1MAX * N1MAX], ty[3][N1MAX * N1MAX];
            for (int c = 0; c < 3; ++c) {
                double v1[N1MAX * N1MAX], v2[N1MAX * N1MAX];
                for (int j = 0; j < n1; ++j) for (int iq = 0; iq < q; ++iq) {
                    double s = 0; for (int i = 0; i < n1; ++i) s += T.B[iq][i] * X[c][slot(n1, i, j, 0)];
                    v1[iq + q * j] = s;
                }
                for (int jq = 0; jq < q; ++jq) for (int iq = 0; iq < q; ++iq) {
                    double s = 0; for (int j = 0; j < n1; ++j) s += T.B[jq][j] * v1[iq + q * j];
                    v2[iq + q * jq] = s;
                }
                for (int jq = 0; jq < q; ++jq) for (int iq = 0; iq < q; ++iq) {
                    double sx = 0, sy = 0;
                    for (int mm = 0; mm < q; ++mm) {
                        sx += T.Dg[iq][mm] * v2[mm + q * jq];
                        sy += T.Dg[jq][mm] * v2[iq + q * mm];
                    }
                    tx[c][iq + q * jq] = sx; ty[c][iq + q * jq] = sy;
                }
            }
            double* FG = &m.fgeo[size_t(f) * 4 * Q2];
            double wn[3][N1MAX * N1MAX];
            for (int fq = 0; fq < Q2; ++fq) {
                double N0 = tx[1][fq] * ty[2][fq] - tx[2][fq] * ty[1][fq];
                double N1 = tx[2][fq] * ty[0][fq] - tx[0][fq] * ty[2][fq];
                double N2 = tx[0][fq] * ty[1][fq] - tx[1][fq] * ty[0][fq];
                double nn = std::sqrt(N0 * N0 + N1 * N1 + N2 * N2);
                double w = T.gaussw[fq % q] * T.gaussw[fq / q];
                FG[0 * Q2 + fq] = w * nn;
                FG[1 * Q2 + fq] = N0 / nn; FG[2 * Q2 + fq] = N1 / nn; FG[3 * Q2 + fq] = N2 / nn;
                wn[0][fq] = w * N0; wn[1][fq] = w * N1; wn[2][fq] = w * N2;
            }
            // int phi_(i,j) n ds at the bottom-plane slots
            for (int c = 0; c < 3; ++c)
                for (int j = 0; j < n1; ++j) for (int i = 0; i < n1; ++i) {
                    double s = 0;
                    for (int jq = 0; jq < q; ++jq) for (int iq = 0; iq < q; ++iq)
                        s += T.B[iq][i] * T.B[jq][j] * wn[c][iq + q * jq];
                    face_nrm[(size_t(f) * 3 + c) * A + slot(n1, i, j, 0)] = s;
                }
        }
    }
    if (inverted) { err = "element with det J <= 0"; return STOKES_E_MESH; }
    // The linearised state stores only the third row of Jinv per quadrature
    // point: x and y must be affine in (xi, eta) on every element, i.e. the
    // first two rows of Jinv diagonal and constant.
    bool not_slab = false;
    #pragma omp parallel for schedule(static) reduction(|| : not_slab)
    for (int64_t e = 0; e < E; ++e) {
        const double* G = &m.geo[size_t(e) * 10 * Q3];
        const double a0 = G[0 * Q3], b0 = G[4 * Q3];
        for (int qp = 0; qp < Q3; ++qp) {
            const double tol = 1e-11 * (std::fabs(a0) + std::fabs(b0));
            if (std::fabs(G[1 * Q3 + qp]) > tol || std::fabs(G[2 * Q3 + qp]) > tol ||
                std::fabs(G[3 * Q3 + qp]) > tol || std::fabs(G[5 * Q3 + qp]) > tol ||
                std::fabs(G[0 * Q3 + qp] - a0) > tol || std::fabs(G[4 * Q3 + qp] - b0) > tol)
                not_slab = true;
        }
    }
    if (not_slab) { err = "internal: element map is not affine in x and y"; return STOKES_E_MESH; }

    // ------------------------------------------------------- basal nodes
    // global nodes on z = 0: every bottom-plane slot of a basal face maps to one
    std::vector<int32_t> bidx(size_t(m.Nv), -1);
    for (int64_t f = 0; f < m.nF; ++f) {
        int64_t e = m.face_elem[f];
        for (int j = 0; j < n1; ++j) for (int i = 0; i < n1; ++i)
            bidx[size_t(m.elem_nodes[size_t(e) * A + slot(n1, i, j, 0)])] = 1;
    }
    m.basal_nodes.clear();
    for (int64_t g = 0; g < m.Nv; ++g)
        if (bidx[g] >= 0) { bidx[g] = int32_t(m.basal_nodes.size()); m.basal_nodes.push_back(int32_t(g)); }
    m.Nb = int64_t(m.basal_nodes.size());
    // face -> basal node map of the bottom-plane slots
    m.fmap.assign(size_t(m.nF) * n1 * n1, -1);
    for (int64_t f = 0; f < m.nF; ++f) {
        int64_t e = m.face_elem[f];
        for (int j = 0; j < n1; ++j) for (int i = 0; i < n1; ++i)
            m.fmap[size_t(f) * n1 * n1 + i + n1 * j] = bidx[size_t(m.elem_nodes[size_t(e) * A + slot(n1, i, j, 0)])];
    }
    // nodal normals: assemble int phi n ds through R^T (hanging transpose on the face)
    std::vector<double> nsum(size_t(m.Nb) * 3, 0.0);
    for (int64_t f = 0; f < m.nF; ++f) {
        int64_t e = m.face_elem[f];
        double v[3][N1MAX * N1MAX];
        for (int c = 0; c < 3; ++c)
            for (int j = 0; j < n1; ++j) for (int i = 0; i < n1; ++i)
                v[c][i + n1 * j] = face_nrm[(size_t(f) * 3 + c) * A + slot(n1, i, j, 0)];
        for (int c = 0; c < 3; ++c) face_hanging_transpose_host(m.elem_hang[e], m.tab, v[c]);
        for (int j = 0; j < n1; ++j) for (int i = 0; i < n1; ++i) {
            int32_t bi = m.fmap[size_t(f) * n1 * n1 + i + n1 * j];
            for (int c = 0; c < 3; ++c) nsum[size_t(bi) * 3 + c] += v[c][i + n1 * j];
        }
    }
    m.basal_P.assign(size_t(m.Nb) * 6, 0.0);
    for (int64_t b = 0; b < m.Nb; ++b) {
        if (m.basal_bc == STOKES_BASE_NOSLIP) continue;   // P = 0
        double n0 = nsum[b * 3], n1v = nsum[b * 3 + 1], n2 = nsum[b * 3 + 2];
        double nn = std::sqrt(n0 * n0 + n1v * n1v + n2 * n2);
        n0 /= nn; n1v /= nn; n2 /= nn;
        double* P = &m.basal_P[size_t(b) * 6];
        P[0] = 1 - n0 * n0; P[1] = 1 - n1v * n1v; P[2] = 1 - n2 * n2;
        P[3] = -n0 * n1v; P[4] = -n0 * n2; P[5] = -n1v * n2;
    }
    // per-element projector rows for bottom-plane slots that gather basal nodes
    m.elem_pidx.assign(E, -1);
    m.pel.clear();
    for (int64_t e = 0; e < E; ++e) {
        bool any = false;
        for (int j = 0; j < n1 && !any; ++j) for (int i = 0; i < n1 && !any; ++i)
            any = bidx[size_t(m.elem_nodes[size_t(e) * A + slot(n1, i, j, 0)])] >= 0;
        if (!any) continue;
        m.elem_pidx[e] = int32_t(m.nP++);
        size_t base = m.pel.size();
        m.pel.resize(base + size_t(6) * n1 * n1, 0.0);
        for (int j = 0; j < n1; ++j) for (int i = 0; i < n1; ++i) {
            int32_t bi = bidx[size_t(m.elem_nodes[size_t(e) * A + slot(n1, i, j, 0)])];
            for (int r = 0; r < 6; ++r) {
                double v = (bi >= 0) ? m.basal_P[size_t(bi) * 6 + r] : (r < 3 ? 1.0 : 0.0);
                m.pel[base + size_t(r) * n1 * n1 + i + n1 * j] = v;
            }
        }
    }
    return STOKES_OK;
}

}  // namespace stokes
