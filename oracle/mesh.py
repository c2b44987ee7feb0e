"""Mesh, global node numbering, hanging-node restriction and geometry (oracle).

TEST INFRASTRUCTURE: plain FP64 restatement, used only by tests, the smoke
check and the CPU-baseline leg of the benchmark.

Definitions followed (Section 3.2.1 and the hanging-node figure of the paper):
  * a coarse hexahedral grid nx x ny x nz (periodic in x, y for the slabs);
    each coarse cell may be split once into 8 children (one refinement
    level, so 2:1 balance holds by construction);
  * element nodes are the tensor GLL nodes of degree k mapped into the cell;
  * global nodes are the element nodes that are not hanging; a node of a
    fine element is hanging when it lies on the closure of an unrefined
    (coarse) cell, and its value is the coarse cell's degree-k Lagrange
    interpolant evaluated at the node;
  * R_i, the restriction of element i, therefore has a unit row for every
    independent node and a row of interpolation weights for every hanging
    node; the global operator is sum_i R_i^T A_i R_i;
  * geometry: x, y affine in the cell index, z = bed + (Z / nz)(surf - bed)
    at the GLL nodes of coarse cells (isoparametric map); refined children
    inherit the parent's map, i.e. their geometry nodes are the parent's
    interpolant evaluated at the child's nodes.

Canonical orderings (shared as a specification, implemented independently by
the library): elements by coarse cell (x fastest, then y, z), a refined cell
replaced by its children in order bx + 2 by + 4 bz; element nodes i + n1 (j +
n1 l); global nodes sorted by (Z, Y, X) reference position with X, Y wrapped
into [0, nx), [0, ny) on periodic meshes; pressure dofs element-major.
"""
import numpy as np
import scipy.sparse as sp

from . import basis

KEYSCALE = 1.0e8


def face_normals(dF, Xb):
    """Area-scaled normal N = t1 x t2 of the basal faces (zeta = -1) at the
    face Gauss points, t_m = dX/dxi_m from the tangential derivative tables
    dF[m] (Section 3.2.1: isoparametric map); |N| = |J_s| and N / |N| is the
    unit normal (sign irrelevant)."""
    t1 = np.einsum("qa,ead->eqd", dF[0], Xb)
    t2 = np.einsum("qa,ead->eqd", dF[1], Xb)
    return np.cross(t1, t2)


def nodal_normals(mesh):
    """int_{Gamma_b} phi_i n ds at the basal nodes, assembled through R (the
    area-weighted nodal normal of the slip condition u . n = 0, Eq. 2.4b)."""
    eb = mesh.basal_elems
    contrib = np.einsum("qa,eqd->ead", mesh.phiF, mesh.nF * mesh.wareaF[..., None])
    full = np.zeros((mesh.E, mesh.A, 3))
    full[eb] = contrib
    nodal = mesh.R.T @ full.reshape(mesh.E * mesh.A, 3)
    return nodal[mesh.basal]


def slip_projector(n):
    """P = I - n n^T at each basal node (n unit): the tangential projector T of
    Eq. 2.4, which imposes u . n = 0 when applied to the basal velocity."""
    return np.eye(3)[None] - n[:, :, None] * n[:, None, :]


class OracleMesh:
    def __init__(self, wl):
        self.wl = wl
        self.k = k = wl.k
        self.n1 = n1 = k + 1
        self.q = q = k + 1
        self.A = n1 ** 3
        self.nx, self.ny, self.nz = wl.nx, wl.ny, wl.nz
        self.periodic = wl.periodic
        self.xi, _ = basis.gauss_lobatto(n1)
        self.g, self.wg = basis.gauss_legendre(q)
        self._build_cells()
        self._build_nodes()
        self._build_geometry()
        self._build_tables()
        self._build_constraints()

    # ------------------------------------------------------------------ cells
    def _build_cells(self):
        wl = self.wl
        mask = wl.refine_mask()
        self.refined = mask.astype(bool)
        origin, size, parent, child = [], [], [], []
        for c in range(wl.n_coarse):
            cx = c % wl.nx
            cy = (c // wl.nx) % wl.ny
            cz = c // (wl.nx * wl.ny)
            if not mask[c]:
                origin.append((cx, cy, cz)); size.append(1.0)
                parent.append(c); child.append((-1, -1, -1))
            else:
                for ch in range(8):
                    bx, by, bz = ch & 1, (ch >> 1) & 1, (ch >> 2) & 1
                    origin.append((cx + 0.5 * bx, cy + 0.5 * by, cz + 0.5 * bz))
                    size.append(0.5); parent.append(c); child.append((bx, by, bz))
        self.origin = np.array(origin, dtype=np.float64)
        self.size = np.array(size)
        self.parent = np.array(parent, dtype=np.int64)
        self.child = np.array(child, dtype=np.int64)
        self.E = len(size)
        self.fine = self.size < 1.0

    def _local_ref(self):
        """Reference offsets (n1^3, 3) of the element nodes, a = i + n1(j + n1 l)."""
        n1 = self.n1
        t = (self.xi + 1.0) / 2.0
        i, j, l = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
        i, j, l = i.transpose(2, 1, 0).ravel(), j.transpose(2, 1, 0).ravel(), l.transpose(2, 1, 0).ravel()
        return np.stack([t[i], t[j], t[l]], axis=1), (i, j, l)

    def _keys(self, P):
        """Integer keys of reference positions, wrapped on periodic axes."""
        K = np.rint(P * KEYSCALE).astype(np.int64)
        if self.periodic:
            K[..., 0] %= int(round(self.nx * KEYSCALE))
            K[..., 1] %= int(round(self.ny * KEYSCALE))
        return K

    # ------------------------------------------------------------------ nodes
    def _build_nodes(self):
        off, (li, lj, ll) = self._local_ref()
        self.local_ijl = (li, lj, ll)
        E, A = self.E, self.A
        P = self.origin[:, None, :] + self.size[:, None, None] * off[None, :, :]
        self.node_ref = P                            # unwrapped reference positions
        hang_cell = np.full((E, A), -1, dtype=np.int64)
        hang_org = np.zeros((E, A, 3))
        if self.fine.any():
            fe = np.nonzero(self.fine)[0]
            Pf = P[fe]                                # (F, A, 3)
            tol = 1e-9
            cands = []
            for d in range(3):
                lo = np.floor(Pf[..., d] - tol).astype(np.int64)
                hi = np.floor(Pf[..., d] + tol).astype(np.int64)
                cands.append((lo, hi))
            found = np.full(Pf.shape[:2], -1, dtype=np.int64)
            forg = np.zeros(Pf.shape)
            for sx in range(2):
                for sy in range(2):
                    for sz in range(2):
                        cx = cands[0][sx]; cy = cands[1][sy]; cz = cands[2][sz]
                        ok = (cz >= 0) & (cz < self.nz)
                        if self.periodic:
                            wx = cx % self.nx; wy = cy % self.ny
                        else:
                            ok &= (cx >= 0) & (cx < self.nx) & (cy >= 0) & (cy < self.ny)
                            wx, wy = cx, cy
                        cell = np.where(ok, wx + self.nx * (wy + self.ny * np.clip(cz, 0, self.nz - 1)), 0)
                        coarse = ok & ~self.refined[np.clip(cell, 0, self.refined.size - 1)]
                        take = coarse & (found < 0)
                        found = np.where(take, cell, found)
                        o = np.stack([cx, cy, cz], axis=-1).astype(np.float64)
                        forg = np.where(take[..., None], o, forg)
            hang_cell[fe] = found
            hang_org[fe] = forg
        self.hang_cell = hang_cell                    # coarse cell constraining the node, -1 if independent
        self.hang_org = hang_org                      # unwrapped origin of that cell
        indep = hang_cell < 0
        keys = self._keys(P)
        ik = keys[indep]
        self._uvals = [np.unique(ik[:, d]) for d in range(3)]
        comb = self._combine(ik)
        uniq_comb, first = np.unique(comb, return_index=True)   # ascending = (Z, Y, X) order
        self.Nv = uniq_comb.size
        self._node_comb = uniq_comb
        self.node_key = ik[first]
        gid = np.full((E, A), -1, dtype=np.int64)
        gid[indep] = self._lookup(ik)
        self.elem_gid = gid
        self._build_R()

    def _combine(self, K):
        """Map integer keys to one int64 whose order is lexicographic in (Z, Y, X)."""
        r = [np.searchsorted(self._uvals[d], K[..., d]) for d in range(3)]
        for d in range(3):
            if not np.all(self._uvals[d][np.clip(r[d], 0, self._uvals[d].size - 1)] == K[..., d]):
                raise KeyError("reference position is not a global node")
        nxu, nyu = self._uvals[0].size, self._uvals[1].size
        return (r[2] * nyu + r[1]) * nxu + r[0]

    def _lookup(self, K):
        c = self._combine(K)
        g = np.searchsorted(self._node_comb, c)
        if not np.all(self._node_comb[np.clip(g, 0, self.Nv - 1)] == c):
            raise KeyError("reference position is not a global node")
        return g

    def _coarse_node_keys(self, org):
        """Keys of all nodes of coarse cells with unwrapped origins org (M, 3)."""
        off, _ = self._local_ref()
        return self._keys(org[:, None, :] + off[None, :, :])

    def _build_R(self):
        E, A, n1 = self.E, self.A, self.n1
        rows, cols, vals = [], [], []
        indep = self.elem_gid >= 0
        r_e, r_a = np.nonzero(indep)
        rows.append(r_e * A + r_a); cols.append(self.elem_gid[indep]); vals.append(np.ones(r_e.size))
        h_e, h_a = np.nonzero(~indep)
        if h_e.size:
            P = self.node_ref[h_e, h_a]               # (H, 3)
            org = self.hang_org[h_e, h_a]
            xi_c = 2.0 * (P - org) - 1.0              # coordinates in the coarse cell
            Lx = basis.lagrange(self.xi, xi_c[:, 0])
            Ly = basis.lagrange(self.xi, xi_c[:, 1])
            Lz = basis.lagrange(self.xi, xi_c[:, 2])
            W = (Lx[:, None, None, :] * Ly[:, None, :, None] * Lz[:, :, None, None]).reshape(h_e.size, A)
            nz = np.abs(W) > 1e-14
            hh, aa = np.nonzero(nz)
            off, _ = self._local_ref()
            ck = self._keys(org[hh] + off[aa])        # keys of the contributing coarse nodes
            rows.append(h_e[hh] * A + h_a[hh]); cols.append(self._lookup(ck)); vals.append(W[hh, aa])
        rows = np.concatenate(rows); cols = np.concatenate(cols); vals = np.concatenate(vals)
        self.R = sp.csr_matrix((vals, (rows, cols)), shape=(E * A, self.Nv))
        # basal nodes: global nodes with Z == 0
        self.basal = np.nonzero(self.node_key[:, 2] == 0)[0]
        self.Nb = self.basal.size
        self.basal_index = np.full(self.Nv, -1, dtype=np.int64)
        self.basal_index[self.basal] = np.arange(self.Nb)

    # --------------------------------------------------------------- geometry
    def _phys(self, Pref):
        """Exact map of reference positions (unwrapped) of coarse cells."""
        wl = self.wl
        x = wl.x0 + wl.Lx * Pref[..., 0] / wl.nx
        y = wl.y0 + wl.Ly * Pref[..., 1] / wl.ny
        b = wl.bed(x, y)
        s = wl.surface(x, y)
        z = b + (Pref[..., 2] / wl.nz) * (s - b)
        return np.stack([x, y, z], axis=-1)

    def _build_geometry(self):
        E, A = self.E, self.A
        X = np.zeros((E, A, 3))
        co = ~self.fine
        X[co] = self._phys(self.node_ref[co])
        if self.fine.any():
            fe = np.nonzero(self.fine)[0]
            pc = self.parent[fe]
            porg = np.stack([pc % self.nx, (pc // self.nx) % self.ny, pc // (self.nx * self.ny)], axis=1).astype(np.float64)
            off, _ = self._local_ref()
            Xp = self._phys(porg[:, None, :] + off[None, :, :])       # parent geometry nodes
            xi_c = 2.0 * (self.node_ref[fe] - porg[:, None, :]) - 1.0  # child nodes in parent coords
            F = fe.size
            Lx = basis.lagrange(self.xi, xi_c[..., 0].ravel()).reshape(F, A, -1)
            Ly = basis.lagrange(self.xi, xi_c[..., 1].ravel()).reshape(F, A, -1)
            Lz = basis.lagrange(self.xi, xi_c[..., 2].ravel()).reshape(F, A, -1)
            W = (Lx[:, :, None, None, :] * Ly[:, :, None, :, None] * Lz[:, :, :, None, None]).reshape(F, A, A)
            X[fe] = np.einsum("fab,fbd->fad", W, Xp)
        self.X = X

    # ----------------------------------------------------------------- tables
    def _build_tables(self):
        n1, q = self.n1, self.q
        B = basis.lagrange(self.xi, self.g)           # (q, n1)
        Dd = basis.lagrange_deriv(self.xi, self.g)
        def k3(a, b, c):
            # table[qp, node] with qp = iq + q (jq + q lq), node = i + n1 (j + n1 l)
            return np.einsum("ai,bj,ck->cbakji", a, b, c).reshape(q ** 3, n1 ** 3)
        self.phi = k3(B, B, B)
        self.dphi = np.stack([k3(Dd, B, B), k3(B, Dd, B), k3(B, B, Dd)])  # (3, Q, A)
        W1 = self.wg
        self.W = np.einsum("a,b,c->cba", W1, W1, W1).ravel()
        # pressure basis at volume qp
        self.modes = basis.pressure_modes(self.k, self.wl.pspace)
        self.npr = len(self.modes)
        T = basis.pressure_1d_tables(self.k, self.wl.pspace, self.g)
        Psi = np.zeros((q ** 3, self.npr))
        for b, (a1, b1, c1) in enumerate(self.modes):
            Psi[:, b] = np.einsum("a,b,c->cba", T[:, a1], T[:, b1], T[:, c1]).ravel()
        self.Psi = Psi
        self.Np = self.E * self.npr
        # geometry at volume qp
        Jm = np.einsum("mqa,ead->eqdm", self.dphi, self.X)  # J[e,q,d,m] = dx_d / dxi_m
        self.detJ = np.linalg.det(Jm)
        self.Jinv = np.linalg.inv(Jm)                       # Jinv[e,q,m,d]
        self.wdetJ = self.detJ * self.W[None, :]
        # basal faces (zeta = -1 on z = 0)
        self.basal_elems = np.nonzero(np.isclose(self.origin[:, 2], 0.0))[0]
        Lm1 = basis.lagrange(self.xi, np.array([-1.0]))      # (1, n1)
        dLm1 = basis.lagrange_deriv(self.xi, np.array([-1.0]))
        def f3(a, b, c):
            return np.einsum("ai,bj,ck->bakji", a, b, c[0:1]).reshape(q * q, n1 ** 3)
        self.phiF = f3(B, B, Lm1)                           # (Qf, A)
        dF = np.stack([f3(Dd, B, Lm1), f3(B, Dd, Lm1)])      # tangential derivatives
        self.WF = np.einsum("a,b->ba", W1, W1).ravel()
        N = face_normals(dF, self.X[self.basal_elems])
        self.areaF = np.linalg.norm(N, axis=-1)              # |J_s|
        self.nF = N / self.areaF[..., None]                  # unit normal (sign irrelevant)
        self.wareaF = self.areaF * self.WF[None, :]

    # ------------------------------------------------------------ constraints
    def _build_constraints(self):
        """Nodal projector P at basal nodes: 0 (no-slip) or I - n n^T (slip).

        The slip normal is the normalised area-weighted nodal normal
        int phi_i n ds, assembled through R.
        """
        nb = nodal_normals(self)
        self.basal_nodal_vec = nb                            # int phi_i n ds (unnormalised)
        self.basal_normal = nb / np.linalg.norm(nb, axis=1)[:, None]
        if self.wl.phys.basal_bc == "noslip":
            self.basal_P = np.zeros((self.Nb, 3, 3))
        else:
            self.basal_P = slip_projector(self.basal_normal)

    # ---------------------------------------------------------------- helpers
    @property
    def ndof(self):
        return 3 * self.Nv + self.Np

    def node_coords(self):
        """Physical coordinates of the global nodes (from any element holding them)."""
        out = np.zeros((self.Nv, 3))
        indep = self.elem_gid >= 0
        out[self.elem_gid[indep]] = self.X[indep]
        if self.periodic:
            for d, L in ((0, self.wl.Lx), (1, self.wl.Ly)):
                out[:, d] = np.mod(out[:, d], L)
                out[L - out[:, d] < 1e-12 * L, d] = 0.0
        return out

    def basal_coords(self):
        return self.node_coords()[self.basal]
