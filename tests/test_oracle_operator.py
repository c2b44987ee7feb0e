"""Pins of the oracle's mesh, residual, Jacobian and gradients.

Each check is fixed by the mathematics of the discretisation, not by the
oracle itself:
  * dof counts (workload statement; periodic lattice closed form);
  * exact volumes, and volume invariance under refinement with inherited
    geometry (Section 3.1: children inherit the parent map);
  * the isoparametric property: rigid-body motions have D(u) = 0 (Section 5:
    rigid modes span the null space of F), constant-strain patch test;
  * hanging nodes (hanging-node figure): Q_k fields reproduced exactly and
    traces continuous across 2:1 faces and edges;
  * Newton linearisation (Eqs. 2.6-2.7): complex-step derivative of the
    residual; linear limit n = 1;
  * energy identity (Appendix A): the velocity residual is the gradient of the
    convex energy;
  * symmetry of the saddle-point matrix (Section 4.1);
  * adjoint parameter products by complex step.
"""
import dataclasses
import os

import numpy as np
import pytest

import stokes_synth as synth
from oracle import OracleMesh, basis, stokes, newton

H = 1e-30
_MESHES = {}


def mesh_of(name):
    if name not in _MESHES:
        _MESHES[name] = OracleMesh(synth.workload(name))
    return _MESHES[name]


def logbeta_of(m):
    lb = m.wl.phys.logbeta
    if lb is None:
        return np.zeros(m.Nb)
    return lb(*m.basal_coords()[:, :2].T)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ------------------------------------------------------------------- counts
def test_dof_counts_golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "dof_counts.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    checked = 0
    for name, nvel, npres in rows:
        wl = synth.workload(name)
        if wl.n_coarse > 5000:
            # closed form only (the oracle mesh would be too large)
            nn = (wl.nx * wl.k) * (wl.ny * wl.k) * (wl.nz * wl.k + 1)
            assert 3 * nn == int(nvel)
            assert wl.n_coarse * basis.n_pressure(wl.k, wl.pspace) == int(npres)
            continue
        m = mesh_of(name)
        assert 3 * m.Nv == int(nvel) and m.Np == int(npres)
        checked += 1
    assert checked >= 2


# ------------------------------------------------------------------ geometry
def test_box_volume_exact():
    m = mesh_of("box_4x4x2_q2p1")
    assert abs(m.wdetJ.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("pair", [("cbox_3x3x2_q2p1", "cforest_3x3x2_q2p1"),
                                  ("cbox_3x3x2_q3q1", "cforest_3x3x2_q3p2")])
def test_refinement_preserves_volume(pair):
    a, b = mesh_of(pair[0]), mesh_of(pair[1])
    assert b.fine.any()
    assert abs(a.wdetJ.sum() - b.wdetJ.sum()) < 1e-13 * a.wdetJ.sum()
    assert np.all(b.detJ > 0)


def test_slab_node_lattice_is_periodic():
    m = mesh_of("slab_8x8x2_q2p1")
    assert m.Nv == (8 * 2) * (8 * 2) * (2 * 2 + 1)
    assert m.Nb == 16 * 16


# ------------------------------------------------------- isoparametric pins
def _no_robin(phys):
    return dataclasses.replace(phys, robin=False)


@pytest.mark.parametrize("name", ["cbox_3x3x2_q2p1", "cforest_3x3x2_q3p2", "cforest_4x3x2_q4p3"])
def test_rigid_body_motion_has_zero_viscous_residual(name):
    m = mesh_of(name)
    rng = np.random.default_rng(1)
    a, w = rng.normal(size=3), rng.normal(size=3)
    X = m.node_coords()
    u = a[None, :] + np.cross(w[None, :], X)
    ue = stokes.gather(m, u)
    # element nodal values reproduce the field at the (isoparametric) geometry nodes
    np.testing.assert_allclose(ue, a + np.cross(w, m.X), atol=1e-12)
    rv, rp = stokes.element_residual(m, _no_robin(m.wl.phys), ue, np.zeros((m.E, m.npr)),
                                     np.zeros(m.Nb), body=False)
    # reference magnitude: residual of a random field
    ur = rng.uniform(-1, 1, size=u.shape)
    rr, _ = stokes.element_residual(m, _no_robin(m.wl.phys), stokes.gather(m, ur),
                                    np.zeros((m.E, m.npr)), np.zeros(m.Nb), body=False)
    assert np.abs(stokes.scatter(m, rv)).max() < 1e-10 * np.abs(stokes.scatter(m, rr)).max()
    assert np.abs(rp).max() < 1e-12


@pytest.mark.parametrize("name", ["cbox_3x3x2_q2p1", "cforest_3x3x2_q2p1", "cforest_3x3x2_q3p2"])
def test_constant_strain_patch(name):
    m = mesh_of(name)
    rng = np.random.default_rng(2)
    G = rng.normal(size=(3, 3))
    G -= np.trace(G) / 3 * np.eye(3)
    X = m.node_coords()
    u = X @ G.T
    p0 = 0.7
    pe = np.zeros((m.E, m.npr))
    if m.wl.pspace == "P":
        pe[:, 0] = p0          # Legendre mode (0,0,0) is the constant 1
    else:
        pe[:, :] = p0          # Lagrange basis: all nodal values
    for n in (1.0, 3.0):
        phys = dataclasses.replace(_no_robin(m.wl.phys), n=n)
        rv, rp = stokes.element_residual(m, phys, stokes.gather(m, u), pe, np.zeros(m.Nb), body=False)
        r = stokes.scatter(m, rv)
        key = m.node_key / 1e8
        interior = np.all((key > 1e-9) & (key < np.array([m.nx, m.ny, m.nz]) - 1e-9), axis=1)
        scale = np.abs(r).max()
        assert scale > 1e-6
        assert np.abs(r[interior]).max() < 1e-11 * scale
        assert np.abs(rp).max() < 1e-12


def _element_interp(m, e, vals, xi):
    L = [basis.lagrange(m.xi, xi[:, d]) for d in range(3)]
    W = (L[0][:, None, None, :] * L[1][:, None, :, None] * L[2][:, :, None, None]).reshape(xi.shape[0], m.A)
    return W @ vals


def test_hanging_nodes_reproduce_qk():
    m = mesh_of("cforest_3x3x2_q3p2")
    rng = np.random.default_rng(3)
    c = [rng.normal(size=m.k + 1) for _ in range(3)]
    f = lambda P: (np.polyval(c[0], P[..., 0]) * np.polyval(c[1], P[..., 1])
                   * np.polyval(c[2], P[..., 2]))
    Pg = np.zeros((m.Nv, 3))
    indep = m.elem_gid >= 0
    Pg[m.elem_gid[indep]] = m.node_ref[indep]
    ue = stokes.gather(m, f(Pg))
    np.testing.assert_allclose(ue, f(m.node_ref), rtol=1e-11, atol=1e-11)
    assert (m.hang_cell >= 0).sum() > 0


def _entity_points(m, f, rng, npts=5):
    """Random points on the 6 faces and 12 edges of element f (reference coords)."""
    out = []
    for d in range(3):
        for s in (-1.0, 1.0):
            xi = rng.uniform(-1, 1, size=(npts, 3)); xi[:, d] = s
            out.append(("face", d, s, xi))
    for d in range(3):                       # edges parallel to axis d
        o = [e for e in range(3) if e != d]
        for s0 in (-1.0, 1.0):
            for s1 in (-1.0, 1.0):
                xi = rng.uniform(-1, 1, size=(npts, 3)); xi[:, o[0]] = s0; xi[:, o[1]] = s1
                out.append(("edge", d, (s0, s1), xi))
    return out


@pytest.mark.parametrize("name", ["cforest_3x3x2_q2p1", "cforest_3x3x2_q3p2", "forest_4x4x2_q2p1"])
def test_traces_continuous_across_nonconforming_interfaces(name):
    m = mesh_of(name)
    rng = np.random.default_rng(4)
    ug = rng.uniform(-1, 1, size=m.Nv)
    ue = stokes.gather(m, ug)
    coarse_elem = {int(m.parent[e]): e for e in range(m.E) if not m.fine[e]}
    nchecked = 0
    for f in np.nonzero(m.fine)[0]:
        for kind, d, s, xi in _entity_points(m, f, rng):
            P = m.origin[f] + m.size[f] * (xi + 1) / 2
            # the coarse cells whose closure contains every sampled point
            cells = None
            for pt in P:
                cs = {tuple(np.floor(pt + np.array([sx, sy, sz]) * 1e-9).astype(int))
                      for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)}
                cells = cs if cells is None else cells & cs
            for cx, cy, cz in cells:
                if not (0 <= cz < m.nz):
                    continue
                wx, wy = (cx % m.nx, cy % m.ny) if m.periodic else (cx, cy)
                if not (0 <= wx < m.nx and 0 <= wy < m.ny):
                    continue
                cell = wx + m.nx * (wy + m.ny * cz)
                if m.refined[cell]:
                    continue
                xc = 2.0 * (P - np.array([cx, cy, cz])) - 1.0
                if np.any(np.abs(xc) > 1 + 1e-9):
                    continue
                vf = _element_interp(m, f, ue[f], xi)
                vc = _element_interp(m, coarse_elem[cell], ue[coarse_elem[cell]], xc)
                np.testing.assert_allclose(vf, vc, atol=1e-12)
                nchecked += 1
    assert nchecked > 10


# --------------------------------------------------------- operator pins
CASES = ["box_4x4x2_q2p1", "cbox_3x3x2_q3q1", "slab_5x3x3_q2p1", "cforest_3x3x2_q3p2",
         "forest_4x4x2_q2p1", "slab_4x4x2_q4p3"]


@pytest.mark.parametrize("name", CASES)
def test_complex_step_jacobian(name):
    m = mesh_of(name)
    lb = logbeta_of(m)
    up = synth.uniform_vector(1, m.ndof)
    x = synth.uniform_vector(1, m.ndof, stream=1)
    y = stokes.jacobian_apply(m, m.wl.phys, up, x, lb)
    yc = stokes.residual(m, m.wl.phys, up + 1j * H * x, lb).imag / H
    assert rel(y, yc) < 1e-13


def test_linear_limit_n1():
    m = mesh_of("cforest_3x3x2_q2p1")
    phys = dataclasses.replace(m.wl.phys, n=1.0)
    lb = logbeta_of(m)
    u1 = synth.uniform_vector(2, m.ndof)
    u2 = synth.uniform_vector(2, m.ndof, stream=2)
    w = synth.uniform_vector(2, m.ndof, stream=3)
    J1 = stokes.jacobian_apply(m, phys, u1, w, lb)
    J2 = stokes.jacobian_apply(m, phys, u2, w, lb)
    assert rel(J1, J2) < 1e-14
    d = stokes.residual(m, phys, u1 + w, lb) - stokes.residual(m, phys, u1, lb)
    assert rel(d, J1) < 1e-12


@pytest.mark.parametrize("name", ["cbox_3x3x2_q2p1", "slab_5x3x3_q2p1", "cforest_3x3x2_q3p2"])
def test_energy_identity(name):
    """grad of the Appendix A energy = velocity residual (p = 0, no constraints)."""
    m = mesh_of(name)
    lb = logbeta_of(m)
    u = synth.uniform_vector(3, 3 * m.Nv).reshape(m.Nv, 3)
    w = synth.uniform_vector(3, 3 * m.Nv, stream=1).reshape(m.Nv, 3)
    dE = stokes.energy(m, m.wl.phys, u + 1j * H * w, lb).imag / H
    rv, _ = stokes.element_residual(m, m.wl.phys, stokes.gather(m, u), np.zeros((m.E, m.npr)), lb)
    r = stokes.scatter(m, rv)
    assert abs(dE - np.sum(r * w)) < 1e-12 * np.abs(r).sum() * np.abs(w).max()


@pytest.mark.parametrize("name", CASES)
def test_jacobian_symmetry_dot(name):
    m = mesh_of(name)
    lb = logbeta_of(m)
    up = synth.uniform_vector(4, m.ndof)
    x = synth.uniform_vector(4, m.ndof, stream=1)
    y = synth.uniform_vector(4, m.ndof, stream=2)
    a = np.dot(y, stokes.jacobian_apply(m, m.wl.phys, up, x, lb))
    b = np.dot(x, stokes.jacobian_apply(m, m.wl.phys, up, y, lb))
    assert abs(a - b) < 1e-12 * (abs(a) + abs(b))


def test_assembled_matrix_symmetric_and_matches_apply():
    m = mesh_of("forest_4x4x2_q2p1")
    lb = logbeta_of(m)
    up = synth.uniform_vector(5, m.ndof)
    J = newton.assemble_jacobian(m, m.wl.phys, up, lb)
    x = synth.uniform_vector(5, m.ndof, stream=1)
    assert rel(J @ x, stokes.jacobian_apply(m, m.wl.phys, up, x, lb)) < 1e-13
    asym = abs(J - J.T).max()
    assert asym < 1e-12 * abs(J).max()


def test_velocity_block_positive_definite():
    """eig(mu') >= mu / n > 0 (Eq. 2.7) plus Robin / constraints: F is SPD."""
    m = mesh_of("cbox_3x3x2_q2p1")
    lb = logbeta_of(m)
    up = synth.uniform_vector(6, m.ndof)
    J = newton.assemble_jacobian(m, m.wl.phys, up, lb).toarray()
    F = J[: 3 * m.Nv, : 3 * m.Nv]
    np.linalg.cholesky(0.5 * (F + F.T))


@pytest.mark.parametrize("name", ["cbox_3x3x2_q2p1", "slab_5x3x3_q2p1", "forest_6x6x2_q3p2"])
def test_param_grad_complex_step(name):
    m = mesh_of(name)
    phys = m.wl.phys
    lb = logbeta_of(m)
    up = synth.uniform_vector(7, m.ndof)
    lam = synth.uniform_vector(7, m.ndof, stream=1)
    g, gA = stokes.param_grad(m, phys, up, lam, lb)
    dlb = synth.uniform_vector(7, m.Nb, stream=2)
    ref = np.dot(lam, stokes.residual(m, phys, up, lb + 1j * H * dlb).imag / H)
    assert abs(np.dot(g, dlb) - ref) < 1e-12 * np.abs(g).sum()
    physc = dataclasses.replace(phys, A=phys.A * (1 + 1j * H))
    refA = np.dot(lam, stokes.residual(m, physc, up, lb).imag / (H * phys.A))
    assert abs(gA - refA) < 1e-12 * abs(refA)


def test_local_mass_conservation_divergence_theorem():
    """Row of B for the constant pressure mode = - boundary flux of u (P_{k-1} contains 1)."""
    m = mesh_of("cforest_3x3x2_q3p2")
    rng = np.random.default_rng(8)
    u = rng.uniform(-1, 1, size=(m.Nv, 3))
    ue = stokes.gather(m, u)
    _, rp = stokes.element_residual(m, _no_robin(m.wl.phys), ue, np.zeros((m.E, m.npr)),
                                    np.zeros(m.Nb), body=False)
    g, wg = basis.gauss_legendre(m.k + 2)
    L = basis.lagrange(m.xi, g)
    dL = basis.lagrange_deriv(m.xi, g)
    Lp = basis.lagrange(m.xi, np.array([-1.0, 1.0]))
    dLp = basis.lagrange_deriv(m.xi, np.array([-1.0, 1.0]))
    def tens(a, b, c):
        return np.einsum("ai,bj,ck->cbakji", a, b, c).reshape(a.shape[0] * b.shape[0] * c.shape[0], m.A)
    for e in rng.choice(m.E, size=12, replace=False):
        flux = 0.0
        for d in range(3):
            for si, s in enumerate((-1.0, 1.0)):
                tabs = [L, L, L]; dtabs = [dL, dL, dL]
                tabs[d] = Lp[si:si + 1]; dtabs[d] = dLp[si:si + 1]
                val = tens(*tabs)
                tang = [o for o in range(3) if o != d]
                t = []
                for o in tang:
                    tt = list(tabs); tt[o] = dtabs[o]
                    t.append(tens(*tt) @ m.X[e])
                N = np.cross(t[0], t[1])
                orient = np.sign(np.einsum("qd,qd->q", N, (tens(*[dtabs[i] if i == d else tabs[i] for i in range(3)]) @ m.X[e])))
                N = N * orient[:, None] * s
                uq = val @ ue[e]
                ww = np.einsum("a,b->ab", wg, wg).ravel()
                flux += np.sum(ww * np.einsum("qd,qd->q", uq, N))
        assert abs(rp[e, 0] + flux) < 1e-11 * max(1.0, abs(flux))
