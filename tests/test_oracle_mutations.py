"""Planted mistakes in the oracle must be caught by its pins.

Each test patches one plausible mistake into the oracle (on the CPU) and
checks that the pin meant to catch it fails.
"""
import dataclasses

import numpy as np
import pytest

import stokes_synth as synth
from oracle import OracleMesh, stokes

H = 1e-30


@pytest.fixture(scope="module")
def cmesh():
    return OracleMesh(synth.workload("cforest_3x3x2_q2p1"))


def _rigid_residual(m):
    rng = np.random.default_rng(1)
    a, w = rng.normal(size=3), rng.normal(size=3)
    u = a + np.cross(w, m.node_coords())
    phys = dataclasses.replace(m.wl.phys, robin=False)
    rv, _ = stokes.element_residual(m, phys, stokes.gather(m, u), np.zeros((m.E, m.npr)),
                                    np.zeros(m.Nb), body=False)
    ur = rng.uniform(-1, 1, size=u.shape)
    rr, _ = stokes.element_residual(m, phys, stokes.gather(m, ur), np.zeros((m.E, m.npr)),
                                    np.zeros(m.Nb), body=False)
    return np.abs(stokes.scatter(m, rv)).max() / np.abs(stokes.scatter(m, rr)).max()


def _cs_error(m):
    lb = m.wl.phys.logbeta(*m.basal_coords()[:, :2].T)
    up = synth.uniform_vector(1, m.ndof)
    x = synth.uniform_vector(1, m.ndof, stream=1)
    y = stokes.jacobian_apply(m, m.wl.phys, up, x, lb)
    yc = stokes.residual(m, m.wl.phys, up + 1j * H * x, lb).imag / H
    return np.linalg.norm(y - yc) / np.linalg.norm(yc)


def _dot_asym(m):
    lb = m.wl.phys.logbeta(*m.basal_coords()[:, :2].T)
    up = synth.uniform_vector(4, m.ndof)
    x = synth.uniform_vector(4, m.ndof, stream=1)
    y = synth.uniform_vector(4, m.ndof, stream=2)
    a = np.dot(y, stokes.jacobian_apply(m, m.wl.phys, up, x, lb))
    b = np.dot(x, stokes.jacobian_apply(m, m.wl.phys, up, y, lb))
    return abs(a - b) / (abs(a) + abs(b))


def test_baseline_pins_hold(cmesh):
    assert _rigid_residual(cmesh) < 1e-10
    assert _cs_error(cmesh) < 1e-13
    assert _dot_asym(cmesh) < 1e-12


def test_transposed_inverse_jacobian_is_caught(cmesh, monkeypatch):
    orig = stokes._grad
    def bad(mesh, ue, sl):
        G = np.einsum("mqa,eac->eqcm", mesh.dphi, ue)
        return np.einsum("eqcm,eqdm->eqcd", G, mesh.Jinv[sl])
    monkeypatch.setattr(stokes, "_grad", bad)
    assert _rigid_residual(cmesh) > 1e-6


def test_dropped_newton_term_is_caught(cmesh, monkeypatch):
    monkeypatch.setattr(stokes, "_pexp", lambda phys: 0.0 * phys.n)
    # residual still uses p_n through _viscosity: restore it there only
    orig_visc = stokes._viscosity
    monkeypatch.setattr(stokes, "_viscosity",
                        lambda phys, DD: phys.viscosity_prefactor()
                        * (phys.gamma * DD + phys.delta) ** ((1.0 - phys.n) / (2.0 * phys.n)))
    assert _cs_error(cmesh) > 1e-6


def test_pressure_sign_error_is_caught(cmesh, monkeypatch):
    orig = stokes.element_jacobian
    def bad(*a, **k):
        yv, yp = orig(*a, **k)
        return yv, -yp
    monkeypatch.setattr(stokes, "element_jacobian", bad)
    assert _dot_asym(cmesh) > 1e-6


def test_wrong_energy_constant_is_caught(cmesh, monkeypatch):
    m = cmesh
    lb = m.wl.phys.logbeta(*m.basal_coords()[:, :2].T)
    u = synth.uniform_vector(3, 3 * m.Nv).reshape(m.Nv, 3)
    w = synth.uniform_vector(3, 3 * m.Nv, stream=1).reshape(m.Nv, 3)
    phys = m.wl.phys
    rv, _ = stokes.element_residual(m, phys, stokes.gather(m, u), np.zeros((m.E, m.npr)), lb)
    ref = np.sum(stokes.scatter(m, rv) * w)
    bad = dataclasses.replace(phys, gamma=2.0 * phys.gamma)   # energy with the wrong gamma
    dE = stokes.energy(m, bad, u + 1j * H * w, lb).imag / H
    assert abs(dE - ref) > 1e-6 * abs(ref)


# ------------------------------------------------------ nonlinear sliding
def _sliding_mesh():
    wl = synth.workload("slab_5x3x3_q2p1")
    return OracleMesh(dataclasses.replace(wl, phys=dataclasses.replace(wl.phys, sliding_m=1.0 / 3.0)))


def _sliding_cs_error(m):
    lb = np.zeros(m.Nb) if m.wl.phys.logbeta is None else m.wl.phys.logbeta(*m.basal_coords()[:, :2].T)
    up = synth.uniform_vector(1, m.ndof)
    x = synth.uniform_vector(1, m.ndof, stream=1)
    y = stokes.jacobian_apply(m, m.wl.phys, up, x, lb)
    yc = stokes.residual(m, m.wl.phys, up + 1j * H * x, lb).imag / H
    return np.linalg.norm(y - yc) / np.linalg.norm(yc)


def test_sliding_derivative_without_its_factor_two_is_caught(monkeypatch):
    m = _sliding_mesh()
    assert _sliding_cs_error(m) < 1e-13
    good = stokes._sliding
    monkeypatch.setattr(stokes, "_sliding", lambda phys, tu: (good(phys, tu)[0], 0.5 * good(phys, tu)[1]))
    assert _sliding_cs_error(m) > 1e-6


def test_sliding_exponent_without_the_half_is_caught(monkeypatch):
    """s(x) = (x + eps)^(m - 1) instead of (x + eps)^((m - 1)/2): the closed
    form of uniform sliding fails."""
    from tests.test_oracle_sliding import test_uniform_sliding_flow_closed_form as closed_form
    closed_form(1.0 / 3.0, 1.7)

    def wrong(phys, tu):
        x = np.einsum("eqc,eqc->eq", tu, tu) + phys.sliding_eps
        mm = phys.sliding_m
        return x ** (mm - 1.0), (mm - 1.0) * x ** (mm - 2.0)

    monkeypatch.setattr(stokes, "_sliding", wrong)
    with pytest.raises(AssertionError):
        closed_form(1.0 / 3.0, 1.7)


def test_doubled_viscosity_stops_the_convergence(monkeypatch):
    """mu -> 2 mu in the oracle's viscous term: the discrete solutions no
    longer converge to the manufactured solution."""
    from tests.test_oracle_convergence import errors
    good = [errors(2, "P", n)[0] for n in (4, 8)]
    assert good[1] < 0.3 * good[0]
    orig = stokes._viscosity
    monkeypatch.setattr(stokes, "_viscosity", lambda phys, DD: 2.0 * orig(phys, DD))
    bad = [errors(2, "P", n)[0] for n in (4, 8)]
    assert bad[1] > 0.6 * bad[0]


def test_infsup_without_the_jacobian_weight_in_k_is_caught(monkeypatch):
    """K assembled without w detJ: the inf-sup constant is no longer
    invariant under a scaling of the domain."""
    from oracle import infsup
    orig = infsup.operators

    def bad(o):
        KI, B, M, I = orig(o)
        return KI / np.mean(o.wdetJ), B, M, I     # drops the volume scaling of K
    b1 = infsup.infsup(infsup.cube_mesh(2, "P", 2, side=1.0))[0]
    b7 = infsup.infsup(infsup.cube_mesh(2, "P", 2, side=7.0))[0]
    assert abs(b1 - b7) <= 1e-10 * b1
    monkeypatch.setattr(infsup, "operators", bad)
    c1 = infsup.infsup(infsup.cube_mesh(2, "P", 2, side=1.0))[0]
    c7 = infsup.infsup(infsup.cube_mesh(2, "P", 2, side=7.0))[0]
    assert abs(c1 - c7) > 1e-3 * c1


# ------------------------------------------------- basal face geometry pins
def _nodal_normal_error(name="cbox_3x3x2_q2p1"):
    from test_oracle_face_geometry import closed_form_nodal_normals
    wl = synth.workload(name)
    m = OracleMesh(wl)
    xs, ys, acc = closed_form_nodal_normals(wl)
    bc = m.basal_coords()
    ref = acc[np.searchsorted(xs, bc[:, 0] - 1e-12), np.searchsorted(ys, bc[:, 1] - 1e-12)]
    nref = ref / np.linalg.norm(ref, axis=1)[:, None]
    return np.abs(m.basal_normal - nref).max()


def _tilted_projector_error():
    from test_oracle_face_geometry import tilted
    alpha, beta = 0.3, -0.2
    m = OracleMesh(tilted("mut", alpha, beta))
    n = np.array([-alpha, -beta, 1.0]) / np.sqrt(1.0 + alpha ** 2 + beta ** 2)
    return np.abs(np.einsum("nij,j->ni", m.basal_P, n)).max()


def test_face_geometry_baseline_pins_hold():
    assert _nodal_normal_error() < 1e-13
    assert _tilted_projector_error() < 1e-14


def test_nodal_normal_without_face_area_is_caught(monkeypatch):
    import oracle.mesh as om

    def bad(mesh):   # weights w instead of w |J_s|
        contrib = np.einsum("qa,eqd->ead", mesh.phiF, mesh.nF * mesh.WF[None, :, None])
        full = np.zeros((mesh.E, mesh.A, 3))
        full[mesh.basal_elems] = contrib
        return (mesh.R.T @ full.reshape(mesh.E * mesh.A, 3))[mesh.basal]
    monkeypatch.setattr(om, "nodal_normals", bad)
    assert _nodal_normal_error() > 1e-6


def test_transposed_tangent_table_is_caught(monkeypatch):
    import oracle.mesh as om

    def bad(dF, Xb):  # face Gauss points of the eta tangent taken in transposed order
        nq = int(round(np.sqrt(dF.shape[1])))
        d1 = dF[1].reshape(nq, nq, -1).transpose(1, 0, 2).reshape(nq * nq, -1)
        t1 = np.einsum("qa,ead->eqd", dF[0], Xb)
        t2 = np.einsum("qa,ead->eqd", d1, Xb)
        return np.cross(t1, t2)
    monkeypatch.setattr(om, "face_normals", bad)
    assert _nodal_normal_error() > 1e-6


def test_projector_from_unnormalised_normal_is_caught(monkeypatch):
    import oracle.mesh as om
    orig_build = om.OracleMesh._build_constraints

    def bad_build(self):   # plant: P = I - v v^T with v = int phi_i n ds, not normalised
        orig_build(self)
        if self.wl.phys.basal_bc != "noslip":
            self.basal_P = om.slip_projector(self.basal_nodal_vec)
    monkeypatch.setattr(om.OracleMesh, "_build_constraints", bad_build)
    assert _tilted_projector_error() > 1e-6
