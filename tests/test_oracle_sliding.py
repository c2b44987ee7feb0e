"""Pins of the nonlinear basal sliding law in the oracle.

Traction beta s(|T u|^2) T u with s(x) = (x + eps_s)^{(m-1)/2} (the linear
law of Eq. 2.4a for m = 1).  Fixed by the mathematics, not by the oracle:
  * a closed form: on a flat periodic slab a uniform tangential velocity U
    has D(u) = 0, so with no body force the only residual is the basal one and
    its x-components sum to beta s(U^2) U times the bed area;
  * the Newton derivative: complex step of the residual (this pins the
    2 s' (T u . T w) T u term and its tangential projection);
  * the energy identity: the velocity residual is the gradient of
    int beta F(|T u|^2), 2 F' = s;
  * the log(beta) adjoint product by complex step;
  * the Picard form, linear in u for frozen s: J_Picard(u) u - r_c(u) = -r_c(0).
"""
import dataclasses

import numpy as np
import pytest

import stokes_synth as synth
from stokes_synth.configs import PhysParams, Workload
from oracle import OracleMesh, stokes

H = 1e-30
M_SLIDE = 1.0 / 3.0
_M = {}


def _mesh(name, m=M_SLIDE):
    key = (name, m)
    if key not in _M:
        wl = synth.workload(name)
        wl = dataclasses.replace(wl, phys=dataclasses.replace(wl.phys, sliding_m=m, robin=True, basal_bc="slip"))
        o = OracleMesh(wl)
        lb = np.zeros(o.Nb) if wl.phys.logbeta is None else wl.phys.logbeta(*o.basal_coords()[:, :2].T)
        _M[key] = (wl, o, lb)
    return _M[key]


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("m", [1.0 / 3.0, 1.0, 3.0])
@pytest.mark.parametrize("U", [0.02, 1.7])
def test_uniform_sliding_flow_closed_form(m, U):
    Lx, Ly = 3.0, 2.0
    phys = PhysParams(n=3.0, A=1.0, C0=1.0, gamma=0.5, delta=1e-6, body=(0.0, 0.0, 0.0),
                      basal_bc="slip", robin=True, logbeta=None, sliding_m=m, sliding_eps=1e-4)
    wl = Workload("flat_sliding", 3, 2, 2, 2, "P", True, Lx, Ly, synth.flat_field(0.0), synth.flat_field(1.0), phys)
    o = OracleMesh(wl)
    u = np.zeros((o.Nv, 3))
    u[:, 0] = U
    up = np.concatenate([u.ravel(), np.zeros(o.Np)])
    r = stokes.residual(o, phys, up)
    rx = r[: 3 * o.Nv].reshape(o.Nv, 3)[:, 0].sum()
    expected = (U * U + 1e-4) ** (0.5 * (m - 1.0)) * U * Lx * Ly if m != 1.0 else U * Lx * Ly
    # rounding floor: the viscous term of the constant field (mu ~ 1e2 at D = 0)
    tol = 1e-12 * abs(expected) + 1e-13
    assert abs(rx - expected) <= tol
    # nothing acts in y, and every x residual sits on the bed
    assert np.abs(r[: 3 * o.Nv].reshape(o.Nv, 3)[:, 1]).max() <= tol
    off_bed = np.setdiff1d(np.arange(o.Nv), o.basal)
    assert np.abs(r[: 3 * o.Nv].reshape(o.Nv, 3)[off_bed, 0]).max() <= tol


@pytest.mark.parametrize("name", ["box_4x4x2_q2p1", "slab_5x3x3_q2p1", "cforest_3x3x2_q3p2"])
def test_sliding_complex_step_jacobian(name):
    wl, o, lb = _mesh(name)
    up = synth.uniform_vector(1, o.ndof)
    x = synth.uniform_vector(1, o.ndof, stream=1)
    y = stokes.jacobian_apply(o, wl.phys, up, x, lb)
    yc = stokes.residual(o, wl.phys, up + 1j * H * x, lb).imag / H
    assert rel(y, yc) < 1e-13
    # the sliding term is active: the linear law gives a different Jacobian
    y1 = stokes.jacobian_apply(o, dataclasses.replace(wl.phys, sliding_m=1.0), up, x, lb)
    assert rel(y, y1) > 1e-6


@pytest.mark.parametrize("name", ["slab_5x3x3_q2p1", "cforest_3x3x2_q3p2"])
def test_sliding_energy_identity(name):
    wl, o, lb = _mesh(name)
    u = synth.uniform_vector(3, 3 * o.Nv).reshape(o.Nv, 3)
    w = synth.uniform_vector(3, 3 * o.Nv, stream=1).reshape(o.Nv, 3)
    dE = stokes.energy(o, wl.phys, u + 1j * H * w, lb).imag / H
    rv, _ = stokes.element_residual(o, wl.phys, stokes.gather(o, u), np.zeros((o.E, o.npr)), lb)
    r = stokes.scatter(o, rv)
    assert abs(dE - np.sum(r * w)) < 1e-12 * np.abs(r).sum() * np.abs(w).max()


@pytest.mark.parametrize("name", ["slab_5x3x3_q2p1", "cforest_3x3x2_q3p2"])
def test_sliding_param_grad_complex_step(name):
    wl, o, lb = _mesh(name)
    up = synth.uniform_vector(7, o.ndof)
    lam = synth.uniform_vector(7, o.ndof, stream=1)
    g, _ = stokes.param_grad(o, wl.phys, up, lam, lb)
    dlb = synth.uniform_vector(7, o.Nb, stream=2)
    ref = np.dot(lam, stokes.residual(o, wl.phys, up, lb + 1j * H * dlb).imag / H)
    assert abs(np.dot(g, dlb) - ref) < 1e-12 * np.abs(g).sum()


@pytest.mark.parametrize("name", ["box_4x4x2_q2p1", "slab_5x3x3_q2p1"])
def test_sliding_picard_operator_reproduces_the_residual(name):
    wl, o, lb = _mesh(name)
    phys = dataclasses.replace(wl.phys, linearization="picard")
    up = synth.uniform_vector(5, o.ndof)
    lhs = stokes.jacobian_apply(o, phys, up, up, lb) - stokes.residual(o, phys, up, lb)
    rhs = -stokes.residual(o, phys, np.zeros(o.ndof), lb)
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(stokes.residual(o, phys, up, lb))
