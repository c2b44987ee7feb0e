"""Exact solutions of the continuous problem that lie in the discrete spaces.

On a flat periodic slab of thickness H with a no-slip base and a
traction-free top, a body force (f_x, 0, f_z) drives a laminar shear flow
u = (u_x(z), 0, 0) with hydrostatic pressure p = f_z (z - H).  For the weak
form of Eq. 2.3, int mu D(u):D(v) - p div v - f.v = 0, the x-momentum
balance is mu D_xz = f_x (H - z), which fixes u_x:

  n = 1 (mu = C):          u_x = (f_x / C) (2 H z - z^2)              (quadratic)
  n = 3, gamma = 1/2, delta -> 0 (mu = C |D_xz|^(-2/3)):
                           u_x = (f_x / C)^3 (H^4 - (H - z)^4) / 2    (quartic)

with C = C0 A^(-1/n).  When u_x lies in Q_k and p in the pressure space,
the interpolant is the discrete solution, and the Gauss rule integrates the
residual exactly: mu D(u) is evaluated pointwise from the exact gradient and
equals the linear stress f_x (H - z), so every integrand is a polynomial of
degree <= 2k - 1 per direction.  The oracle's residual must vanish to
rounding.  A wrong factor in the viscous term (2 mu D vs mu D), a wrong
viscosity exponent or gamma convention, a wrong sign of p or f, or a wrong
top boundary treatment each leave a residual of the size of the body-force
term.
"""
import dataclasses

import numpy as np
import pytest

import stokes_synth as synth
from stokes_synth.configs import PhysParams, Workload
from oracle import OracleMesh, stokes as ostokes

H = 1.0
FX, FZ = 0.7, -2.0


def _slab(k, pspace, n, nz=3):
    phys = PhysParams(n=n, A=1.0, C0=1.3, gamma=0.5, delta=1e-30 if n != 1 else 1e-6,
                      body=(FX, 0.0, FZ), basal_bc="noslip", robin=False, logbeta=None)
    return Workload(f"flat_{k}{pspace}_n{n}", 2, 2, nz, k, pspace, True, 3.0, 2.0,
                    synth.flat_field(0.0), synth.flat_field(H), phys)


def _exact_state(o, wl):
    phys = wl.phys
    C = phys.viscosity_prefactor()
    z = o.node_coords()[:, 2]
    if phys.n == 1:
        ux = (FX / C) * (2 * H * z - z * z)
    else:
        ux = (FX / C) ** 3 * (H ** 4 - (H - z) ** 4) / 2.0
    u = np.zeros((o.Nv, 3))
    u[:, 0] = ux
    # pressure: L2 projection of f_z (z - H) on each element's pressure space
    zq = np.einsum("qa,ea->eq", o.phi, o.X[..., 2])
    pq = FZ * (zq - H)
    M = np.einsum("qa,q,qb->ab", o.Psi, o.W, o.Psi)
    p = np.linalg.solve(M, np.einsum("qa,q,eq->ae", o.Psi, o.W, pq)).T
    return np.concatenate([u.ravel(), p.ravel()])


def _body_scale(o, wl):
    return np.linalg.norm(ostokes.residual(o, wl.phys, np.zeros(o.ndof)))


@pytest.mark.parametrize("k,pspace,n", [(2, "P", 1.0), (3, "Q", 1.0), (3, "P", 1.0), (4, "P", 3.0)])
def test_laminar_slab_flow_is_a_discrete_solution(k, pspace, n):
    wl = _slab(k, pspace, n)
    o = OracleMesh(wl)
    up = _exact_state(o, wl)
    r = ostokes.residual(o, wl.phys, up)
    # rounding: the n = 3 stress C |D|^(1/3) is formed from D ~ 1e-6 near the
    # traction-free top, computed from nodal values of order 0.1
    assert np.linalg.norm(r) <= 1e-10 * _body_scale(o, wl)


def test_glen_flow_is_not_a_solution_of_the_linear_law():
    """The quartic n = 3 profile does not solve the n = 1 problem (the check
    above is not vacuous)."""
    wl = _slab(4, "P", 3.0)
    o = OracleMesh(wl)
    up = _exact_state(o, wl)
    lin = dataclasses.replace(wl.phys, n=1.0, delta=1e-6)
    r = ostokes.residual(o, lin, up)
    assert np.linalg.norm(r) >= 1e-3 * _body_scale(o, dataclasses.replace(wl, phys=lin))


def test_wrong_gamma_convention_leaves_a_residual():
    wl = _slab(4, "P", 3.0)
    o = OracleMesh(wl)
    up = _exact_state(o, wl)
    r = ostokes.residual(o, dataclasses.replace(wl.phys, gamma=1.0), up)
    assert np.linalg.norm(r) >= 1e-2 * _body_scale(o, wl)


def test_doubled_velocity_leaves_a_residual():
    wl = _slab(2, "P", 1.0)
    o = OracleMesh(wl)
    up = _exact_state(o, wl)
    up[: 3 * o.Nv] *= 2.0
    assert np.linalg.norm(ostokes.residual(o, wl.phys, up)) >= 0.1 * _body_scale(o, wl)


@pytest.mark.gpu
@pytest.mark.parametrize("k,pspace,n", [(2, "P", 1.0), (3, "Q", 1.0), (4, "P", 3.0)])
def test_gpu_residual_vanishes_at_the_exact_solution(k, pspace, n):
    """The CUDA residual (FP64) at the same exact state also vanishes."""
    torch = pytest.importorskip("torch")
    from paper_1406_6573_gb300 import capi
    from paper_1406_6573_gb300.mesh import Mesh, params
    wl = _slab(k, pspace, n)
    o = OracleMesh(wl)
    up = _exact_state(o, wl)
    m = Mesh(wl, device=0)
    assert (m.Nv, m.Np) == (o.Nv, o.Np)
    p = params(wl.phys, torch.zeros(m.Nb, dtype=torch.float64, device="cuda"))
    r = torch.empty(o.ndof, dtype=torch.float64, device="cuda")
    capi.stokes_residual(m.handle, p, torch.as_tensor(up, device="cuda"), r, capi.STOKES_F64)
    assert float(r.norm()) <= 1e-10 * _body_scale(o, wl)
