"""Convergence orders of the discretisation (linear Stokes, n = 1) against a
manufactured solution, computed with the oracle's assembled operator.

Domain: periodic in x and y, [0, 1]^2 x [0, 1], no-slip base, traction-free
top (the natural boundary condition of the weak form Eq. 2.5, with the
paper's int mu D(v):D(u), i.e. traction (mu D(u) - p I) n).  Solution from
the stream function psi = cos(2 pi x) f(z):
    u = (cos(2 pi x) f'(z), 0, 2 pi sin(2 pi x) f(z))   (divergence-free)
    p = 2 pi mu f'(1) sin(2 pi x)
with f(z) = z^2 + a z^3, f(0) = f'(0) = 0 (no slip) and
f''(1) + 4 pi^2 f(1) = 0 (no shear traction at the top; p gives zero
normal traction there).  Body force b = -(mu/2) Lap u + grad p.
The discrete solution of Q_k x P_{k-1} converges like h^k in the velocity
H1 seminorm and the pressure L2 norm; Q_k x Q_{k-2} like h^(k-1)
(standard mixed-FEM estimates; Section 3.1 contrasts the two pairings).
A dropped or doubled viscous factor, a wrong pressure sign or a wrong
treatment of the top boundary each stop the convergence.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import stokes_synth as synth
from stokes_synth.configs import PhysParams, Workload
from oracle import OracleMesh, newton, stokes

TWO_PI = 2.0 * np.pi
A_COEF = -(2.0 + 4.0 * np.pi ** 2) / (6.0 + 4.0 * np.pi ** 2)
MU = 1.0


def f(z, d=0):
    a = A_COEF
    return [z * z + a * z ** 3, 2 * z + 3 * a * z * z, 2 + 6 * a * z, 6 * a + 0 * z][d]


def u_exact(x):
    X, Z = x[..., 0], x[..., 2]
    c, s = np.cos(TWO_PI * X), np.sin(TWO_PI * X)
    u = np.stack([c * f(Z, 1), 0 * X, TWO_PI * s * f(Z)], axis=-1)
    g = np.zeros(x.shape[:-1] + (3, 3))         # g[..., c, d] = d u_c / d x_d
    g[..., 0, 0] = -TWO_PI * s * f(Z, 1)
    g[..., 0, 2] = c * f(Z, 2)
    g[..., 2, 0] = TWO_PI ** 2 * c * f(Z)
    g[..., 2, 2] = TWO_PI * s * f(Z, 1)
    return u, g


def p_exact(x):
    return TWO_PI * MU * f(1.0, 1) * np.sin(TWO_PI * x[..., 0])


def body(x):
    X, Z = x[..., 0], x[..., 2]
    c, s = np.cos(TWO_PI * X), np.sin(TWO_PI * X)
    lap_ux = c * (f(Z, 3) - TWO_PI ** 2 * f(Z, 1))
    lap_uz = TWO_PI * s * (f(Z, 2) - TWO_PI ** 2 * f(Z))
    dpdx = TWO_PI ** 2 * MU * f(1.0, 1) * c
    return np.stack([-0.5 * MU * lap_ux + dpdx, 0 * X, -0.5 * MU * lap_uz], axis=-1)


def errors(k, pspace, n):
    phys = PhysParams(n=1.0, A=1.0, C0=MU, gamma=0.5, delta=1e-6, body=(0.0, 0.0, 0.0),
                      basal_bc="noslip", robin=False, logbeta=None)
    wl = Workload("mms", n, 1, n, k, pspace, True, 1.0, 1.0, synth.flat_field(0.0), synth.flat_field(1.0), phys)
    o = OracleMesh(wl)
    xq = np.einsum("qa,eac->eqc", o.phi, o.X)                      # physical Gauss points
    Fe = np.einsum("eq,qa,eqc->eac", o.wdetJ, o.phi, body(xq))
    F = np.concatenate([stokes.scatter(o, Fe).ravel(), np.zeros(o.Np)])
    J = newton.assemble_jacobian(o, phys, np.zeros(o.ndof))
    P = newton.projector_matrix(o)
    up = spla.spsolve(J.tocsc(), P @ F)
    u, p = stokes.split(o, up)
    g = stokes._grad(o, stokes.gather(o, u), slice(0, o.E))
    _, g_ex = u_exact(xq)
    eu = np.sqrt(np.sum(o.wdetJ * np.sum((g - g_ex) ** 2, axis=(2, 3))))
    pq = np.einsum("qb,eb->eq", o.Psi, p)
    ep = np.sqrt(np.sum(o.wdetJ * (pq - p_exact(xq)) ** 2))
    return eu, ep


def test_manufactured_solution_satisfies_the_boundary_conditions():
    z = np.array([1.0])
    assert abs(f(z, 2)[0] + TWO_PI ** 2 * f(z)[0]) < 1e-12          # no shear traction at the top
    assert f(0.0) == 0.0 and f(0.0, 1) == 0.0


@pytest.mark.parametrize("k,pspace,order", [(2, "P", 2), (2, "Q", 1), (3, "P", 3), (3, "Q", 2)])
def test_convergence_orders(k, pspace, order):
    levels = (2, 4, 8) if k == 2 else (2, 4, 6)
    eu, ep = zip(*(errors(k, pspace, n) for n in levels))
    h = np.array([1.0 / n for n in levels])
    ru = np.log(eu[-2] / eu[-1]) / np.log(h[-2] / h[-1])
    rp = np.log(ep[-2] / ep[-1]) / np.log(h[-2] / h[-1])
    assert abs(ru - order) < 0.35, (eu, ru)
    assert rp > order - 0.35, (ep, rp)
    assert eu[-1] < eu[0] and ep[-1] < ep[0]
