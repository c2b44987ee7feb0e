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
treatment of the top boundary each stop the convergence.  The same flow with
the Glen law (n = 3, delta = 0.1) and its body force derived symbolically
checks the nonlinear operator the same way.
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


# ------------------------------------------------ Glen law (n = 3)
def _glen_manufactured(delta):
    """Body force, velocity gradient and pressure of the same flow for the
    Glen viscosity mu = (D:D / 2 + delta)^(-1/3) (C0 = A = 1, gamma = 1/2),
    derived symbolically: b = -div(mu D(u)) + grad p, p = mu D_zz at z = 1."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z", real=True)
    X = [x, y, z]
    fz = z ** 2 + A_COEF * z ** 3
    u = [sp.cos(2 * sp.pi * x) * sp.diff(fz, z), sp.Integer(0), 2 * sp.pi * sp.sin(2 * sp.pi * x) * fz]
    G = sp.Matrix(3, 3, lambda c, d: sp.diff(u[c], X[d]))
    D = (G + G.T) / 2
    DD = sum(D[i, j] ** 2 for i in range(3) for j in range(3))
    mu = (DD / 2 + delta) ** sp.Rational(-1, 3)
    p = (mu * D[2, 2]).subs(z, 1)
    b = [-sum(sp.diff(mu * D[c, d], X[d]) for d in range(3)) + sp.diff(p, X[c]) for c in range(3)]
    lam = lambda e: sp.lambdify((x, y, z), e, "numpy")
    fb = [lam(e) for e in b]
    fg = [[lam(G[c, d]) for d in range(3)] for c in range(3)]
    fp = lam(p)

    def ev(fn, xq):
        return np.broadcast_to(fn(xq[..., 0], xq[..., 1], xq[..., 2]), xq.shape[:-1])

    def body_fn(xq):
        return np.stack([ev(fn, xq) for fn in fb], -1)

    def grad_fn(xq):
        return np.stack([np.stack([ev(fg[c][d], xq) for d in range(3)], -1) for c in range(3)], -2)

    def p_fn(xq):
        return ev(fp, xq)

    return body_fn, grad_fn, p_fn


def glen_errors(k, pspace, n, delta, fns):
    body_fn, grad_fn, p_fn = fns
    phys = PhysParams(n=3.0, A=1.0, C0=1.0, gamma=0.5, delta=delta, body=(0.0, 0.0, 0.0),
                      basal_bc="noslip", robin=False, logbeta=None)
    wl = Workload("mms3", n, 1, n, k, pspace, True, 1.0, 1.0, synth.flat_field(0.0), synth.flat_field(1.0), phys)
    o = OracleMesh(wl)
    xq = np.einsum("qa,eac->eqc", o.phi, o.X)
    Fe = np.einsum("eq,qa,eqc->eac", o.wdetJ, o.phi, body_fn(xq))
    PF = newton.projector_matrix(o) @ np.concatenate([stokes.scatter(o, Fe).ravel(), np.zeros(o.Np)])
    res = lambda v: stokes.residual(o, phys, v) - PF
    up = np.zeros(o.ndof)
    r = res(up)
    r0 = np.linalg.norm(r)
    for _ in range(40):                        # damped Newton on r_c(u) - P F
        if np.linalg.norm(r) <= 1e-11 * r0:
            break
        d = spla.spsolve(newton.assemble_jacobian(o, phys, up).tocsc(), -r)
        alpha = 1.0
        while alpha > 1e-4 and np.linalg.norm(res(up + alpha * d)) > (1 - 1e-4 * alpha) * np.linalg.norm(r):
            alpha *= 0.5
        up = up + alpha * d
        r = res(up)
    assert np.linalg.norm(r) <= 1e-10 * r0
    u, p = stokes.split(o, up)
    g = stokes._grad(o, stokes.gather(o, u), slice(0, o.E))
    eu = np.sqrt(np.sum(o.wdetJ * np.sum((g - grad_fn(xq)) ** 2, axis=(2, 3))))
    ep = np.sqrt(np.sum(o.wdetJ * (np.einsum("qb,eb->eq", o.Psi, p) - p_fn(xq)) ** 2))
    return eu, ep


@pytest.mark.parametrize("k,pspace,order", [(2, "P", 2), (2, "Q", 1)])
def test_glen_law_convergence_orders(k, pspace, order):
    """The nonlinear operator (n = 3) converges at the same orders as the
    linear one on a smooth solution (delta = 0.1 keeps mu smooth)."""
    fns = _glen_manufactured(0.1)
    levels = (2, 4, 8)
    eu, ep = zip(*(glen_errors(k, pspace, n, 0.1, fns) for n in levels))
    ru = np.log(eu[-2] / eu[-1]) / np.log(2.0)
    rp = np.log(ep[-2] / ep[-1]) / np.log(2.0)
    # still pre-asymptotic at h = 1/8 (observed 2.07 / 1.68 for P1, 1.30 / 0.82
    # for Q0); a wrong operator gives no convergence at all
    assert abs(ru - order) < 0.5, (eu, ru)
    assert rp > order - 0.5, (ep, rp)
