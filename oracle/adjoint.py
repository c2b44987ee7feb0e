"""Misfit gradient by the adjoint method (FP64 oracle).

TEST INFRASTRUCTURE: only tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module.

J(u) = 1/2 sum over top-surface velocity nodes of |u - u_obs|^2 (nodal l2);
u solves the constrained residual r_c(u; log beta, A) = 0.  Implicit function
theorem: dJ/dm = -lambda^T d r_c/dm with J_c^T lambda = dJ/du (Sections 2.3
and 8.3: the adjoint equations carry the same linearised operator).  The
Newton solve and the adjoint solve use sparse direct factorisations.
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import newton, stokes


def top_nodes(mesh):
    """Global nodes on the top surface (largest reference Z)."""
    kz = mesh.node_key[:, 2]
    return np.nonzero(kz == kz.max())[0]


def misfit(mesh, up, u_obs, top):
    u, _ = stokes.split(mesh, up)
    d = u[top] - u_obs
    return 0.5 * np.sum(d * d)


def gradient(mesh, phys, logbeta, u_obs, top, rtol=1e-13, up0=None):
    """Returns (J, dJ/dlog(beta) [Nb], dJ/dA, up)."""
    up, _ = newton.newton_solve(mesh, phys, logbeta, rtol=rtol, up0=up0)
    u, _ = stokes.split(mesh, up)
    dJdu = np.zeros(mesh.ndof)
    dJdu[: 3 * mesh.Nv].reshape(mesh.Nv, 3)[top] = u[top] - u_obs
    Jc = newton.assemble_jacobian(mesh, phys, up, logbeta)
    lam = spla.spsolve(Jc.T.tocsc(), dJdu)
    g, gA = stokes.param_grad(mesh, phys, up, lam, logbeta)
    return misfit(mesh, up, u_obs, top), -g, -gA, up


def misfit_complex_step(mesh, phys, logbeta, dlogbeta, u_obs, top, h=1e-30, up0=None):
    """Im J(log beta + i h dlog beta) / h: directional derivative through a
    complex Newton solve (the residual is analytic in u and log beta)."""
    lb = logbeta + 1j * h * dlogbeta
    up = np.zeros(mesh.ndof, dtype=complex) if up0 is None else up0.astype(complex)
    r = stokes.residual(mesh, phys, up, lb)
    r0 = np.linalg.norm(r)
    for _ in range(60):
        J = newton.assemble_jacobian_complex(mesh, phys, up, lb)
        d = spla.spsolve(J.tocsc(), -r)
        alpha = 1.0
        while True:
            rn = stokes.residual(mesh, phys, up + alpha * d, lb)
            if np.linalg.norm(rn) <= (1 - 1e-4 * alpha) * np.linalg.norm(r) or alpha < 1e-4:
                break
            alpha *= 0.5
        up = up + alpha * d
        r = rn
        if np.linalg.norm(r) <= 1e-13 * r0 and alpha == 1.0:
            break
    u, _ = stokes.split(mesh, up)
    dd = u[top] - u_obs
    return np.imag(0.5 * np.sum(dd * dd)) / h
