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


def misfit_complex_step(mesh, phys, logbeta, dlogbeta, u_obs, top, up0, h=1e-30, steps=4):
    """Im J(log beta + i h dlog beta) / h: directional derivative through a
    complex Newton solve of the forward problem (the residual is analytic in u
    and log beta).  Starts from the converged real solution up0, so that only
    the O(h) imaginary part is unresolved; full Newton steps (a line search
    on |r| cannot see an O(h) part next to the real part's round-off)."""
    lb = logbeta + 1j * h * dlogbeta
    up = up0.astype(complex)
    for _ in range(steps):
        r = stokes.residual(mesh, phys, up, lb)
        J = newton.assemble_jacobian_complex(mesh, phys, up, lb)
        up = up + spla.spsolve(J.tocsc(), -r)
    u, _ = stokes.split(mesh, up)
    dd = u[top] - u_obs
    return np.imag(0.5 * np.sum(dd * dd)) / h
