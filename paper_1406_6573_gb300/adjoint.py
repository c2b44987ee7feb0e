"""Adjoint gradients of a surface-velocity misfit with respect to log(beta) and A.

The forward map log(beta) -> u(log beta) is the Newton solve of the
constrained residual r_c(u; log beta, A) = 0 (Eq. 2.5 with the basal sliding
law of Eq. 2.4; Section 4.1).  By the implicit function theorem the gradient
of a functional J(u) is

    dJ/dm = -lambda^T d r_c / d m,     J_c(u)^T lambda = dJ/du,

i.e. one adjoint solve with the Jacobian transpose (the "adjoint equations"
of Sections 2.3 and 8.3) and one parameter-Jacobian product
(stokes_param_grad).  Everything runs in the CUDA library through the C-ABI;
this module only wires the calls into torch.autograd.
"""
import numpy as np
import torch

from . import capi
from .mesh import params


class StokesForward(torch.autograd.Function):
    """u = solve(r_c(u; log beta, A) = 0); backward: adjoint solve + param grad.

    forward(logbeta, A, ctxobj) with logbeta a CUDA FP64 tensor [Nb] and A a
    0-d FP64 tensor; ctxobj carries the mesh, physics, solver and tolerances.
    Returns the converged state vector up [3 Nv + Np] (FP64, CUDA).
    """

    @staticmethod
    def forward(ctx, logbeta, A, cobj):
        phys = cobj.phys_with_A(float(A))
        p = params(phys, logbeta.contiguous())
        up = torch.zeros(cobj.mesh.ndof, dtype=torch.float64, device=logbeta.device)
        rc, rep = capi.stokes_newton_solve(cobj.solver, p, up)
        if rc != 0:
            raise RuntimeError(f"forward Newton solve did not converge: {rep}")
        cobj.last_forward = rep
        ctx.cobj = cobj
        ctx.scale = rep["constraint_scale"]
        ctx.save_for_backward(logbeta, up)
        ctx.A = float(A)
        return up

    @staticmethod
    def backward(ctx, grad_up):
        logbeta, up = ctx.saved_tensors
        cobj = ctx.cobj
        phys = cobj.phys_with_A(ctx.A)
        p = params(phys, logbeta.contiguous(), constraint_scale=ctx.scale)
        lam = torch.zeros_like(up)
        rhs = grad_up.contiguous().to(torch.float64)
        rc, rep = capi.stokes_linear_solve(cobj.solver, p, up, rhs, lam, transpose=True,
                                           rtol=cobj.adjoint_rtol)
        if rc != 0:
            raise RuntimeError(f"adjoint solve did not converge: {rep}")
        cobj.last_adjoint = rep
        g = torch.empty_like(logbeta)
        gA = torch.empty(1, dtype=torch.float64, device=up.device)
        capi.stokes_param_grad(cobj.mesh.handle, p, up, lam, g, gA)
        return -g, -gA[0], None


class StokesProblem:
    """Mesh + physics + solver bundle used by StokesForward."""

    def __init__(self, mesh, phys, inner_prec=capi.STOKES_F32, rtol=1e-12, adjoint_rtol=1e-10,
                 restart=30, max_krylov=4000, max_newton=60, velocity_mg=1, eta_max=1e-4):
        import dataclasses
        self.mesh = mesh
        self.phys = phys
        self._replace = dataclasses.replace
        op = capi.stokes_solver_opts()
        op.inner_prec = inner_prec
        op.restart = restart
        op.max_krylov = max_krylov
        op.max_newton = max_newton
        op.rtol = rtol
        op.eta_max = eta_max
        op.velocity_mg = velocity_mg     # multigrid velocity block where the mesh allows it
        self.solver = capi.stokes_solver_create(mesh.handle, op)
        self.adjoint_rtol = adjoint_rtol
        self.last_forward = None
        self.last_adjoint = None

    def phys_with_A(self, A):
        return self._replace(self.phys, A=A)

    def close(self):
        if getattr(self, "solver", None) is not None:
            capi.stokes_solver_destroy(self.solver)
            self.solver = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def top_nodes(mesh):
    """Indices of the top-surface velocity nodes of a conforming slab mesh.

    Global nodes are ordered by reference Z first, so on a conforming lattice
    the top layer is the last block of nodes, as many as the basal layer."""
    if mesh.n_hanging:
        raise ValueError("top_nodes needs a conforming (unrefined) slab mesh")
    return torch.arange(mesh.Nv - mesh.Nb, mesh.Nv, device="cuda")


def surface_velocity(up, mesh, top):
    return up[: 3 * mesh.Nv].view(mesh.Nv, 3)[top]


def misfit(up, u_obs, mesh, top):
    """J = 1/2 sum over top-surface velocity nodes of |u - u_obs|^2 (nodal l2)."""
    d = surface_velocity(up, mesh, top) - u_obs
    return 0.5 * (d * d).sum()
