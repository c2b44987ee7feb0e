"""Assembled Jacobian and damped Newton solve (FP64 oracle).

TEST INFRASTRUCTURE: only tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module.

Section 4.1: Newton's method on the discrete residual, whose Jacobian is the
exact derivative of the discretisation (discretise-then-differentiate), with a
line search that makes the residual norm decrease.  The oracle assembles the
constrained Jacobian P J P + (I - P) as a sparse matrix, A = sum_i R_i^T A_i
R_i, with the element matrices A_i obtained column by column from the element
Jacobian action, and solves each Newton system with a sparse direct solver.
The line search is plain backtracking on ||r||_2 (the paper's weak-Wolfe
details are not given); the stopping rule is ||r_j|| / ||r_0|| <= rtol.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import stokes


def _restriction_full(mesh):
    """Sparse map from global dofs to stacked element dofs [vel (A*3), pres (npr)]."""
    E, A, npr, Nv = mesh.E, mesh.A, mesh.npr, mesh.Nv
    nde = 3 * A + npr
    R = mesh.R.tocoo()
    e, a = np.divmod(R.row, A)
    rows, cols, vals = [], [], []
    for c in range(3):
        rows.append(e * nde + 3 * a + c); cols.append(3 * R.col + c); vals.append(R.data)
    ee, bb = np.meshgrid(np.arange(E), np.arange(npr), indexing="ij")
    rows.append((ee * nde + 3 * A + bb).ravel())
    cols.append((3 * Nv + ee * npr + bb).ravel())
    vals.append(np.ones(E * npr))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(E * nde, mesh.ndof))


def element_matrices(mesh, phys, up, logbeta=None):
    """Element Jacobians K[e] (nde x nde), nde = 3 A + npr, at the state up."""
    logbeta = stokes._logbeta(mesh, phys, logbeta)
    u, _ = stokes.split(mesh, up)
    ue = stokes.gather(mesh, stokes.project(mesh, u))
    E, A, npr = mesh.E, mesh.A, mesh.npr
    nde = 3 * A + npr
    K = np.zeros((E, nde, nde), dtype=np.result_type(up, logbeta, np.float64))
    for j in range(nde):
        we = np.zeros((E, A, 3)); qe = np.zeros((E, npr))
        if j < 3 * A:
            we[:, j // 3, j % 3] = 1.0
        else:
            qe[:, j - 3 * A] = 1.0
        yv, yp = stokes.element_jacobian(mesh, phys, ue, we, qe, logbeta)
        K[:, : 3 * A, j] = yv.reshape(E, 3 * A)
        K[:, 3 * A:, j] = yp
    return K


def projector_matrix(mesh):
    """The nodal constraint projector P as a sparse ndof x ndof matrix."""
    n = mesh.ndof
    P = sp.lil_matrix((n, n))
    d = np.ones(n)
    d[np.concatenate([3 * mesh.basal + c for c in range(3)])] = 0.0
    P.setdiag(d)
    P = P.tocsr()
    rows, cols, vals = [], [], []
    for i, g in enumerate(mesh.basal):
        for a in range(3):
            for b in range(3):
                rows.append(3 * g + a); cols.append(3 * g + b); vals.append(mesh.basal_P[i, a, b])
    return P + sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def assemble_jacobian_complex(mesh, phys, up, logbeta=None):
    """Same as assemble_jacobian for complex states / parameters."""
    return assemble_jacobian(mesh, phys, up, logbeta)


def assemble_jacobian(mesh, phys, up, logbeta=None):
    """Constrained global Jacobian P (sum_i R_i^T A_i R_i) P + s (I - P), sparse."""
    K = element_matrices(mesh, phys, up, logbeta)
    E, nde = K.shape[0], K.shape[1]
    e, i, j = np.meshgrid(np.arange(E), np.arange(nde), np.arange(nde), indexing="ij")
    Kb = sp.csr_matrix((K.ravel(), ((e * nde + i).ravel(), (e * nde + j).ravel())),
                       shape=(E * nde, E * nde), dtype=K.dtype)
    Rf = _restriction_full(mesh)
    J = (Rf.T @ Kb @ Rf).tocsr()
    P = projector_matrix(mesh)
    I = sp.identity(mesh.ndof, format="csr")
    return (P @ J @ P + phys.constraint_scale * (I - P)).tocsr()


def newton_solve(mesh, phys, logbeta=None, rtol=1e-10, maxit=60, up0=None, verbose=False):
    """Damped Newton from up0 (default 0) until ||r|| <= rtol ||r_0||.

    Returns (up, history of ||r_j||).
    """
    up = np.zeros(mesh.ndof) if up0 is None else up0.copy()
    r = stokes.residual(mesh, phys, up, logbeta)
    hist = [np.linalg.norm(r)]
    for _ in range(maxit):
        if hist[-1] <= rtol * hist[0]:
            break
        J = assemble_jacobian(mesh, phys, up, logbeta)
        d = spla.spsolve(J.tocsc(), -r)
        alpha, nr = 1.0, np.inf
        while alpha > 1e-6:
            r_new = stokes.residual(mesh, phys, up + alpha * d, logbeta)
            nr = np.linalg.norm(r_new)
            if nr <= (1.0 - 1e-4 * alpha) * hist[-1]:
                break
            alpha *= 0.5
        up = up + alpha * d
        r = r_new
        hist.append(nr)
        if verbose:
            print(f"newton {len(hist) - 1}: |r| = {nr:.3e}  alpha = {alpha:g}")
    return up, np.array(hist)
