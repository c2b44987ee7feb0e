"""Discrete inf-sup constants of Q_k x P_{k-1}^disc and Q_k x Q_{k-2}^disc
against the element aspect ratio (Section 3.1: the P_{k-1} pairing's
constant degrades with the aspect ratio, the Q_{k-2} pairing's does not).

TEST INFRASTRUCTURE: only tests (and this module run as a script, to print
the table) use it.

  beta_h = inf_q sup_v (q, div v) / (|v|_1 ||q||_0)

over velocities v in Q_k^3 vanishing on the whole boundary of the unit cube
and discontinuous pressures q orthogonal to the constants.  beta_h^2 is the
smallest non-zero eigenvalue of  (B K^{-1} B^T) q = lambda M q  with K the
vector H^1 seminorm matrix on the interior nodes, B the divergence coupling
(q, div v) and M the pressure mass matrix; the zero eigenvalue belongs to the
constant pressure.  The cube is split into n x n x (n phi) elements, so the
elements have aspect ratio phi (width / height) on a fixed domain (a thin
domain would add its own, continuous, loss of inf-sup stability).
Element integrals use the oracle's Gauss rule and basis tables (the ones the
operator pins fix).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from stokes_synth import flat_field
from stokes_synth.configs import PhysParams, Workload

from .mesh import OracleMesh


def cube_mesh(k, pspace, phi, n=2, side=1.0):
    """Cube [0, side]^3 split into n x n x (n phi) elements of Q_k x pspace."""
    phys = PhysParams(n=1.0, A=1.0, C0=1.0, basal_bc="noslip", robin=False, logbeta=None)
    wl = Workload("infsup_cube", n, n, n * phi, k, pspace, False, side, side, flat_field(0.0),
                  flat_field(side), phys)
    return OracleMesh(wl)


def operators(o):
    """(K_I, [B_c restricted to interior nodes for c = 0, 1, 2], M, interior node list)."""
    G = np.einsum("mqa,eqmd->eqad", o.dphi, o.Jinv)           # physical basis gradients
    Ke = np.einsum("eq,eqad,eqbd->eab", o.wdetJ, G, G)
    Be = np.einsum("eq,qp,eqac->ecpa", o.wdetJ, o.Psi, G)      # (psi_p, d phi_a / d x_c)
    Me = np.einsum("eq,qp,qr->epr", o.wdetJ, o.Psi, o.Psi)
    R = o.R.tocsr()
    K = (R.T @ sp.block_diag([sp.csr_matrix(m) for m in Ke]) @ R).toarray()
    x = o.node_coords()
    lo, hi = x.min(axis=0), x.max(axis=0)
    tol = 1e-9 * float(np.max(hi - lo))
    on_boundary = np.any((np.abs(x - lo) < tol) | (np.abs(x - hi) < tol), axis=1)
    interior = np.where(~on_boundary)[0]
    KI = K[np.ix_(interior, interior)]
    B = [(sp.block_diag([sp.csr_matrix(Be[e, c]) for e in range(o.E)]) @ R).toarray()[:, interior]
         for c in range(3)]
    M = sla.block_diag(*Me)
    return KI, B, M, interior


def infsup(o):
    """(beta_h, the two smallest eigenvalues of (B K^{-1} B^T, M))."""
    KI, B, M, _ = operators(o)
    cf = sla.cho_factor(KI)
    S = sum(Bc @ sla.cho_solve(cf, Bc.T) for Bc in B)
    lam = sla.eigh(S, M, eigvals_only=True)
    return float(np.sqrt(max(lam[1], 0.0))), lam[:2]


def constant_pressure(o):
    """Coefficients of q = 1 in the pressure basis (element L2 projection)."""
    Me = np.einsum("eq,qp,qr->epr", o.wdetJ, o.Psi, o.Psi)
    rhs = np.einsum("eq,qp->ep", o.wdetJ, o.Psi)
    return np.concatenate([np.linalg.solve(Me[e], rhs[e]) for e in range(o.E)])


def table(phis=(1, 2, 4, 8, 16), degrees=(2, 3)):
    rows = []
    for k in degrees:
        for ps in ("P", "Q"):
            rows.append((k, ps, [infsup(cube_mesh(k, ps, phi))[0] for phi in phis]))
    return phis, rows


if __name__ == "__main__":
    phis, rows = table()
    print("k pressure " + " ".join(f"phi={p:<5d}" for p in phis))
    for k, ps, vals in rows:
        name = {"P": f"P{k - 1}", "Q": f"Q{k - 2}"}[ps]
        print(f"{k} {name:8s} " + " ".join(f"{v:9.4f}" for v in vals))
