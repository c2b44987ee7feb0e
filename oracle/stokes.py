"""Residual, Newton Jacobian, parameter gradients and energy (FP64 oracle).

TEST INFRASTRUCTURE: only tests, the smoke check and the CPU-baseline leg of
the benchmark may import this module.  Parity unpinned: none (see the pins in
tests/test_oracle_*.py).

Definitions followed, with dense basis tables at the quadrature points (no sum
factorisation, no fusion):

  viscosity (Eq. 2.2 / Section 2.2, generalised):
      mu(u) = C (gamma D(u):D(u) + delta)^{(1-n)/(2n)},   C = C0 A^{-1/n}
      (the paper's form is gamma = 1/2, delta = eps, C = B = A^{-1/n})
  residual (weak form, Eq. 2.5), velocity test v = phi_a e_c:
      r_{a,c} = int mu D(v):D(u) - p div v - b . v dx + int_{Gamma_b} beta T v . T u ds
  pressure test q = psi_b:   r_b = - int q div u dx
  Newton linearisation (Eqs. 2.6-2.7, generalised to gamma, delta):
      mu'(u) E = mu (E + 2 gamma p_n (D(u):E) / (gamma D(u):D(u) + delta) D(u)),
      p_n = (1 - n) / (2n)
  constraints at the basal nodes (no-slip or u . n = 0, Eq. 2.4b): nodal
  projector P, constrained residual r_c(u) = P r(P u) + s (I - P) u and its
  exact Jacobian P J(P u) P + s (I - P), s = phys.constraint_scale > 0 (the
  solution does not depend on s).
  beta = exp(log beta) with log beta the basal nodal field interpolated by
  the face basis.
  basal sliding (Eq. 2.3: the traction T(sigma n) balances a function of
  |T u|; the linear law beta T u is Eq. 2.4a): traction
      beta s(|T u|^2) T u,   s(x) = (x + eps_s)^{(m-1)/2},
  m = phys.sliding_m, eps_s = phys.sliding_eps; s = 1 for m = 1 (the linear
  law, exactly).  Its Newton derivative in the direction w is
      beta (s T w + 2 s'(|T u|^2) (T u . T w) T u),
  the Picard form keeps s and drops s'.

Every function accepts complex arrays (only analytic operations are used), so
complex-step derivatives of the residual are available to the tests.
"""
import numpy as np

CHUNK = 2048


def _pexp(phys):
    return (1.0 - phys.n) / (2.0 * phys.n)


def split(mesh, up):
    u = up[: 3 * mesh.Nv].reshape(mesh.Nv, 3)
    p = up[3 * mesh.Nv:].reshape(mesh.E, mesh.npr)
    return u, p


def project(mesh, u, transpose=False):
    """Apply the nodal constraint projector P to a velocity array (Nv, 3)."""
    out = u.copy()
    b = mesh.basal
    Pm = mesh.basal_P.transpose(0, 2, 1) if transpose else mesh.basal_P
    out[b] = np.einsum("nij,nj->ni", Pm, u[b])
    return out


def gather(mesh, u):
    """Element nodal values R_i u, shape (E, A, 3) (or (E, A) for scalars)."""
    if u.ndim == 1:
        return (mesh.R @ u).reshape(mesh.E, mesh.A)
    return (mesh.R @ u).reshape(mesh.E, mesh.A, u.shape[1])


def scatter(mesh, ye):
    """Assemble element contributions: sum_i R_i^T y_i."""
    E, A = ye.shape[:2]
    if ye.ndim == 2:
        return mesh.R.T @ ye.reshape(E * A)
    return mesh.R.T @ ye.reshape(E * A, ye.shape[2])


def _grad(mesh, ue, sl):
    """Physical velocity gradient grad[e, q, c, d] = d u_c / d x_d."""
    G = np.einsum("mqa,eac->eqcm", mesh.dphi, ue)
    return np.einsum("eqcm,eqmd->eqcd", G, mesh.Jinv[sl])


def _sym(g):
    return 0.5 * (g + np.swapaxes(g, -1, -2))


def _frob(a, b):
    return np.einsum("...cd,...cd->...", a, b)


def _viscosity(phys, DD):
    return phys.viscosity_prefactor() * (phys.gamma * DD + phys.delta) ** _pexp(phys)


def _integrate(mesh, sl, S_phys, S_val):
    """Element vector sum_q wdetJ [ sum_d dphi_a/dx_d S_phys[c,d] + phi_a S_val[c] ]."""
    wdj = mesh.wdetJ[sl]
    S_ref = np.einsum("eqmd,eqcd->eqcm", mesh.Jinv[sl], S_phys) * wdj[:, :, None, None]
    out = np.einsum("mqa,eqcm->eac", mesh.dphi, S_ref)
    if S_val is not None:
        out = out + np.einsum("qa,eqc->eac", mesh.phi, S_val * wdj[:, :, None])
    return out


def _logbeta_nodal(mesh, logbeta):
    """Scatter the basal nodal log(beta) into a full nodal array (zeros elsewhere)."""
    full = np.zeros(mesh.Nv, dtype=np.result_type(logbeta, np.float64))
    full[mesh.basal] = logbeta
    return full


def _face_terms(mesh, phys, ue, logbeta):
    """Basal face quantities for the basal elements: (elements, beta*w|Js|, n, u at face qp)."""
    eb = mesh.basal_elems
    lbe = gather(mesh, _logbeta_nodal(mesh, logbeta))[eb]
    beta = np.exp(np.einsum("qa,ea->eq", mesh.phiF, lbe))
    uf = np.einsum("qa,eac->eqc", mesh.phiF, ue[eb])
    return eb, beta * mesh.wareaF, mesh.nF, uf


def _tang(n, v):
    return v - n * np.einsum("eqc,eqc->eq", n, v)[..., None]


def _sliding(phys, tu):
    """s and ds/dx at x = |T u|^2 of the sliding law (s = 1, ds = 0 when m = 1)."""
    m = phys.sliding_m
    if m == 1.0:
        return 1.0, 0.0
    x = np.einsum("eqc,eqc->eq", tu, tu) + phys.sliding_eps
    return x ** (0.5 * (m - 1.0)), 0.5 * (m - 1.0) * x ** (0.5 * (m - 3.0))


def element_residual(mesh, phys, ue, pe, logbeta, body=True):
    """Unconstrained element residual vectors (velocity (E,A,3), pressure (E,npr))."""
    dt = np.result_type(ue, pe, logbeta, phys.A, np.float64)
    rv = np.zeros((mesh.E, mesh.A, 3), dtype=dt)
    rp = np.zeros((mesh.E, mesh.npr), dtype=dt)
    bvec = np.asarray(phys.body, dtype=np.float64)
    for s0 in range(0, mesh.E, CHUNK):
        sl = slice(s0, min(s0 + CHUNK, mesh.E))
        g = _grad(mesh, ue[sl], sl)
        D = _sym(g)
        mu = _viscosity(phys, _frob(D, D))
        pq = np.einsum("qb,eb->eq", mesh.Psi, pe[sl])
        sig = mu[..., None, None] * D - pq[..., None, None] * np.eye(3)
        Sval = None
        if body:
            Sval = np.broadcast_to(-bvec, g.shape[:2] + (3,))
        rv[sl] = _integrate(mesh, sl, sig, Sval)
        div = np.einsum("eqcc->eq", g)
        rp[sl] = -np.einsum("qb,eq->eb", mesh.Psi, div * mesh.wdetJ[sl])
    if phys.robin:
        eb, bw, n, uf = _face_terms(mesh, phys, ue, logbeta)
        tu = _tang(n, uf)
        s, _ = _sliding(phys, tu)
        t = tu * (bw * s)[..., None]
        rv[eb] += np.einsum("qa,eqc->eac", mesh.phiF, t)
    return rv, rp


def element_jacobian(mesh, phys, ue, we, qe, logbeta):
    """Element Newton Jacobian action at ue on the direction (we, qe)."""
    dt = np.result_type(ue, we, qe, logbeta, phys.A, np.float64)
    yv = np.zeros((mesh.E, mesh.A, 3), dtype=dt)
    yp = np.zeros((mesh.E, mesh.npr), dtype=dt)
    pn = _pexp(phys)
    for s0 in range(0, mesh.E, CHUNK):
        sl = slice(s0, min(s0 + CHUNK, mesh.E))
        Du = _sym(_grad(mesh, ue[sl], sl))
        gw = _grad(mesh, we[sl], sl)
        Dw = _sym(gw)
        DD = _frob(Du, Du)
        mu = _viscosity(phys, DD)
        # Newton (Eq. 2.7); the Picard linearisation freezes mu and drops this term
        coef = 2.0 * phys.gamma * pn * _frob(Du, Dw) / (phys.gamma * DD + phys.delta)
        if phys.linearization == "picard":
            coef = 0.0 * coef
        stress = mu[..., None, None] * (Dw + coef[..., None, None] * Du)
        pq = np.einsum("qb,eb->eq", mesh.Psi, qe[sl])
        sig = stress - pq[..., None, None] * np.eye(3)
        yv[sl] = _integrate(mesh, sl, sig, None)
        div = np.einsum("eqcc->eq", gw)
        yp[sl] = -np.einsum("qb,eq->eb", mesh.Psi, div * mesh.wdetJ[sl])
    if phys.robin:
        eb, bw, n, wf = _face_terms(mesh, phys, we, logbeta)
        tw = _tang(n, wf)
        t = tw * bw[..., None]
        if phys.sliding_m != 1.0:
            tu = _tang(n, np.einsum("qa,eac->eqc", mesh.phiF, ue[eb]))
            s, ds = _sliding(phys, tu)
            if phys.linearization == "picard":
                ds = 0.0 * ds
            t = bw[..., None] * (s[..., None] * tw + (2.0 * ds * np.einsum("eqc,eqc->eq", tu, tw))[..., None] * tu)
        yv[eb] += np.einsum("qa,eqc->eac", mesh.phiF, t)
    return yv, yp


def _logbeta(mesh, phys, logbeta):
    if logbeta is None:
        return np.zeros(mesh.Nb)
    return logbeta


def residual(mesh, phys, up, logbeta=None):
    """Constrained residual r_c(u, p) = [P r_u(P u, p) + s (I - P) u ; r_p(P u)]."""
    logbeta = _logbeta(mesh, phys, logbeta)
    u, p = split(mesh, up)
    uP = project(mesh, u)
    rv, rp = element_residual(mesh, phys, gather(mesh, uP), p, logbeta)
    ru = scatter(mesh, rv)
    ru = project(mesh, ru, transpose=True) + phys.constraint_scale * (u - project(mesh, u))
    return np.concatenate([ru.ravel(), rp.ravel()])


def jacobian_apply(mesh, phys, up, x, logbeta=None):
    """Constrained Newton Jacobian action  (P J(P u) P + s (I - P)) x; with
    phys.linearization == 'picard' the fixed-viscosity operator instead."""
    logbeta = _logbeta(mesh, phys, logbeta)
    u, _ = split(mesh, up)
    w, qv = split(mesh, x)
    uP = project(mesh, u)
    wP = project(mesh, w)
    yv, yp = element_jacobian(mesh, phys, gather(mesh, uP), gather(mesh, wP), qv, logbeta)
    yu = scatter(mesh, yv)
    yu = project(mesh, yu, transpose=True) + phys.constraint_scale * (w - project(mesh, w))
    return np.concatenate([yu.ravel(), yp.ravel()])


def param_grad(mesh, phys, up, lam, logbeta=None):
    """Adjoint products with the parameter Jacobians of r_c.

    g_logbeta[j] = lam^T d r_c / d log(beta_j)
                 = int_{Gamma_b} beta s(|T P u|^2) phi_j (T P lam) . (T P u) ds
    g_A          = lam^T d r_c / d A = -(1/(n A)) int mu(P u) D(P lam) : D(P u) dx
    (d mu / d A = -mu / (n A) because C = C0 A^{-1/n}).
    """
    logbeta = _logbeta(mesh, phys, logbeta)
    u, _ = split(mesh, up)
    l, _ = split(mesh, lam)
    ue = gather(mesh, project(mesh, u))
    le = gather(mesh, project(mesh, l))
    gA = 0.0
    for s0 in range(0, mesh.E, CHUNK):
        sl = slice(s0, min(s0 + CHUNK, mesh.E))
        Du = _sym(_grad(mesh, ue[sl], sl))
        Dl = _sym(_grad(mesh, le[sl], sl))
        mu = _viscosity(phys, _frob(Du, Du))
        gA = gA + np.sum(mesh.wdetJ[sl] * mu * _frob(Dl, Du))
    gA = -gA / (phys.n * phys.A)
    g = np.zeros(mesh.Nb, dtype=np.result_type(up, lam, logbeta, phys.A, np.float64))
    if phys.robin:
        eb, bw, n, uf = _face_terms(mesh, phys, ue, logbeta)
        lf = np.einsum("qa,eac->eqc", mesh.phiF, le[eb])
        tu = _tang(n, uf)
        sl_s, _ = _sliding(phys, tu)
        s = bw * sl_s * np.einsum("eqc,eqc->eq", _tang(n, lf), tu)
        full = np.zeros((mesh.E, mesh.A), dtype=g.dtype)
        full[eb] = np.einsum("qa,eq->ea", mesh.phiF, s)
        g = scatter(mesh, full)[mesh.basal]
    return g, gA


def energy(mesh, phys, u, logbeta=None):
    """Convex energy whose gradient is the velocity residual (Appendix A).

    E(u) = int C / (2 gamma (1 + p_n)) (gamma D:D + delta)^{1 + p_n} dx
           + int_{Gamma_b} beta F(|T u|^2) ds - int b . u dx,
    F(x) = x / 2 for the linear sliding law (m = 1), else
    F(x) = (x + eps_s)^{(m+1)/2} / (m + 1), so that 2 F'(x) = s(x)
    (unconstrained, velocity only; u has shape (Nv, 3)).
    """
    logbeta = _logbeta(mesh, phys, logbeta)
    ue = gather(mesh, u)
    pn = _pexp(phys)
    C = phys.viscosity_prefactor()
    bvec = np.asarray(phys.body, dtype=np.float64)
    total = 0.0
    for s0 in range(0, mesh.E, CHUNK):
        sl = slice(s0, min(s0 + CHUNK, mesh.E))
        D = _sym(_grad(mesh, ue[sl], sl))
        dens = C / (2.0 * phys.gamma * (1.0 + pn)) * (phys.gamma * _frob(D, D) + phys.delta) ** (1.0 + pn)
        total = total + np.sum(mesh.wdetJ[sl] * dens)
        uq = np.einsum("qa,eac->eqc", mesh.phi, ue[sl])
        total = total - np.sum(mesh.wdetJ[sl] * np.einsum("eqc,c->eq", uq, bvec))
    if phys.robin:
        eb, bw, n, uf = _face_terms(mesh, phys, ue, logbeta)
        tu = _tang(n, uf)
        x = np.einsum("eqc,eqc->eq", tu, tu)
        if phys.sliding_m == 1.0:
            total = total + 0.5 * np.sum(bw * x)
        else:
            m = phys.sliding_m
            total = total + np.sum(bw * (x + phys.sliding_eps) ** (0.5 * (m + 1.0)) / (m + 1.0))
    return total
