"""Pins of the oracle's basal face geometry and slip projector on non-flat beds.

What the mathematics fixes (Eq. 2.4: u . n = 0 and T = I - n n^T on the bed;
Section 3.2.1: isoparametric map with x, y affine in each cell):

  * tilted planar bed z = alpha x + beta y + c: the isoparametric map
    reproduces the plane exactly, so every basal nodal normal equals
    (-alpha, -beta, 1) / sqrt(1 + alpha^2 + beta^2), the projector
    annihilates it, and sum_q w |J_s| equals the plane's area
    Lx Ly sqrt(1 + alpha^2 + beta^2) (also on 2:1 forests);
  * curved bed, graph surface z = b_h(x, y) with b_h the Q_k interpolant of
    the bed: n ds = (-d b_h/dx, -d b_h/dy, 1) dx dy, so the unnormalised
    nodal normal int phi_i n ds of each element is a sum of products of the
    1-D integrals int l_a l_c and int l_a l_c' of GLL Lagrange polynomials,
    computed here by exact polynomial integration (numpy.polynomial), with
    no quadrature table of the oracle;
  * curved bed: the discrete bed area sum_q w |J_s| converges to
    int sqrt(1 + b_x^2 + b_y^2) dx dy, the derivatives of the cosine series
    taken analytically and the integral by a fine tensor Gauss rule.
"""
import dataclasses
import math

import numpy as np
import pytest
from numpy.polynomial import Polynomial, legendre

import stokes_synth as synth
from oracle import OracleMesh


class Plane:
    """z = alpha x + beta y + c (a bed or surface callable like ModalField)."""

    def __init__(self, alpha, beta, c):
        self.alpha, self.beta, self.c = alpha, beta, c

    def __call__(self, x, y):
        return self.alpha * np.asarray(x, dtype=np.float64) + self.beta * np.asarray(y, dtype=np.float64) + self.c


def tilted(name, alpha, beta, k=2, pspace="P", refine=0.0, n=(3, 2, 2)):
    base = synth.workload("cbox_3x3x2_q2p1")
    return dataclasses.replace(base, name=f"tilted_{name}", nx=n[0], ny=n[1], nz=n[2], k=k, pspace=pspace,
                               bed=Plane(alpha, beta, 0.1), surface=Plane(alpha, beta, 1.1),
                               refine_frac=refine, refine_seed=3)


PLANES = [
    ("q2", 0.3, -0.2, 2, "P", 0.0),
    ("q3", -0.45, 0.15, 3, "Q", 0.0),
    ("q2_forest", 0.25, 0.35, 2, "P", 0.4),
    ("q3_forest", -0.1, 0.5, 3, "P", 0.4),
]


@pytest.mark.parametrize("name,alpha,beta,k,ps,refine", PLANES)
def test_tilted_plane_nodal_normals_and_projector(name, alpha, beta, k, ps, refine):
    m = OracleMesh(tilted(name, alpha, beta, k, ps, refine))
    exact = np.array([-alpha, -beta, 1.0]) / math.sqrt(1.0 + alpha ** 2 + beta ** 2)
    n = m.basal_normal * np.sign(m.basal_normal[:, 2:3])
    assert np.abs(n - exact[None]).max() < 1e-14
    # the slip projector annihilates the normal and keeps the tangent plane
    P = m.basal_P
    assert np.abs(np.einsum("nij,j->ni", P, exact)).max() < 1e-14
    t1 = np.array([1.0, 0.0, alpha])
    t2 = np.array([0.0, 1.0, beta])
    assert np.abs(np.einsum("nij,j->ni", P, t1) - t1).max() < 1e-14
    assert np.abs(np.einsum("nij,j->ni", P, t2) - t2).max() < 1e-14
    # symmetric and idempotent
    assert np.abs(P - P.transpose(0, 2, 1)).max() < 1e-15
    assert np.abs(np.einsum("nij,njk->nik", P, P) - P).max() < 1e-14


@pytest.mark.parametrize("name,alpha,beta,k,ps,refine", PLANES)
def test_tilted_plane_face_area(name, alpha, beta, k, ps, refine):
    wl = tilted(name, alpha, beta, k, ps, refine)
    m = OracleMesh(wl)
    exact = wl.Lx * wl.Ly * math.sqrt(1.0 + alpha ** 2 + beta ** 2)
    assert abs(m.wareaF.sum() - exact) / exact < 1e-14
    # pointwise: the unit normal at every face Gauss point is the plane's
    nrm = np.array([-alpha, -beta, 1.0]) / math.sqrt(1.0 + alpha ** 2 + beta ** 2)
    nF = m.nF * np.sign(m.nF[..., 2:3])
    assert np.abs(nF - nrm).max() < 1e-14


# ------------------------------------------------------------ curved beds
def _gll_nodes(n1):
    """GLL nodes: +-1 and the roots of P_k' (k = n1 - 1)."""
    r = legendre.Legendre.basis(n1 - 1).deriv().roots().real
    return np.sort(np.concatenate([[-1.0], r, [1.0]]))


def _lagrange_polys(nodes):
    out = []
    for a, xa in enumerate(nodes):
        p = Polynomial([1.0])
        for j, xj in enumerate(nodes):
            if j != a:
                p = p * Polynomial([-xj, 1.0]) / (xa - xj)
        out.append(p)
    return out


def _int11(p):
    P = p.integ()
    return P(1.0) - P(-1.0)


def closed_form_nodal_normals(wl):
    """Unnormalised nodal normals int phi_i n ds on the basal node lattice of a
    conforming, non-periodic mesh, from exact 1-D polynomial integrals.

    On the element [x0, x0 + hx] x [y0, y0 + hy] with bed nodal values
    B[c, d] (tensor GLL nodes), n ds = (-(hy/2) d_xi b_h, -(hx/2) d_eta b_h,
    hx hy / 4) d xi d eta, so node (a, b) receives
        x: -(hy/2) sum_cd B[c,d] Mp[a,c] M[b,d]
        y: -(hx/2) sum_cd B[c,d] M[a,c] Mp[b,d]
        z:  (hx hy / 4) m[a] m[b]
    with M[a,c] = int l_a l_c, Mp[a,c] = int l_a l_c', m[a] = int l_a.
    """
    k = wl.k
    n1 = k + 1
    nodes = _gll_nodes(n1)
    ell = _lagrange_polys(nodes)
    M = np.array([[_int11(ell[a] * ell[c]) for c in range(n1)] for a in range(n1)])
    Mp = np.array([[_int11(ell[a] * ell[c].deriv()) for c in range(n1)] for a in range(n1)])
    mv = np.array([_int11(ell[a]) for a in range(n1)])
    hx, hy = wl.Lx / wl.nx, wl.Ly / wl.ny
    NX, NY = wl.nx * k + 1, wl.ny * k + 1
    xs, ys = np.zeros(NX), np.zeros(NY)
    for cx in range(wl.nx):
        xs[cx * k:cx * k + n1] = wl.x0 + cx * hx + hx * (nodes + 1.0) / 2.0
    for cy in range(wl.ny):
        ys[cy * k:cy * k + n1] = wl.y0 + cy * hy + hy * (nodes + 1.0) / 2.0
    acc = np.zeros((NX, NY, 3))
    for cx in range(wl.nx):
        for cy in range(wl.ny):
            sx, sy = slice(cx * k, cx * k + n1), slice(cy * k, cy * k + n1)
            X, Y = np.meshgrid(xs[sx], ys[sy], indexing="ij")
            B = wl.bed(X, Y)
            acc[sx, sy, 0] += -(hy / 2.0) * np.einsum("cd,ac,bd->ab", B, Mp, M)
            acc[sx, sy, 1] += -(hx / 2.0) * np.einsum("cd,ac,bd->ab", B, M, Mp)
            acc[sx, sy, 2] += (hx * hy / 4.0) * np.outer(mv, mv)
    return xs, ys, acc


@pytest.mark.parametrize("name", ["cbox_3x3x2_q2p1", "cbox_3x3x2_q3q1"])
def test_curved_bed_nodal_normals_closed_form(name):
    wl = synth.workload(name)
    m = OracleMesh(wl)
    xs, ys, acc = closed_form_nodal_normals(wl)
    bc = m.basal_coords()
    I = np.searchsorted(xs, bc[:, 0] - 1e-12)
    J = np.searchsorted(ys, bc[:, 1] - 1e-12)
    assert np.allclose(xs[I], bc[:, 0], atol=1e-13) and np.allclose(ys[J], bc[:, 1], atol=1e-13)
    ref = acc[I, J]
    assert ref.shape == m.basal_nodal_vec.shape
    assert np.abs(m.basal_nodal_vec - ref).max() / np.abs(ref).max() < 1e-13
    nref = ref / np.linalg.norm(ref, axis=1)[:, None]
    assert np.abs(m.basal_normal - nref).max() < 1e-13
    # the projector of the slip condition is built from the unit normal
    P = m.basal_P
    assert np.abs(np.einsum("nij,nj->ni", P, nref)).max() < 1e-13
    assert np.abs(np.einsum("nij,njk->nik", P, P) - P).max() < 1e-13


def _bed_area(bed, Lx, Ly, cells=40, pts=40):
    """int_0^Lx int_0^Ly sqrt(1 + b_x^2 + b_y^2), derivatives of the cosine
    series analytically, composite Gauss-Legendre rule."""
    g, w = legendre.leggauss(pts)
    xs = ((np.arange(cells)[:, None] + (g[None, :] + 1.0) / 2.0).ravel() / cells) * Lx
    ys = ((np.arange(cells)[:, None] + (g[None, :] + 1.0) / 2.0).ravel() / cells) * Ly
    wx = np.tile(w / 2.0, cells) / cells * Lx
    wy = np.tile(w / 2.0, cells) / cells * Ly
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    bx, by = np.zeros_like(X), np.zeros_like(X)
    for a, kx, ky, ph in zip(bed.amp, bed.kx, bed.ky, bed.phase):
        s = np.sin(kx * X + ky * Y + ph)
        bx -= a * kx * s
        by -= a * ky * s
    return float(np.sum(np.outer(wx, wy) * np.sqrt(1.0 + bx ** 2 + by ** 2)))


@pytest.mark.parametrize("k", [2, 3])
def test_curved_bed_area_converges(k):
    base = synth.workload("cbox_3x3x2_q2p1")
    exact = _bed_area(base.bed, base.Lx, base.Ly)
    errs = []
    for n in (4, 8, 16):
        m = OracleMesh(dataclasses.replace(base, nx=n, ny=n, nz=1, k=k, pspace="P"))
        errs.append(abs(m.wareaF.sum() - exact) / exact)
    errs = np.array(errs)
    assert np.all(errs[1:] < errs[:-1])
    # isoparametric Q_k bed: over h = 1/4 -> 1/16 the area error falls at
    # least as h^(k+1) (observed about h^4 for k = 2, h^4.8 for k = 3)
    rate = np.log2(errs[0] / errs[-1]) / 2.0
    assert rate > k + 0.75, (errs, rate)
    assert errs[-1] < (5e-6 if k == 2 else 1e-8)
