"""GPU parity: the CUDA library (through the C-ABI) against the FP64 oracle.

Tolerances (norm-wise, per block: velocity rows and pressure rows separately):
  FP64 kernels  ||y_gpu - y_ora|| / ||y_ora|| <= 1e-12
  FP32 kernels  ||y_gpu - y_ora|| / ||y_ora|| <= 1e-5
The FP32 bound: the sum-factorised element operator accumulates O(k)-term
dot products in FP32 (unit roundoff 6e-8) through about ten chained stages,
and atomics add up to 8 element contributions per node in arbitrary order,
so errors of a few 1e-7 relative to the block norm are expected; 1e-5 leaves
a margin for the ill-conditioned anisotropic elements (aspect ratio up to 25).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import stokes_synth as synth
from oracle import OracleMesh, stokes as ostokes
from paper_1406_6573_gb300 import capi
from paper_1406_6573_gb300.mesh import Mesh, State, params

TOL64 = 1e-12
TOL32 = 1e-5

CASES = [
    "box_4x4x2_q2p1",      # conforming box, no-slip base (the 1215 + 128 dof workload)
    "slab_5x3x3_q2p1",     # periodic slab, ragged sizes, slip + Robin
    "slab_8x8x2_q2p1",     # log(beta) random field
    "slab_6x6x2_q3q1",     # Q3 x Q1 pressure
    "slab_3x3x2_q3p2",     # Q3 x P2
    "slab_4x4x2_q4p3",     # Q4 x P3
    "cbox_3x3x2_q3q1",     # curved non-periodic box, slip base
    "forest_4x4x2_q2p1",   # hanging faces and edges, periodic
    "forest_6x6x2_q3p2",   # hanging nodes + random log(beta)
    "cforest_3x3x2_q3p2",  # hanging nodes on a curved box
    "cforest_4x3x2_q4p3",  # hanging nodes, degree 4
    # Q_k x Q_(k-2) pressure (Section 3.2.2), the pairing preferred on anisotropic meshes
    "slab_5x3x3_q2q0",     # Q2 x Q0: component-per-lane kernel with Q pressure
    "cbox_3x3x2_q2q0",     # Q2 x Q0 on a curved box, slip base
    "forest_4x4x2_q2q0",   # Q2 x Q0 with hanging faces and edges
    "slab_4x4x2_q4q2",     # Q4 x Q2
    "cforest_4x3x2_q4q2",  # Q4 x Q2 with hanging nodes on a curved box
]

_cache = {}


def setup(name):
    if name not in _cache:
        wl = synth.workload(name)
        o = OracleMesh(wl)
        m = Mesh(wl, device=0)
        lb = np.zeros(o.Nb) if wl.phys.logbeta is None else wl.phys.logbeta(*o.basal_coords()[:, :2].T)
        _cache[name] = (wl, o, m, lb)
    return _cache[name]


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def blocks(o, v):
    return v[: 3 * o.Nv], v[3 * o.Nv:]


def assert_close(o, got, ref, tol, what):
    for part, (g, r) in zip(("velocity", "pressure"), zip(blocks(o, got), blocks(o, ref))):
        nr = np.linalg.norm(r)
        if nr == 0:
            assert np.linalg.norm(g) <= tol, (what, part)
            continue
        err = np.linalg.norm(g - r) / nr
        assert err <= tol, f"{what} {part}: rel err {err:.3e} > {tol:g} (max-entry {np.abs(g - r).max() / np.abs(r).max():.3e})"


def inputs(o, seed):
    up = synth.uniform_vector(seed, o.ndof)
    x = synth.uniform_vector(seed, o.ndof, stream=1)
    return up, x


@pytest.mark.parametrize("name", CASES)
def test_residual_f64(name):
    wl, o, m, lb = setup(name)
    up, _ = inputs(o, 11)
    ref = ostokes.residual(o, wl.phys, up, lb)
    r = torch.empty(o.ndof, dtype=torch.float64, device="cuda")
    lbd = dev(lb)
    capi.stokes_residual(m.handle, params(wl.phys, lbd), dev(up), r, capi.STOKES_F64)
    assert_close(o, r.cpu().numpy(), ref, TOL64, "residual f64")


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("trans", [False, True])
def test_jacobian_fused_f64(name, trans):
    wl, o, m, lb = setup(name)
    up, x = inputs(o, 12)
    ref = ostokes.jacobian_apply(o, wl.phys, up, x, lb)
    y = torch.empty(o.ndof, dtype=torch.float64, device="cuda")
    lbd = dev(lb)
    f = capi.stokes_jacobian_apply_transpose if trans else capi.stokes_jacobian_apply
    f(m.handle, params(wl.phys, lbd), dev(up), dev(x), y, capi.STOKES_F64)
    assert_close(o, y.cpu().numpy(), ref, TOL64, f"jacobian f64 trans={trans}")


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("prec", [capi.STOKES_F64, capi.STOKES_F32])
def test_state_apply(name, prec):
    wl, o, m, lb = setup(name)
    up, x = inputs(o, 13)
    ref = ostokes.jacobian_apply(o, wl.phys, up, x, lb)
    dt = torch.float64 if prec == capi.STOKES_F64 else torch.float32
    lbd = dev(lb)
    st = State(m, prec)
    st.linearize(params(wl.phys, lbd), dev(up))
    y = torch.empty(o.ndof, dtype=dt, device="cuda")
    st.apply(dev(x, dt), y)
    tol = TOL64 if prec == capi.STOKES_F64 else TOL32
    assert_close(o, y.double().cpu().numpy(), ref, tol, f"state apply prec={prec}")
    yt = torch.empty_like(y)
    st.apply_transpose(dev(x, dt), yt)
    assert_close(o, yt.double().cpu().numpy(), ref, tol, f"state apply^T prec={prec}")


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("prec", [capi.STOKES_F64, capi.STOKES_F32])
def test_state_pressure_block(name, prec):
    """y = J_c (0, x_p): against the oracle Jacobian applied to x with its
    velocity part zeroed (velocity rows P B^T x_p, pressure rows zero)."""
    wl, o, m, lb = setup(name)
    up, x = inputs(o, 17)
    xp = x.copy()
    xp[: 3 * o.Nv] = 0.0
    ref = ostokes.jacobian_apply(o, wl.phys, up, xp, lb)
    assert np.linalg.norm(ref[3 * o.Nv:]) == 0.0
    dt = torch.float64 if prec == capi.STOKES_F64 else torch.float32
    st = State(m, prec)
    st.linearize(params(wl.phys, dev(lb)), dev(up))
    y = torch.full((o.ndof,), float("nan"), dtype=dt, device="cuda")
    st.apply_pressure_block(dev(x, dt), y)
    tol = TOL64 if prec == capi.STOKES_F64 else TOL32
    assert_close(o, y.double().cpu().numpy(), ref, tol, f"pressure block prec={prec}")


@pytest.mark.parametrize("name", CASES)
def test_fused_f32(name):
    wl, o, m, lb = setup(name)
    up, x = inputs(o, 14)
    ref_r = ostokes.residual(o, wl.phys, up, lb)
    ref_j = ostokes.jacobian_apply(o, wl.phys, up, x, lb)
    lbd = dev(lb)
    p = params(wl.phys, lbd)
    r = torch.empty(o.ndof, dtype=torch.float32, device="cuda")
    capi.stokes_residual(m.handle, p, dev(up, torch.float32), r, capi.STOKES_F32)
    assert_close(o, r.double().cpu().numpy(), ref_r, TOL32, "residual f32")
    y = torch.empty(o.ndof, dtype=torch.float32, device="cuda")
    capi.stokes_jacobian_apply(m.handle, p, dev(up, torch.float32), dev(x, torch.float32), y, capi.STOKES_F32)
    assert_close(o, y.double().cpu().numpy(), ref_j, TOL32, "jacobian f32")


@pytest.mark.parametrize("name", CASES)
def test_param_grad_f64(name):
    wl, o, m, lb = setup(name)
    up, lam = inputs(o, 15)
    g_ref, gA_ref = ostokes.param_grad(o, wl.phys, up, lam, lb)
    lbd = dev(lb)
    g = torch.empty(o.Nb, dtype=torch.float64, device="cuda")
    gA = torch.empty(1, dtype=torch.float64, device="cuda")
    capi.stokes_param_grad(m.handle, params(wl.phys, lbd), dev(up), dev(lam), g, gA)
    g = g.cpu().numpy()
    if np.linalg.norm(g_ref) > 0:
        assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) <= TOL64
    else:
        assert np.abs(g).max() == 0
    assert abs(gA.item() - gA_ref) <= TOL64 * abs(gA_ref)


def test_dot_product_transpose_f64():
    """<y, J x> = <J^T y, x> on a hanging-node mesh (Section 4.1 symmetry)."""
    wl, o, m, lb = setup("forest_6x6x2_q3p2")
    up, x = inputs(o, 16)
    yv = synth.uniform_vector(16, o.ndof, stream=5)
    lbd = dev(lb)
    p = params(wl.phys, lbd)
    Jx = torch.empty(o.ndof, dtype=torch.float64, device="cuda")
    JTy = torch.empty_like(Jx)
    capi.stokes_jacobian_apply(m.handle, p, dev(up), dev(x), Jx, capi.STOKES_F64)
    capi.stokes_jacobian_apply_transpose(m.handle, p, dev(up), dev(yv), JTy, capi.STOKES_F64)
    a = float(np.dot(yv, Jx.cpu().numpy()))
    b = float(np.dot(JTy.cpu().numpy(), x))
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))


def test_empty_hanging_free_paths_agree():
    """Forcing the general node numbering (all-zero refinement mask) gives the same operator."""
    wl = synth.workload("slab_5x3x3_q2p1")
    a = Mesh(wl, device=0)
    b = Mesh(wl, device=0, force_general=True)
    o = OracleMesh(wl)
    lb = wl.phys.logbeta(*o.basal_coords()[:, :2].T)
    up, x = inputs(o, 17)
    lbd = dev(lb)
    p = params(wl.phys, lbd)
    ya = torch.empty(o.ndof, dtype=torch.float64, device="cuda")
    yb = torch.empty_like(ya)
    capi.stokes_jacobian_apply(a.handle, p, dev(up), dev(x), ya, capi.STOKES_F64)
    capi.stokes_jacobian_apply(b.handle, p, dev(up), dev(x), yb, capi.STOKES_F64)
    assert torch.allclose(ya, yb, rtol=1e-13, atol=0)


@pytest.mark.parametrize("name", ["box_4x4x2_q2p1", "slab_8x8x2_q2p1", "forest_6x6x2_q3p2", "slab_4x4x2_q4p3"])
@pytest.mark.parametrize("prec", [capi.STOKES_F64, capi.STOKES_F32])
def test_picard_operators(name, prec):
    """Picard (fixed-viscosity) linearisation: stored-state and fused applies
    against the oracle's Picard operator."""
    import dataclasses
    wl, o, m, lb = setup(name)
    phys = dataclasses.replace(wl.phys, linearization="picard")
    up, x = inputs(o, 23)
    ref = ostokes.jacobian_apply(o, phys, up, x, lb)
    dt = torch.float64 if prec == capi.STOKES_F64 else torch.float32
    tol = TOL64 if prec == capi.STOKES_F64 else TOL32
    lbd = dev(lb)
    p = params(phys, lbd)
    st = State(m, prec)
    st.linearize(p, dev(up))
    y = torch.empty(o.ndof, dtype=dt, device="cuda")
    st.apply(dev(x, dt), y)
    assert_close(o, y.double().cpu().numpy(), ref, tol, f"picard state apply prec={prec}")
    yf = torch.empty(o.ndof, dtype=dt, device="cuda")
    capi.stokes_jacobian_apply(m.handle, p, dev(up, dt), dev(x, dt), yf, prec)
    assert_close(o, yf.double().cpu().numpy(), ref, tol, f"picard fused apply prec={prec}")


def test_picard_identity_on_the_gpu():
    """J_Picard(u) u - r_c(u) = -r_c(0) with the GPU operators (FP64)."""
    import dataclasses
    wl, o, m, lb = setup("cforest_3x3x2_q3p2")
    phys = dataclasses.replace(wl.phys, linearization="picard")
    up = synth.uniform_vector(9, o.ndof)
    up[: 3 * o.Nv] *= 50.0
    lbd = dev(lb)
    p = params(phys, lbd)
    u = dev(up)
    ju = torch.empty_like(u)
    capi.stokes_jacobian_apply(m.handle, p, u, u, ju, capi.STOKES_F64)
    r = torch.empty_like(u)
    capi.stokes_residual(m.handle, p, u, r, capi.STOKES_F64)
    r0 = torch.empty_like(u)
    capi.stokes_residual(m.handle, p, torch.zeros_like(u), r0, capi.STOKES_F64)
    err = float((ju - r + r0).norm())
    assert err <= 1e-12 * float(r.norm()), err / float(r.norm())


@pytest.mark.parametrize("name", ["cbox_3x3x2_q2p1", "slab_5x3x3_q2p1"])
def test_gridded_bed_operators(name):
    """Geometry from heights on the horizontal GLL lattice (a random gridded
    bed): residual, fused Jacobian and FP32 state apply against the oracle
    built on the same heights."""
    import dataclasses
    from test_library import _GridLookup
    wl = synth.workload(name)
    host = Mesh(wl, device=-1)
    bxy = host.node_coords()[host.basal_nodes(), :2]
    surf = wl.surface(bxy[:, 0], bxy[:, 1])
    bed = wl.bed(bxy[:, 0], bxy[:, 1])
    rbed = bed + np.random.default_rng(21).uniform(-0.03, 0.03, size=bed.shape) * (surf - bed)
    per = (wl.Lx, wl.Ly) if wl.periodic else None
    gw = dataclasses.replace(wl, bed=_GridLookup(bxy, rbed, per), surface=_GridLookup(bxy, surf, per))
    o = OracleMesh(gw)
    m = Mesh(wl, device=0, grid=(rbed, surf))
    lb = np.zeros(o.Nb) if wl.phys.logbeta is None else wl.phys.logbeta(*o.basal_coords()[:, :2].T)
    up, x = inputs(o, 27)
    p = params(wl.phys, dev(lb))
    r = torch.empty(o.ndof, dtype=torch.float64, device="cuda")
    capi.stokes_residual(m.handle, p, dev(up), r, capi.STOKES_F64)
    assert_close(o, r.cpu().numpy(), ostokes.residual(o, wl.phys, up, lb), TOL64, "gridded residual")
    ref = ostokes.jacobian_apply(o, wl.phys, up, x, lb)
    y = torch.empty(o.ndof, dtype=torch.float64, device="cuda")
    capi.stokes_jacobian_apply(m.handle, p, dev(up), dev(x), y, capi.STOKES_F64)
    assert_close(o, y.cpu().numpy(), ref, TOL64, "gridded jacobian")
    st = State(m, capi.STOKES_F32)
    st.linearize(p, dev(up))
    y32 = torch.empty(o.ndof, dtype=torch.float32, device="cuda")
    st.apply(dev(x, torch.float32), y32)
    assert_close(o, y32.double().cpu().numpy(), ref, TOL32, "gridded state apply")
