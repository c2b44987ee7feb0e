"""GPU parity of the nonlinear basal sliding law against the FP64 oracle.

Traction beta s(|T u|^2) T u, s(x) = (x + eps_s)^{(m-1)/2}, m = 1/3 (the
oracle's pins: tests/test_oracle_sliding.py).  The same tolerances as the
linear operators (tests/test_gpu_parity.py): 1e-12 for FP64, 1e-5 for FP32,
norm-wise per block.  Covered: the residual (face term with u = x), the
fused Jacobian (face term linearised at u), the stored-state applies (the
linearisation kept per basal Gauss point, read by the stored-state kernels'
basal tail), the log(beta) adjoint product, the Picard form, and a Newton
solve that reaches the oracle's solution.
"""
import dataclasses

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
M_SLIDE = 1.0 / 3.0
CASES = ["slab_5x3x3_q2p1", "slab_8x8x2_q2p1", "forest_6x6x2_q3p2", "cforest_3x3x2_q3p2", "slab_4x4x2_q4p3"]

_cache = {}


def setup(name):
    if name not in _cache:
        wl = synth.workload(name)
        wl = dataclasses.replace(wl, phys=dataclasses.replace(wl.phys, sliding_m=M_SLIDE, robin=True,
                                                              basal_bc="slip"))
        o = OracleMesh(wl)
        m = Mesh(wl, device=0)
        lb = np.zeros(o.Nb) if wl.phys.logbeta is None else wl.phys.logbeta(*o.basal_coords()[:, :2].T)
        _cache[name] = (wl, o, m, lb)
    return _cache[name]


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def assert_close(o, got, ref, tol, what):
    for part, sl in (("velocity", slice(0, 3 * o.Nv)), ("pressure", slice(3 * o.Nv, None))):
        g, r = got[sl], ref[sl]
        nr = np.linalg.norm(r)
        if nr == 0:
            assert np.linalg.norm(g) <= tol, (what, part)
            continue
        err = np.linalg.norm(g - r) / nr
        assert err <= tol, f"{what} {part}: rel err {err:.3e} > {tol:g}"


def inputs(o, seed):
    return synth.uniform_vector(seed, o.ndof), synth.uniform_vector(seed, o.ndof, stream=1)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("prec", [capi.STOKES_F64, capi.STOKES_F32])
def test_sliding_residual(name, prec):
    wl, o, m, lb = setup(name)
    up, _ = inputs(o, 21)
    ref = ostokes.residual(o, wl.phys, up, lb)
    # the sliding term matters: the linear law gives another residual
    lin = ostokes.residual(o, dataclasses.replace(wl.phys, sliding_m=1.0), up, lb)
    assert np.linalg.norm(ref - lin) > 1e-6 * np.linalg.norm(ref)
    dt = torch.float64 if prec == capi.STOKES_F64 else torch.float32
    r = torch.empty(o.ndof, dtype=dt, device="cuda")
    capi.stokes_residual(m.handle, params(wl.phys, dev(lb)), dev(up, dt), r, prec)
    assert_close(o, r.double().cpu().numpy(), ref, TOL64 if prec == capi.STOKES_F64 else TOL32, "residual")


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("trans", [False, True])
def test_sliding_fused_jacobian_f64(name, trans):
    wl, o, m, lb = setup(name)
    up, x = inputs(o, 22)
    ref = ostokes.jacobian_apply(o, wl.phys, up, x, lb)
    y = torch.empty(o.ndof, dtype=torch.float64, device="cuda")
    f = capi.stokes_jacobian_apply_transpose if trans else capi.stokes_jacobian_apply
    f(m.handle, params(wl.phys, dev(lb)), dev(up), dev(x), y, capi.STOKES_F64)
    assert_close(o, y.cpu().numpy(), ref, TOL64, f"fused jacobian trans={trans}")


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("prec", [capi.STOKES_F64, capi.STOKES_F32])
@pytest.mark.parametrize("lin", ["newton", "picard"])
def test_sliding_state_apply(name, prec, lin):
    wl, o, m, lb = setup(name)
    phys = dataclasses.replace(wl.phys, linearization=lin)
    up, x = inputs(o, 23)
    ref = ostokes.jacobian_apply(o, phys, up, x, lb)
    dt = torch.float64 if prec == capi.STOKES_F64 else torch.float32
    st = State(m, prec)
    st.linearize(params(phys, dev(lb)), dev(up))
    tol = TOL64 if prec == capi.STOKES_F64 else TOL32
    y = torch.empty(o.ndof, dtype=dt, device="cuda")
    st.apply(dev(x, dt), y)
    assert_close(o, y.double().cpu().numpy(), ref, tol, f"state apply {lin} prec={prec}")
    yt = torch.empty_like(y)
    st.apply_transpose(dev(x, dt), yt)
    assert_close(o, yt.double().cpu().numpy(), ref, tol, f"state apply^T {lin} prec={prec}")


@pytest.mark.parametrize("name", CASES)
def test_sliding_param_grad_f64(name):
    wl, o, m, lb = setup(name)
    up, lam = inputs(o, 24)
    g_ref, gA_ref = ostokes.param_grad(o, wl.phys, up, lam, lb)
    g = torch.empty(o.Nb, dtype=torch.float64, device="cuda")
    gA = torch.empty(1, dtype=torch.float64, device="cuda")
    capi.stokes_param_grad(m.handle, params(wl.phys, dev(lb)), dev(up), dev(lam), g, gA)
    assert np.linalg.norm(g.cpu().numpy() - g_ref) <= TOL64 * np.linalg.norm(g_ref)
    assert abs(gA.item() - gA_ref) <= TOL64 * abs(gA_ref)


# (On the forest_6x6x2_q3p2 mesh with nonlinear sliding the column
# preconditioner leaves the FGMRES solves at their iteration cap and Newton
# stalls, although exact Newton converges there in 15 steps: a preconditioner
# limit, not an operator error; the operators are covered above on that mesh.)
@pytest.mark.parametrize("name", ["slab_5x3x3_q2p1", "slab_8x8x2_q2p1"])
@pytest.mark.parametrize("inner", [capi.STOKES_F64, capi.STOKES_F32])
def test_sliding_newton_reaches_oracle_solution(name, inner):
    wl, o, m, lb = setup(name)
    op = capi.stokes_solver_opts()
    op.inner_prec = inner
    op.restart = 30
    op.max_krylov = 3000
    op.max_newton = 60
    op.rtol = 1e-11
    op.eta_max = 0.1
    s = capi.stokes_solver_create(m.handle, op)
    try:
        up = torch.zeros(o.ndof, dtype=torch.float64, device="cuda")
        rc, rep = capi.stokes_newton_solve(s, params(wl.phys, dev(lb)), up)
        assert rc == 0 and rep["converged"], rep
        r0 = np.linalg.norm(ostokes.residual(o, wl.phys, np.zeros(o.ndof), lb))
        r = np.linalg.norm(ostokes.residual(o, wl.phys, up.cpu().numpy(), lb))
        assert r <= 1e-10 * r0, (r / r0, rep)
    finally:
        capi.stokes_solver_destroy(s)


@pytest.mark.parametrize("name", ["slab_8x8x2_q2p1", "forest_6x6x2_q3p2"])
@pytest.mark.parametrize("inner", [capi.STOKES_F64, capi.STOKES_F32])
def test_sliding_newton_multigrid(name, inner):
    """Nonlinear sliding with the multigrid velocity block: on the Q3 forest,
    where the column blocks alone stall, the base-level correction carries the
    horizontal couplings and Newton reaches the oracle's solution."""
    wl, o, m, lb = setup(name)
    op = capi.stokes_solver_opts()
    op.inner_prec = inner
    op.restart = 30
    op.max_krylov = 3000
    op.max_newton = 60
    op.rtol = 1e-11
    op.eta_max = 1e-4
    op.velocity_mg = 1
    s = capi.stokes_solver_create(m.handle, op)
    try:
        up = torch.zeros(o.ndof, dtype=torch.float64, device="cuda")
        rc, rep = capi.stokes_newton_solve(s, params(wl.phys, dev(lb)), up)
        assert rc == 0 and rep["converged"] and rep["mg_levels"] >= 2, rep
        r0 = np.linalg.norm(ostokes.residual(o, wl.phys, np.zeros(o.ndof), lb))
        r = np.linalg.norm(ostokes.residual(o, wl.phys, up.cpu().numpy(), lb))
        assert r <= 1e-10 * r0, (r / r0, rep)
    finally:
        capi.stokes_solver_destroy(s)


def test_sliding_parameters_are_checked():
    wl, o, m, lb = setup("slab_5x3x3_q2p1")
    bad = dataclasses.replace(wl.phys, sliding_eps=0.0)
    r = torch.empty(o.ndof, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.StokesError, match="sliding"):
        capi.stokes_residual(m.handle, params(bad, dev(lb)), dev(np.zeros(o.ndof)), r, capi.STOKES_F64)
