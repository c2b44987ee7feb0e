"""Velocity degrees k = 5 .. 9 on the GPU (block-per-element kernels) against
the FP64 oracle: residual, fused Jacobian and its transpose, linearised
state (FP64 and FP32) with its apply and pressure block, parameter
gradients, and a Newton solve whose end point the oracle's residual
accepts.  The paper runs k = 3, 6, 9 in its independence study (Section 5).

Tolerances as in tests/test_gpu_parity.py: norm-wise per block, 1e-12 for
FP64 and 1e-5 for FP32.
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

CASES = [("box_4x4x2_q2p1", 5, "P"),        # no-slip box
         ("slab_5x3x3_q2p1", 6, "Q"),       # periodic slab, slip + Robin, Q_(k-2) pressure
         ("cforest_3x3x2_q3p2", 5, "P"),    # hanging faces and edges on a curved box
         ("cbox_3x3x2_q2p1", 7, "P"),       # curved box, slip
         ("box_3x2x2_q3q1", 9, "Q")]        # degree 9

_cache = {}


def setup(base, k, ps):
    key = (base, k, ps)
    if key not in _cache:
        wl = dataclasses.replace(synth.workload(base), name=f"{base}_k{k}{ps}", k=k, pspace=ps)
        o = OracleMesh(wl)
        m = Mesh(wl, device=0)
        lb = np.zeros(o.Nb) if wl.phys.logbeta is None else wl.phys.logbeta(*o.basal_coords()[:, :2].T)
        _cache[key] = (wl, o, m, lb)
    return _cache[key]


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def close(o, got, ref, tol, what):
    nu = 3 * o.Nv
    for part, g, r in (("velocity", got[:nu], ref[:nu]), ("pressure", got[nu:], ref[nu:])):
        nr = np.linalg.norm(r)
        err = np.linalg.norm(g - r) / nr if nr > 0 else np.linalg.norm(g)
        assert err <= tol, f"{what} {part}: {err:.3e}"


@pytest.mark.parametrize("base,k,ps", CASES)
def test_residual_and_fused_jacobian(base, k, ps):
    wl, o, m, lb = setup(base, k, ps)
    up = synth.uniform_vector(5, o.ndof)
    x = synth.uniform_vector(5, o.ndof, stream=1)
    p = params(wl.phys, dev(lb))
    r = torch.empty(o.ndof, dtype=torch.float64, device="cuda")
    capi.stokes_residual(m.handle, p, dev(up), r, capi.STOKES_F64)
    close(o, r.cpu().numpy(), ostokes.residual(o, wl.phys, up, lb), 1e-12, "residual f64")
    ref = ostokes.jacobian_apply(o, wl.phys, up, x, lb)
    for f in (capi.stokes_jacobian_apply, capi.stokes_jacobian_apply_transpose):
        y = torch.empty_like(r)
        f(m.handle, p, dev(up), dev(x), y, capi.STOKES_F64)
        close(o, y.cpu().numpy(), ref, 1e-12, f"{f.__name__} f64")
    y32 = torch.empty(o.ndof, dtype=torch.float32, device="cuda")
    capi.stokes_jacobian_apply(m.handle, p, dev(up, torch.float32), dev(x, torch.float32), y32, capi.STOKES_F32)
    close(o, y32.double().cpu().numpy(), ref, 1e-5, "jacobian f32")
    r32 = torch.empty(o.ndof, dtype=torch.float32, device="cuda")
    capi.stokes_residual(m.handle, p, dev(up, torch.float32), r32, capi.STOKES_F32)
    close(o, r32.double().cpu().numpy(), ostokes.residual(o, wl.phys, up, lb), 1e-5, "residual f32")


@pytest.mark.parametrize("base,k,ps", CASES)
@pytest.mark.parametrize("prec", [capi.STOKES_F64, capi.STOKES_F32])
def test_state_apply_and_pressure_block(base, k, ps, prec):
    wl, o, m, lb = setup(base, k, ps)
    up = synth.uniform_vector(6, o.ndof)
    x = synth.uniform_vector(6, o.ndof, stream=1)
    dt = torch.float64 if prec == capi.STOKES_F64 else torch.float32
    tol = 1e-12 if prec == capi.STOKES_F64 else 1e-5
    p = params(wl.phys, dev(lb))
    st = State(m, prec)
    st.linearize(p, dev(up))
    ref = ostokes.jacobian_apply(o, wl.phys, up, x, lb)
    y = torch.empty(o.ndof, dtype=dt, device="cuda")
    st.apply(dev(x, dt), y)
    close(o, y.double().cpu().numpy(), ref, tol, "state apply")
    xp = x.copy()
    xp[: 3 * o.Nv] = 0.0
    refp = ostokes.jacobian_apply(o, wl.phys, up, xp, lb)
    st.apply_pressure_block(dev(x, dt), y)
    close(o, y.double().cpu().numpy(), refp, tol, "pressure block")


@pytest.mark.parametrize("base,k,ps", CASES)
def test_param_grad(base, k, ps):
    wl, o, m, lb = setup(base, k, ps)
    up = synth.uniform_vector(7, o.ndof)
    lam = synth.uniform_vector(7, o.ndof, stream=1)
    g_ref, gA_ref = ostokes.param_grad(o, wl.phys, up, lam, lb)
    g = torch.empty(o.Nb, dtype=torch.float64, device="cuda")
    gA = torch.empty(1, dtype=torch.float64, device="cuda")
    capi.stokes_param_grad(m.handle, params(wl.phys, dev(lb)), dev(up), dev(lam), g, gA)
    if np.linalg.norm(g_ref) > 0:
        assert np.linalg.norm(g.cpu().numpy() - g_ref) <= 1e-12 * np.linalg.norm(g_ref)
    assert abs(gA.item() - gA_ref) <= 1e-12 * abs(gA_ref)


@pytest.mark.parametrize("inner", [capi.STOKES_F64, capi.STOKES_F32])
def test_newton_degree_five(inner):
    """Newton on a thin periodic slab at k = 5 (the column-block velocity
    preconditioner suits the column-dominated coupling of thin ice; on the
    isotropic unit box its linear solves stall at this degree)."""
    wl, o, m, lb = setup("slab_5x3x3_q2p1", 5, "P")
    p = params(wl.phys, dev(lb))
    op = capi.stokes_solver_opts()
    op.inner_prec = inner
    op.restart = 30
    op.max_krylov = 4000
    op.max_newton = 60
    op.rtol = 1e-11
    op.eta_max = 0.1
    s = capi.stokes_solver_create(m.handle, op)
    try:
        up = torch.zeros(o.ndof, dtype=torch.float64, device="cuda")
        rc, rep = capi.stokes_newton_solve(s, p, up, check=False)
        assert rc == 0 and rep["converged"], (rc, rep)
        r0 = np.linalg.norm(ostokes.residual(o, wl.phys, np.zeros(o.ndof), lb))
        r = np.linalg.norm(ostokes.residual(o, wl.phys, up.cpu().numpy(), lb))
        assert r <= 1e-10 * r0, r / r0
    finally:
        capi.stokes_solver_destroy(s)
