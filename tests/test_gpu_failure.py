"""Failure paths on the GPU, injected on the host (no kernel is made to fault,
trap or hang).

* Expired waits: the stored-state applies wait, with a bounded number of
  polls, for the bulk copy of each element group's state.  The test hook
  stokes_debug_wait_limit(mesh, 0) makes the first of those waits give up at
  once; the warps then set the mesh's status word, wait (at the normal limit)
  for the copies they issued and return.  stokes_mesh_status must report
  STOKES_E_CUDA once, the solvers must return STOKES_E_CUDA instead of a
  result built on the incomplete product, and with the default limit restored
  the next apply must be parity-green against the oracle.
* Allocation failures: stokes_debug_fail_alloc_after(n) lets the library's
  next n device allocations succeed and fails the one after; every entry
  point that allocates must return STOKES_E_NOMEM, free what it had taken,
  and leave the library usable.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import stokes_synth as synth
from oracle import OracleMesh, stokes as ostokes
from paper_1406_6573_gb300 import capi
from paper_1406_6573_gb300.mesh import Mesh, State, params

E_NOMEM, E_CUDA = -3, -4


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# slab: component-per-lane kernel (FP32) and the warp-per-group kernel (FP64);
# forest: the warp-per-group kernel with hanging nodes, both precisions
@pytest.mark.parametrize("name", ["slab_5x3x3_q2p1", "forest_4x4x2_q2p1", "slab_4x4x2_q4p3"])
@pytest.mark.parametrize("prec", [capi.STOKES_F32, capi.STOKES_F64])
def test_expired_wait_is_reported_and_the_next_apply_is_exact(name, prec):
    wl = synth.workload(name)
    o = OracleMesh(wl)
    m = Mesh(wl, device=0)
    lb = wl.phys.logbeta(*o.basal_coords()[:, :2].T)
    up = synth.uniform_vector(3, o.ndof)
    x = synth.uniform_vector(3, o.ndof, stream=1)
    ref = ostokes.jacobian_apply(o, wl.phys, up, x, lb)
    dt = torch.float32 if prec == capi.STOKES_F32 else torch.float64
    p = params(wl.phys, torch.as_tensor(lb, device="cuda"))
    st = State(m, prec)
    st.linearize(p, torch.as_tensor(up, device="cuda"))
    xd = torch.as_tensor(x, dtype=dt, device="cuda")
    y = torch.empty(o.ndof, dtype=dt, device="cuda")
    capi.stokes_mesh_status(m.handle)                       # clean start
    capi.stokes_debug_wait_limit(m.handle, 0)
    try:
        st.apply(xd, y)
        torch.cuda.synchronize()
        with pytest.raises(capi.StokesError) as e:
            capi.stokes_mesh_status(m.handle)
        assert e.value.code == E_CUDA
        # the incomplete product differs from J x
        assert _rel(y.double().cpu().numpy(), ref) > 0.5
    finally:
        capi.stokes_debug_wait_limit(m.handle, capi.STOKES_WAIT_POLLS_DEFAULT)
    capi.stokes_mesh_status(m.handle)                       # reported once, then clear
    st.apply(xd, y)
    capi.stokes_mesh_status(m.handle)
    tol = 1e-5 if prec == capi.STOKES_F32 else 1e-12
    got = y.double().cpu().numpy()
    nu = 3 * o.Nv
    assert _rel(got[:nu], ref[:nu]) <= tol and _rel(got[nu:], ref[nu:]) <= tol


def test_solver_returns_e_cuda_when_a_wait_expires():
    wl = synth.workload("slab_5x3x3_q2p1")
    m = Mesh(wl, device=0)
    o = OracleMesh(wl)
    lb = wl.phys.logbeta(*o.basal_coords()[:, :2].T)
    p = params(wl.phys, torch.as_tensor(lb, device="cuda"))
    s = capi.stokes_solver_create(m.handle)
    try:
        up = torch.zeros(m.ndof, dtype=torch.float64, device="cuda")
        b = torch.as_tensor(synth.uniform_vector(5, m.ndof), device="cuda")
        xs = torch.zeros_like(b)
        capi.stokes_debug_wait_limit(m.handle, 0)
        try:
            rc, rep = capi.stokes_linear_solve(s, p, up, b, xs, rtol=1e-8, check=False)
            assert rc == E_CUDA, (rc, rep)
            rc, rep = capi.stokes_newton_solve(s, p, up, check=False)
            assert rc == E_CUDA, (rc, rep)
        finally:
            capi.stokes_debug_wait_limit(m.handle, capi.STOKES_WAIT_POLLS_DEFAULT)
        # the solver cleared the word; a normal solve converges
        capi.stokes_mesh_status(m.handle)
        up.zero_()
        rc, rep = capi.stokes_newton_solve(s, p, up, check=False)
        assert rc == 0 and rep["converged"], rep
    finally:
        capi.stokes_solver_destroy(s)


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_allocation_failures_are_reported_and_leak_nothing():
    wl = synth.workload("forest_4x4x2_q2p1")
    # warm-up: the first mesh on a device uploads tables and creates the context
    Mesh(wl, device=0).close()
    free0 = _free_bytes()
    failures = {"mesh": 0, "state": 0, "solver": 0}
    try:
        for n in range(0, 40):
            capi.stokes_debug_fail_alloc_after(n)
            try:
                m = Mesh(wl, device=0)
            except capi.StokesError as e:
                assert e.code == E_NOMEM, e
                failures["mesh"] += 1
                continue
            try:
                try:
                    st = State(m, capi.STOKES_F32)
                    st.close()
                except capi.StokesError as e:
                    assert e.code == E_NOMEM
                    failures["state"] += 1
                    continue
                try:
                    s = capi.stokes_solver_create(m.handle)
                    capi.stokes_solver_destroy(s)
                except capi.StokesError as e:
                    assert e.code == E_NOMEM
                    failures["solver"] += 1
            finally:
                m.close()
    finally:
        assert capi.stokes_debug_fail_alloc_after(-1) >= -1
    assert failures["mesh"] > 5 and failures["state"] >= 1 and failures["solver"] > 5, failures
    # everything taken before a failure was given back
    assert abs(_free_bytes() - free0) < (8 << 20)
    # and the library still works
    m = Mesh(wl, device=0)
    st = State(m, capi.STOKES_F32)
    st.close()
    m.close()
