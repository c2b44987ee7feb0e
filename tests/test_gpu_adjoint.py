"""GPU adjoint gradient (torch.autograd.Function over the C-ABI) against the
oracle's adjoint gradient (itself pinned by a complex-step derivative of the
forward solve) and against central finite differences of GPU forward solves.

The forward Newton tolerance is 1e-11 relative: on this 3x3x2 box the FP64
residual of the constrained system stalls near 1e-13 absolute (about 1e-12
of the initial residual), the rounding floor of the assembled terms."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import stokes_synth as synth
from oracle import OracleMesh, adjoint as oadjoint
from paper_1406_6573_gb300 import capi
from paper_1406_6573_gb300.adjoint import StokesForward, StokesProblem, misfit, top_nodes
from paper_1406_6573_gb300.mesh import Mesh


def _problem(name):
    wl = synth.workload(name)
    o = OracleMesh(wl)
    lb_ref = wl.phys.logbeta(*o.basal_coords()[:, :2].T)
    lb_true = lb_ref + 0.3 * np.cos(2 * np.pi * o.basal_coords()[:, 0] / wl.Lx)
    top_o = oadjoint.top_nodes(o)
    _, _, _, up_true = oadjoint.gradient(o, wl.phys, lb_true, np.zeros((top_o.size, 3)), top_o)
    u_obs = up_true[: 3 * o.Nv].reshape(o.Nv, 3)[top_o]
    return wl, o, lb_ref, u_obs, top_o


@pytest.mark.parametrize("name", ["cbox_3x3x2_q2p1", "slab_5x3x3_q2p1"])
@pytest.mark.parametrize("inner", [capi.STOKES_F64, capi.STOKES_F32])
def test_adjoint_gradient_matches_oracle(name, inner):
    """cbox: curved box, unit-scale parameters; slab: periodic ice slab in SI
    units (A = 1e-16, slip + Robin), the physics of the large slab workloads."""
    wl, o, lb_ref, u_obs, top_o = _problem(name)
    J_o, g_o, gA_o, _ = oadjoint.gradient(o, wl.phys, lb_ref, u_obs, top_o)
    m = Mesh(wl, device=0)
    prob = StokesProblem(m, wl.phys, inner_prec=inner, rtol=1e-11, adjoint_rtol=1e-11)
    top = top_nodes(m)
    assert np.array_equal(top.cpu().numpy(), top_o)
    lb = torch.as_tensor(lb_ref, dtype=torch.float64, device="cuda").requires_grad_(True)
    A = torch.tensor(wl.phys.A, dtype=torch.float64, device="cuda", requires_grad=True)
    up = StokesForward.apply(lb, A, prob)
    J = misfit(up, torch.as_tensor(u_obs, device="cuda"), m, top)
    J.backward()
    # J is small (u is close to u_obs), so its relative error is the
    # forward solution error over |u - u_obs|, not over |u|
    assert abs(J.item() - J_o) <= 1e-7 * J_o
    g = lb.grad.cpu().numpy()
    assert np.linalg.norm(g - g_o) <= 1e-7 * np.linalg.norm(g_o), np.linalg.norm(g - g_o) / np.linalg.norm(g_o)
    assert abs(A.grad.item() - gA_o) <= 1e-7 * abs(gA_o)
    prob.close()


def test_adjoint_gradient_central_differences():
    wl, o, lb_ref, u_obs, top_o = _problem("cbox_3x3x2_q2p1")
    m = Mesh(wl, device=0)
    prob = StokesProblem(m, wl.phys, inner_prec=capi.STOKES_F32, rtol=1e-11, adjoint_rtol=1e-11)
    top = top_nodes(m)
    uo = torch.as_tensor(u_obs, device="cuda")
    A = torch.tensor(wl.phys.A, dtype=torch.float64, device="cuda")
    lb = torch.as_tensor(lb_ref, dtype=torch.float64, device="cuda").requires_grad_(True)
    J = misfit(StokesForward.apply(lb, A, prob), uo, m, top)
    J.backward()
    g = lb.grad.clone()
    rng = np.random.default_rng(3)
    h = 1e-4
    for _ in range(3):
        d = torch.as_tensor(rng.uniform(-1, 1, size=m.Nb), device="cuda")
        with torch.no_grad():
            Jp = misfit(StokesForward.apply(lb + h * d, A, prob), uo, m, top).item()
            Jm = misfit(StokesForward.apply(lb - h * d, A, prob), uo, m, top).item()
        fd = (Jp - Jm) / (2 * h)
        ad = float((g * d).sum())
        assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)
    prob.close()


@pytest.mark.parametrize("inner", [capi.STOKES_F32])
def test_adjoint_gradient_on_a_block_of_the_largest_slab(inner):
    """The 512 x 512 x 8 slab's generators (random log(beta) field, SI units)
    on a 4 x 4 x 8 column block: the GPU gradient through the multigrid
    forward and adjoint solves against the oracle's adjoint gradient, with
    u_obs = 0 (J = 1/2 |u_top|^2)."""
    wl = synth.sub_block(synth.workload("slab_512x512x8_q2p1"), 100, 37, 4, 4)
    o = OracleMesh(wl)
    lb_ref = wl.phys.logbeta(*o.basal_coords()[:, :2].T)
    top_o = oadjoint.top_nodes(o)
    u_obs = np.zeros((top_o.size, 3))
    J_o, g_o, gA_o, _ = oadjoint.gradient(o, wl.phys, lb_ref, u_obs, top_o, rtol=1e-12)
    m = Mesh(wl, device=0)
    prob = StokesProblem(m, wl.phys, inner_prec=inner, rtol=1e-11, adjoint_rtol=1e-11)
    top = top_nodes(m)
    assert np.array_equal(top.cpu().numpy(), top_o)
    lb = torch.as_tensor(lb_ref, dtype=torch.float64, device="cuda").requires_grad_(True)
    A = torch.tensor(wl.phys.A, dtype=torch.float64, device="cuda", requires_grad=True)
    J = misfit(StokesForward.apply(lb, A, prob), torch.as_tensor(u_obs, device="cuda"), m, top)
    J.backward()
    assert prob.last_forward["mg_levels"] == 2 and prob.last_adjoint["mg_levels"] == 2
    assert abs(J.item() - J_o) <= 1e-8 * J_o
    g = lb.grad.cpu().numpy()
    assert np.linalg.norm(g - g_o) <= 1e-7 * np.linalg.norm(g_o), np.linalg.norm(g - g_o) / np.linalg.norm(g_o)
    assert abs(A.grad.item() - gA_o) <= 1e-7 * abs(gA_o)
    prob.close()
