"""Pin of the oracle's adjoint gradient: the adjoint formula (implicit
function theorem, Sections 2.3/8.3) must equal the complex-step derivative of
the misfit through a complex Newton solve of the forward problem, in random
directions of log(beta)."""
import numpy as np

import stokes_synth as synth
from oracle import OracleMesh, adjoint


def test_adjoint_gradient_equals_complex_step_of_forward_solve():
    wl = synth.workload("cbox_3x3x2_q2p1")
    m = OracleMesh(wl)
    top = adjoint.top_nodes(m)
    assert top.size == m.Nb
    lb_ref = wl.phys.logbeta(*m.basal_coords()[:, :2].T)
    # observations from a perturbed reference field
    lb_true = lb_ref + 0.3 * np.cos(2 * np.pi * m.basal_coords()[:, 0] / wl.Lx)
    _, _, _, up_true = adjoint.gradient(m, wl.phys, lb_true, np.zeros((top.size, 3)), top)
    u_obs = up_true[: 3 * m.Nv].reshape(m.Nv, 3)[top]
    J, g, gA, up = adjoint.gradient(m, wl.phys, lb_ref, u_obs, top)
    assert J > 0
    rng = np.random.default_rng(0)
    for _ in range(1):
        d = rng.uniform(-1, 1, size=m.Nb)
        cs = adjoint.misfit_complex_step(m, wl.phys, lb_ref, d, u_obs, top, up0=up)
        assert abs(np.dot(g, d) - cs) <= 1e-7 * abs(cs), (np.dot(g, d), cs)
