"""Newton solve of the oracle (Section 4.1): residual decrease, quadratic
convergence near the solution, and a unique end point (Appendix A)."""
import numpy as np

import stokes_synth as synth
from oracle import OracleMesh, stokes, newton


def test_newton_config1_converges_quadratically():
    wl = synth.workload("box_4x4x2_q2p1")
    m = OracleMesh(wl)
    up, hist = newton.newton_solve(m, wl.phys, rtol=1e-10)
    assert hist[-1] <= 1e-10 * hist[0]
    assert np.all(np.diff(hist) < 0)
    # observed convergence order of the last steps: log(r_{j+1}/r_j) / log(r_j/r_{j-1})
    r = hist / hist[0]
    order = np.log(r[-1] / r[-2]) / np.log(r[-2] / r[-3])
    assert order > 1.6
    assert np.linalg.norm(stokes.residual(m, wl.phys, up)) <= 1e-10 * hist[0]


def test_newton_end_point_unique():
    wl = synth.workload("cforest_3x3x2_q2p1")
    m = OracleMesh(wl)
    lb = wl.phys.logbeta(*m.basal_coords()[:, :2].T)
    up1, h1 = newton.newton_solve(m, wl.phys, lb, rtol=1e-12)
    start = 0.1 * synth.uniform_vector(9, m.ndof)
    up2, h2 = newton.newton_solve(m, wl.phys, lb, rtol=1e-12, up0=start)
    assert np.linalg.norm(up1 - up2) <= 1e-8 * np.linalg.norm(up1)
