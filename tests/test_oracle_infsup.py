"""The inf-sup study of Section 3.1 (oracle/infsup.py).

Pins of the computation, fixed by the mathematics:
  * the constant pressure is orthogonal to the divergence of every velocity
    vanishing on the boundary (divergence theorem): B^T 1 = 0, and the
    smallest eigenvalue is zero;
  * beta_h is invariant under a uniform scaling of the domain (catches a
    missing or doubled Jacobian factor in K or B).
Then the paper's statement itself: on a fixed domain, beta_h of
Q_k x Q_{k-2} stays bounded as the element aspect ratio phi grows, beta_h of
Q_k x P_{k-1} decays.
"""
import numpy as np
import pytest

from oracle import infsup


@pytest.mark.parametrize("k,ps", [(2, "P"), (2, "Q"), (3, "P"), (3, "Q")])
def test_constant_pressure_is_the_null_mode(k, ps):
    o = infsup.cube_mesh(k, ps, 2)
    _, B, M, _ = infsup.operators(o)
    one = infsup.constant_pressure(o)
    scale = max(np.abs(Bc).max() for Bc in B) * np.abs(one).max()
    for Bc in B:
        assert np.abs(one @ Bc).max() <= 1e-13 * scale * Bc.shape[0]
    beta, lam = infsup.infsup(o)
    assert abs(lam[0]) <= 1e-12 * lam[1]
    assert 0.05 < beta < 1.0


@pytest.mark.parametrize("k,ps", [(2, "P"), (3, "Q")])
def test_infsup_constant_is_scale_invariant(k, ps):
    b1, _ = infsup.infsup(infsup.cube_mesh(k, ps, 4, side=1.0))
    b7, _ = infsup.infsup(infsup.cube_mesh(k, ps, 4, side=7.0))
    assert abs(b1 - b7) <= 1e-10 * b1


def test_q_pressure_is_uniform_and_p_pressure_degrades_with_aspect_ratio():
    for k, phi in ((2, 16), (3, 8)):
        bq = [infsup.infsup(infsup.cube_mesh(k, "Q", f))[0] for f in (1, phi)]
        bp = [infsup.infsup(infsup.cube_mesh(k, "P", f))[0] for f in (1, phi)]
        assert bq[1] >= 0.8 * bq[0], (k, bq)
        assert bp[1] <= 0.7 * bp[0], (k, bp)
        assert bp[1] < bq[1], (k, bp, bq)
