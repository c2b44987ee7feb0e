"""Pins of the Picard (fixed-viscosity) linearisation.

With mu frozen at u the operator is A(u) w = int mu(u) D(v):D(w) - p div v
- q div w + Robin, and the residual is r(u) = A(u) u - f.  For the
constrained forms (P A P + s (I - P) and P r(P u) + s (I - P) u) this gives
the exact identity  J_Picard(u) u - r_c(u) = -r_c(0)  for every state u.
For n = 1 the viscosity does not depend on u and Picard equals Newton.
"""
import dataclasses

import numpy as np
import pytest

import stokes_synth as synth
from oracle import OracleMesh, newton as onewton, stokes as ostokes

_M = {}


def _mesh(name):
    if name not in _M:
        wl = synth.workload(name)
        o = OracleMesh(wl)
        lb = None if wl.phys.logbeta is None else wl.phys.logbeta(*o.basal_coords()[:, :2].T)
        _M[name] = (wl, o, lb)
    return _M[name]


@pytest.mark.parametrize("name", ["box_4x4x2_q2p1", "cforest_3x3x2_q2p1", "slab_3x3x2_q3p2"])
def test_picard_operator_reproduces_the_residual(name):
    wl, o, lb = _mesh(name)
    phys = dataclasses.replace(wl.phys, linearization="picard")
    up = synth.uniform_vector(5, o.ndof)
    up[: 3 * o.Nv] *= 50.0
    lhs = ostokes.jacobian_apply(o, phys, up, up, lb) - ostokes.residual(o, phys, up, lb)
    rhs = -ostokes.residual(o, phys, np.zeros(o.ndof), lb)
    assert np.linalg.norm(lhs - rhs) <= 1e-12 * np.linalg.norm(ostokes.residual(o, phys, up, lb))


def test_picard_equals_newton_for_linear_viscosity():
    wl, o, lb = _mesh("cforest_3x3x2_q2p1")
    lin = dataclasses.replace(wl.phys, n=1.0)
    up = synth.uniform_vector(6, o.ndof)
    x = synth.uniform_vector(6, o.ndof, stream=1)
    jn = ostokes.jacobian_apply(o, lin, up, x, lb)
    jp = ostokes.jacobian_apply(o, dataclasses.replace(lin, linearization="picard"), up, x, lb)
    assert np.linalg.norm(jn - jp) <= 1e-13 * np.linalg.norm(jn)


def test_picard_differs_from_newton_for_glen_flow():
    wl, o, lb = _mesh("box_4x4x2_q2p1")
    up = synth.uniform_vector(7, o.ndof)
    x = synth.uniform_vector(7, o.ndof, stream=1)
    jn = ostokes.jacobian_apply(o, wl.phys, up, x, lb)
    jp = ostokes.jacobian_apply(o, dataclasses.replace(wl.phys, linearization="picard"), up, x, lb)
    assert np.linalg.norm(jn - jp) >= 1e-2 * np.linalg.norm(jn)


def test_picard_iteration_reaches_the_newton_solution():
    """Both iterations solve r(u) = 0 (unique solution); Picard converges
    linearly, Newton quadratically."""
    wl, o, lb = _mesh("box_4x4x2_q2p1")
    un, hn = onewton.newton_solve(o, wl.phys, lb, rtol=1e-10)
    picard = dataclasses.replace(wl.phys, linearization="picard")
    up, hp = onewton.newton_solve(o, picard, lb, rtol=1e-9, maxit=200)
    assert hp[-1] <= 1e-9 * hp[0]
    assert len(hp) > len(hn)
    assert np.linalg.norm(up - un) <= 1e-6 * np.linalg.norm(un)
