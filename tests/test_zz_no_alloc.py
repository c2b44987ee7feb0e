"""The fixed-order A-gradient that allocates nothing, against stokes_param_grad.

stokes_param_grad_A_fixed_order keeps its per-warp partial sums in a static
device array of the library (no allocation).  It must give the A-gradient of
stokes_param_grad up to summation order, give bitwise the same value on two
calls in a row (nothing left over in the scratch from the first call changes
the second), and refuse meshes that need more partials than the array holds.
This file sorts last so that it also runs after every other GPU test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import stokes_synth as synth
from paper_1406_6573_gb300 import capi
from paper_1406_6573_gb300.mesh import Mesh, params


def _inputs(m, wl, seed):
    up = torch.as_tensor(synth.uniform_vector(seed, m.ndof), device="cuda")
    up[: 3 * m.Nv] *= 100.0
    lam = torch.as_tensor(synth.uniform_vector(seed, m.ndof, stream=2), device="cuda")
    xyz = m.node_coords()
    bn = m.basal_nodes()
    lb = torch.as_tensor(wl.phys.logbeta(xyz[bn, 0], xyz[bn, 1]) if wl.phys.logbeta is not None
                         else np.zeros(m.Nb), device="cuda")
    return up, lam, params(wl.phys, lb)


@pytest.mark.parametrize("name", ["cforest_3x3x2_q2p1", "slab_6x6x2_q3q1", "slab_4x4x2_q4p3",
                                  "slab_128x128x8_q2p1"])
def test_fixed_order_matches_param_grad_twice(name):
    wl = synth.workload(name)
    m = Mesh(wl, device=0)
    up, lam, p = _inputs(m, wl, 17)
    ref = torch.empty(1, dtype=torch.float64, device="cuda")
    capi.stokes_param_grad(m.handle, p, up, lam, None, ref)
    got = []
    for _ in range(2):
        g = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        capi.stokes_param_grad_A_fixed_order(m.handle, p, up, lam, g)
        torch.cuda.synchronize()
        got.append(g.item())
    r = ref.item()
    assert np.isfinite(r) and r != 0.0
    assert abs(got[0] - r) <= 1e-12 * abs(r), (got[0], r)
    assert got[1] == got[0]
    capi.stokes_mesh_status(m.handle)


def test_fixed_order_after_other_inputs():
    """A call on other inputs in between leaves no trace in the next result."""
    wl = synth.workload("slab_8x8x2_q2p1")
    m = Mesh(wl, device=0)
    up, lam, p = _inputs(m, wl, 3)
    up2, lam2, _ = _inputs(m, wl, 4)
    g = torch.empty(1, dtype=torch.float64, device="cuda")
    capi.stokes_param_grad_A_fixed_order(m.handle, p, up, lam, g)
    first = g.item()
    capi.stokes_param_grad_A_fixed_order(m.handle, p, up2, lam2, g)
    other = g.item()
    capi.stokes_param_grad_A_fixed_order(m.handle, p, up, lam, g)
    assert g.item() == first and other != first


def test_fixed_order_rejects_meshes_beyond_the_scratch():
    wl = synth.workload("slab_512x512x8_q2p1")       # 2,097,152 Q2 elements: 699,052 partials
    m = Mesh(wl, device=0)
    up = torch.zeros(m.ndof, dtype=torch.float64, device="cuda")
    p = params(wl.phys, torch.zeros(m.Nb, dtype=torch.float64, device="cuda"))
    g = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.StokesError) as e:
        capi.stokes_param_grad_A_fixed_order(m.handle, p, up, up, g)
    assert e.value.code == -1      # STOKES_E_INVAL
    assert g.item() == 7.0
