"""Parity at the full benchmark sizes.

The 128x128x8 Q2xP1 slab, the 64x64x4 Q3xQ1 and Q4xP3 slabs and the
64x64x4 forest with 30 % refined cells (Q3xP2, hanging faces and edges) are
compared entry by entry with the oracle run on the whole mesh.  The
512x512x8 slab (62M dofs) is compared on sampled rows: the oracle builds the
column block around the sampled nodes (same element shapes and fields), whose
interior rows depend only on elements it contains.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

import stokes_synth as synth
from oracle import OracleMesh, stokes as ostokes
from paper_1406_6573_gb300 import capi
from paper_1406_6573_gb300.mesh import Mesh, State, params


def rel_blocks(o, got, ref):
    nu = 3 * o.Nv
    out = []
    for g, r in ((got[:nu], ref[:nu]), (got[nu:], ref[nu:])):
        out.append(np.linalg.norm(g - r) / np.linalg.norm(r))
    return out


@pytest.mark.parametrize("name", ["slab_128x128x8_q2p1", "slab_128x128x8_q2q0", "slab_64x64x4_q3q1",
                                  "slab_64x64x4_q4p3", "forest_64x64x4_q3p2"])
def test_full_size_parity(name):
    wl = synth.workload(name)
    o = OracleMesh(wl)
    lb = wl.phys.logbeta(*o.basal_coords()[:, :2].T)
    scale = np.concatenate([np.full(3 * o.Nv, 100.0), np.full(o.Np, 1e5)])
    up = synth.uniform_vector(31, o.ndof) * scale
    x = synth.uniform_vector(31, o.ndof, stream=1)
    r_ref = ostokes.residual(o, wl.phys, up, lb)
    j_ref = ostokes.jacobian_apply(o, wl.phys, up, x, lb)
    m = Mesh(wl, device=0)
    assert (m.Nv, m.Np) == (o.Nv, o.Np)
    lbd = torch.as_tensor(lb, device="cuda")
    p = params(wl.phys, lbd)
    upd = torch.as_tensor(up, device="cuda")
    r = torch.empty(o.ndof, dtype=torch.float64, device="cuda")
    capi.stokes_residual(m.handle, p, upd, r, capi.STOKES_F64)
    for err in rel_blocks(o, r.cpu().numpy(), r_ref):
        assert err <= 1e-12, err
    st = State(m, capi.STOKES_F32)
    st.linearize(p, upd)
    y = torch.empty(o.ndof, dtype=torch.float32, device="cuda")
    st.apply(torch.as_tensor(x, dtype=torch.float32, device="cuda"), y)
    for err in rel_blocks(o, y.double().cpu().numpy(), j_ref):
        assert err <= 1e-5, err
    capi.stokes_mesh_status(m.handle)


def test_largest_slab_sampled_rows():
    wl = synth.workload("slab_512x512x8_q2p1")
    k = wl.k
    NX, NY = wl.nx * k, wl.ny * k
    m = Mesh(wl, device=0)
    assert m.Nv == NX * NY * (wl.nz * k + 1)
    xyz = m.node_coords()
    bn = m.basal_nodes()
    lb_full = wl.phys.logbeta(xyz[bn, 0], xyz[bn, 1])
    up = torch.as_tensor(synth.uniform_vector(41, m.ndof), device="cuda")
    up[: 3 * m.Nv] *= 100.0
    up[3 * m.Nv:] *= 1e5
    x = torch.as_tensor(synth.uniform_vector(41, m.ndof, stream=1), device="cuda")
    p = params(wl.phys, torch.as_tensor(lb_full, device="cuda"))
    r = torch.empty(m.ndof, dtype=torch.float64, device="cuda")
    capi.stokes_residual(m.handle, p, up, r, capi.STOKES_F64)
    st = State(m, capi.STOKES_F32)
    st.linearize(p, up)
    y = torch.empty(m.ndof, dtype=torch.float32, device="cuda")
    st.apply(x.float(), y)
    capi.stokes_mesh_status(m.handle)
    r = r.cpu().numpy()
    y = y.double().cpu().numpy()
    up_h = up.cpu().numpy()
    x_h = x.cpu().numpy()
    del st
    rng = np.random.default_rng(5)
    nb = 6
    for ox, oy in [(0, 0), (wl.nx - 3, wl.ny - 2),
                   (int(rng.integers(1, wl.nx - nb)), int(rng.integers(1, wl.ny - nb)))]:
        sb = synth.sub_block(wl, ox, oy, nb, nb)
        o = OracleMesh(sb)
        # sub-block node (I', J', L) -> full lattice node (periodic wrap)
        NXs, NYs = nb * k + 1, nb * k + 1
        g = np.arange(o.Nv)
        Is, Js, Ls = g % NXs, (g // NXs) % NYs, g // (NXs * NYs)
        gf = ((Is + ox * k) % NX) + NX * (((Js + oy * k) % NY) + NY * Ls)
        ex = np.arange(o.E)
        cx, cy, cz = ex % nb, (ex // nb) % nb, ex // (nb * nb)
        ef = ((cx + ox) % wl.nx) + wl.nx * (((cy + oy) % wl.ny) + wl.ny * cz)

        def sub(v):
            return np.concatenate([v[: 3 * m.Nv].reshape(-1, 3)[gf].ravel(),
                                   v[3 * m.Nv:].reshape(-1, m.npr)[ef].ravel()])

        lb_sub = wl.phys.logbeta(*o.basal_coords()[:, :2].T)
        r_sub = ostokes.residual(o, sb.phys, sub(up_h), lb_sub)
        j_sub = ostokes.jacobian_apply(o, sb.phys, sub(up_h), sub(x_h), lb_sub)
        inner = (Is > k) & (Is < NXs - 1 - k) & (Js > k) & (Js < NYs - 1 - k)
        einner = (cx > 0) & (cx < nb - 1) & (cy > 0) & (cy < nb - 1)
        for full, ref, tol in ((r, r_sub, 1e-12), (y, j_sub, 1e-5)):
            rv = ref[: 3 * o.Nv].reshape(-1, 3)[inner]
            gv = full[: 3 * m.Nv].reshape(-1, 3)[gf[inner]]
            assert np.linalg.norm(gv - rv) <= tol * np.linalg.norm(rv), (ox, oy, tol)
            rp = ref[3 * o.Nv:].reshape(-1, m.npr)[einner]
            gp = full[3 * m.Nv:].reshape(-1, m.npr)[ef[einner]]
            assert np.linalg.norm(gp - rp) <= tol * np.linalg.norm(rp), (ox, oy, tol)
