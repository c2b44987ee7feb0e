"""CPU checks of the CUDA library: it loads, exports every symbol of
include/stokes.h, rejects bad arguments, and its host mesh builder agrees
with the oracle's independent construction (node count and coordinates,
basal node set, element count)."""
import dataclasses
import re

import numpy as np
import pytest

import stokes_synth as synth
from oracle import OracleMesh
from paper_1406_6573_gb300 import capi
from paper_1406_6573_gb300.mesh import Mesh, mesh_desc


def _header_symbols():
    src = open(capi.os.path.join(capi.HERE, "..", "include", "stokes.h")).read()
    return sorted(set(re.findall(r"\b(stokes_[A-Za-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = capi.lib()
    names = _header_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(capi._SIGS)


def test_invalid_arguments_are_rejected():
    wl = synth.workload("box_4x4x2_q2p1")
    d, keep = mesh_desc(wl, device=-1)
    d.k = 10
    with pytest.raises(capi.StokesError) as e:
        capi.stokes_mesh_create(d)
    assert e.value.code == -1 and "degree" in str(e.value)
    d.k = 2
    d.nx = 0
    with pytest.raises(capi.StokesError):
        capi.stokes_mesh_create(d)
    # host-only meshes refuse compute calls
    m = Mesh(wl, device=-1)
    p = capi.stokes_params()
    with pytest.raises(capi.StokesError) as e:
        capi.stokes_residual(m.handle, p, None, None, capi.STOKES_F64, 0)
    assert e.value.code == -1


def _periodic_dist(a, b, L):
    d = a - b
    return np.abs(d - L * np.round(d / L))


MESHES = ["box_4x4x2_q2p1", "slab_8x8x2_q2p1", "slab_5x3x3_q2p1", "forest_4x4x2_q2p1",
          "cforest_3x3x2_q3p2", "forest_6x6x2_q3p2", "cforest_4x3x2_q4p3", "slab_4x4x2_q4p3",
          "cbox_3x3x2_q3q1", "slab_6x6x2_q3q1", "slab_5x3x3_q2q0", "forest_4x4x2_q2q0",
          "slab_4x4x2_q4q2", "cforest_4x3x2_q4q2", "cbox_3x3x2_q2q0"]


HIGH_K = [("box_4x4x2_q2p1", 5, "P"), ("slab_5x3x3_q2p1", 6, "Q"), ("cforest_3x3x2_q3p2", 6, "P"),
          ("box_4x4x2_q2p1", 9, "Q")]


def _high_k(base, k, ps):
    import dataclasses
    wl = synth.workload(base)
    return dataclasses.replace(wl, name=f"{base}_k{k}{ps}", k=k, pspace=ps)


@pytest.mark.parametrize("base,k,ps", HIGH_K)
def test_host_mesh_matches_oracle_high_degree(base, k, ps):
    """Degrees 5..9 (the paper's range, Section 7): the host mesh builder and
    the oracle agree on counts, coordinates and basal nodes, including
    hanging nodes (device meshes of these degrees run the block-per-element
    kernels, tests/test_gpu_high_degree.py)."""
    _compare_with_oracle(_high_k(base, k, ps))


@pytest.mark.parametrize("name", MESHES)
def test_host_mesh_matches_oracle(name):
    _compare_with_oracle(synth.workload(name))


def _compare_with_oracle(wl):
    m = Mesh(wl, device=-1)
    o = OracleMesh(wl)
    assert (m.E, m.Nv, m.Np, m.Nb) == (o.E, o.Nv, o.Np, o.Nb)
    a, b = m.node_coords(), o.node_coords()
    scale = max(wl.Lx, wl.Ly)
    for d, L in ((0, wl.Lx), (1, wl.Ly)):
        dd = _periodic_dist(a[:, d], b[:, d], L) if wl.periodic else np.abs(a[:, d] - b[:, d])
        assert dd.max() < 1e-12 * scale
    assert np.abs(a[:, 2] - b[:, 2]).max() < 1e-10 * max(1.0, np.abs(b[:, 2]).max())
    np.testing.assert_array_equal(m.basal_nodes(), o.basal)
    assert (m.n_hanging > 0) == bool(o.fine.any() and (o.hang_cell >= 0).any())


def test_general_numbering_equals_lattice_numbering():
    wl = synth.workload("slab_5x3x3_q2p1")
    a = Mesh(wl, device=-1)
    b = Mesh(wl, device=-1, force_general=True)
    assert a.Nv == b.Nv
    np.testing.assert_allclose(a.node_coords(), b.node_coords(), rtol=0, atol=1e-9)


@pytest.mark.parametrize("name", ["slab_128x128x8_q2p1", "slab_64x64x4_q3q1", "slab_64x64x4_q4p3"])
def test_full_size_counts(name):
    wl = synth.workload(name)
    m = Mesh(wl, device=-1)
    assert m.Nv == (wl.nx * wl.k) * (wl.ny * wl.k) * (wl.nz * wl.k + 1)
    assert m.Nb == (wl.nx * wl.k) * (wl.ny * wl.k)
    assert m.E == wl.n_coarse and m.Np == m.E * m.npr


def test_forest_full_size_builds():
    wl = synth.workload("forest_64x64x4_q3p2")
    m = Mesh(wl, device=-1)
    nref = int(wl.refine_mask().sum())
    assert m.E == wl.n_coarse + 7 * nref
    assert m.n_hanging > 0 and m.Np == m.E * 10


def test_allocation_failure_hook_settings():
    """The allocation-failure hook is process-wide and returns its previous
    setting; host-only meshes allocate no device memory and are unaffected."""
    prev = capi.stokes_debug_fail_alloc_after(0)
    try:
        assert prev == -1
        m = Mesh(synth.workload("box_4x4x2_q2p1"), device=-1)
        m.close()
        assert capi.stokes_debug_fail_alloc_after(7) == 0
        assert capi.stokes_debug_fail_alloc_after(-5) == 7
    finally:
        capi.stokes_debug_fail_alloc_after(-1)
    assert capi.stokes_debug_fail_alloc_after(-1) == -1


def test_wait_limit_hook_needs_a_device_mesh():
    m = Mesh(synth.workload("box_4x4x2_q2p1"), device=-1)
    with pytest.raises(capi.StokesError) as e:
        capi.stokes_debug_wait_limit(m.handle, 0)
    assert e.value.code == -1


class _GridLookup:
    """Bed or surface heights given at the horizontal lattice points (x, y)
    of a mesh, looked up by position (a callable like a modal field)."""

    def __init__(self, xy, values, period=None):
        self.period = period
        self.table = {(round(float(x), 9), round(float(y), 9)): float(v) for (x, y), v in zip(xy, values)}

    def __call__(self, x, y):
        x, y = np.broadcast_arrays(np.asarray(x, dtype=np.float64), np.asarray(y, dtype=np.float64))
        if self.period is not None:      # periodic meshes evaluate at x = Lx, y = Ly too
            x = np.where(np.isclose(x, self.period[0]), 0.0, x)
            y = np.where(np.isclose(y, self.period[1]), 0.0, y)
        out = np.array([self.table[(round(float(a), 9), round(float(b), 9))] for a, b in zip(x.ravel(), y.ravel())])
        return out.reshape(x.shape)


@pytest.mark.parametrize("name", ["cbox_3x3x2_q2p1", "slab_5x3x3_q2p1", "cbox_3x3x2_q3q1"])
def test_gridded_geometry(name):
    """Heights given on the horizontal GLL lattice (stokes_mesh_desc.bed_nodes,
    surface_nodes): sampled from the modal fields they give the modal mesh
    exactly; a random gridded bed gives the oracle's mesh built on the same
    heights."""
    import dataclasses
    wl = synth.workload(name)
    a = Mesh(wl, device=-1)
    xyz = a.node_coords()
    bxy = xyz[a.basal_nodes(), :2]            # the lattice, [Y][X] order (X fastest)
    bed = wl.bed(bxy[:, 0], bxy[:, 1])
    surf = wl.surface(bxy[:, 0], bxy[:, 1])
    b = Mesh(wl, device=-1, grid=(bed, surf))
    # equal up to the rounding of the modal series at x = Lx vs its wrapped x = 0
    np.testing.assert_allclose(a.node_coords(), b.node_coords(), rtol=0,
                               atol=1e-12 * max(wl.Lx, np.abs(surf).max()))
    rng = np.random.default_rng(9)
    rbed = bed + rng.uniform(-0.02, 0.02, size=bed.shape) * (surf - bed)
    c = Mesh(wl, device=-1, grid=(rbed, surf))
    per = (wl.Lx, wl.Ly) if wl.periodic else None
    o = OracleMesh(dataclasses.replace(wl, bed=_GridLookup(bxy, rbed, per), surface=_GridLookup(bxy, surf, per)))
    assert c.Nv == o.Nv
    assert np.abs(c.node_coords()[:, 2] - o.node_coords()[:, 2]).max() < 1e-12 * max(1.0, np.abs(surf).max())
    np.testing.assert_array_equal(c.basal_nodes(), o.basal)
    with pytest.raises(capi.StokesError):
        d, keep = mesh_desc(wl, device=-1, grid=(rbed, surf))
        d.surface_nodes = None
        capi.stokes_mesh_create(d)


def test_offset_sub_block_geometry():
    """A column block of a slab (origin x0, y0 != 0) builds the geometry of
    its physical position: the node heights equal the oracle's."""
    wl = synth.sub_block(synth.workload("slab_512x512x8_q2p1"), 100, 37, 3, 2)
    m = Mesh(wl, device=-1)
    o = OracleMesh(wl)
    a, b = m.node_coords(), o.node_coords()
    np.testing.assert_allclose(a[:, 0] + wl.x0, b[:, 0], rtol=0, atol=1e-9 * wl.Lx)
    np.testing.assert_allclose(a[:, 2], b[:, 2], rtol=0, atol=1e-9 * np.abs(b[:, 2]).max())


@pytest.mark.parametrize("name", ["forest_4x4x2_q2p1", "forest_6x6x2_q3p2", "cforest_3x3x2_q2p1",
                                  "cforest_4x3x2_q4p3", "forest_4x4x2_q2q0"])
def test_forest_multigrid_prolongation(name):
    """The forest multigrid's first coarse level is the unrefined base mesh;
    its prolongation (base Q_k functions evaluated at the forest's
    independent nodes) reproduces the forest's node coordinates from the
    base's (the children inherit the parent map), and has unit row sums."""
    wl = synth.workload(name)
    f = Mesh(wl, device=-1)
    b = Mesh(dataclasses.replace(wl, refine_frac=0.0), device=-1)
    nnz, err = capi.stokes_debug_forest_prolongation(f.handle, b.handle)
    assert nnz >= f.Nv and err < 1e-12, (nnz, err)
    # a base mesh that is not the forest's: refused
    other = Mesh(dataclasses.replace(wl, refine_frac=0.0, nz=wl.nz + 1), device=-1)
    with pytest.raises(capi.StokesError):
        capi.stokes_debug_forest_prolongation(f.handle, other.handle)


def _gll(k):
    """GLL nodes of degree k on [-1, 1]: the end points and the roots of P_k'."""
    from numpy.polynomial import legendre as L
    inner = np.sort(L.legroots(L.legder([0] * k + [1]))) if k > 1 else np.array([])
    return np.concatenate([[-1.0], inner, [1.0]])


def _lattice_x(n_el, k, scale):
    """Node positions of a non-periodic degree-k lattice of n_el elements of
    length `scale` (element e, local node i at e + (g_i + 1) / 2)."""
    g = _gll(k)
    x = [scale * (e + 0.5 * (g[i] + 1.0)) for e in range(n_el) for i in range(k)]
    return np.array(x + [scale * n_el])


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("nf", [4, 6])
def test_multigrid_transfer_tables(k, nf):
    """The velocity multigrid's 1-D transfers: P interpolates degree-k data
    of the coarse lattice (nf / 2 elements of length 2) at the fine nodes
    exactly, R is exactly P^T, J interpolates degree-k data of the fine
    lattice at the coarse nodes exactly; the periodic P is the non-periodic
    one with the end nodes identified."""
    xf = _lattice_x(nf, k, 1.0)
    xc = _lattice_x(nf // 2, k, 2.0)
    P = capi.stokes_debug_mg_transfer(nf, k, False, 0)
    R = capi.stokes_debug_mg_transfer(nf, k, False, 1)
    J = capi.stokes_debug_mg_transfer(nf, k, False, 2)
    assert P.shape == (len(xf), len(xc)) and R.shape == J.shape == (len(xc), len(xf))
    for j in range(k + 1):
        fc, ff = (xc / nf) ** j, (xf / nf) ** j
        assert np.max(np.abs(P @ fc - ff)) < 1e-13, (k, nf, j)
        assert np.max(np.abs(J @ ff - fc)) < 1e-13, (k, nf, j)
    assert np.array_equal(R, P.T)
    # a degree-(k + 1) function is not reproduced: the tables are of degree k
    assert np.max(np.abs(P @ (xc / nf) ** (k + 1) - (xf / nf) ** (k + 1))) > 1e-6
    Pp = capi.stokes_debug_mg_transfer(nf, k, True, 0)
    fold = P[:-1].copy()
    fold[:, 0] += fold[:, -1]
    assert np.allclose(Pp, fold[:, :-1], rtol=0, atol=1e-15)
    assert np.array_equal(capi.stokes_debug_mg_transfer(nf, k, True, 1), Pp.T)


def test_multigrid_transfer_tables_reject_bad_shapes():
    with pytest.raises(capi.StokesError):
        capi.stokes_debug_mg_transfer(5, 2, False, 0)       # odd element count
    with pytest.raises(capi.StokesError):
        capi.stokes_debug_mg_transfer(4, 5, False, 0)       # degree above 4
