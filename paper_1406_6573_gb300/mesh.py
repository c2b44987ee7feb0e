"""Mesh and parameter handles over the C-ABI (argument marshalling only)."""
import ctypes as C

import numpy as np
import torch

from . import capi


def _field(f, keep, x0=0.0, y0=0.0):
    """stokes_field from an object with mean/amp/kx/ky/phase (numpy arrays);
    (x0, y0): physical position of the mesh origin, folded into the phases
    (f(x0 + x, y0 + y) is the same cosine series with phases + kx x0 + ky y0)."""
    arrs = [np.ascontiguousarray(getattr(f, n), dtype=np.float64) for n in ("amp", "kx", "ky", "phase")]
    if x0 or y0:
        arrs[3] = arrs[3] + arrs[1] * x0 + arrs[2] * y0
    keep.extend(arrs)
    P = C.POINTER(C.c_double)
    ptrs = [a.ctypes.data_as(P) if a.size else None for a in arrs]
    return capi.stokes_field(float(f.mean), int(arrs[0].size), *ptrs)


def mesh_desc(wl, device=0, force_general=False, grid=None):
    """stokes_mesh_desc of a workload (stokes_synth.Workload); returns (desc, keepalive).
    grid: optional (bed_nodes, surface_nodes) height arrays on the horizontal GLL
    lattice ([NY][NX], X fastest), used instead of the workload's modal fields."""
    keep = []
    d = capi.stokes_mesh_desc()
    d.nx, d.ny, d.nz, d.k = wl.nx, wl.ny, wl.nz, wl.k
    d.pressure_space = capi.STOKES_PRESSURE_P if wl.pspace == "P" else capi.STOKES_PRESSURE_Q
    d.periodic_xy = 1 if wl.periodic else 0
    d.Lx, d.Ly = wl.Lx, wl.Ly
    x0, y0 = getattr(wl, "x0", 0.0), getattr(wl, "y0", 0.0)
    d.bed = _field(wl.bed, keep, x0, y0)
    d.surface = _field(wl.surface, keep, x0, y0)
    mask = wl.refine_mask()
    if mask.any() or force_general:
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        keep.append(mask)
        d.refine = mask.ctypes.data_as(C.POINTER(C.c_uint8))
    d.basal_bc = capi.STOKES_BASE_NOSLIP if wl.phys.basal_bc == "noslip" else capi.STOKES_BASE_SLIP
    d.device = device
    if grid is not None:
        P = C.POINTER(C.c_double)
        arrs = [np.ascontiguousarray(g, dtype=np.float64).ravel() for g in grid]
        keep.extend(arrs)
        d.bed_nodes, d.surface_nodes = (a.ctypes.data_as(P) for a in arrs)
    return d, keep


class Mesh:
    """Owns a stokes_mesh handle (device = -1: host-only, for inspection)."""

    def __init__(self, wl, device=0, force_general=False, grid=None):
        self.wl = wl
        d, keep = mesh_desc(wl, device, force_general, grid)
        self.handle = capi.stokes_mesh_create(d)
        del keep
        s = capi.stokes_mesh_sizes(self.handle)
        self.E, self.Nv, self.Np, self.Nb = s.E, s.Nv, s.Np, s.Nb
        self.k, self.npr, self.n_hanging = s.k, s.npr, s.n_hanging_elems
        self.device = device

    @property
    def ndof(self):
        return 3 * self.Nv + self.Np

    def node_coords(self):
        out = np.zeros((self.Nv, 3))
        capi.stokes_mesh_node_coords(self.handle, out)
        return out

    def basal_nodes(self):
        out = np.zeros(self.Nb, dtype=np.int64)
        capi.stokes_mesh_basal_nodes(self.handle, out)
        return out

    def close(self):
        if getattr(self, "handle", None) is not None:
            capi.stokes_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def params(phys, logbeta=None, constraint_scale=None):
    """stokes_params from stokes_synth.PhysParams; logbeta: device FP64 tensor [Nb] or None."""
    p = capi.stokes_params()
    p.n, p.A, p.C0, p.gamma, p.delta = phys.n, phys.A, phys.C0, phys.gamma, phys.delta
    for c in range(3):
        p.body[c] = phys.body[c]
    p.robin = 1 if phys.robin else 0
    if logbeta is not None:
        if not (logbeta.is_cuda and logbeta.dtype == torch.float64 and logbeta.is_contiguous()):
            raise ValueError("logbeta must be a contiguous CUDA float64 tensor")
        p.logbeta = C.c_void_p(logbeta.data_ptr())
    else:
        p.logbeta = None
    # the struct holds a raw device pointer: keep the tensor alive with it
    p._logbeta_tensor = logbeta
    p.constraint_scale = phys.constraint_scale if constraint_scale is None else constraint_scale
    p.linearization = capi.STOKES_LIN_PICARD if phys.linearization == "picard" else capi.STOKES_LIN_NEWTON
    p.sliding_m = getattr(phys, "sliding_m", 1.0)
    p.sliding_eps = getattr(phys, "sliding_eps", 1.0e-4)
    return p


class State:
    """Linearised per-quadrature-point Newton state (stokes_state)."""

    def __init__(self, mesh, prec):
        self.mesh = mesh
        self.prec = prec
        self.handle = capi.stokes_state_create(mesh.handle, prec)

    def linearize(self, p, up_lin, stream=None):
        capi.stokes_linearize(self.handle, p, up_lin, stream)
        self._params = p     # the state keeps params' device pointers (log beta)

    def apply(self, x, y, stream=None):
        capi.stokes_state_apply(self.handle, x, y, stream)

    def apply_transpose(self, x, y, stream=None):
        capi.stokes_state_apply_transpose(self.handle, x, y, stream)

    def apply_pressure_block(self, x, y, stream=None):
        capi.stokes_state_apply_pressure_block(self.handle, x, y, stream)

    def close(self):
        if getattr(self, "handle", None) is not None:
            capi.stokes_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
