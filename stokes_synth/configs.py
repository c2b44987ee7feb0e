"""Workload definitions: mesh sizes, discretisation and physical constants.

The large slab workloads restate the paper's thin periodic ice slabs
(Section 4.3 test problem, Section 7 ice stream constants): periodic in x
and y, free top surface, Robin sliding plus no-penetration at the base, Glen
flow law with n = 3 and A = 1e-16 Pa^-3 a^-1, rho = 910 kg m^-3,
g = 9.81 m s^-2, eps = 1e-6 a^-2, a 0.5 degree pitch of gravity along x.
Units are metres, years and pascals.
"""
from dataclasses import dataclass, field
import math
import numpy as np

from .fields import ModalField, flat_field, surface_field, bed_field, logbeta_field

RHO_ICE = 910.0
G_ACC = 9.81
SLAB_L = 100.0e3


@dataclass(frozen=True)
class PhysParams:
    n: float = 3.0            # Glen exponent
    A: float = 1.0e-16        # flow-law prefactor; B = A^(-1/n)
    C0: float = 1.0           # viscosity: mu = C0 * A^(-1/n) * (gamma*D:D + delta)^((1-n)/(2n))
    gamma: float = 0.5
    delta: float = 1.0e-6
    body: tuple = (0.0, 0.0, -RHO_ICE * G_ACC)
    basal_bc: str = "slip"    # 'noslip' (Dirichlet) or 'slip' (u.n = 0 plus Robin)
    robin: bool = True        # basal Robin term  int beta T v . T u
    logbeta: ModalField = None
    constraint_scale: float = 1.0   # s of the constraint rows s (I - P)
    linearization: str = "newton"   # Jacobian: 'newton' (Eq. 2.7) or 'picard' (viscosity frozen)
    # basal sliding law: traction beta (|T u|^2 + sliding_eps)^((m - 1)/2) T u,
    # m = sliding_m; m = 1 is the linear law beta T u of Eq. 2.4a
    sliding_m: float = 1.0
    sliding_eps: float = 1.0e-4

    def viscosity_prefactor(self):
        return self.C0 * self.A ** (-1.0 / self.n)


@dataclass(frozen=True)
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    k: int
    pspace: str               # 'P' -> P_{k-1}^disc, 'Q' -> Q_{k-2}^disc
    periodic: bool
    Lx: float
    Ly: float
    bed: ModalField
    surface: ModalField
    phys: PhysParams
    refine_frac: float = 0.0
    refine_seed: int = 0
    seed: int = 0
    x0: float = 0.0           # physical offset of the mesh origin (sub-blocks of a larger slab)
    y0: float = 0.0

    @property
    def n_coarse(self):
        return self.nx * self.ny * self.nz

    def refine_mask(self):
        """uint8 per coarse cell (x fastest, then y, then z): 1 = split into 8."""
        m = np.zeros(self.n_coarse, dtype=np.uint8)
        nref = int(round(self.refine_frac * self.n_coarse))
        if nref > 0:
            rng = np.random.default_rng([self.refine_seed, 505])
            m[rng.permutation(self.n_coarse)[:nref]] = 1
        return m


def _box(name, nx, ny, nz, k, pspace):
    phys = PhysParams(n=3.0, A=1.0, C0=0.5, gamma=1.0, delta=1.0e-12,
                      body=(0.0, 0.0, -1.0), basal_bc="noslip", robin=False,
                      logbeta=None)
    return Workload(name, nx, ny, nz, k, pspace, False, 1.0, 1.0,
                    flat_field(0.0), flat_field(1.0), phys)


def _cbox(name, nx, ny, nz, k, pspace, refine_frac=0.0, seed=11):
    """Unit box with a curved bed and surface (non-periodic): exercises curved
    isoparametric maps, slip normals and hanging nodes where rigid-body
    motions and linear fields are still admissible."""
    tp = 2.0 * math.pi
    bed = ModalField(0.0, np.array([0.08, 0.05]), np.array([tp, 0.0]),
                     np.array([0.0, tp]), np.array([0.3, 1.1]))
    surf = ModalField(1.0, np.array([0.06]), np.array([tp]), np.array([tp]),
                      np.array([0.7]))
    phys = PhysParams(n=3.0, A=1.0, C0=0.5, gamma=1.0, delta=1.0e-12,
                      body=(0.0, 0.0, -1.0), basal_bc="slip", robin=True,
                      logbeta=ModalField(0.0, np.array([0.5]), np.array([tp]),
                                         np.array([tp]), np.array([0.2])))
    return Workload(name, nx, ny, nz, k, pspace, False, 1.0, 1.0, bed, surf, phys,
                    refine_frac=refine_frac, refine_seed=seed, seed=seed)


def _slab(name, nx, ny, nz, k, pspace, seed=0, refine_frac=0.0, grf_beta=False,
          L=SLAB_L):
    theta = math.radians(0.5)
    rg = RHO_ICE * G_ACC
    if grf_beta:
        lb = logbeta_field(seed, L, L)
    else:
        lb = flat_field(math.log(1.0e3))
    phys = PhysParams(n=3.0, A=1.0e-16, C0=1.0, gamma=0.5, delta=1.0e-6,
                      body=(rg * math.sin(theta), 0.0, -rg * math.cos(theta)),
                      basal_bc="slip", robin=True, logbeta=lb)
    return Workload(name, nx, ny, nz, k, pspace, True, L, L,
                    bed_field(seed, L, L), surface_field(seed, L, L), phys,
                    refine_frac=refine_frac, refine_seed=seed, seed=seed)


def _build():
    w = {}
    # the five workloads of the benchmark plan
    w["box_4x4x2_q2p1"] = _box("box_4x4x2_q2p1", 4, 4, 2, 2, "P")
    w["slab_128x128x8_q2p1"] = _slab("slab_128x128x8_q2p1", 128, 128, 8, 2, "P")
    w["slab_64x64x4_q3q1"] = _slab("slab_64x64x4_q3q1", 64, 64, 4, 3, "Q")
    w["slab_64x64x4_q4p3"] = _slab("slab_64x64x4_q4p3", 64, 64, 4, 4, "P")
    w["forest_64x64x4_q3p2"] = _slab("forest_64x64x4_q3p2", 64, 64, 4, 3, "P",
                                      refine_frac=0.3, grf_beta=True)
    w["slab_512x512x8_q2p1"] = _slab("slab_512x512x8_q2p1", 512, 512, 8, 2, "P",
                                      grf_beta=True)
    w["slab_32x32x4_q2p1"] = _slab("slab_32x32x4_q2p1", 32, 32, 4, 2, "P",
                                    grf_beta=True)
    # small cases the oracle finishes in seconds (several tiles + ragged tails)
    w["slab_8x8x2_q2p1"] = _slab("slab_8x8x2_q2p1", 8, 8, 2, 2, "P", grf_beta=True)
    w["slab_5x3x3_q2p1"] = _slab("slab_5x3x3_q2p1", 5, 3, 3, 2, "P", seed=7)
    w["slab_6x6x2_q3q1"] = _slab("slab_6x6x2_q3q1", 6, 6, 2, 3, "Q")
    w["slab_4x4x2_q4p3"] = _slab("slab_4x4x2_q4p3", 4, 4, 2, 4, "P")
    w["slab_3x3x2_q3p2"] = _slab("slab_3x3x2_q3p2", 3, 3, 2, 3, "P")
    w["forest_6x6x2_q3p2"] = _slab("forest_6x6x2_q3p2", 6, 6, 2, 3, "P",
                                    refine_frac=0.3, grf_beta=True, seed=3)
    w["forest_4x4x2_q2p1"] = _slab("forest_4x4x2_q2p1", 4, 4, 2, 2, "P",
                                    refine_frac=0.3, seed=5)
    w["box_3x2x2_q3q1"] = _box("box_3x2x2_q3q1", 3, 2, 2, 3, "Q")
    # the aspect-robust Q_k x Q_(k-2) pairing (Section 3.2.2) at k = 2 and 4
    w["slab_128x128x8_q2q0"] = _slab("slab_128x128x8_q2q0", 128, 128, 8, 2, "Q")
    w["slab_5x3x3_q2q0"] = _slab("slab_5x3x3_q2q0", 5, 3, 3, 2, "Q", seed=7)
    w["slab_4x4x2_q4q2"] = _slab("slab_4x4x2_q4q2", 4, 4, 2, 4, "Q", grf_beta=True, seed=2)
    w["forest_4x4x2_q2q0"] = _slab("forest_4x4x2_q2q0", 4, 4, 2, 2, "Q",
                                    refine_frac=0.3, grf_beta=True, seed=6)
    # curved non-periodic boxes (conforming and with hanging nodes)
    w["cbox_3x3x2_q2p1"] = _cbox("cbox_3x3x2_q2p1", 3, 3, 2, 2, "P")
    w["cbox_3x3x2_q3q1"] = _cbox("cbox_3x3x2_q3q1", 3, 3, 2, 3, "Q")
    w["cforest_3x3x2_q2p1"] = _cbox("cforest_3x3x2_q2p1", 3, 3, 2, 2, "P", refine_frac=0.4)
    w["cforest_3x3x2_q3p2"] = _cbox("cforest_3x3x2_q3p2", 3, 3, 2, 3, "P", refine_frac=0.4)
    w["cforest_4x3x2_q4p3"] = _cbox("cforest_4x3x2_q4p3", 4, 3, 2, 4, "P", refine_frac=0.3, seed=4)
    w["cbox_3x3x2_q2q0"] = _cbox("cbox_3x3x2_q2q0", 3, 3, 2, 2, "Q")
    w["cforest_4x3x2_q4q2"] = _cbox("cforest_4x3x2_q4q2", 4, 3, 2, 4, "Q", refine_frac=0.3, seed=4)
    return w


WORKLOADS = _build()


def workload(name):
    return WORKLOADS[name]


def sub_block(wl, ox, oy, sx, sy):
    """The sx x sy x nz column block of a conforming slab workload starting at
    coarse cell (ox, oy): same element shapes and fields, not periodic."""
    import dataclasses
    hx, hy = wl.Lx / wl.nx, wl.Ly / wl.ny
    return dataclasses.replace(wl, name=f"{wl.name}[{ox}:{ox + sx},{oy}:{oy + sy}]", nx=sx, ny=sy,
                               Lx=sx * hx, Ly=sy * hy, periodic=False,
                               x0=wl.x0 + ox * hx, y0=wl.y0 + oy * hy)
