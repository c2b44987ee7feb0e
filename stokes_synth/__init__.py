"""Seeded synthetic inputs shared by the oracle tests and the GPU path.

This package holds only input generation: the workload configurations
(grid sizes, degrees, physical constants), the coefficients of the smooth
random surface, bed and basal-friction fields, and seeded random vectors.
It contains none of the finite element arithmetic; both the oracle and the
CUDA library evaluate these inputs with code of their own.
"""
from .fields import ModalField, surface_field, bed_field, logbeta_field, flat_field
from .configs import Workload, PhysParams, workload, WORKLOADS, sub_block
from .vectors import uniform_vector

__all__ = [
    "ModalField", "surface_field", "bed_field", "logbeta_field", "flat_field",
    "Workload", "PhysParams", "workload", "WORKLOADS", "sub_block", "uniform_vector",
]
