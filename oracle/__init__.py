"""Plain, slow FP64 CPU oracle of the matrix-free nonlinear Stokes operator.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import anything under oracle/.
The oracle shares no code with the CUDA library; the two meet only through
the seeded inputs of stokes_synth.
"""
from .mesh import OracleMesh
from . import basis, stokes, newton

__all__ = ["OracleMesh", "basis", "stokes", "newton"]
