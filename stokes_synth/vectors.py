"""Seeded random vectors (inputs to residual and operator evaluations)."""
import numpy as np


def uniform_vector(seed, n, lo=-1.0, hi=1.0, stream=0):
    """n values ~ U(lo, hi) from numpy's PCG64 stream keyed by (seed, stream)."""
    rng = np.random.default_rng([seed, 404, stream])
    return rng.uniform(lo, hi, size=int(n))
