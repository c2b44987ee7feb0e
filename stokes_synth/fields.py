"""Smooth seeded random fields on the periodic (x, y) plane.

Every field is a finite cosine series
    f(x, y) = mean + sum_m amp[m] * cos(kx[m] x + ky[m] y + phase[m]),
with wavenumbers on the lattice 2*pi*(j/Lx, l/Ly) so that the field is
periodic on [0, Lx) x [0, Ly).  The recipes follow the paper's synthetic
workloads: the random Fourier series of Section 4.3 (Eq. 4.2, decay
|(j,k)|^-gamma) for beds, a sum of 16 sinusoids for the
surface, and a Gaussian random field realised by random Fourier features
for log(beta).
"""
from dataclasses import dataclass
import numpy as np


@dataclass(frozen=True)
class ModalField:
    mean: float
    amp: np.ndarray
    kx: np.ndarray
    ky: np.ndarray
    phase: np.ndarray

    def __call__(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        out = np.full(np.broadcast(x, y).shape, self.mean, dtype=np.float64)
        for a, kx, ky, ph in zip(self.amp, self.kx, self.ky, self.phase):
            out = out + a * np.cos(kx * x + ky * y + ph)
        return out

    @property
    def n_modes(self):
        return int(self.amp.size)


def flat_field(value):
    z = np.zeros(0)
    return ModalField(float(value), z, z, z, z)


def _rescale(mean, amp, kx, ky, ph, Lx, Ly, max_dev):
    """Scale the amplitudes so that max |f - mean| on a 512^2 grid is max_dev."""
    f = ModalField(0.0, amp, kx, ky, ph)
    xs = np.linspace(0.0, Lx, 512, endpoint=False)
    ys = np.linspace(0.0, Ly, 512, endpoint=False)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    m = float(np.max(np.abs(f(X, Y))))
    s = max_dev / m if m > 0 else 0.0
    return ModalField(float(mean), amp * s, kx, ky, ph)


def _merge(amp, kx, ky, ph):
    """Combine terms with the same wavevector: sum a_m cos(t + p_m) = |S| cos(t + arg S)."""
    groups = {}
    for a, x, y, p in zip(amp, kx, ky, ph):
        groups[(x, y)] = groups.get((x, y), 0.0) + a * np.exp(1j * p)
    keys = sorted(groups)
    S = np.array([groups[q] for q in keys])
    keep = np.abs(S) > 0
    S = S[keep]
    kxy = np.array(keys)[keep]
    return np.abs(S), kxy[:, 0].copy(), kxy[:, 1].copy(), np.angle(S)


def surface_field(seed, Lx, Ly, mean=1000.0, max_dev=50.0, n_modes=16):
    """Surface elevation: 16 sinusoids, integer wavenumbers j, l in 1..4."""
    rng = np.random.default_rng([seed, 101])
    j = rng.integers(1, 5, size=n_modes)
    l = rng.integers(1, 5, size=n_modes)
    amp = rng.uniform(-1.0, 1.0, size=n_modes)
    ph = rng.uniform(0.0, 2.0 * np.pi, size=n_modes)
    kx = 2.0 * np.pi * j / Lx
    ky = 2.0 * np.pi * l / Ly
    return _rescale(mean, amp, kx, ky, ph, Lx, Ly, max_dev)


def bed_field(seed, Lx, Ly, max_dev=100.0, N=10, gamma=1.5):
    """Bed elevation from the random Fourier series of the paper's test problems.

    s = sum_{(j,k) != (0,0), 0 <= j,k <= N} (a cos cos + b cos sin + c sin cos
        + d sin sin) |(j,k)|^-gamma with a, b, c, d ~ U(-1, 1); the pointwise
    noise term of that recipe is left out (a bed must be smooth).  Each
    product of a cosine/sine pair is rewritten as two cosines of the sum and
    difference wavevectors.
    """
    rng = np.random.default_rng([seed, 202])
    amps, kxs, kys, phs = [], [], [], []
    for jj in range(N + 1):
        for kk in range(N + 1):
            if jj == 0 and kk == 0:
                continue
            a, b, c, d = rng.uniform(-1.0, 1.0, size=4)
            decay = (jj * jj + kk * kk) ** (-gamma / 2.0)
            wx = 2.0 * np.pi * jj / Lx
            wy = 2.0 * np.pi * kk / Ly
            # cos A cos B = 1/2 [cos(A-B) + cos(A+B)]
            # cos A sin B = 1/2 [sin(A+B) - sin(A-B)]
            # sin A cos B = 1/2 [sin(A+B) + sin(A-B)]
            # sin A sin B = 1/2 [cos(A-B) - cos(A+B)]
            # sin(t) = cos(t - pi/2)
            half = 0.5 * decay
            terms = [
                (half * a, wx, -wy, 0.0), (half * a, wx, wy, 0.0),
                (half * b, wx, wy, -np.pi / 2), (-half * b, wx, -wy, -np.pi / 2),
                (half * c, wx, wy, -np.pi / 2), (half * c, wx, -wy, -np.pi / 2),
                (half * d, wx, -wy, 0.0), (-half * d, wx, wy, 0.0),
            ]
            for t in terms:
                amps.append(t[0]); kxs.append(t[1]); kys.append(t[2]); phs.append(t[3])
    amp, kx, ky, ph = _merge(np.array(amps), np.array(kxs), np.array(kys), np.array(phs))
    return _rescale(0.0, amp, kx, ky, ph, Lx, Ly, max_dev)


def logbeta_field(seed, Lx, Ly, mean=np.log(1.0e3), std=1.0, corr_len=1.0e4, M=256):
    """Gaussian random field by random Fourier features (M cosines).

    omega ~ N(0, corr_len^-2 I), rounded to the periodic wavenumber lattice so
    the field is periodic; phase ~ U(0, 2 pi); amplitude std * sqrt(2 / M).
    """
    rng = np.random.default_rng([seed, 303])
    om = rng.normal(0.0, 1.0 / corr_len, size=(M, 2))
    j = np.rint(om[:, 0] * Lx / (2.0 * np.pi))
    l = np.rint(om[:, 1] * Ly / (2.0 * np.pi))
    ph = rng.uniform(0.0, 2.0 * np.pi, size=M)
    amp = np.full(M, std * np.sqrt(2.0 / M))
    return ModalField(float(mean), amp, 2.0 * np.pi * j / Lx, 2.0 * np.pi * l / Ly, ph)
