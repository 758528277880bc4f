"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds no arithmetic of the method: it only draws numbers.  The white-noise
field omega(q) of Sec. 2.1 (Eq. 6: any real white noise on the Lagrangian lattice) is
i.i.d. N(0, 1), drawn by a counter-based generator: SplitMix64 (Steele, Lea & Flood 2014)
of seed * 2^40 + counter, two 53-bit uniforms per pair, Box-Muller transform in float64,
then rounded to float32 so that every consumer sees the same bytes.

Cosmologies for batched ensembles are drawn uniformly from the ranges of the batched
workload (Omega_m in [0.25, 0.35], A_s in [1.8, 2.4]e-9, n_s in [0.94, 0.99], Omega_b =
0.049, h = 0.68).
"""
import numpy as np

THETA_FIDUCIAL = (2.1e-9, 0.965, 0.31, 0.049, 0.68)   # (A_s, n_s, Omega_m, Omega_b, h)

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _splitmix64(counter):
    z = counter * _GAMMA + _GAMMA
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform01(seed, count, offset=0):
    """``count`` float64 uniforms in (0, 1] from stream ``seed``, counters offset.."""
    base = np.uint64(seed) << np.uint64(40)
    ctr = base + np.arange(offset, offset + count, dtype=np.uint64)
    bits = _splitmix64(ctr) >> np.uint64(11)
    return (bits.astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def white_noise(n, seed, chunk=1 << 24):
    """float32 array (n, n, n) of i.i.d. standard normals for stream ``seed``."""
    total = n ** 3
    out = np.empty(total, dtype=np.float32)
    pairs = (total + 1) // 2
    for start in range(0, pairs, chunk):
        m = min(chunk, pairs - start)
        u = uniform01(seed, 2 * m, offset=2 * start)
        r = np.sqrt(-2.0 * np.log(u[0::2]))
        phi = 2.0 * np.pi * u[1::2]
        z = np.empty(2 * m)
        z[0::2] = r * np.cos(phi)
        z[1::2] = r * np.sin(phi)
        lo = 2 * start
        hi = min(total, lo + 2 * m)
        out[lo:hi] = z[: hi - lo]
    return out.reshape(n, n, n)


def ensemble_theta(batch, seed=1000):
    """(batch, 5) float64 cosmologies drawn uniformly, one stream per instance."""
    th = np.empty((batch, 5))
    for b in range(batch):
        u = uniform01(seed + b, 3)
        th[b] = (1.8e-9 + 0.6e-9 * u[0], 0.94 + 0.05 * u[1], 0.25 + 0.10 * u[2], 0.049, 0.68)
    return th


def cross_target(n_mesh, half_width=1.5, amplitude=2.0):
    """Synthetic target pattern for the white-noise optimisation (the paper's target image
    is not available): overdensity ``amplitude`` in three orthogonal bars of half-width
    ``half_width`` cells through the box centre, mean subtracted; float64 (n, n, n)."""
    c = np.arange(n_mesh) - n_mesh / 2 + 0.5
    x, y, z = np.meshgrid(c, c, c, indexing="ij")
    near = lambda u: np.abs(u) < half_width
    inside = (near(y) & near(z)) | (near(x) & near(z)) | (near(x) & near(y))
    return amplitude * (inside - inside.mean())
