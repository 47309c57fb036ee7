"""Seeded synthetic particle systems for the 2D log-potential FMM.

This module draws random numbers only; it holds none of the method's
arithmetic, so the FP64 CPU oracle and the CUDA path can both be fed from it.

The generator is SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: value i of stream s under seed S is mix(S' + (i + 1) * gamma) with
S' a per-(S, s) key.  Uniform doubles take the top 53 bits; Gaussians use the
Box-Muller transform.

Workload families follow the paper's setup (charges scattered randomly in a
square box of side 5, Sec. 2.1 item 1 and Sec. 3) with charges q ~ U[-1, 1]:

* ``uniform``   -- positions uniform in [0, box]^2;
* ``gmm``       -- a mixture of K isotropic Gaussians, centres uniform in
                   [0.5, 4.5]^2, sigma log-uniform in [sigma_lo, sigma_hi],
                   equal weights; draws outside the box are redrawn (a
                   truncated normal) rather than clamped, so no duplicate
                   points pile up on the box edges;
* ``annulus``   -- radius uniform in [1, 2] about (2.5, 2.5), angle uniform;
* ``paper_cube``  -- the paper's own experiments (Sec. 3): charges +1 or -1 with equal
                   probability scattered uniformly in a cube (D = 3) or square (D = 2) of
                   side 5.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = _mix(np.array([(int(seed) * 0x100000001B3 + int(stream) * 0x2545F4914F6CDD1D) & 0xFFFFFFFFFFFFFFFF],
                          dtype=np.uint64))
    return k[0]


def u01(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniform doubles in [0, 1) from counters offset .. offset+n-1 of (seed, stream)."""
    ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix(_key(seed, stream) + ctr * _GAMMA)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n standard normals by Box-Muller from counter pairs of (seed, stream)."""
    m = (n + 1) // 2
    u1 = u01(seed, stream, m, offset)
    u2 = u01(seed, stream + 1_000_003, m, offset)
    r = np.sqrt(-2.0 * np.log1p(-u1))           # 1 - u1 in (0, 1]
    t = 2.0 * np.pi * u2
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(t)
    out[1::2] = r * np.sin(t)
    return out[:n]


def charges(n: int, seed: int) -> np.ndarray:
    """q ~ U[-1, 1]."""
    return 2.0 * u01(seed, 7, n) - 1.0


def uniform(n: int, seed: int, box: float = 5.0):
    """Positions uniform in [0, box)^2 and q ~ U[-1, 1]; returns (xy [n,2] f64, q [n] f64)."""
    xy = np.empty((n, 2))
    xy[:, 0] = box * u01(seed, 1, n)
    xy[:, 1] = box * u01(seed, 2, n)
    return xy, charges(n, seed)


def gmm(n: int, seed: int, k: int = 32, sigma_lo: float = 0.01, sigma_hi: float = 0.3,
        box: float = 5.0, centre_lo: float = 0.5, centre_hi: float = 4.5):
    """Mixture of k isotropic Gaussians, out-of-box draws redrawn; returns (xy, q)."""
    cx = centre_lo + (centre_hi - centre_lo) * u01(seed, 11, k)
    cy = centre_lo + (centre_hi - centre_lo) * u01(seed, 12, k)
    sig = np.exp(np.log(sigma_lo) + (np.log(sigma_hi) - np.log(sigma_lo)) * u01(seed, 13, k))
    comp = np.minimum((u01(seed, 14, n) * k).astype(np.int64), k - 1)
    xy = np.empty((n, 2))
    todo = np.arange(n)
    rnd = 0
    while todo.size:
        gx = normal(seed, 100 + 4 * rnd, n)[todo]
        gy = normal(seed, 102 + 4 * rnd, n)[todo]
        c = comp[todo]
        x = cx[c] + sig[c] * gx
        y = cy[c] + sig[c] * gy
        xy[todo, 0], xy[todo, 1] = x, y
        bad = ~((x >= 0.0) & (x < box) & (y >= 0.0) & (y < box))
        todo = todo[bad]
        rnd += 1
    return xy, charges(n, seed)


def annulus(n: int, seed: int, r_lo: float = 1.0, r_hi: float = 2.0, centre: float = 2.5):
    """Radius uniform in [r_lo, r_hi] about (centre, centre), angle uniform; returns (xy, q)."""
    r = r_lo + (r_hi - r_lo) * u01(seed, 21, n)
    t = 2.0 * np.pi * u01(seed, 22, n)
    xy = np.empty((n, 2))
    xy[:, 0] = centre + r * np.cos(t)
    xy[:, 1] = centre + r * np.sin(t)
    return xy, charges(n, seed)


def signs(n: int, seed: int) -> np.ndarray:
    """q = +1 or -1, each with probability 1/2."""
    return np.where(u01(seed, 8, n) < 0.5, -1.0, 1.0)


def paper_cube(n: int, seed: int, dim: int = 3, box: float = 5.0):
    """Positions uniform in [0, box)^dim and q = +-1; returns (pos [n, dim] f64, q [n] f64)."""
    pos = np.empty((n, dim))
    for a in range(dim):
        pos[:, a] = box * u01(seed, 31 + a, n)
    return pos, signs(n, seed)


def config_seed(config: int, replicate: int = 0) -> int:
    """Seed convention for the benchmark configurations: 20090767 + 1000 * config + replicate."""
    return 20090767 + 1000 * int(config) + int(replicate)
