"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method itself (no energy, no
rasterisation, no solver step): it only draws fracture descriptions and
random vectors from seeded numpy generators (PCG64), so that both sides of
every parity check receive byte-identical inputs.

Fracture rows (host arrays, float64):

* ``LINE2D``  -> ``[cx, cy, theta, half_length]``: a straight crack segment,
  the 2D "smooth rectangle" of Sec. 5.2 before regularisation.
* ``DISC3D``  -> ``[cx, cy, cz, nx, ny, nz, radius]``: a penny-shaped crack
  with unit normal ``n`` (the 3D workload's fracture shape).
* ``BOX3D``   -> ``[cx, cy, cz, nx, ny, nz, ax, ay, az, bx, by, bz, ha, hb]``:
  a rectangular plate with unit normal ``n``, orthonormal in-plane axes
  ``a``, ``b`` and half-lengths ``ha``, ``hb`` (the paper's 3D "smooth
  parallelepipeds" once widened to the band).

Workload recipes (Sec. 5.2 describes the paper's generator: uniform
hypocentres, bounded orientations, power-law lengths; the sizes here are the
workloads this library is benchmarked on):

* centred straight crack of half-length 0.1 in the unit square;
* ``n`` discs with radius U[rmin, rmax], centre U[0,1]^3, normal uniform on
  the sphere (normalised Gaussian triple);
* ``n`` line segments in two orientation families +-30 deg with +-10 deg
  uniform jitter, half-lengths log-uniform in [lmin, lmax]/2, centres U[0,1]^2.
"""
from __future__ import annotations

import numpy as np

LINE2D = 0
DISC3D = 1
BOX3D = 2

# seed convention: 1000 + 100 * workload + instance
SEED_2D_PLAIN = 1000
SEED_3D_PLAIN = 1100
SEED_3D_MIXED = 1200
SEED_2D_BATCHED = 1300
SEED_2D_LEARNED = 1400
SEED_3D_PAPER = 1500


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def centred_crack_2d(half_length: float = 0.1) -> np.ndarray:
    """One horizontal crack through the centre of the unit square."""
    return np.array([[0.5, 0.5, 0.0, half_length]], dtype=np.float64)


def disc_network_3d(seed: int, n: int, rmin: float = 0.03, rmax: float = 0.1) -> np.ndarray:
    g = rng(seed)
    out = np.empty((n, 7), dtype=np.float64)
    for k in range(n):
        r = g.uniform(rmin, rmax)
        cen = g.uniform(0.0, 1.0, size=3)
        nv = g.standard_normal(3)
        nv = nv / np.sqrt(np.dot(nv, nv))
        out[k, 0:3] = cen
        out[k, 3:6] = nv
        out[k, 6] = r
    return out


def box_network_3d(seed: int, n: int, lmin: float = 0.05, lmax: float = 0.25,
                   exponent: float = 2.0) -> np.ndarray:
    """n rectangular plates: centre U[0,1]^3, normal uniform on the sphere
    (normalised Gaussian triple), in-plane axis at a uniform angle, side
    length from the power law p(l) ~ l^-exponent on [lmin, lmax] (inverse
    transform), second side U[0.5, 1] times the first."""
    g = rng(seed)
    out = np.empty((n, 14), dtype=np.float64)
    for k in range(n):
        cen = g.uniform(0.0, 1.0, size=3)
        nv = g.standard_normal(3)
        nv = nv / np.sqrt(np.dot(nv, nv))
        # an orthonormal pair in the plane, then a uniform rotation in it
        helper = np.array([1.0, 0.0, 0.0]) if abs(nv[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
        e1 = helper - np.dot(helper, nv) * nv
        e1 = e1 / np.sqrt(np.dot(e1, e1))
        e2 = np.cross(nv, e1)
        phi = g.uniform(0.0, np.pi)
        av = np.cos(phi) * e1 + np.sin(phi) * e2
        bv = np.cross(nv, av)
        u = g.uniform()
        a1 = 1.0 - exponent
        length = (lmin ** a1 + u * (lmax ** a1 - lmin ** a1)) ** (1.0 / a1)
        width = length * g.uniform(0.5, 1.0)
        out[k, 0:3] = cen
        out[k, 3:6] = nv
        out[k, 6:9] = av
        out[k, 9:12] = bv
        out[k, 12] = 0.5 * length
        out[k, 13] = 0.5 * width
    return out


def line_network_2d(seed: int, n: int, lmin: float = 0.01, lmax: float = 0.1,
                    family_deg: float = 30.0, jitter_deg: float = 10.0) -> np.ndarray:
    g = rng(seed)
    out = np.empty((n, 4), dtype=np.float64)
    for k in range(n):
        fam = family_deg if g.uniform() < 0.5 else -family_deg
        th = np.deg2rad(fam + g.uniform(-jitter_deg, jitter_deg))
        length = np.exp(g.uniform(np.log(lmin), np.log(lmax)))
        cen = g.uniform(0.0, 1.0, size=2)
        out[k] = (cen[0], cen[1], th, 0.5 * length)
    return out


def batched_grid_draw(seed: int, n_instances: int = 64,
                      sizes=(129, 257, 513, 1025), balanced: bool = True):
    """Grid sizes and fracture counts for the uneven 2D batch."""
    g = rng(seed)
    if balanced:
        per = n_instances // len(sizes)
        grid = [s for s in sizes for _ in range(per)]
    else:
        grid = [int(sizes[g.integers(0, len(sizes))]) for _ in range(n_instances)]
    counts = [int(round(np.exp(g.uniform(np.log(10), np.log(1000))))) for _ in range(n_instances)]
    return grid, counts


def random_state(seed: int, dim: int, n_nodes: int, u_scale: float = 1e-2,
                 c_lo: float = 0.0, c_hi: float = 0.9) -> np.ndarray:
    """A random iterate: d displacement planes then the phase-field plane."""
    g = rng(seed)
    x = np.empty((dim + 1) * n_nodes, dtype=np.float64)
    x[: dim * n_nodes] = g.uniform(-u_scale, u_scale, size=dim * n_nodes)
    x[dim * n_nodes:] = g.uniform(c_lo, c_hi, size=n_nodes)
    return x


def random_direction(seed: int, n: int, scale: float = 1.0) -> np.ndarray:
    return rng(seed).uniform(-scale, scale, size=n)
