"""Seeded synthetic inputs shared by the tests and the benchmark.

Holds none of the PIC method's arithmetic: only random fields and random particle sets (numpy
PCG64 generators, FP64) in the physical form (absolute grid-unit positions, full momenta u = gamma v,
weights, charges, ids). The beam initial state of the paper's runs is not made here: the CUDA
library and the oracle each draw it from Philox4x32-10 themselves.
"""
from __future__ import annotations

import math

import numpy as np

FIELDS = ("ex", "ey", "ez", "bx", "by", "bz")


def random_fields(shape, seed: int, scale: float = 1e-2, smooth: int = 0) -> dict:
    """Six field arrays of the given (nz, ny, nx) shape, N(0, scale^2); `smooth` box passes per axis
    make them spatially correlated (periodic)."""
    rng = np.random.default_rng(seed)
    out = {}
    for n in FIELDS:
        a = rng.normal(0.0, scale, size=shape)
        for _ in range(smooth):
            for ax in range(3):
                if a.shape[ax] > 1:
                    a = (np.roll(a, 1, ax) + a + np.roll(a, -1, ax)) / 3.0
        out[n] = np.ascontiguousarray(a)
    return out


def random_particles(ndim: int, nx: int, ny: int, nz: int, n: int, seed: int, gamma: float = 130.0,
                     spread: float = 0.05, weight: float = 0.01, per_particle_weight: bool = False) -> dict:
    """n particles uniformly in the periodic box with momenta (N, N, u0 + N) * spread, random charges +-1."""
    rng = np.random.default_rng(seed)
    u0 = math.sqrt(gamma * gamma - 1.0)
    p = {
        "x": rng.uniform(0, nx, n),
        "y": rng.uniform(0, ny, n) if ndim == 3 else np.zeros(n),
        "z": rng.uniform(0, nz, n),
        "ux": rng.normal(0, spread, n),
        "uy": rng.normal(0, spread, n),
        "uz": u0 + rng.normal(0, spread, n),
        "w": weight * (rng.uniform(0.5, 1.5, n) if per_particle_weight else np.ones(n)),
        "q": rng.choice([-1.0, 1.0], n),
        "id": np.arange(n, dtype=np.int64),
    }
    return p


def clustered_particles(ndim: int, nx: int, ny: int, nz: int, n: int, seed: int, corner=(0, 0, 0), size: int = 2,
                        gamma: float = 130.0, spread: float = 0.05, weight: float = 0.01) -> dict:
    """n particles uniformly in the block of size^ndim cells whose lowest corner is the cell `corner`
    (x, y, z), with momenta (N, N, u0 + N) * spread and random charges +-1: far more particles per cell
    than a uniform load, for the full-bin paths of the particle storage."""
    rng = np.random.default_rng(seed)
    u0 = math.sqrt(gamma * gamma - 1.0)
    x0, y0, z0 = corner
    return {
        "x": (x0 + rng.uniform(0, size, n)) % nx,
        "y": ((y0 + rng.uniform(0, size, n)) % ny) if ndim == 3 else np.zeros(n),
        "z": (z0 + rng.uniform(0, size, n)) % nz,
        "ux": rng.normal(0, spread, n),
        "uy": rng.normal(0, spread, n),
        "uz": u0 + rng.normal(0, spread, n),
        "w": weight * np.ones(n),
        "q": rng.choice([-1.0, 1.0], n),
        "id": np.arange(n, dtype=np.int64),
    }


def edge_particles(ndim: int, nx: int, ny: int, nz: int, gamma: float = 130.0) -> dict:
    """Hand-placed particles on the awkward spots: exactly on cell faces and nodes, next to the periodic
    wrap on both sides, at the last representable offset below a face, moving backwards."""
    u0 = math.sqrt(gamma * gamma - 1.0)
    pts = [
        (0.0, 0.0, 0.0, 0.0, 0.0, u0),
        (nx - 1e-7, 0.5, nz - 1e-7, 0.3, -0.2, u0),
        (1.0, 0.25, 2.0, -0.5, 0.1, -u0),
        (0.5, 0.5, 0.5, 5.0, 0.0, 0.0),
        (nx - 0.5, 0.0, 1.0 - 2.0 ** -30, -5.0, 0.0, 1.0),
        (3.0 - 2.0 ** -40, 0.75, 4.0, 0.0, 0.0, -0.5 * u0),
    ]
    n = len(pts)
    a = np.array(pts, dtype=np.float64)
    return {"x": a[:, 0] % nx, "y": (a[:, 1] % max(ny, 1)) if ndim == 3 else np.zeros(n), "z": a[:, 2] % nz,
            "ux": a[:, 3], "uy": a[:, 4], "uz": a[:, 5], "w": np.full(n, 0.02), "q": np.array([-1.0, 1.0] * 3),
            "id": np.arange(n, dtype=np.int64)}
