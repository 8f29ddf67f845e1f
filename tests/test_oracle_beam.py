"""Pins of the seeded beam recipe: Philox4x32-10 known answers, lattice layout, co-located pairs,
charge neutrality and the statistics of the thermal draw."""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert O.philox4x32_10(ctr, key) == out


@pytest.mark.parametrize("ndim,ppc,dims", [(2, 4, (2, 1, 2)), (2, 16, (4, 1, 4)), (2, 8, (2, 1, 4)),
                                           (3, 8, (2, 2, 2)), (3, 1, (1, 1, 1)), (3, 12, (2, 2, 3))])
def test_lattice_dims(ndim, ppc, dims):
    assert O.lattice_dims(ndim, ppc) == dims


@pytest.mark.parametrize("ndim", [2, 3])
def test_beam_layout_and_statistics(ndim):
    ppc = 4 if ndim == 2 else 8
    sim = O.Sim(ndim=ndim, nx=12, ny=6 if ndim == 3 else 1, nz=20, dt=0.5)
    sim.init_beam(ppc=ppc, gamma=130.0, seed=7, jitter=0.1, u_th=1e-4)
    nz, ny, nx = sim.shape
    n = nx * ny * nz * ppc * 2
    P = sim.part
    assert len(P["x"]) == n
    # species alternate, electrons first; each positron sits exactly on its electron
    np.testing.assert_array_equal(P["q"][0::2], -1.0)
    np.testing.assert_array_equal(P["q"][1::2], 1.0)
    for a in ("x", "z") + (("y",) if ndim == 3 else ()):
        np.testing.assert_array_equal(P[a][0::2], P[a][1::2])
    # position = cell + lattice offset + jitter within +-0.1
    L = O.lattice_dims(ndim, ppc)
    pid = np.arange(n) // 2
    cell = pid // ppc
    lat = pid % ppc
    i, j, k = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    lx, ly, lz = lat % L[0], (lat // L[0]) % L[1], lat // (L[0] * L[1])
    dx = (P["x"] - (i + (lx + 0.5) / L[0]) + nx / 2) % nx - nx / 2
    dz = (P["z"] - (k + (lz + 0.5) / L[2]) + nz / 2) % nz - nz / 2
    assert np.abs(dx).max() <= 0.1 and np.abs(dz).max() <= 0.1
    assert np.abs(dx).max() > 0.09  # the jitter is really there
    # thermal draw: mean and spread within statistical error
    u0 = math.sqrt(130.0 ** 2 - 1)
    for comp, mean in (("ux", 0.0), ("uy", 0.0), ("uz", u0)):
        v = P[comp] - mean
        assert abs(v.mean()) < 5 * 1e-4 / math.sqrt(n)
        assert abs(v.std() / 1e-4 - 1) < 5 / math.sqrt(2 * n)
    # independent draws per species
    assert not np.array_equal(P["ux"][0::2], P["ux"][1::2])
    # charge neutral to roundoff
    assert np.abs(sim.rho()).max() < 1e-15
    # weight: omega_p^2 dV / (2 ppc)
    np.testing.assert_allclose(P["w"], 0.3868 ** 2 / (2 * ppc), rtol=1e-15)


def test_beam_gaussian_weight():
    sim = O.Sim(ndim=3, nx=16, ny=16, nz=4, dt=0.5)
    sim.init_beam(ppc=8, sigma_perp=3.0, seed=3)
    P = sim.part
    r2 = (P["x"] - 8) ** 2 + (P["y"] - 8) ** 2
    np.testing.assert_allclose(P["w"], 0.3868 ** 2 / 16 * np.exp(-r2 / 18.0), rtol=1e-14)


def test_beam_seed_changes_draws():
    a = O.Sim(ndim=2, nx=4, nz=4)
    b = O.Sim(ndim=2, nx=4, nz=4)
    a.init_beam(ppc=4, seed=1)
    b.init_beam(ppc=4, seed=2)
    assert not np.array_equal(a.part["ux"], b.part["ux"])
