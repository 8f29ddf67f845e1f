"""Pins of the oracle's charge density and field divergence, the two sides of the Gauss-law residual
div E - F rho (charge conservation of the Esirkepov deposit cited in Sec. 2): rho on the integer nodes
node by node against the centred B-spline written out from its piecewise definition with every
periodic image, and div E of a sampled plane wave on the Yee mesh against its closed form."""
import math

import numpy as np
import pytest

import oracle as O


def _spline(order, d):
    # centred cardinal B-splines of order 1 (hat) and 3 (cubic), from their piecewise definitions
    a = np.abs(d)
    if order == 1:
        return np.maximum(0.0, 1.0 - a)
    return np.where(a < 1.0, 2.0 / 3.0 - a * a + 0.5 * a ** 3, np.where(a < 2.0, (2.0 - a) ** 3 / 6.0, 0.0))


def _nearest_image(node, x, n):
    # node - x folded into [-n/2, n/2]: on grids of 5 or more cells only the nearest image of a
    # particle reaches a node through shapes of support 2 or less
    d = node - x
    return d - n * np.round(d / n)


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("order", [1, 3])
def test_rho_brute_force(ndim, order):
    # rho(node) = sum_p q_p w_p S(i - x_p) S(j - y_p) S(k - z_p) / dV, positions in cell units, on a
    # grid with unequal cell sizes; particles on the first and last cells exercise the wrap
    rng = np.random.default_rng(31 + 10 * ndim + order)
    nx, ny, nz = 7, (6 if ndim == 3 else 1), 9
    dx, dy, dz = 1.1, (0.9 if ndim == 3 else 1.0), 1.3
    sim = O.Sim(ndim=ndim, nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, order=order)
    n = 40
    x, z = rng.uniform(0, nx, n), rng.uniform(0, nz, n)
    y = rng.uniform(0, ny, n) if ndim == 3 else None
    x[:4] = (0.0, 0.25, nx - 0.2, nx - 1e-9)
    z[:4] = (nz - 1e-9, 0.0, 0.6, nz - 0.5)
    w = rng.uniform(0.5, 2.0, n)
    q = rng.choice([-1.0, 1.0], n)
    zero = np.zeros(n)
    sim.set_particles(x, y, z, zero, zero, zero, w, q)
    got = sim.rho()

    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    want = np.zeros((nz, ny, nx))
    for p in range(n):
        s = _spline(order, _nearest_image(ii, x[p], nx)) * _spline(order, _nearest_image(kk, z[p], nz))
        if ndim == 3:
            s = s * _spline(order, _nearest_image(jj, y[p], ny))
        want += q[p] * w[p] * s / (dx * dy * dz)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(want).max())
    # the shapes are partitions of unity: the total charge is sum q w
    assert abs(got.sum() * dx * dy * dz - (q * w).sum()) < 1e-12


def test_rho_single_particle_values():
    # one unit charge at offsets (0.25, 0.5) inside cell (2, 3) of a unit 2D grid: the hat gives the
    # nodes (2, 3), (3, 3), (2, 4), (3, 4) the weights 0.75*0.5, 0.25*0.5, 0.75*0.5, 0.25*0.5; the cubic
    # B-spline at offset 1/2 has node weights (1/48, 23/48, 23/48, 1/48) and at 1/4 (27/384, 235/384,
    # 121/384, 1/384)
    for order, wx, wz in ((1, [0.75, 0.25], [0.5, 0.5]),
                          (3, [27 / 384, 235 / 384, 121 / 384, 1 / 384], [1 / 48, 23 / 48, 23 / 48, 1 / 48])):
        sim = O.Sim(ndim=2, nx=8, nz=10, order=order)
        sim.set_particles(np.array([2.25]), None, np.array([3.5]), np.zeros(1), np.zeros(1), np.zeros(1),
                          np.ones(1), np.ones(1))
        got = sim.rho()[:, 0, :]
        lo = 2 if order == 1 else 1
        loz = 3 if order == 1 else 2
        want = np.zeros((10, 8))
        want[loz:loz + len(wz), lo:lo + len(wx)] = np.outer(wz, wx)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("ndim", [2, 3])
def test_div_e_of_a_plane_wave(ndim):
    # Ex at (i+1/2, j, k), Ey at (i, j+1/2, k), Ez at (i, j, k+1/2) sampled from A_c sin(k.r); the
    # backward differences onto the node (i, j, k) give exactly
    # cos(k.r_node) * sum_c 2 A_c sin(k_c d_c / 2) / d_c
    nx, ny, nz = 12, (10 if ndim == 3 else 1), 16
    dx, dy, dz = 1.1, (0.9 if ndim == 3 else 1.0), 1.3
    kx, kz = 2 * math.pi * 3 / (nx * dx), 2 * math.pi * 5 / (nz * dz)
    ky = 2 * math.pi * 2 / (ny * dy) if ndim == 3 else 0.0
    a = (0.7, -0.4, 1.2)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X, Y, Z = ii * dx, jj * dy, kk * dz
    sim = O.Sim(ndim=ndim, nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz)
    sim.f.update({"ex": a[0] * np.sin(kx * (X + dx / 2) + ky * Y + kz * Z),
                  "ey": a[1] * np.sin(kx * X + ky * (Y + dy / 2) + kz * Z),
                  "ez": a[2] * np.sin(kx * X + ky * Y + kz * (Z + dz / 2))})
    amp = (2 * a[0] * math.sin(kx * dx / 2) / dx + 2 * a[1] * math.sin(ky * dy / 2) / dy
           + 2 * a[2] * math.sin(kz * dz / 2) / dz)
    want = amp * np.cos(kx * X + ky * Y + kz * Z)
    np.testing.assert_allclose(sim.div_e(), want, rtol=0, atol=1e-13)
