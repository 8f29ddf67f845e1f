"""Pins of the oracle's Cole-Karkkainen field solver (the CK solver that Sec. 2 names for Fig. 1,
beta_z = 1/8, c dt/dz = 0.9), 2D x-z.

The B update's curl of E averages each forward difference over the two transverse neighbours with
weights (beta, 1 - 2 beta, beta); the E update is Yee's. Pinned against closed forms that do not
come from the stencil itself: the Fourier symbol of one B update, the exact discrete solution of a
vacuum plane wave (sin^2(w dt / 2) = dt^2 [sz^2 (1 - 4 beta_z sx^2) / dz^2 + sx^2 (1 - 4 beta_x sz^2)
/ dx^2] with sx = sin(kx dx / 2), sz = sin(kz dz / 2)), the Courant limit c dt = dx = dz at
beta = 1/8, the beta = 0 special case (Yee) and the invariant that the CK curl conserves.
"""
import math

import numpy as np
import pytest

import oracle as O


def _mode(shape, kx, kz, sx=0.0, sz=0.0, f=np.cos):
    nz, _, nx = shape
    k, i = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    return f(kx * (i + sx) + kz * (k + sz))[:, None, :]


def _theta(dt, dx, dz, bx, bz, kx, kz):
    sx, sz = math.sin(kx / 2), math.sin(kz / 2)
    s2 = dt * dt * (sz * sz * (1 - 4 * bz * sx * sx) / dz ** 2 + sx * sx * (1 - 4 * bx * sz * sz) / dx ** 2)
    return 2 * math.asin(math.sqrt(s2))


def test_ck_symbol_of_one_b_update():
    # Ey = cos(kx i + kz k) at Ey's nodes (i, k). One update B -= h curl_CK E gives
    #   Bx(i, k+1/2) = -h (2/dz) sin(kz/2) (1 - 4 beta_z sin^2(kx/2)) sin(kx i + kz (k + 1/2))
    #   Bz(i+1/2, k) = +h (2/dx) sin(kx/2) (1 - 4 beta_x sin^2(kz/2)) sin(kx (i + 1/2) + kz k)
    # (unequal betas and cell sizes, so that a swapped weight or axis fails).
    nx, nz, dx, dz, h = 20, 28, 0.9, 1.3, 0.37
    bx, bz = 0.09, 0.13
    sim = O.Sim(ndim=2, nx=nx, nz=nz, dx=dx, dz=dz, dt=0.5, solver=O.CK, ck_beta=(bx, bz))
    kx, kz = 2 * math.pi * 3 / nx, 2 * math.pi * 5 / nz
    sim.f["ey"] = _mode(sim.shape, kx, kz)
    sim.yee_b(h)
    ax = -h * 2 / dz * math.sin(kz / 2) * (1 - 4 * bz * math.sin(kx / 2) ** 2)
    az = h * 2 / dx * math.sin(kx / 2) * (1 - 4 * bx * math.sin(kz / 2) ** 2)
    np.testing.assert_allclose(sim.f["bx"], ax * _mode(sim.shape, kx, kz, sz=0.5, f=np.sin), atol=1e-14)
    np.testing.assert_allclose(sim.f["bz"], az * _mode(sim.shape, kx, kz, sx=0.5, f=np.sin), atol=1e-14)
    assert np.abs(sim.f["by"]).max() == 0.0
    # TM part: Ex and Ez feed By = -h (D*_z Ex - D*_x Ez)
    sim2 = O.Sim(ndim=2, nx=nx, nz=nz, dx=dx, dz=dz, dt=0.5, solver=O.CK, ck_beta=(bx, bz))
    sim2.f["ex"] = _mode(sim2.shape, kx, kz, sx=0.5)
    sim2.f["ez"] = 0.7 * _mode(sim2.shape, kx, kz, sz=0.5)
    sim2.yee_b(h)
    # forward z difference of Ex at (i+1/2, k+1/2) and forward x difference of Ez there
    dzex = -2 / dz * math.sin(kz / 2) * (1 - 4 * bz * math.sin(kx / 2) ** 2)
    dxez = -0.7 * 2 / dx * math.sin(kx / 2) * (1 - 4 * bx * math.sin(kz / 2) ** 2)
    ref = -h * (dzex - dxez) * _mode(sim2.shape, kx, kz, sx=0.5, sz=0.5, f=np.sin)
    np.testing.assert_allclose(sim2.f["by"], ref, atol=1e-14)


@pytest.mark.parametrize("pol", ["TE", "TM"])
@pytest.mark.parametrize("dt,dx,dz,bx,bz", [(0.9, 1.0, 1.0, 0.125, 0.125), (0.8, 1.1, 0.95, 0.08, 0.15)])
def test_ck_vacuum_dispersion(pol, dt, dx, dz, bx, bz):
    # A plane wave started with B = 0 evolves as cos(n theta) exactly under the split-B leapfrog; theta
    # from the CK dispersion relation (c dt/dz = 0.9 is above Yee's 2D limit 1/sqrt(2)).
    nx, nz = 24, 40
    sim = O.Sim(ndim=2, nx=nx, nz=nz, dx=dx, dz=dz, dt=dt, solver=O.CK, ck_beta=(bx, bz))
    kx, kz = 2 * math.pi * 5 / nx, 2 * math.pi * 11 / nz
    if pol == "TE":
        sim.f["ey"] = _mode(sim.shape, kx, kz)
    else:  # the transverse eigenvector (Yee divergence-free, since the E update is Yee's)
        sim.f["ex"] = math.sin(kz / 2) / dz * _mode(sim.shape, kx, kz, sx=0.5)
        sim.f["ez"] = -math.sin(kx / 2) / dx * _mode(sim.shape, kx, kz, sz=0.5)
    e0 = {n: sim.f[n].copy() for n in ("ex", "ey", "ez")}
    th = _theta(dt, dx, dz, bx, bz, kx, kz)
    nsteps = 60
    for _ in range(nsteps):
        sim.yee_b(0.5 * dt)
        sim.yee_e(dt)
        sim.yee_b(0.5 * dt)
    for n in ("ex", "ey", "ez"):
        np.testing.assert_allclose(sim.f[n], math.cos(nsteps * th) * e0[n], atol=1e-12)


def test_ck_axis_wave_at_unit_courant_is_exact():
    # Along z (kx = 0) the CK z difference is Yee's, and at c dt = dz the discrete wave moves exactly
    # one cell per step: theta = kz dz.
    nx, nz, dt = 8, 32, 1.0
    sim = O.Sim(ndim=2, nx=nx, nz=nz, dt=dt, solver=O.CK)
    kz = 2 * math.pi * 7 / nz
    sim.f["ey"] = _mode(sim.shape, 0.0, kz)
    e0 = sim.f["ey"].copy()
    for _ in range(13):
        sim.yee_b(0.5 * dt)
        sim.yee_e(dt)
        sim.yee_b(0.5 * dt)
    np.testing.assert_allclose(sim.f["ey"], math.cos(13 * kz) * e0, atol=1e-12)


def test_ck_beta_zero_is_yee():
    rng = np.random.default_rng(5)
    a = O.Sim(ndim=2, nx=9, nz=13, dt=0.6)
    b = O.Sim(ndim=2, nx=9, nz=13, dt=0.6, solver=O.CK, ck_beta=(0.0, 0.0))
    for n in ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz"):
        a.f[n] = rng.normal(size=a.shape)
        b.f[n] = a.f[n].copy()
    for _ in range(5):
        for s in (a, b):
            s.yee_b(0.3)
            s.yee_e(0.6)
            s.yee_b(0.3)
    for n in ("ex", "ey", "ez", "bx", "by", "bz"):
        assert np.array_equal(a.f[n], b.f[n])


def _vacuum_growth(dt, solver, nsteps=200):
    rng = np.random.default_rng(11)
    sim = O.Sim(ndim=2, nx=16, nz=16, dt=dt, solver=solver)
    for n in ("ex", "ey", "ez"):
        sim.f[n] = rng.normal(size=sim.shape)
    m0 = max(np.abs(sim.f[n]).max() for n in ("ex", "ey", "ez"))
    for _ in range(nsteps):
        sim.yee_b(0.5 * dt)
        sim.yee_e(dt)
        sim.yee_b(0.5 * dt)
    return max(np.abs(sim.f[n]).max() for n in ("ex", "ey", "ez")) / m0


def test_ck_courant_limit():
    # beta = 1/8, dx = dz: stable up to c dt = 1 (the corner mode sx = sz = 1 reaches sin^2 = dt^2),
    # unstable just above; Yee at the same 0.9 is past its 1/sqrt(2) limit.
    assert _vacuum_growth(0.99, O.CK) < 10.0
    assert _vacuum_growth(1.02, O.CK) > 1e6
    assert _vacuum_growth(0.9, O.YEE) > 1e6


def test_ck_conserves_its_own_divergence_of_b():
    # The CK curl commutes with the averaged divergence A_x d_x Bx + A_z d_z Bz (periodic, shift
    # invariant operators), so starting from B = 0 that divergence stays at rounding level; the plain
    # Yee divergence of B does not (the solver really averages).
    rng = np.random.default_rng(2)
    bxw, bzw = 0.1, 0.125
    sim = O.Sim(ndim=2, nx=10, nz=14, dt=0.6, solver=O.CK, ck_beta=(bxw, bzw))
    for n in ("ex", "ey", "ez", "jx", "jy", "jz"):
        sim.f[n] = rng.normal(size=sim.shape)
    for _ in range(10):
        sim.yee_b(0.3)
        sim.yee_e(0.6)
        sim.yee_b(0.3)
    bx, bz = sim.f["bx"][:, 0, :], sim.f["bz"][:, 0, :]  # (z, x)
    avg_z = lambda f, w: (1 - 2 * w) * f + w * (np.roll(f, 1, 0) + np.roll(f, -1, 0))  # noqa: E731
    avg_x = lambda f, w: (1 - 2 * w) * f + w * (np.roll(f, 1, 1) + np.roll(f, -1, 1))  # noqa: E731
    dxf = lambda f: np.roll(f, -1, 1) - f  # noqa: E731
    dzf = lambda f: np.roll(f, -1, 0) - f  # noqa: E731
    div_ck = dxf(avg_z(bx, bxw)) + dzf(avg_x(bz, bzw))
    assert np.abs(div_ck).max() < 1e-12 * np.abs(bx).max()
    assert np.abs(sim.div_b()).max() > 1e-3


def test_ck_is_2d_only():
    with pytest.raises(ValueError):
        O.Sim(ndim=3, nx=4, ny=4, nz=4, solver=O.CK)
