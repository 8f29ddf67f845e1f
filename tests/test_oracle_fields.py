"""Pins of the oracle's field operators: Psi z-stencil and Eq. 6 filter on Fourier modes, gather copies,
Yee vacuum dispersion (exact discrete solution of a plane wave), div B and Gauss's law invariants."""
import math

import numpy as np
import pytest

import oracle as O


def _mode(shape, kx, ky, kz, sx=0.0, sy=0.0, sz=0.0):
    nz, ny, nx = shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.cos(kx * (i + sx) + ky * (j + sy) + kz * (k + sz))


def _filter_symbol(k, nbin, ncomp, a):
    c2 = math.cos(k / 2) ** 2
    return c2 ** nbin * (a - (a - 1) * (2 * c2 - 1)) ** ncomp


@pytest.mark.parametrize("nbin,ncomp,alpha", [(1, 1, 3.0), (2, 2, 3.0), (2, 1, 2.0), (1, 0, 3.0)])
def test_filter_transfer(nbin, ncomp, alpha):
    # Eq. 6 per direction: cos^4 (5 - 4 cos^2)^2 for two bilinear + two compensation passes;
    # its square root cos^2 (5 - 4 cos^2) for one of each (Sec. 4). Written here in terms of cos^2(k/2).
    sim = O.Sim(ndim=2, nx=24, nz=32, f_nbin=nbin, f_ncomp=ncomp, f_alpha=alpha)
    for mx, mz in [(0, 0), (1, 3), (5, 7), (12, 16), (7, 0)]:
        kx, kz = 2 * math.pi * mx / 24, 2 * math.pi * mz / 32
        f = _mode(sim.shape, kx, 0, kz)
        g = sim.filter(f)
        expect = _filter_symbol(kx, nbin, ncomp, alpha) * _filter_symbol(kz, nbin, ncomp, alpha)
        np.testing.assert_allclose(g, expect * f, atol=1e-13)


def test_eq6_literal_form():
    # (2,2,3) is Eq. 6 literally: cos^4(s)(5-4cos^2 s)^2 per direction, peak gain 2.44 at cos^2 = 5/8.
    for s in np.linspace(0, math.pi / 2, 11):
        c2 = math.cos(s) ** 2
        assert abs(_filter_symbol(2 * s, 2, 2, 3.0) - c2 ** 2 * (5 - 4 * c2) ** 2) < 1e-13
    c2 = 5 / 8
    assert abs(c2 ** 2 * (5 - 4 * c2) ** 2 - 2.44140625) < 1e-12


def test_filter_3d_transfer():
    sim = O.Sim(ndim=3, nx=8, ny=12, nz=16, f_nbin=1, f_ncomp=1)
    kx, ky, kz = 2 * math.pi * 3 / 8, 2 * math.pi * 5 / 12, 2 * math.pi * 2 / 16
    f = _mode(sim.shape, kx, ky, kz)
    g = sim.filter(f)
    e = _filter_symbol(kx, 1, 1, 3) * _filter_symbol(ky, 1, 1, 3) * _filter_symbol(kz, 1, 1, 3)
    np.testing.assert_allclose(g, e * f, atol=1e-13)


def test_gather_copies_symbols():
    # Copies seen by the particles: Psi_E(xi_z) on Ex, Ey; Psi_B(xi_z) on Ez, Bx, By, Bz; times the filter.
    _, pe, pb = O.rational_coeffs(O.GALERKIN, 0.5)
    sim = O.Sim(ndim=2, nx=16, nz=32, psi_e=pe, psi_b=pb, f_nbin=1, f_ncomp=1)
    kx, kz = 2 * math.pi * 3 / 16, 2 * math.pi * 5 / 32
    base = _mode(sim.shape, kx, 0, kz)
    for n in ("ex", "ey", "ez", "bx", "by", "bz"):
        sim.f[n] = base.copy()
    out = sim.gather_copies()
    fx = _filter_symbol(kx, 1, 1, 3) * _filter_symbol(kz, 1, 1, 3)
    xi = math.sin(kz / 2) ** 2
    for c in range(6):
        psi = np.polyval((pe if c < 2 else pb)[::-1], xi)
        np.testing.assert_allclose(out[c], psi * fx * base, atol=1e-12)
    # the Yee fields themselves are untouched
    np.testing.assert_array_equal(sim.f["ex"], base)


def _dispersion_theta(dt, kx, ky, kz, dx=1.0, dy=1.0, dz=1.0):
    # Yee vacuum dispersion: sin^2(w dt/2)/dt^2 = sum sin^2(k d/2)/d^2
    s = dt * math.sqrt(math.sin(kx * dx / 2) ** 2 / dx ** 2 + math.sin(ky * dy / 2) ** 2 / dy ** 2
                       + math.sin(kz * dz / 2) ** 2 / dz ** 2)
    return 2 * math.asin(s)


@pytest.mark.parametrize("pol", ["TE", "TM"])
def test_yee_vacuum_dispersion_2d(pol):
    # A single plane wave started with B = 0 evolves as cos(n w dt) exactly for the split-B leapfrog,
    # with w from the Yee dispersion relation.
    nx, nz, dt, dx, dz = 32, 48, 0.45, 1.0, 1.3
    sim = O.Sim(ndim=2, nx=nx, nz=nz, dt=dt, dx=dx, dz=dz)
    kx, kz = 2 * math.pi * 3 / nx, 2 * math.pi * 5 / nz
    if pol == "TE":
        sim.f["ey"] = _mode(sim.shape, kx, 0, kz)
    else:  # discrete divergence-free (Ex, Ez)
        ax, az = math.sin(kz / 2) / dz, -math.sin(kx / 2) / dx
        sim.f["ex"] = ax * _mode(sim.shape, kx, 0, kz, sx=0.5)
        sim.f["ez"] = az * _mode(sim.shape, kx, 0, kz, sz=0.5)
    e0 = {n: sim.f[n].copy() for n in ("ex", "ey", "ez")}
    s = dt * math.sqrt(math.sin(kx / 2) ** 2 / dx ** 2 + math.sin(kz / 2) ** 2 / dz ** 2)
    th = 2 * math.asin(s)
    nsteps = 40
    for _ in range(nsteps):
        sim.yee_b(0.5 * dt)
        sim.yee_e(dt)
        sim.yee_b(0.5 * dt)
    for n in ("ex", "ey", "ez"):
        np.testing.assert_allclose(sim.f[n], math.cos(nsteps * th) * e0[n], atol=1e-12)


def test_yee_vacuum_dispersion_3d():
    nx, ny, nz, dt = 12, 10, 16, 0.4
    sim = O.Sim(ndim=3, nx=nx, ny=ny, nz=nz, dt=dt)
    kx, ky, kz = 2 * math.pi * 2 / nx, 2 * math.pi * 1 / ny, 2 * math.pi * 3 / nz
    # divergence-free E: amplitudes a with sum a_d sin(k_d/2) = 0
    sx, sy, sz = math.sin(kx / 2), math.sin(ky / 2), math.sin(kz / 2)
    a = np.cross([sx, sy, sz], [1.0, 0.3, -0.2])
    sim.f["ex"] = a[0] * _mode(sim.shape, kx, ky, kz, sx=0.5)
    sim.f["ey"] = a[1] * _mode(sim.shape, kx, ky, kz, sy=0.5)
    sim.f["ez"] = a[2] * _mode(sim.shape, kx, ky, kz, sz=0.5)
    assert np.abs(sim.div_e()).max() < 1e-13
    e0 = {n: sim.f[n].copy() for n in ("ex", "ey", "ez")}
    th = _dispersion_theta(dt, kx, ky, kz)
    for _ in range(25):
        sim.yee_b(0.5 * dt)
        sim.yee_e(dt)
        sim.yee_b(0.5 * dt)
    for n in ("ex", "ey", "ez"):
        np.testing.assert_allclose(sim.f[n], math.cos(25 * th) * e0[n], atol=1e-12)


@pytest.mark.parametrize("ndim", [2, 3])
def test_div_b_stays_zero(ndim):
    rng = np.random.default_rng(1)
    sim = O.Sim(ndim=ndim, nx=10, ny=6, nz=14, dt=0.4)
    for n in ("ex", "ey", "ez", "jx", "jy", "jz"):
        sim.f[n] = rng.normal(size=sim.shape)
    for _ in range(10):
        sim.yee_b(0.2)
        sim.yee_e(0.4)
        sim.yee_b(0.2)
    assert np.abs(sim.div_b()).max() < 1e-12
    assert np.abs(sim.f["bx"]).max() > 0.1


def test_curl_adjointness():
    # The discrete curls are adjoint on the periodic Yee mesh: <curl_E(E), B> = <E, curl_B(B)>.
    rng = np.random.default_rng(3)
    sim = O.Sim(ndim=3, nx=6, ny=5, nz=7, dt=1.0)
    E = {n: rng.normal(size=sim.shape) for n in ("ex", "ey", "ez")}
    B = {n: rng.normal(size=sim.shape) for n in ("bx", "by", "bz")}
    s1 = O.Sim(ndim=3, nx=6, ny=5, nz=7)
    s1.f.update({k: v.copy() for k, v in E.items()})
    s1.yee_b(-1.0)  # B = curl E
    lhs = sum((s1.f[n] * B[n]).sum() for n in ("bx", "by", "bz"))
    s2 = O.Sim(ndim=3, nx=6, ny=5, nz=7)
    s2.f.update({k: v.copy() for k, v in B.items()})
    s2.yee_e(1.0)  # E = curl B
    rhs = sum((s2.f[n] * E[n.replace("b", "e")]).sum() for n in ("ex", "ey", "ez"))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
