"""Pins of the oracle's exact rational multiplier (Sec. 2: Psi_B applied by inversion; Sec. 3's
variant with Psi_E / Psi_B on the transverse E copies only): the circulant inverse on Fourier modes,
the round trip through Psi_B's own stencil, the copies' transfer functions, and Gauss's law over
whole steps."""
import numpy as np
import pytest

import oracle as O


def _coeffs(alpha=0.6, scheme=O.GALERKIN):
    st, pe, pb = O.rational_coeffs(scheme, alpha)
    assert st == 0
    return pe, pb


def _poly(c, xi):
    return sum(c[n] * xi ** n for n in range(5))


@pytest.mark.parametrize("nz", [16, 33])
def test_inverse_on_fourier_modes(nz):
    pe, pb = _coeffs()
    sim = O.Sim(ndim=2, nx=5, nz=nz, psi_e=pe, psi_b=pb)
    k = np.arange(nz)[:, None, None] * np.ones((1, 1, 5))
    for m in (0, 1, 3, nz // 2):
        for ph in (0.0, 0.7):
            f = np.cos(2 * np.pi * m * k / nz + ph)
            g = sim.inverse_psi_z(f)
            xi = np.sin(np.pi * m / nz) ** 2
            np.testing.assert_allclose(g, f / _poly(pb, xi), atol=1e-12)


def test_inverse_round_trip_through_the_stencil():
    # Psi_B(D_z) applied (9-tap stencil) to Psi_B(D_z)^-1 f gives f back
    pe, pb = _coeffs(0.45, O.UNIFORM)
    sim = O.Sim(ndim=2, nx=7, nz=24, psi_e=pe, psi_b=pb)
    f = np.random.default_rng(3).normal(size=sim.shape)
    g = sim.inverse_psi_z(f)
    back = sim.conv_axis(g, 2, O.psi_taps(pb))
    np.testing.assert_allclose(back, f, atol=1e-12)


def test_copies_transfer_functions_rational_mode():
    # corr_mode 1: Ex, Ey copies carry Psi_E / Psi_B times the gather filter; Ez, B copies the filter only
    pe, pb = _coeffs()
    nx, nz = 8, 32
    sim = O.Sim(ndim=2, nx=nx, nz=nz, psi_e=pe, psi_b=pb, corr_mode=1)
    kz, kx = 3, 1
    k, _, i = np.meshgrid(np.arange(nz), np.arange(1), np.arange(nx), indexing="ij")
    mode = np.cos(2 * np.pi * (kz * k / nz + kx * i / nx))
    for n in ("ex", "ey", "ez", "bx", "by", "bz"):
        sim.f[n][...] = mode
    G = sim.gather_copies()
    sz, sx = np.sin(np.pi * kz / nz) ** 2, np.sin(np.pi * kx / nx) ** 2
    filt = lambda s: (1 - s) * (5 - 4 * (1 - s))  # one bilinear and one compensation pass (a = 3)
    fz, fx = filt(sz), filt(sx)
    rat = _poly(pe, sz) / _poly(pb, sz)
    for c in range(6):
        expect = mode * fz * fx * (rat if c < 2 else 1.0)
        np.testing.assert_allclose(G[c], expect, atol=1e-12)


def test_gauss_law_rational_mode():
    pe, pb = _coeffs()
    sim = O.Sim(ndim=2, nx=12, nz=20, dt=0.6, psi_e=pe, psi_b=pb, corr_mode=1)
    sim.init_beam(ppc=4, u_th=1e-2, seed=5)
    rng = np.random.default_rng(6)
    for n in ("ex", "ey", "ez", "bx", "by", "bz"):
        sim.f[n][...] = 1e-2 * rng.standard_normal(sim.shape)
    g0 = sim.div_e() - sim.filter(sim.rho())
    for _ in range(4):
        sim.step(1)
    g = sim.div_e() - sim.filter(sim.rho())
    assert np.abs(g - g0).max() < 1e-12 * max(np.abs(sim.part["w"]).max(), np.abs(g0).max())
