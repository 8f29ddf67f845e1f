"""Pins of the oracle's energy sums (the observables of the Fig. 2 and Fig. 4 captions: field energy,
its transverse part W_perp, and the kinetic energy) against closed forms, not against a restatement of
the sums.

Fields: a staggered plane wave A cos(k . r) of an integer mode (0 < m < N/2 along an axis) sampled on
its Yee points of a periodic N-cell grid has sum cos^2 = N / 2 exactly (discrete orthogonality,
whatever the half-cell shift), so the energy of one component is A^2 N dV / 4 with dV = dx dy dz.
Unequal cell sizes make a dropped dV visible, a dropped 1/2 doubles the value, and one component at a
time shows which sum (W_E, W_B, W_perp = Ex, Ey, Bx, By) it enters.
Particles: momenta with exactly known Lorentz factors, gamma^2 = 1 + |u|^2 (u = 4/3 gives gamma = 5/3;
u = (12/5, 0, 0) ... gamma = 13/5; the gamma = 130 beam drift gamma - 1 = 129), so K = sum w (gamma - 1)
is known in closed form; a sum of w gamma would be off by sum w, and the no-cancellation form keeps full
relative precision for the thermal momenta (|u| = 1e-4: gamma - 1 = u^2 / 2 - u^4 / 8 + ...)."""
import math

import numpy as np
import pytest

import oracle as O

COMPONENTS = ("ex", "ey", "ez", "bx", "by", "bz")
# (in W_E, in W_B, in W_perp)
ROLE = {"ex": (1, 0, 1), "ey": (1, 0, 1), "ez": (1, 0, 0), "bx": (0, 1, 1), "by": (0, 1, 1), "bz": (0, 1, 0)}
# half-cell offsets of each component on the Yee mesh (x, y, z)
STAGGER = {"ex": (0.5, 0, 0), "ey": (0, 0.5, 0), "ez": (0, 0, 0.5), "bx": (0, 0.5, 0.5), "by": (0.5, 0, 0.5),
           "bz": (0.5, 0.5, 0)}


def _sim(ndim):
    if ndim == 2:
        return O.Sim(ndim=2, nx=12, nz=20, dx=0.7, dz=1.3, dt=0.3)
    return O.Sim(ndim=3, nx=8, ny=6, nz=10, dx=0.7, dy=1.1, dz=1.3, dt=0.2)


def _wave(sim, comp, amp, mode):
    nz, ny, nx = sim.shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    sx, sy, sz = STAGGER[comp]
    mx, my, mz = mode
    phase = 2 * np.pi * (mx * (i + sx) / nx + my * (j + sy) / max(ny, 1) + mz * (k + sz) / nz)
    return amp * np.cos(phase)


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("comp", COMPONENTS)
def test_single_component_plane_wave(ndim, comp):
    sim = _sim(ndim)
    nz, ny, nx = sim.shape
    n = nx * ny * nz
    dv = 0.7 * 1.3 * (1.1 if ndim == 3 else 1.0)
    amp = 0.37
    mode = (2, 1 if ndim == 3 else 0, 3)
    for c in COMPONENTS:
        sim.f[c] = np.zeros(sim.shape)
    sim.f[comp] = _wave(sim, comp, amp, mode)
    we, wb, wp, k, tot = sim.energy()
    expect = amp * amp * n * dv / 4.0
    in_e, in_b, in_p = ROLE[comp]
    assert we == pytest.approx(in_e * expect, rel=1e-13, abs=1e-15)
    assert wb == pytest.approx(in_b * expect, rel=1e-13, abs=1e-15)
    assert wp == pytest.approx(in_p * expect, rel=1e-13, abs=1e-15)
    assert k == 0.0
    assert tot == pytest.approx(we + wb, rel=1e-15)


def test_two_waves_add_and_uniform_field():
    # orthogonal modes add their energies; a uniform field E0 in every cell gives E0^2 N dV / 2
    sim = _sim(2)
    nz, ny, nx = sim.shape
    n = nx * ny * nz
    dv = 0.7 * 1.3
    for c in COMPONENTS:
        sim.f[c] = np.zeros(sim.shape)
    sim.f["by"] = _wave(sim, "by", 0.2, (1, 0, 2)) + _wave(sim, "by", 0.5, (3, 0, 1))
    sim.f["ey"] = np.full(sim.shape, 0.25)
    we, wb, wp, _, _ = sim.energy()
    assert wb == pytest.approx((0.2 ** 2 + 0.5 ** 2) * n * dv / 4.0, rel=1e-13)
    assert we == pytest.approx(0.25 ** 2 * n * dv / 2.0, rel=1e-13)
    assert wp == pytest.approx(we + wb, rel=1e-13)


def test_kinetic_energy_exact_gammas():
    sim = _sim(2)
    for c in COMPONENTS:
        sim.f[c] = np.zeros(sim.shape)
    u0 = math.sqrt(130.0 ** 2 - 1.0)
    # (ux, uy, uz, w, exact gamma - 1)
    cases = [
        (0.0, 0.0, 4.0 / 3.0, 0.5, 2.0 / 3.0),
        (0.0, 12.0 / 5.0, 0.0, 0.25, 8.0 / 5.0),
        (3.0 / 5.0 * 4.0 / 3.0, 0.0, 4.0 / 5.0 * 4.0 / 3.0, 2.0, 2.0 / 3.0),  # |u| = 4/3 split over x, z
        (0.0, 0.0, u0, 0.125, 129.0),
        (0.0, 0.0, -u0, 1.5, 129.0),
        (0.0, 0.0, 0.0, 3.0, 0.0),
    ]
    ux, uy, uz, w, gm1 = (np.array(c) for c in zip(*cases))
    n = len(cases)
    sim.set_particles(np.linspace(0.5, 10.5, n), None, np.linspace(1.5, 15.5, n), ux, uy, uz, w,
                      np.where(np.arange(n) % 2 == 0, -1.0, 1.0))
    we, wb, wp, k, tot = sim.energy()
    assert we == wb == wp == 0.0
    assert k == pytest.approx(float(np.sum(w * gm1)), rel=1e-15)
    assert tot == pytest.approx(k, rel=1e-15)


def test_kinetic_energy_thermal_momenta_keep_precision():
    # |u| = 1e-4 (the beam's thermal spread): gamma - 1 = u^2/2 - u^4/8 + u^6/16 - ..., which a plain
    # sqrt(1 + u^2) - 1 would give to only ~1e-8 relative
    sim = _sim(2)
    for c in COMPONENTS:
        sim.f[c] = np.zeros(sim.shape)
    u = 1e-4
    sim.set_particles(np.array([1.5]), None, np.array([2.5]), np.array([u]), np.array([0.0]), np.array([0.0]),
                      np.array([1.0]), np.array([-1.0]))
    k = sim.energy()[3]
    series = u * u / 2 - u ** 4 / 8 + u ** 6 / 16
    assert k == pytest.approx(series, rel=1e-14)
