"""Whole-step pins of the oracle: Gauss's law with the filtered current, div B, momentum of a
field-free beam, the growth fit on synthetic curves, and (slow) the Cherenkov contrast."""
import math

import numpy as np
import pytest

import oracle as O
from oracle.fit import growth_rate


def _beam(alpha=0.5, scheme=O.GALERKIN, corr=True, nx=16, nz=24, ndim=2, ny=1, ppc=4, f_targets=3, seed=1):
    st, pe, pb = O.rational_coeffs(scheme, alpha)
    sim = O.Sim(ndim=ndim, nx=nx, ny=ny, nz=nz, dt=alpha, scheme=scheme, psi_e=pe if corr else None,
                psi_b=pb if corr else None, f_nbin=1, f_ncomp=1, f_targets=f_targets)
    sim.init_beam(ppc=ppc, seed=seed, u_th=1e-2)
    return sim


@pytest.mark.parametrize("ndim", [2, 3])
def test_gauss_law_with_filtered_current(ndim):
    # div(F J) = F div J, so div E - F rho stays constant step after step (F = the J filter).
    sim = _beam(ndim=ndim, nx=10, ny=6 if ndim == 3 else 1, nz=14, ppc=4 if ndim == 2 else 1,
                alpha=0.5 if ndim == 2 else 0.45)
    g0 = sim.div_e() - sim.filter(sim.rho())
    scale = np.abs(sim.part["w"]).max()
    for _ in range(6):
        sim.step(1)
        g = sim.div_e() - sim.filter(sim.rho())
        assert np.abs(g - g0).max() < 1e-12 * scale
    assert sim.energy()[0] > 0
    assert np.abs(sim.div_b()).max() < 1e-14


def test_gauss_law_unfiltered():
    sim = _beam(f_targets=0)
    g0 = sim.div_e() - sim.rho()
    for _ in range(5):
        sim.step(1)
    assert np.abs(sim.div_e() - sim.rho() - g0).max() < 1e-13


def test_single_particle_free_streaming():
    # no fields, one particle: u unchanged, x advances by dt u / gamma.
    sim = O.Sim(ndim=2, nx=8, nz=8, dt=0.5, f_targets=0)
    sim.set_particles([1.3], None, [6.9], [0.1], [0.2], [5.0], [1e-12], [1.0])
    g = math.sqrt(1 + 0.01 + 0.04 + 25)
    sim.step(1)
    assert abs(sim.part["x"][0] - (1.3 + 0.5 * 0.1 / g)) < 1e-14
    assert abs(sim.part["z"][0] - ((6.9 + 0.5 * 5.0 / g) % 8)) < 1e-14


def test_growth_fit_recovers_rate():
    t = np.arange(200) * 0.5
    gam = 0.037
    noise = 1e-8 * (1 + 0.1 * np.sin(t))
    w = noise + 1e-9 * np.exp(2 * gam * t)
    w = np.minimum(w, 1e3)  # saturation
    g, i0, i1 = growth_rate(t, w)
    assert abs(g - gam) < 0.02 * gam
    assert i1 > i0 + 5


def test_growth_fit_fallback_window():
    # a curve that never gets two decades above its floor: fallback to the steepest 20 % window
    t = np.arange(100) * 1.0
    w = 1.0 + 0.5 * (t > 50) * (t - 50) / 50
    g, i0, i1 = growth_rate(t, w)
    assert i0 >= 10 and i1 - i0 + 1 == 20
    assert g > 0


@pytest.mark.slow
def test_cherenkov_growth_and_suppression():
    # Sec. 3/4, qualitative: without correction or filter the transverse field energy of the beam
    # grows exponentially (numerical Cherenkov); with the Psi correction and the filter it ends far lower.
    nsteps = 500
    runs = {}
    for label, corr, filt in (("off", False, 0), ("on", True, 3)):
        sim = _beam(alpha=0.7, corr=corr, nx=32, nz=64, f_targets=filt)
        sim.init_beam(ppc=4, seed=1)  # cold: u_th = 1e-4
        w = []
        for _ in range(nsteps // 10):
            sim.step(10)
            w.append(sim.energy()[2])
        runs[label] = np.array(w)
    t = np.arange(1, nsteps // 10 + 1) * 10 * 0.7
    g_off, _, _ = growth_rate(t, runs["off"])
    assert runs["off"][-1] > 1e3 * runs["off"][5]   # clear exponential growth
    assert g_off > 0.01
    assert runs["on"][-1] < 1e-2 * runs["off"][-1]
