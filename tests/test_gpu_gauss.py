"""GPU parity of the Gauss-law diagnostic pic_charge_residual (charge conservation of the Esirkepov
deposit with the filtered current, Sec. 2 / Eq. 6) against the oracle's div E - F rho of the same state,
and its size after steps from the seeded beam."""
import math

import numpy as np
import pytest

import oracle as O
import synth
from tests._pic import P, Pair, make_cfg, uniform_weight

pytestmark = pytest.mark.gpu

FIELDS = ("ex", "ey", "ez", "bx", "by", "bz")


def _oracle_residual(pair, cfg):
    """(max, rms, max |F rho|) of div E - F rho by the oracle, from the handle's exported state."""
    f, p = pair.gpu_state()
    o = O.Sim(ndim=cfg.ndim, nx=cfg.nx, ny=cfg.ny, nz=cfg.nz, dx=cfg.dx, dy=cfg.dy, dz=cfg.dz, dt=cfg.dt,
              f_nbin=cfg.filter_nbin, f_ncomp=cfg.filter_ncomp, f_alpha=cfg.filter_comp_alpha,
              order=cfg.shape_order)
    o.set_particles(p["x"], p["y"] if cfg.ndim == 3 else None, p["z"], p["ux"], p["uy"], p["uz"], p["w"], p["q"])
    o.f.update({n: f[n].reshape(o.shape).copy() for n in FIELDS})
    rho = o.rho()
    frho = o.filter(rho) if cfg.filter_targets & P.PIC_FILTER_J else rho
    g = o.div_e() - frho
    return np.abs(g).max(), math.sqrt(np.mean(g ** 2)), np.abs(frho).max()


def _handle_pair(cfg):
    pair = object.__new__(Pair)
    pair.cfg, pair.T = cfg, np.float32 if cfg.precision == 0 else np.float64
    pair.u0 = math.sqrt(cfg.gamma ** 2 - 1)
    pair.o = O.Sim(ndim=cfg.ndim, nx=cfg.nx, ny=cfg.ny, nz=cfg.nz, dt=cfg.dt)
    return pair


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("order,targets", [(1, 3), (3, 3), (1, 2)])
def test_residual_matches_oracle(precision, order, targets):
    # an arbitrary E (not the one Gauss's law would give) over the particles of a few beam steps: the
    # residual is large, and the library's FP64 evaluation equals the oracle's of the same state
    # (ragged 2D grid, both species, 8 ppc; filter on J or not)
    cfg = make_cfg(nx=37, nz=70, dt=0.5, precision=precision, ppc=8, init_beam=1, seed=5, order=order,
                   targets=targets, cap=48 if order == 3 else 0)
    h = P.pic_create(cfg)
    try:
        pair = _handle_pair(cfg)
        pair.h = h
        P.pic_step(h, 2)
        fields = synth.random_fields((cfg.nz, 1, cfg.nx), seed=17, scale=1e-2, smooth=1)
        fn = {n: np.ascontiguousarray(fields[n].astype(pair.T)) for n in FIELDS}
        s = P.make_state(P.PIC_HOST, fn, None)
        s.np = -1  # fields only: the particles stay
        P.pic_set_state(h, s)
        got = P.pic_charge_residual(h)
        mx, rms, scale = _oracle_residual(pair, cfg)
    finally:
        P.pic_destroy(h)
    # the pairs have barely separated, so F rho is a cancellation of O(one) terms: its bar is absolute,
    # in units of one particle's charge density; the residual (dominated by div E) is compared relatively
    one = uniform_weight(cfg)
    assert mx > 1e-4
    assert abs(got["max"] - mx) <= 1e-12 * mx, (got, mx)
    assert abs(got["rms"] - rms) <= 1e-12 * rms, (got, rms)
    assert abs(got["rho_max"] - scale) <= 1e-12 * one, (got, scale)


@pytest.mark.parametrize("precision,order", [(1, 1), (1, 3), (0, 1)])
def test_residual_is_conserved_by_the_step(precision, order):
    # a non-neutral random particle set with E = B = 0: the residual field is -F rho (large) and the
    # step must leave it unchanged node by node, so its max and RMS keep their values while the
    # particles move (FP64: to 1e-11 relative; FP32: the positions and the current carry FP32 rounding)
    nx, nz = 48, 80
    cfg = make_cfg(nx=nx, nz=nz, dt=0.5, precision=precision, ppc=4, order=order, track_ids=1,
                   cap=64 if order == 3 else 0)
    part = synth.random_particles(2, nx, 1, nz, 12000, seed=23)
    pair = Pair(cfg, psi=P.pic_compute_correction_coeffs(0, 0.5), part=part)
    try:
        r0 = P.pic_charge_residual(pair.h)
        P.pic_step(pair.h, 30)
        r1 = P.pic_charge_residual(pair.h)
        mx, rms, scale = _oracle_residual(pair, cfg)
    finally:
        pair.close()
    assert r0["max"] > 0.1 * uniform_weight(cfg)
    tol = 1e-11 if precision == 1 else 2e-5
    assert abs(r1["max"] - r0["max"]) <= tol * r0["max"], (r0, r1)
    assert abs(r1["rms"] - r0["rms"]) <= tol * r0["rms"], (r0, r1)
    # and the final value is the oracle's evaluation of the final state
    assert abs(r1["max"] - mx) <= 1e-12 * mx and abs(r1["rms"] - rms) <= 1e-12 * rms, (r1, mx, rms)


@pytest.mark.parametrize("precision,order", [(1, 1), (1, 3), (0, 1)])
def test_residual_stays_at_roundoff_from_the_beam(precision, order):
    # steps from the seeded neutral beam with E = B = 0 and the Psi correction and the filter on:
    # div E - F rho stays at rounding level, in units of one particle's charge density
    cfg = make_cfg(nx=64, nz=128, dt=0.5, precision=precision, ppc=4, init_beam=1, seed=3, order=order,
                   track_ids=0, cap=48 if order == 3 else 0)
    h = P.pic_create(cfg)
    try:
        P.pic_set_correction_stencil(h, *P.pic_compute_correction_coeffs(0, 0.5))
        P.pic_step(h, 40)
        got = P.pic_charge_residual(h)
    finally:
        P.pic_destroy(h)
    one = uniform_weight(cfg)
    assert got["max"] < (1e-11 if precision == 1 else 1e-4) * one, got
