"""GPU parity of the Cole-Karkkainen field solver (the CK solver named in Sec. 2 for Fig. 1: beta_z =
1/8, c dt/dz = 0.9, above Yee's 2D limit) against the FP64 oracle, through the C ABI.

Bars as in the Yee parity tests: FP64 <= 1e-10 and FP32 <= 1e-5 relative per step; the growth rate of
the uncorrected gamma = 130 beam within 5 % of the oracle run from the same state.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth
from oracle.fit import growth_rate
from tests._pic import P, Pair, make_cfg, rel_l2, uniform_weight
from tests.test_gpu_parity import FIELDS, TOL, _compare

pytestmark = pytest.mark.gpu


def _ck_pair(precision, nx, nz, npart, alpha=0.9, scheme=0, seed=0, psi=True, beta=(0.125, 0.125), field_scale=2e-2,
             dx=1.0, dz=1.0):
    cfg = make_cfg(nx=nx, nz=nz, dt=alpha, scheme=scheme, precision=precision, solver=P.PIC_CK, ck_beta=beta,
                   dx=dx, dz=dz)
    fields = synth.random_fields((nz, 1, nx), seed=seed + 100, scale=field_scale, smooth=1)
    part = synth.random_particles(2, nx, 1, nz, npart, seed=seed + 200) if npart else None
    coeffs = P.pic_compute_correction_coeffs(scheme, alpha) if psi else None
    return Pair(cfg, psi=coeffs, fields=fields, part=part)


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("nx,nz", [(40, 72), (33, 70), (5, 7), (1, 2)])
def test_ck_vacuum(precision, nx, nz):
    # field-only steps; grids from several tiles with ragged edges down to halos that wrap many times
    pair = _ck_pair(precision, nx, nz, 0)
    try:
        pair.step(10)
        _compare(pair, TOL[precision] * (10 if precision == 0 else 1), particles=False)
    finally:
        pair.close()


def test_ck_anisotropic_weights_and_cells():
    # unequal beta_x, beta_z and dx != dz (a swapped weight or axis fails)
    pair = _ck_pair(1, 48, 40, 0, alpha=0.8, beta=(0.08, 0.15), dx=1.1, dz=0.95)
    try:
        pair.step(6)
        _compare(pair, 1e-10, particles=False)
    finally:
        pair.close()


def test_ck_plane_wave_closed_form():
    # A vacuum plane wave started with B = 0 evolves as cos(n theta) E0 with theta from the CK
    # dispersion relation sin^2(theta/2) = dt^2 [sz^2 (1 - 4 bz sx^2) + sx^2 (1 - 4 bx sz^2)] (dx = dz = 1)
    nx, nz, dt, n = 64, 96, 0.9, 80
    cfg = make_cfg(nx=nx, nz=nz, dt=dt, precision=1, solver=P.PIC_CK, targets=0)
    kx, kz = 2 * math.pi * 5 / nx, 2 * math.pi * 17 / nz
    k, i = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    ey = np.cos(kx * i + kz * k)[:, None, :]
    zero = np.zeros_like(ey)
    h = P.pic_create(cfg)
    try:
        P.pic_set_state(h, P.make_state(P.PIC_HOST, {"ex": zero, "ey": ey, "ez": zero, "bx": zero, "by": zero,
                                                     "bz": zero}, None))
        P.pic_step(h, n)
        out = {c: np.zeros(nx * nz) for c in ("ex", "ey", "ez", "bx", "by", "bz")}
        P.pic_get_state(h, P.make_state(P.PIC_HOST, out, None))
    finally:
        P.pic_destroy(h)
    sx, sz = math.sin(kx / 2), math.sin(kz / 2)
    th = 2 * math.asin(dt * math.sqrt(sz * sz * (1 - 0.5 * sx * sx) + sx * sx * (1 - 0.5 * sz * sz)))
    np.testing.assert_allclose(out["ey"].reshape(ey.shape), math.cos(n * th) * ey, atol=1e-10)
    assert np.abs(out["ex"]).max() == 0.0 and np.abs(out["ez"]).max() == 0.0


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("scheme", [0, 1])
def test_ck_step(precision, scheme):
    # whole steps with particles and the Psi correction at c dt/dz = 0.9
    pair = _ck_pair(precision, 40, 72, 20000, scheme=scheme)
    try:
        pair.step(1)
        _compare(pair, TOL[precision])
    finally:
        pair.close()


def test_ck_multi_step_fp64():
    pair = _ck_pair(1, 32, 48, 12000, seed=3)
    try:
        for _ in range(5):
            pair.step(1)
        _compare(pair, 1e-10)
    finally:
        pair.close()


def test_ck_zero_beta_is_yee():
    # beta = 0 turns the CK curl into Yee's (c dt/dz below Yee's limit)
    a = _ck_pair(1, 40, 72, 8000, alpha=0.6, beta=(0.0, 0.0), seed=5)
    cfg = make_cfg(nx=40, nz=72, dt=0.6, precision=1)
    fields = synth.random_fields((72, 1, 40), seed=105, scale=2e-2, smooth=1)
    part = synth.random_particles(2, 40, 1, 72, 8000, seed=205)
    b = Pair(cfg, psi=P.pic_compute_correction_coeffs(0, 0.6), fields=fields, part=part)
    try:
        a.step(3)
        b.step(3)
        fa, _ = a.gpu_state()
        fb, _ = b.gpu_state()
        for n in FIELDS:
            assert rel_l2(fa[n], fb[n]) <= 1e-13, n
    finally:
        a.close()
        b.close()


def test_ck_gauss_law_beam_fp32():
    # the E update is Yee's, so div E - F rho stays at roundoff with the Esirkepov deposit (256x512
    # seeded beam, 16 ppc/species, FP32, c dt/dz = 0.9, Galerkin + Psi + filter)
    nx, nz = 256, 512
    cfg = make_cfg(nx=nx, nz=nz, dt=0.9, precision=0, ppc=16, init_beam=1, seed=4, track_ids=0, solver=P.PIC_CK)
    h = P.pic_create(cfg)
    try:
        P.pic_set_correction_stencil(h, *P.pic_compute_correction_coeffs(0, 0.9))
        P.pic_step(h, 20)
        pair = object.__new__(Pair)
        pair.cfg, pair.h, pair.T = cfg, h, np.float32
        pair.u0 = math.sqrt(cfg.gamma ** 2 - 1)
        pair.o = O.Sim(ndim=2, nx=nx, nz=nz, dt=0.9)
        f, p = pair.gpu_state()
        assert len(p["x"]) == nx * nz * 32
        o = pair.o
        o.set_particles(p["x"], None, p["z"], p["ux"], p["uy"], p["uz"], p["w"], p["q"])
        o.f.update({n: f[n].reshape(o.shape).copy() for n in FIELDS})
        g = o.div_e() - o.filter(o.rho())
        assert np.abs(g).max() < 2e-3 * uniform_weight(cfg)
    finally:
        P.pic_destroy(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_ck_growth_rate_matches_oracle(precision):
    # the uncorrected, unfiltered gamma = 130 beam at c dt/dz = 0.9 (2D 64x128, 4 ppc/species): the fitted
    # growth rate of W_perp agrees with the oracle's run from the same initial state
    alpha, nx, nz, steps, every = 0.9, 64, 128, 400, 10
    cfg = make_cfg(nx=nx, nz=nz, dt=alpha, precision=precision, ppc=4, init_beam=1, seed=1, targets=0, track_ids=1,
                   solver=P.PIC_CK)
    cfg.diag_every = every
    h = P.pic_create(cfg)
    try:
        pair = object.__new__(Pair)
        pair.cfg, pair.h = cfg, h
        pair.T = np.float32 if precision == 0 else np.float64
        pair.u0 = math.sqrt(cfg.gamma ** 2 - 1)
        pair.o = O.Sim(ndim=2, nx=nx, nz=nz, dt=alpha)
        _, p0 = pair.gpu_state()
        o = O.Sim(ndim=2, nx=nx, nz=nz, dt=alpha, f_targets=0, solver=O.CK)
        o.set_particles(p0["x"], None, p0["z"], p0["ux"], p0["uy"], p0["uz"], p0["w"], p0["q"], pid=p0["id"])
        w_o = []
        for _ in range(steps // every):
            o.step(every)
            w_o.append(o.energy()[2])
        P.pic_step(h, steps)
        w_g = [e["w_perp"] for e in P.pic_energy_history(h, 4096)]
    finally:
        P.pic_destroy(h)
    t = np.arange(1, steps // every + 1) * every * alpha
    g_o, a, b = growth_rate(t, w_o)
    assert w_o[-1] > 1e3 * w_o[5]
    sel = slice(a, b + 1)
    tt, lw = t[sel], np.log(np.asarray(w_g)[sel])
    g_same = 0.5 * float(((tt - tt.mean()) * (lw - lw.mean())).sum() / ((tt - tt.mean()) ** 2).sum())
    assert abs(g_same / g_o - 1) < 0.05, (g_same, g_o, (a, b))
    # and over the window the fit rule picks on the GPU run's own history
    g_g, c, d = growth_rate(t, w_g)
    assert abs(g_g / g_o - 1) < 0.05, (g_g, g_o, (a, b), (c, d))


@pytest.mark.parametrize("scheme", [0, 1])
def test_ck_cubic_correction_suppresses_growth_past_yee_limit(scheme):
    # The setting of Fig. 2 past Yee's 2D limit: CK solver, cubic shapes, 128x128, gamma = 130, the
    # Eq. 6 filter. With the Psi correction the fitted growth rate of W_perp stays at the floor at
    # c dt/dz = 0.8 and 0.95, far below the uncorrected run's.
    steps, every = 2000, 10
    rates = {}
    for alpha in (0.8, 0.95):
        for corr in (False, True):
            cfg = make_cfg(nx=128, nz=128, dt=alpha, scheme=scheme, precision=0, ppc=4, init_beam=1, seed=7,
                           track_ids=0, order=3, cap=96, solver=P.PIC_CK)
            cfg.diag_every = every
            h = P.pic_create(cfg)
            try:
                if corr:
                    P.pic_set_correction_stencil(h, *P.pic_compute_correction_coeffs(scheme, alpha))
                P.pic_step(h, steps)
                w = [e["w_perp"] for e in P.pic_energy_history(h, 4096)]
            finally:
                P.pic_destroy(h)
            t = np.arange(1, len(w) + 1) * every * alpha
            rates[(alpha, corr)] = P.pic_fit_growth_rate(t, w)[0]
    for alpha in (0.8, 0.95):
        assert rates[(alpha, False)] > 0.01, rates
        assert rates[(alpha, True)] < 0.25 * rates[(alpha, False)], rates
        assert rates[(alpha, True)] < 0.006, rates
