"""GPU tests of batched runs: a batch of uneven independent runs (different grids, particles per
cell, c dt/dz, gamma, correction on and off) must evolve like the FP64 oracle run from the same
imported state (FP64 1e-10, FP32 1e-5 per step; one run crowded past its bins, so the batched spill
path runs too) and exactly like the same runs stepped one by one through pic_step (FP64: 1e-10; the
only difference is the order of the deposit's atomics), also after the autotuner (which puts the runs
back into their seeded initial state)."""
import math

import numpy as np
import pytest

import oracle as O
import synth
from oracle.fit import growth_rate
from tests._pic import P, Pair, make_cfg, periodic_diff, rel_l2
from tests.test_gpu_parity import TOL
from tests.test_gpu_parity import _compare as _compare_oracle

ORACLE_RUNS = [  # nx, nz, alpha, gamma, correction, particles, crowded into four cells
    (40, 72, 0.5, 130.0, True, 5000, False),
    (32, 48, 0.3, 10.0, False, 3000, False),
    (24, 40, 0.7, 50.0, True, 700, True),
    (48, 32, 0.2, 130.0, True, 2000, False),
]


@pytest.mark.parametrize("precision", [1, 0])
def test_batch_matches_oracle(precision):
    # each run imports its own random state (fields and particles), the batch advances them together
    # (lead steps, then graph replays), and each run is compared with the oracle run from that state
    steps = 6
    cfgs = [make_cfg(nx=nx, nz=nz, dt=a, gamma=g, precision=precision, init_beam=0, track_ids=1)
            for (nx, nz, a, g, _, _, _) in ORACLE_RUNS]
    b = P.pic_batch_create(cfgs)
    pairs = []
    try:
        for i, (nx, nz, a, g, corr, n, crowded) in enumerate(ORACLE_RUNS):
            coeffs = P.pic_compute_correction_coeffs(0, a) if corr else None
            if coeffs is not None:
                P.pic_batch_set_correction_stencil(b, i, *coeffs)
            fields = synth.random_fields((nz, 1, nx), seed=40 + i, scale=2e-2, smooth=1)
            if crowded:
                part = synth.clustered_particles(2, nx, 1, nz, n, seed=50 + i, corner=(9, 0, 11), size=2,
                                                 gamma=g)
            else:
                part = synth.random_particles(2, nx, 1, nz, n, seed=50 + i, gamma=g)
            pairs.append(Pair(cfgs[i], psi=coeffs, fields=fields, part=part, handle=P.pic_batch_run(b, i)))
        P.pic_batch_step(b, steps)
        P.pic_batch_sync(b)
        for pair in pairs:
            pair.o.step(steps)
            _compare_oracle(pair, TOL[precision])
            assert P.pic_num_particles(pair.h) == pair.npart
        # the crowded run's bins grew at the synchronising calls above; the batch re-uploads its tables
        P.pic_batch_step(b, 2)
        for pair in pairs:
            pair.o.step(2)
            _compare_oracle(pair, TOL[precision])
    finally:
        for pair in pairs:
            pair.close()
        P.pic_batch_destroy(b)

pytestmark = pytest.mark.gpu

RUNS = [  # nx, nz, ppc, alpha, gamma, correction
    (48, 80, 4, 0.3, 10.0, True),
    (64, 128, 8, 0.5, 50.0, False),
    (32, 96, 16, 0.7, 130.0, True),
]


def _cfgs(precision, diag_every=2):
    cfgs = []
    for i, (nx, nz, ppc, a, g, _) in enumerate(RUNS):
        c = make_cfg(nx=nx, nz=nz, dt=a, gamma=g, precision=precision, ppc=ppc, init_beam=1, seed=10 + i,
                     track_ids=1, u_th=1e-2)
        c.diag_every = diag_every
        cfgs.append(c)
    return cfgs


def _state(cfg, h):
    pair = object.__new__(Pair)
    pair.cfg, pair.h = cfg, h
    pair.T = np.float32 if cfg.precision == 0 else np.float64
    pair.u0 = math.sqrt(cfg.gamma ** 2 - 1)
    pair.o = O.Sim(ndim=2, nx=cfg.nx, nz=cfg.nz, dt=cfg.dt)
    return pair.gpu_state()


def _compare(cfg, hb, hs, tol):
    fb, pb = _state(cfg, hb)
    fs, ps = _state(cfg, hs)
    gross = math.sqrt(cfg.nx * cfg.nz) * cfg.dt * cfg.omega_p_dz ** 2 / 2
    for n in fb:
        assert rel_l2(fb[n], fs[n], floor=gross) < tol, n
    np.testing.assert_array_equal(pb["id"], ps["id"])
    assert np.abs(periodic_diff(pb["x"], ps["x"], cfg.nx)).max() < tol
    assert np.abs(periodic_diff(pb["z"], ps["z"], cfg.nz)).max() < tol
    for c in ("ux", "uy", "uz"):
        assert rel_l2(pb[c], ps[c]) < tol, c


def _run_both(precision, steps, autotune=False):
    cfgs = _cfgs(precision)
    b = P.pic_batch_create(cfgs)
    singles = []
    try:
        for i, (_, _, _, a, _, corr) in enumerate(RUNS):
            if corr:
                P.pic_batch_set_correction_stencil(b, i, *P.pic_compute_correction_coeffs(0, a))
        if autotune:
            lpcs = P.pic_batch_autotune(b, trial_steps=2)
            assert all(v in (0, 4, 8, 16) for v in lpcs)
        for i, c in enumerate(cfgs):
            h = P.pic_create(c)
            if RUNS[i][5]:
                P.pic_set_correction_stencil(h, *P.pic_compute_correction_coeffs(0, RUNS[i][3]))
            singles.append(h)
        P.pic_batch_step(b, steps)
        P.pic_batch_sync(b)
        for h in singles:
            P.pic_step(h, steps)
        return cfgs, b, singles
    except Exception:
        P.pic_batch_destroy(b)
        for h in singles:
            P.pic_destroy(h)
        raise


@pytest.mark.parametrize("autotune", [False, True])
def test_batch_matches_single_runs_fp64(autotune):
    cfgs, b, singles = _run_both(1, 14, autotune=autotune)
    try:
        assert P.pic_batch_size(b) == len(RUNS)
        for i, c in enumerate(cfgs):
            _compare(c, P.pic_batch_run(b, i), singles[i], 1e-10)
            hb = P.pic_batch_energy_history(b, i)
            hs = P.pic_energy_history(singles[i])
            assert len(hb) == len(hs) == 7
            for eb, es in zip(hb, hs):
                assert eb["np"] == es["np"] == c.nx * c.nz * c.ppc_per_species * 2
                assert abs(eb["w_perp"] - es["w_perp"]) <= 1e-9 * es["w_perp"] + 1e-300
                assert abs(eb["k"] - es["k"]) <= 1e-12 * es["k"]
    finally:
        P.pic_batch_destroy(b)
        for h in singles:
            P.pic_destroy(h)


def test_batch_matches_single_runs_fp32():
    # Two FP32 runs that differ only in the order of the deposit's atomics: their rounding
    # differences grow over the 10 steps of this warm (u_th = 1e-2) beam, so the bar is the per-step
    # FP32 bar (1e-5) accumulated over the steps; observed 0.5-2e-5 of the gross scale
    steps = 10
    cfgs, b, singles = _run_both(0, steps)
    try:
        for i, c in enumerate(cfgs):
            _compare(c, P.pic_batch_run(b, i), singles[i], 1e-5 * steps)
    finally:
        P.pic_batch_destroy(b)
        for h in singles:
            P.pic_destroy(h)


def test_batch_growth_rates_per_run():
    # each run's growth rate, fitted from its own device history, equals the single run's fit
    cfgs = _cfgs(1, diag_every=10)
    b = P.pic_batch_create(cfgs)
    try:
        P.pic_batch_step(b, 200)
        for i, c in enumerate(cfgs):
            h = P.pic_create(c)
            try:
                P.pic_step(h, 200)
                wb = [e["w_perp"] for e in P.pic_batch_energy_history(b, i)]
                ws = [e["w_perp"] for e in P.pic_energy_history(h)]
                t = np.arange(1, 21) * 10 * c.dt
                gb = P.pic_fit_growth_rate(t, wb)
                gs = P.pic_fit_growth_rate(t, ws)
                assert gb[1:] == gs[1:] and abs(gb[0] - gs[0]) <= 1e-6 * abs(gs[0])
            finally:
                P.pic_destroy(h)
    finally:
        P.pic_batch_destroy(b)


def test_batch_rejects_mismatched_settings():
    cfgs = _cfgs(1)
    cfgs[1].filter_nbin = 2
    with pytest.raises(P.PicError) as e:
        P.pic_batch_create(cfgs)
    assert e.value.code == P.PIC_E_ARG
