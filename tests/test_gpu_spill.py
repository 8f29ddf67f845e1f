"""GPU tests of the particle storage under crowding: a particle whose cell bin is full is never
dropped. It waits in the handle's spill list, the next step pushes it there with the same gather,
Boris push, move and Esirkepov deposit as the particles in bins, and the next synchronising call
re-bins every particle into larger bins.

Parity with the FP64 oracle, element by element (FP64 1e-10, FP32 1e-5), on particles crowded into a
few cells far past the initial bins (every push path: linear Galerkin / Uniform, momentum-conserving,
cubic, 2D and 3D), and conservation of every particle through the uncorrected beam run of the paper's
Sec. 3 setting, whose numerical Cherenkov instability bunches the beam past the default capacity."""
import numpy as np
import pytest

import synth
from tests._pic import P, Pair, make_cfg
from tests.test_gpu_parity import TOL, _compare

pytestmark = pytest.mark.gpu


def _crowded_pair(ndim, precision, order, scheme, n=600, seed=3):
    nx, ny, nz = (24, 1, 40) if ndim == 2 else (12, 10, 16)
    cfg = make_cfg(ndim=ndim, nx=nx, ny=ny, nz=nz, dt=0.5, scheme=scheme, precision=precision, order=order)
    shape = (nz, ny, nx)
    fields = synth.random_fields(shape, seed=seed + 100, scale=2e-2, smooth=1)
    # the block of 2^ndim cells at (10, 4, 18) holds n particles: about 75 (2D) or 38 (3D) per cell and
    # species, against initial bins of 8 (FP64) or 16 (FP32) slots
    part = synth.clustered_particles(ndim, nx, ny, nz, n, seed=seed + 200, corner=(10, 4, 18), size=2)
    coeffs = P.pic_compute_correction_coeffs(0, 0.5)
    return Pair(cfg, psi=coeffs, fields=fields, part=part)


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("ndim,order,scheme", [(2, 1, 0), (2, 1, 1), (2, 1, 2), (2, 3, 0), (2, 3, 2), (3, 1, 0),
                                               (3, 1, 1), (3, 3, 2)])
def test_crowded_cells_match_oracle(precision, ndim, order, scheme):
    pair = _crowded_pair(ndim, precision, order, scheme)
    try:
        cap0, spilled0 = P.pic_bin_stats(pair.h)
        assert spilled0 > pair.npart // 2  # most of the imported particles went to the spill list
        # three steps in one call: the bins stay full, the excess is pushed from the spill list each step
        pair.step(3)
        _compare(pair, TOL[precision])
        assert P.pic_num_particles(pair.h) == pair.npart
        assert P.pic_bin_stats(pair.h)[0] > cap0  # the synchronising calls above grew the bins
        # two more steps from the grown bins (the particles keep drifting together in z)
        pair.step(2)
        _compare(pair, TOL[precision])
    finally:
        pair.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_one_overfull_cell_keeps_every_particle(precision):
    # 80 particles (about 40 per species) imported into one cell whose bins hold 8 or 16: nothing is
    # refused or dropped, the count is exact before and after steps, and the bins grow once
    cfg = make_cfg(nx=16, nz=16, precision=precision, cap=8)
    h = P.pic_create(cfg)
    try:
        T = np.float32 if precision == 0 else np.float64
        rng = np.random.default_rng(0)
        n = 80
        part = {"cell": np.full(n, 37, np.int32), "species": (np.arange(n) % 2).astype(np.int32),
                "ox": (0.1 + 0.8 * rng.random(n)).astype(T), "oy": None,
                "oz": (0.1 + 0.8 * rng.random(n)).astype(T), "dux": (1e-3 * rng.standard_normal(n)).astype(T),
                "duy": (1e-3 * rng.standard_normal(n)).astype(T), "duz": np.zeros(n, T), "w": None,
                "id": np.arange(n, dtype=np.uint32)}
        cap0 = P.pic_bin_stats(h)[0]
        P.pic_set_state(h, P.make_state(P.PIC_HOST, None, part))
        P.pic_sync(h)
        assert P.pic_num_particles(h) == n
        cap1, spilled = P.pic_bin_stats(h)
        assert cap1 >= 40 > cap0 and spilled == n - 2 * cap0
        P.pic_step(h, 2)
        P.pic_sync(h)
        assert P.pic_num_particles(h) == n
    finally:
        P.pic_destroy(h)


def test_default_capacity_beam_run_keeps_every_particle():
    # The uncorrected linear Galerkin beam (128 x 128, 4 particles per cell and species, gamma = 130,
    # c dt/dz = 0.5, FP32) with the default bins of 2 ppc + 8 = 16 slots: the numerical Cherenkov
    # instability bunches the beam until cells hold more than 16 particles of a species. The excess
    # waits in the spill list, so every recorded step pushes every particle (the count in each history
    # sample is the step's own count of pushed particles), and the run ends with all of them.
    cfg = make_cfg(nx=128, nz=128, dt=0.5, scheme=0, precision=0, ppc=4, init_beam=1, seed=7, track_ids=0)
    cfg.diag_every = 10
    total = 128 * 128 * 4 * 2
    h = P.pic_create(cfg)
    try:
        P.pic_step(h, 2000)
        hist = P.pic_energy_history(h, 4096)
        assert len(hist) == 200
        assert all(e["np"] == total for e in hist)
        assert P.pic_num_particles(h) == total
        assert P.pic_bin_stats(h)[1] > 0  # the beam did bunch past the initial bins
        w = [e["w_perp"] for e in hist]
        assert w[-1] > 1e3 * w[20]  # and the instability grew
    finally:
        P.pic_destroy(h)
