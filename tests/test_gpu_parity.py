"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on the same seeded inputs.

Bars: FP64 GPU vs FP64 oracle <= 1e-10 relative per step (atomic ordering is the only difference);
FP32 GPU vs FP64 oracle <= 1e-5 relative per step. Particles are matched by id; positions are
compared as absolute periodic differences in cells, the rest as relative L2 norms per array.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth
from tests._pic import P, Pair, make_cfg, periodic_diff, rel_l2, uniform_weight

pytestmark = pytest.mark.gpu

TOL = {1: 1e-10, 0: 1e-5}
FIELDS = ("ex", "ey", "ez", "bx", "by", "bz")


def _coeffs(scheme, alpha):
    return P.pic_compute_correction_coeffs(scheme, alpha)


def _compare(pair, tol, fields=True, particles=True, field_floor=0.0):
    f, p = pair.gpu_state()
    out = {}
    if fields:
        for n in FIELDS:
            e = rel_l2(f[n], pair.o.f[n], floor=field_floor)
            out[n] = e
            assert e <= tol, (n, e)
    if particles and pair.npart:
        o = pair.o
        order = np.argsort(o.pid, kind="stable")
        assert len(p["id"]) == len(order), (len(p["id"]), len(order))
        np.testing.assert_array_equal(p["id"], o.pid[order])
        nz, ny, nx = o.shape
        dx = periodic_diff(p["x"], o.part["x"][order], nx)
        dz = periodic_diff(p["z"], o.part["z"][order], nz)
        pos_err = max(np.abs(dx).max(), np.abs(dz).max())
        if pair.cfg.ndim == 3:
            pos_err = max(pos_err, np.abs(periodic_diff(p["y"], o.part["y"][order], ny)).max())
        out["pos"] = pos_err
        assert pos_err <= tol, ("pos", pos_err)
        for c in ("ux", "uy", "uz"):
            e = rel_l2(p[c], o.part[c][order])
            out[c] = e
            assert e <= tol, (c, e)
        np.testing.assert_array_equal(p["q"], o.part["q"][order])
    return out


def _random_pair(ndim, precision, scheme=0, nx=40, ny=12, nz=72, npart=20000, seed=0, psi=True, alpha=0.5,
                 targets=3, nbin=1, ncomp=1, calpha=3.0, sigma=0.0, field_scale=2e-2, order=1, corr_mode=0,
                 coeffs=None):
    dt = alpha if ndim == 2 else min(alpha, 0.55)
    cfg = make_cfg(ndim=ndim, nx=nx, ny=ny, nz=nz, dt=dt, scheme=scheme, precision=precision, targets=targets,
                   nbin=nbin, ncomp=ncomp, calpha=calpha, sigma_perp=sigma, order=order, corr_mode=corr_mode)
    shape = (nz, ny if ndim == 3 else 1, nx)
    fields = synth.random_fields(shape, seed=seed + 100, scale=field_scale, smooth=1)
    part = synth.random_particles(ndim, nx, ny if ndim == 3 else 1, nz, npart, seed=seed + 200,
                                  per_particle_weight=sigma > 0)
    if coeffs is None and psi:
        coeffs = _coeffs(scheme, alpha)
    return Pair(cfg, psi=coeffs, fields=fields, part=part)


# ---------------------------------------------------------------------------------------------
# stage-level parity
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("nbin,ncomp,calpha,targets", [(1, 1, 3.0, 3), (2, 1, 2.0, 3), (2, 2, 3.0, 2), (0, 0, 3.0, 0)])
def test_gather_copies(precision, ndim, nbin, ncomp, calpha, targets):
    # Psi_E / Psi_B z-stencils and the gather filter (Sec. 2, Eq. 6): one step with no particles,
    # then the copies the particles would have seen.
    pair = _random_pair(ndim, precision, npart=0, nx=40, ny=10, nz=36, nbin=nbin, ncomp=ncomp, calpha=calpha,
                        targets=targets)
    try:
        expect = pair.o.gather_copies()
        P.pic_step(pair.h, 1)
        T = pair.T
        outs = [np.zeros(pair.o.shape, dtype=T) for _ in range(6)]
        P.pic_debug_gather_copies(pair.h, P.PIC_HOST, outs)
        for c in range(6):
            assert rel_l2(outs[c], expect[c]) <= TOL[precision], c
    finally:
        pair.close()


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("ndim", [2, 3])
def test_step_on_grids_staged_by_tma(precision, ndim):
    # Grids that span the tiles the stencil and Yee kernels stage by one bulk tensor copy (TMA) in
    # every direction, with ragged edge tiles (200 = 128 + 72 columns, 100 = 3 x 32 + 4 rows): a box's
    # elements outside the grid read as zero and are replaced by their periodic images. The copies the
    # particles see after the first step, then every field and particle after three steps.
    nx, ny, nz = (200, 1, 100) if ndim == 2 else (48, 16, 24)
    pair = _random_pair(ndim, precision, nx=nx, ny=ny, nz=nz, npart=8000, sigma=1.0 if ndim == 3 else 0.0)
    try:
        expect = pair.o.gather_copies()
        pair.step(1)
        outs = [np.zeros(pair.o.shape, dtype=pair.T) for _ in range(6)]
        P.pic_debug_gather_copies(pair.h, P.PIC_HOST, outs)
        for c in range(6):
            assert rel_l2(outs[c], expect[c]) <= TOL[precision], c
        _compare(pair, TOL[precision])
        pair.step(2)
        _compare(pair, TOL[precision])
    finally:
        pair.close()


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("ndim", [2, 3])
def test_yee_vacuum(precision, ndim):
    # field-only steps (no particles, J = 0)
    pair = _random_pair(ndim, precision, npart=0, nx=24, ny=8, nz=40)
    try:
        pair.step(10)
        _compare(pair, TOL[precision] * (10 if precision == 0 else 1), particles=False)
    finally:
        pair.close()


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("scheme", [0, 1])
def test_current_deposit(precision, ndim, scheme):
    # Esirkepov current of one step from zero fields (pure drift), filtered
    pair = _random_pair(ndim, precision, scheme=scheme, npart=6000, nx=20, ny=10, nz=36, field_scale=0.0)
    try:
        pair.step(1)
        T = pair.T
        outs = [np.zeros(pair.o.shape, dtype=T) for _ in range(3)]
        P.pic_debug_current(pair.h, P.PIC_HOST, outs)
        for c, n in enumerate(("jx", "jy", "jz")):
            assert rel_l2(outs[c], pair.o.f[n]) <= TOL[precision], n
    finally:
        pair.close()


# ---------------------------------------------------------------------------------------------
# whole-step parity
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("nx,nz", [(40, 72), (16, 16), (7, 33)])
def test_step_2d(precision, scheme, nx, nz):
    pair = _random_pair(2, precision, scheme=scheme, nx=nx, nz=nz, npart=min(20000, nx * nz * 8))
    try:
        pair.step(1)
        _compare(pair, TOL[precision])
    finally:
        pair.close()


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("scheme", [0, 1])
def test_step_3d(precision, scheme):
    pair = _random_pair(3, precision, scheme=scheme, nx=20, ny=12, nz=28, npart=15000, sigma=1.0)
    try:
        pair.step(1)
        _compare(pair, TOL[precision])
    finally:
        pair.close()


def test_multi_step_fp64():
    # several steps in FP64 stay within the per-step bar (errors grow only by roundoff)
    pair = _random_pair(2, 1, nx=32, nz=48, npart=12000)
    try:
        for _ in range(5):
            pair.step(1)
        _compare(pair, 1e-10)
    finally:
        pair.close()


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("ndim", [2, 3])
def test_edge_particles(precision, ndim):
    # particles on faces, nodes, next to the wrap on either side, moving backwards
    nx, ny, nz = 12, 6, 16
    cfg = make_cfg(ndim=ndim, nx=nx, ny=ny, nz=nz, dt=0.5, precision=precision)
    part = synth.edge_particles(ndim, nx, ny if ndim == 3 else 1, nz)
    fields = synth.random_fields((nz, ny if ndim == 3 else 1, nx), seed=3, scale=0.05)
    pair = Pair(cfg, psi=_coeffs(0, 0.5), fields=fields, part=part)
    try:
        for _ in range(3):
            pair.step(1)
            _compare(pair, TOL[precision])
    finally:
        pair.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_tile_with_more_leavers_than_its_buffer(precision):
    # 1200 particles in the top cell row of one particle tile, all moving up: every one leaves the
    # tile in the first step, more than the 512 the tile buffers in shared memory, so the rest take
    # the direct path into the global leaver list. On this 32x48 grid the 4x64 tiles are spread to
    # 4x4 cells (96 tiles), so x in [0, 4), z in [15.6, 16) is the top row of the tile [0, 4) x [12, 16).
    nx, nz, n = 32, 48, 1200
    cfg = make_cfg(nx=nx, nz=nz, dt=0.5, precision=precision, cap=192)
    rng = np.random.default_rng(31)
    u0 = math.sqrt(cfg.gamma ** 2 - 1)
    part = {"x": rng.uniform(0, 3.999, n), "y": np.zeros(n), "z": rng.uniform(15.6, 15.999, n),
            "ux": rng.normal(0, 1e-3, n), "uy": rng.normal(0, 1e-3, n), "uz": u0 + rng.normal(0, 1e-3, n),
            "w": np.ones(n), "q": rng.choice([-1.0, 1.0], n), "id": np.arange(n, dtype=np.int64)}
    fields = synth.random_fields((nz, 1, nx), seed=33, scale=1e-3)
    pair = Pair(cfg, psi=_coeffs(0, 0.5), fields=fields, part=part)
    try:
        pair.step(1)
        _compare(pair, TOL[precision])
        assert P.pic_num_particles(pair.h) == n
        pair.step(2)
        _compare(pair, TOL[precision])
    finally:
        pair.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_empty_and_single(precision):
    cfg = make_cfg(nx=16, nz=16, precision=precision)
    pair = Pair(cfg, fields=synth.random_fields((16, 1, 16), seed=1))
    try:
        pair.step(2)
        _compare(pair, TOL[precision], particles=False)
        assert P.pic_num_particles(pair.h) == 0
    finally:
        pair.close()
    part = synth.random_particles(2, 16, 1, 16, 1, seed=9)
    pair = Pair(cfg, part=part, fields=synth.random_fields((16, 1, 16), seed=2))
    try:
        pair.step(3)
        _compare(pair, TOL[precision])
    finally:
        pair.close()


# ---------------------------------------------------------------------------------------------
# beam initialisation and energies
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("ndim", [2, 3])
def test_beam_init_matches_oracle(precision, ndim):
    nx, ny, nz, ppc = (20, 1, 36, 4) if ndim == 2 else (10, 8, 12, 8)
    cfg = make_cfg(ndim=ndim, nx=nx, ny=ny, nz=nz, dt=0.5, precision=precision, ppc=ppc, init_beam=1, seed=11,
                   sigma_perp=3.0 if ndim == 3 else 0.0)
    h = P.pic_create(cfg)
    try:
        from tests._pic import Pair as _P
        pair = object.__new__(_P)
        pair.cfg, pair.h, pair.T = cfg, h, (np.float32 if precision == 0 else np.float64)
        pair.u0 = math.sqrt(cfg.gamma ** 2 - 1)
        pair.o = O.Sim(ndim=ndim, nx=nx, ny=ny, nz=nz, dt=0.5)
        _, p = _P.gpu_state(pair)
        o = pair.o
        o.init_beam(ppc=ppc, seed=11, sigma_perp=3.0 if ndim == 3 else 0.0)
        n = nx * ny * nz * ppc * 2
        assert len(p["id"]) == n
        np.testing.assert_array_equal(p["id"], np.arange(n))
        tol = 1e-14 if precision == 1 else 1e-6
        assert np.abs(periodic_diff(p["x"], o.part["x"], nx)).max() < tol * 10
        assert np.abs(periodic_diff(p["z"], o.part["z"], nz)).max() < tol * 10
        for c in ("ux", "uy", "uz"):
            assert rel_l2(p[c], o.part[c]) < tol
        if ndim == 3:
            assert rel_l2(p["w"], o.part["w"]) < tol
        else:
            np.testing.assert_allclose(p["w"], uniform_weight(cfg), rtol=tol)
    finally:
        P.pic_destroy(h)


@pytest.mark.parametrize("precision", [1, 0])
def test_energies(precision):
    pair = _random_pair(2, precision, nx=24, nz=40, npart=5000)
    try:
        pair.step(2)
        e = P.pic_energy(pair.h)
        ref = pair.o.energy()
        tol = 1e-12 if precision == 1 else 1e-5
        assert abs(e["w_e"] - ref[0]) <= tol * ref[0]
        assert abs(e["w_b"] - ref[1]) <= tol * ref[1]
        assert abs(e["w_perp"] - ref[2]) <= tol * ref[2]
        assert abs(e["k"] - ref[3]) <= tol * ref[3]
        assert e["np"] == 5000
    finally:
        pair.close()


def test_beam_run_fp64_config1_size():
    # the 2D 64x128, 4 ppc, gamma = 130, alpha = 0.5, Galerkin + Psi beam: 20 FP64 steps vs the oracle
    cfg = make_cfg(nx=64, nz=128, dt=0.5, precision=1, ppc=4, init_beam=1, seed=1)
    psi = _coeffs(0, 0.5)
    h = P.pic_create(cfg)
    P.pic_set_correction_stencil(h, *psi)
    o = O.Sim(ndim=2, nx=64, nz=128, dt=0.5, psi_e=psi[0], psi_b=psi[1])
    o.init_beam(ppc=4, seed=1)
    try:
        # start the oracle from the GPU's own initial state (identical up to FP64 roundoff)
        pair = object.__new__(Pair)
        pair.cfg, pair.h, pair.T, pair.o = cfg, h, np.float64, o
        pair.u0 = math.sqrt(cfg.gamma ** 2 - 1)
        pair.npart = 65536
        _, p0 = pair.gpu_state()
        o.set_particles(p0["x"], None, p0["z"], p0["ux"], p0["uy"], p0["uz"], p0["w"], p0["q"], pid=p0["id"])
        for _ in range(4):
            P.pic_step(h, 5)
            o.step(5)
        # The pair plasma is neutral and co-moving: each species carries a current density
        # n_s c = omega_p^2 / 2 while the net current is ~1e-6 of that, so the summation order of the
        # deposit (atomics) moves the net fields by FP64 roundoff of the per-species current. Errors
        # are therefore normalised by the field change one step of one species' current makes.
        f, p = pair.gpu_state()
        gross = math.sqrt(64 * 128) * 0.5 * 0.3868 ** 2 / 2
        for n in FIELDS:
            assert rel_l2(f[n], o.f[n], floor=gross) < 1e-10, (n, rel_l2(f[n], o.f[n], floor=gross))
        order = np.argsort(o.pid)
        assert np.abs(periodic_diff(p["z"], o.part["z"][order], 128)).max() < 1e-10
        for c in ("ux", "uy", "uz"):
            assert rel_l2(p[c], o.part[c][order]) < 1e-10
        e, ref = P.pic_energy(h), o.energy()
        assert abs(e["w_perp"] - ref[2]) < 1e-8 * ref[2]
    finally:
        P.pic_destroy(h)


def test_step_full_size_fp32():
    # the benchmark workload at full size (2D 512x1024, 16 ppc/species, 16.8M particles, FP32, Psi at
    # alpha = 0.5, the 2-bilinear + 1-compensation (a = 2) filter, the launch configuration bench.py
    # times): after 3 steps from the seeded beam, one more step of the same state in the library and in
    # the FP64 oracle, every field and every particle compared. The pair plasma's net fields are a
    # cancellation of the two species' currents, so field errors are normalised by the field change one
    # step of one species' current makes (as in the FP64 beam test); particles at the FP32 bar.
    nx, nz = 512, 1024
    cfg = make_cfg(nx=nx, nz=nz, dt=0.5, precision=0, ppc=16, init_beam=1, seed=2, nbin=2, ncomp=1, calpha=2.0,
                   track_ids=1)
    psi = _coeffs(0, 0.5)
    h = P.pic_create(cfg)
    try:
        P.pic_set_correction_stencil(h, *psi)
        P.pic_step(h, 3)
        pair = object.__new__(Pair)
        pair.cfg, pair.h, pair.T = cfg, h, np.float32
        pair.u0 = math.sqrt(cfg.gamma ** 2 - 1)
        pair.o = O.Sim(ndim=2, nx=nx, nz=nz, dt=0.5, psi_e=psi[0], psi_b=psi[1], f_nbin=2, f_ncomp=1, f_alpha=2.0)
        pair.npart = nx * nz * 32
        f0, p0 = pair.gpu_state()
        assert len(p0["x"]) == pair.npart
        o = pair.o
        o.set_particles(p0["x"], None, p0["z"], p0["ux"], p0["uy"], p0["uz"], p0["w"], p0["q"], pid=p0["id"])
        o.f.update({n: f0[n].reshape(o.shape).copy() for n in FIELDS})
        P.pic_step(h, 1)
        o.step(1)
        f, p = pair.gpu_state()
        gross = math.sqrt(nx * nz) * 0.5 * 0.3868 ** 2 / 2
        for n in FIELDS:
            assert rel_l2(f[n], o.f[n], floor=gross) < 1e-6, (n, rel_l2(f[n], o.f[n], floor=gross))
        order = np.argsort(o.pid, kind="stable")
        np.testing.assert_array_equal(p["id"], o.pid[order])
        assert np.abs(periodic_diff(p["x"], o.part["x"][order], nx)).max() < 1e-5
        assert np.abs(periodic_diff(p["z"], o.part["z"][order], nz)).max() < 1e-5
        for c in ("ux", "uy"):
            assert rel_l2(p[c], o.part[c][order]) < 1e-5, c
        # uz carries u0 = 130: compare the deviation from the drift, which FP32 stores
        assert rel_l2(p["uz"] - pair.u0, o.part["uz"][order] - pair.u0) < 1e-5
    finally:
        P.pic_destroy(h)


def test_gauss_law_full_size_fp32():
    # full benchmark size (2D 512x1024, 16 ppc/species, 16.8M particles, FP32): after steps from the
    # seeded beam, div E - F rho (oracle rho of the GPU particles, oracle filter) stays at roundoff
    cfg = make_cfg(nx=512, nz=1024, dt=0.5, precision=0, ppc=16, init_beam=1, seed=2, nbin=2, ncomp=1, calpha=2.0,
                   track_ids=0)
    psi = _coeffs(0, 0.5)
    h = P.pic_create(cfg)
    try:
        P.pic_set_correction_stencil(h, *psi)
        P.pic_step(h, 3)
        pair = object.__new__(Pair)
        pair.cfg, pair.h, pair.T = cfg, h, np.float32
        pair.u0 = math.sqrt(cfg.gamma ** 2 - 1)
        pair.o = O.Sim(ndim=2, nx=512, nz=1024, dt=0.5, f_nbin=2, f_ncomp=1, f_alpha=2.0)
        f, p = pair.gpu_state()
        assert len(p["x"]) == 512 * 1024 * 32
        o = pair.o
        o.set_particles(p["x"], None, p["z"], p["ux"], p["uy"], p["uz"], p["w"], p["q"])
        o.f.update({n: f[n].reshape(o.shape).copy() for n in FIELDS})
        g = o.div_e() - o.filter(o.rho())
        scale = uniform_weight(cfg)  # one macro-particle's charge density
        assert np.abs(g).max() < 2e-3 * scale
    finally:
        P.pic_destroy(h)


def test_push_sampled_full_size_3d_fp32():
    # the 3D workload at full size (128x128x512, 8 ppc/species, 134M particles, Gaussian transverse
    # weights, FP32, correction + filter): after 2 steps, one more step; 4096 particles drawn at random
    # are pushed one by one by the oracle (its copies of the exported fields, its gather, its Boris,
    # the move x + dt u / gamma) and compared by id with the library's step
    nx, ny, nz = 128, 128, 512
    cfg = make_cfg(ndim=3, nx=nx, ny=ny, nz=nz, dt=0.5, precision=0, ppc=8, init_beam=1, seed=3,
                   sigma_perp=20.0, track_ids=1)
    psi = _coeffs(0, 0.5)
    h = P.pic_create(cfg)
    try:
        P.pic_set_correction_stencil(h, *psi)
        P.pic_step(h, 2)
        pair = object.__new__(Pair)
        pair.cfg, pair.h, pair.T = cfg, h, np.float32
        pair.u0 = math.sqrt(cfg.gamma ** 2 - 1)
        pair.o = O.Sim(ndim=3, nx=nx, ny=ny, nz=nz, dt=0.5)
        f0, p0 = pair.gpu_state()  # sorted by id; ids are 0 .. N-1
        n = len(p0["x"])
        assert n == nx * ny * nz * 16 and p0["id"][-1] == n - 1
        sample = np.sort(np.random.default_rng(7).choice(n, 4096, replace=False))
        ps = {k: v[sample].copy() for k, v in p0.items()}
        del p0
        o = O.Sim(ndim=3, nx=nx, ny=ny, nz=nz, dt=0.5, psi_e=psi[0], psi_b=psi[1])
        o.f.update({k: f0[k].reshape(o.shape).copy() for k in FIELDS})
        F = o.gather(o.gather_copies(), ps["x"], ps["y"], ps["z"])
        want = {k: np.zeros(len(sample)) for k in ("x", "y", "z", "ux", "uy", "uz")}
        for i in range(len(sample)):
            u = O.boris(ps["q"][i], 0.5, [F[0][i], F[1][i], F[2][i]], [F[3][i], F[4][i], F[5][i]],
                        [ps["ux"][i], ps["uy"][i], ps["uz"][i]])
            g = math.sqrt(1.0 + u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
            for c, k in enumerate(("x", "y", "z")):
                want[k][i] = ps[k][i] + 0.5 * u[c] / g
            want["ux"][i], want["uy"][i], want["uz"][i] = u
        P.pic_step(h, 1)
        _, p1 = pair.gpu_state()
        got = {k: v[sample] for k, v in p1.items()}
        del p1
    finally:
        P.pic_destroy(h)
    np.testing.assert_array_equal(got["id"], sample)
    for k, m in (("x", nx), ("y", ny), ("z", nz)):
        assert np.abs(periodic_diff(got[k], want[k], m)).max() < 1e-5, k
    for k in ("ux", "uy"):
        assert rel_l2(got[k], want[k]) < 1e-5, (k, rel_l2(got[k], want[k]))
    assert rel_l2(got["uz"] - pair.u0, want["uz"] - pair.u0) < 1e-5


def test_gauss_law_full_size_3d_fp32():
    # the 3D workload at full size (128x128x512, 8 ppc/species, 134M particles, Gaussian transverse
    # weights, FP32, correction + filter): after steps from the seeded beam, div E - F rho (oracle rho
    # of the GPU particles, oracle filter) stays at roundoff, and no particle is lost
    cfg = make_cfg(ndim=3, nx=128, ny=128, nz=512, dt=0.5, precision=0, ppc=8, init_beam=1, seed=3,
                   sigma_perp=20.0, track_ids=0)
    psi = _coeffs(0, 0.5)
    h = P.pic_create(cfg)
    try:
        P.pic_set_correction_stencil(h, *psi)
        n0 = P.pic_num_particles(h)
        assert n0 == 128 * 128 * 512 * 16
        P.pic_step(h, 2)
        pair = object.__new__(Pair)
        pair.cfg, pair.h, pair.T = cfg, h, np.float32
        pair.u0 = math.sqrt(cfg.gamma ** 2 - 1)
        pair.o = O.Sim(ndim=3, nx=128, ny=128, nz=512, dt=0.5)
        f, p = pair.gpu_state()
        assert len(p["x"]) == n0
        o = pair.o
        o.set_particles(p["x"], p["y"], p["z"], p["ux"], p["uy"], p["uz"], p["w"], p["q"])
        del p
        o.f.update({n: f[n].reshape(o.shape).copy() for n in FIELDS})
        g = o.div_e() - o.filter(o.rho())
        scale = uniform_weight(cfg)  # one macro-particle's (peak) charge density
        assert np.abs(g).max() < 2e-3 * scale
    finally:
        P.pic_destroy(h)
