"""Failure detection on the GPU without a fault. A device allocation that fails is returned as
PIC_E_OOM. The kernels turn an invalid imported particle and a non-finite particle into error flags,
with every access in bounds: the import checks cell, species and offsets, and the push stops a
particle whose displacement is not finite. The host reads the flags as status codes at the next
synchronising call and clears them; the handle stays usable. (A full particle bin is not an error:
tests/test_gpu_spill.py.)"""
import numpy as np
import pytest

from tests._pic import P, make_cfg

pytestmark = pytest.mark.gpu

FIELDS = ("ex", "ey", "ez", "bx", "by", "bz")


def _particles(cfg, n, cell, seed=0):
    T = np.float32 if cfg.precision == 0 else np.float64
    rng = np.random.default_rng(seed)
    return {"cell": np.full(n, cell, np.int32), "species": (np.arange(n) % 2).astype(np.int32),
            "ox": (0.1 + 0.8 * rng.random(n)).astype(T), "oy": None, "oz": (0.1 + 0.8 * rng.random(n)).astype(T),
            "dux": (1e-3 * rng.standard_normal(n)).astype(T), "duy": (1e-3 * rng.standard_normal(n)).astype(T),
            "duz": np.zeros(n, T), "w": None, "id": np.arange(n, dtype=np.uint32)}


def _import(h, part):
    P.pic_set_state(h, P.make_state(P.PIC_HOST, None, part))


def _fields(h, cfg):
    out = {c: np.zeros(cfg.nx * cfg.ny * cfg.nz, np.float32 if cfg.precision == 0 else np.float64) for c in FIELDS}
    P.pic_get_state(h, P.make_state(P.PIC_HOST, out, None))
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_invalid_imported_particles_are_reported_and_skipped(precision):
    # a cell index past the grid, a negative cell, a species other than 0 / 1 and an offset of 1e30
    # cells: each is refused (PIC_E_ARG at the next synchronising call), the other 6 particles land
    cfg = make_cfg(nx=16, nz=16, precision=precision)
    h = P.pic_create(cfg)
    try:
        part = _particles(cfg, 10, cell=21)
        part["cell"][1] = 16 * 16
        part["cell"][4] = -1
        part["species"][6] = 2
        part["oz"][8] = 1e30
        _import(h, part)
        with pytest.raises(P.PicError) as e:
            P.pic_sync(h)
        assert e.value.code == P.PIC_E_ARG
        assert P.pic_num_particles(h) == 6
        P.pic_step(h, 1)
        P.pic_sync(h)
    finally:
        P.pic_destroy(h)


@pytest.mark.parametrize("precision,order,scheme", [(0, 1, 0), (1, 1, 0), (0, 1, 2), (0, 3, 0)])
def test_non_finite_momentum_is_reported_and_stopped(precision, order, scheme):
    # one particle with a NaN momentum among 8: the import accepts it (it checks positions only); the
    # push flags it (PIC_E_NONFINITE) and stops it, so no NaN reaches the current or the fields and
    # the next step is clean (the linear push, the momentum-conserving gather, cubic shapes)
    cfg = make_cfg(nx=16, nz=16, precision=precision, order=order, scheme=scheme, cap=48 if order == 3 else 0)
    h = P.pic_create(cfg)
    try:
        part = _particles(cfg, 8, cell=40)
        part["dux"][3] = np.nan
        _import(h, part)
        P.pic_sync(h)
        P.pic_step(h, 1)
        with pytest.raises(P.PicError) as e:
            P.pic_sync(h)
        assert e.value.code == P.PIC_E_NONFINITE
        P.pic_step(h, 1)
        P.pic_sync(h)
        assert P.pic_num_particles(h) == 8
        f = _fields(h, cfg)
        assert all(np.isfinite(f[c]).all() for c in FIELDS)
        assert max(np.abs(f[c]).max() for c in FIELDS) > 0  # the other particles did deposit
    finally:
        P.pic_destroy(h)


def test_allocation_failure_is_reported_and_other_handles_keep_working():
    # a run whose particle bins would need about 1 TB per array: pic_create frees what it allocated
    # and returns PIC_E_OOM; a live handle on the same thread still counts (a launch outside the
    # per-kernel wrapper, which would see a stale allocation error) and steps
    ok = make_cfg(nx=16, nz=16, precision=0)
    h = P.pic_create(ok)
    try:
        _import(h, _particles(ok, 8, cell=40))
        with pytest.raises(P.PicError) as e:
            P.pic_create(make_cfg(nx=128, nz=128, precision=0, cap=1 << 24))
        assert e.value.code == P.PIC_E_OOM
        assert "allocation" in P.pic_last_error(None)
        assert P.pic_num_particles(h) == 8
        P.pic_step(h, 1)
        P.pic_sync(h)
    finally:
        P.pic_destroy(h)
