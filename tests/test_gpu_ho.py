"""GPU parity of the particle step with cubic shapes (the Sec. 3 setting) and with the
momentum-conserving gather (the scheme of Eq. 5), against the FP64 oracle on the same seeded
inputs: FP64 <= 1e-10 and FP32 <= 1e-5 relative per step, and Gauss's law on a beam run."""
import math

import numpy as np
import pytest

import oracle as O
from tests._pic import P, Pair, make_cfg, uniform_weight
from tests.test_gpu_parity import FIELDS, TOL, _compare, _random_pair

pytestmark = pytest.mark.gpu

SCHEMES = [(0, 3), (1, 3), (2, 3), (2, 1)]  # (scheme, shape order)


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("scheme,order", SCHEMES)
@pytest.mark.parametrize("nx,nz", [(40, 72), (7, 33)])
def test_ho_step_2d(precision, scheme, order, nx, nz):
    pair = _random_pair(2, precision, scheme=scheme, order=order, nx=nx, nz=nz, npart=min(16000, nx * nz * 8))
    try:
        pair.step(1)
        _compare(pair, TOL[precision])
    finally:
        pair.close()


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("scheme,order", SCHEMES)
def test_ho_step_3d(precision, scheme, order):
    pair = _random_pair(3, precision, scheme=scheme, order=order, nx=20, ny=12, nz=28, npart=12000, sigma=1.0)
    try:
        pair.step(1)
        _compare(pair, TOL[precision])
    finally:
        pair.close()


@pytest.mark.parametrize("scheme,order", SCHEMES)
def test_ho_multi_step_fp64(scheme, order):
    pair = _random_pair(2, 1, scheme=scheme, order=order, nx=32, nz=48, npart=12000)
    try:
        for _ in range(5):
            pair.step(1)
        _compare(pair, 1e-10)
    finally:
        pair.close()


@pytest.mark.parametrize("scheme,order", SCHEMES)
def test_ho_beam_gauss_law(scheme, order):
    # seeded beam, correction + filter, 4 steps in FP32: div E - F rho (oracle rho with the same shape
    # order from the GPU particles, oracle filter) stays at roundoff
    cfg = make_cfg(nx=64, nz=128, dt=0.5, scheme=scheme, precision=0, ppc=4, init_beam=1, seed=4, track_ids=0,
                   order=order)
    h = P.pic_create(cfg)
    try:
        P.pic_set_correction_stencil(h, *P.pic_compute_correction_coeffs(scheme, 0.5))
        P.pic_step(h, 4)
        pair = object.__new__(Pair)
        pair.cfg, pair.h, pair.T = cfg, h, np.float32
        pair.u0 = math.sqrt(cfg.gamma ** 2 - 1)
        pair.o = O.Sim(ndim=2, nx=64, nz=128, dt=0.5, scheme=scheme, order=order)
        f, p = pair.gpu_state()
        assert len(p["x"]) == 64 * 128 * 8
        o = pair.o
        o.set_particles(p["x"], None, p["z"], p["ux"], p["uy"], p["uz"], p["w"], p["q"])
        o.f.update({n: f[n].reshape(o.shape).copy() for n in FIELDS})
        g = o.div_e() - o.filter(o.rho())
        assert np.abs(g).max() < 2e-3 * uniform_weight(cfg)
    finally:
        P.pic_destroy(h)


def test_ho_rejected_where_not_covered():
    cfg = make_cfg(nx=16, nz=16, precision=1, init_beam=1, order=3)
    with pytest.raises(P.PicError) as e:
        P.pic_batch_create([cfg])
    assert e.value.code == P.PIC_E_ARG
    h = P.pic_create(cfg)
    with pytest.raises(P.PicError) as e:
        P.pic_adjoint_forward(h, 2, 1)
    assert e.value.code == P.PIC_E_ARG
    P.pic_destroy(h)
