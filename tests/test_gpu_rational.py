"""GPU parity of the exact rational multiplier mode (Sec. 2: Psi_B applied by inverting it along z;
Sec. 3's variant with Psi_E / Psi_B on the transverse E copies only) against the FP64 oracle, which
inverts Psi_B(D_z) as a circulant by direct DFT: the field copies, whole steps, and errors."""
import numpy as np
import pytest

from tests._pic import P, make_cfg, rel_l2
from tests.test_gpu_parity import TOL, _compare, _random_pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("scheme,alpha", [(0, 0.6), (1, 0.45)])
def test_rational_copies(precision, ndim, scheme, alpha):
    pair = _random_pair(ndim, precision, scheme=scheme, alpha=alpha, npart=0, nx=24, ny=10, nz=36, corr_mode=1)
    try:
        expect = pair.o.gather_copies()
        P.pic_step(pair.h, 1)
        outs = [np.zeros(pair.o.shape, dtype=pair.T) for _ in range(6)]
        P.pic_debug_gather_copies(pair.h, P.PIC_HOST, outs)
        for c in range(6):
            assert rel_l2(outs[c], expect[c]) <= TOL[precision], c
    finally:
        pair.close()


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("nx,nz", [(5, 7), (13, 33), (9, 100), (11, 1024), (3, 1600), (2, 2000)])
def test_rational_copies_line_lengths(precision, nx, nz):
    # the z-line solve at line lengths below one warp, with ragged and empty lane chunks, at the
    # workload's 1024, near the shared-memory limit of the warp-per-line kernel (1600) and past it
    # (2000: the thread-per-line kernel); line counts that leave a partial block
    pair = _random_pair(2, precision, scheme=0, alpha=0.6, npart=0, nx=nx, nz=nz, corr_mode=1)
    try:
        expect = pair.o.gather_copies()
        P.pic_step(pair.h, 1)
        outs = [np.zeros(pair.o.shape, dtype=pair.T) for _ in range(6)]
        P.pic_debug_gather_copies(pair.h, P.PIC_HOST, outs)
        for c in range(2):  # the transverse E copies carry the inverse
            assert rel_l2(outs[c], expect[c]) <= TOL[precision], (c, rel_l2(outs[c], expect[c]))
    finally:
        pair.close()


@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("scheme", [0, 1])
def test_rational_step(precision, scheme):
    pair = _random_pair(2, precision, scheme=scheme, alpha=0.6 if scheme == 0 else 0.45, nx=32, nz=48, npart=12000,
                        corr_mode=1)
    try:
        for _ in range(2):
            pair.step(1)
        _compare(pair, TOL[precision])
    finally:
        pair.close()


def test_rational_constant_denominator_and_errors():
    # a constant Psi_B = 2 halves the transverse E copies; a Psi_B with a zero on [0, 1] has no inverse
    coeffs = (np.array([1.0, 0, 0, 0, 0]), np.array([2.0, 0, 0, 0, 0]))
    pair = _random_pair(2, 1, npart=0, nx=16, nz=20, corr_mode=1, coeffs=coeffs)
    try:
        expect = pair.o.gather_copies()
        P.pic_step(pair.h, 1)
        outs = [np.zeros(pair.o.shape) for _ in range(6)]
        P.pic_debug_gather_copies(pair.h, P.PIC_HOST, outs)
        for c in range(6):
            assert rel_l2(outs[c], expect[c]) <= 1e-12, c
        with pytest.raises(P.PicError) as e:
            P.pic_set_correction_stencil(pair.h, [1.0, 0, 0, 0, 0], [1.0, -1.5, 0, 0, 0])  # zero at xi = 2/3
        assert e.value.code == P.PIC_E_SINGULAR
    finally:
        pair.close()
    cfg = make_cfg(nx=16, nz=16, precision=1, init_beam=1, corr_mode=1)
    with pytest.raises(P.PicError) as e:
        P.pic_batch_create([cfg])
    assert e.value.code == P.PIC_E_ARG
