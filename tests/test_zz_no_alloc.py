"""GPU test of pic_field_energy_noalloc, the entry point for callers that cannot allocate device
memory (it keeps its partial sums in a fixed array of the library's own device memory).

Its results must equal those of pic_energy, the regular entry point that computes the same field
energies with handle-owned scratch, within the FP64 parity tolerance of the other tests, on two
calls in a row. This file is collected last so that a run stopping at the first failure has already
run every other test; it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

import synth
from tests._pic import P, make_cfg

pytestmark = pytest.mark.gpu

TOL = 1e-10  # FP64 sums of the same values in another order


def _energies_via_handle(cfg, fields_dev):
    h = P.pic_create(cfg)
    try:
        P.pic_set_state(h, P.make_state(P.PIC_DEVICE, fields_dev, None))
        e = P.pic_energy(h)
        return e["w_e"], e["w_b"], e["w_perp"]
    finally:
        P.pic_destroy(h)


@pytest.mark.parametrize("precision", [P.PIC_FP64, P.PIC_FP32] if P else [1, 0])
def test_noalloc_energy_matches_pic_energy(precision):
    torch = pytest.importorskip("torch")
    nx, nz = 96, 160
    cfg = make_cfg(nx=nx, nz=nz, precision=precision, ppc=4)
    dt = torch.float64 if precision == P.PIC_FP64 else torch.float32
    for seed in (21, 22):  # two calls in a row, on different fields
        host = synth.random_fields((nz, 1, nx), seed=seed, scale=0.3)
        dev = {k: torch.tensor(v, dtype=dt, device="cuda").contiguous() for k, v in host.items()}
        torch.cuda.synchronize()
        ref = _energies_via_handle(cfg, dev)
        got = P.pic_field_energy_noalloc([dev[k] for k in ("ex", "ey", "ez", "bx", "by", "bz")], nx * nz,
                                         precision, cfg.dx * cfg.dy * cfg.dz)
        for a, b in zip(got, ref):
            assert abs(a - b) <= TOL * abs(b), (got, ref)
        again = P.pic_field_energy_noalloc([dev[k] for k in ("ex", "ey", "ez", "bx", "by", "bz")], nx * nz,
                                           precision, cfg.dx * cfg.dy * cfg.dz)
        assert again == got  # deterministic: fixed chunks summed in a fixed order


@pytest.mark.parametrize("nx,nz", [(329, 249), (4096, 4096)])
def test_noalloc_partial_last_chunk_and_largest_size(nx, nz):
    # 81,921 = 4096 * 20 + 1 cells: the last of the fixed 4096-cell chunks holds one cell; 16,777,216
    # cells: every one of the 4096 partial-sum slots of the fixed array is used (the largest size)
    torch = pytest.importorskip("torch")
    cfg = make_cfg(nx=nx, nz=nz, precision=P.PIC_FP32, ppc=0)
    host = synth.random_fields((nz, 1, nx), seed=23, scale=0.3)
    dev = {k: torch.tensor(v, dtype=torch.float32, device="cuda").contiguous() for k, v in host.items()}
    torch.cuda.synchronize()
    ref = _energies_via_handle(cfg, dev)
    for _ in range(2):
        got = P.pic_field_energy_noalloc([dev[k] for k in ("ex", "ey", "ez", "bx", "by", "bz")], nx * nz,
                                         P.PIC_FP32, cfg.dx * cfg.dy * cfg.dz)
        for a, b in zip(got, ref):
            assert abs(a - b) <= TOL * abs(b), (got, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    with pytest.raises(P.PicError) as e:
        P.pic_field_energy_noalloc([1, 1, 1, 1, 1, 1], 16_777_216 + 1, P.PIC_FP32, 1.0)
    assert e.value.code == P.PIC_E_ARG
