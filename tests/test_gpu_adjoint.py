"""GPU adjoint of the 2D step (pic_adjoint_forward / pic_adjoint_backward) against the oracle-side
gradient (oracle/torch_step.py, pinned to orc_step and to finite differences of the C oracle) and
against central finite differences of the library's own FP64 forward run."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from oracle import torch_step as TS
from tests._pic import P, Pair, make_cfg

pytestmark = pytest.mark.gpu
FN = ("ex", "ey", "ez", "bx", "by", "bz")


def _beam_pair(scheme=0, nx=16, nz=32, ppc=4, gamma=3.0, alpha=0.5, u_th=5e-2, field_amp=2e-2, seed=5,
               precision=1, targets=3):
    cfg = make_cfg(nx=nx, nz=nz, dt=alpha, gamma=gamma, scheme=scheme, precision=precision, ppc=ppc,
                   targets=targets, u_th=u_th, seed=seed)
    st, pe, pb = O.rational_coeffs(scheme, alpha)
    o = O.Sim(ndim=2, nx=nx, nz=nz, dt=alpha)
    o.init_beam(ppc=ppc, gamma=gamma, u_th=u_th, seed=seed)
    part = dict(o.part)
    part["id"] = o.pid.copy()
    rng = np.random.default_rng(seed)
    fields = {n: field_amp * rng.standard_normal((nz, 1, nx)) for n in FN}
    pair = Pair(cfg, psi=(pe, pb), fields=fields, part=part)
    return pair, np.asarray(pe), np.asarray(pb)


def _gpu_grad(h, cfg, nsteps, every, dtype=torch.float64):
    w = P.pic_adjoint_forward(h, nsteps, every)
    gf = [torch.empty(cfg.nz * cfg.nx, dtype=dtype, device="cuda") for _ in range(6)]
    ge, gb = P.pic_adjoint_backward(h, 1.0, gf)
    return w, ge, gb, [g.cpu().numpy().reshape(cfg.nz, cfg.nx) for g in gf]


def _oracle_grad(pair, pe, pb, nsteps):
    g, F, Pt = TS.from_sim(pair.o)
    F = [f.clone().requires_grad_(True) for f in F]
    a_e = torch.tensor(pe, requires_grad=True)
    a_b = torch.tensor(pb, requires_grad=True)
    w = TS.run_w_perp(g, a_e, a_b, F, Pt, nsteps)
    w.backward()
    return w.item(), a_e.grad.numpy(), a_b.grad.numpy(), [f.grad.numpy() for f in F]


@pytest.mark.parametrize("scheme", [0, 1])
def test_adjoint_fp64_matches_oracle_gradient(scheme):
    nsteps = 6
    pair, pe, pb = _beam_pair(scheme=scheme)
    w, ge, gb, gf = _gpu_grad(pair.h, pair.cfg, nsteps, 2)
    wo, ge_o, gb_o, gf_o = _oracle_grad(pair, pe, pb, nsteps)
    assert abs(w - wo) <= 1e-10 * wo
    for a, b in ((ge, ge_o), (gb, gb_o)):
        assert np.abs(b).max() > 1e-4 * wo
        assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max(), (a, b)
    for q in range(6):
        scale = max(np.abs(gf_o[q]).max(), 1e-12 * wo)
        assert np.abs(gf[q] - gf_o[q]).max() <= 1e-9 * scale, FN[q]


def test_adjoint_filters_off_and_unfiltered_current():
    pair, pe, pb = _beam_pair(targets=0, nx=20, nz=24)
    w, ge, gb, gf = _gpu_grad(pair.h, pair.cfg, 5, 5)
    wo, ge_o, gb_o, gf_o = _oracle_grad(pair, pe, pb, 5)
    assert abs(w - wo) <= 1e-10 * wo
    assert np.abs(ge - ge_o).max() <= 1e-9 * np.abs(ge_o).max()
    assert np.abs(gb - gb_o).max() <= 1e-9 * np.abs(gb_o).max()
    for q in range(6):
        assert np.abs(gf[q] - gf_o[q]).max() <= 1e-9 * max(np.abs(gf_o[q]).max(), 1e-12 * wo)


def test_checkpoint_interval_does_not_change_the_gradient():
    res = []
    for every in (1, 3, 7):
        pair, pe, pb = _beam_pair(nx=24, nz=40, seed=7)
        res.append(_gpu_grad(pair.h, pair.cfg, 7, every))
    for r in res[1:]:
        assert abs(r[0] - res[0][0]) <= 1e-13 * res[0][0]  # the forward's atomics may reorder sums
        assert np.abs(r[1] - res[0][1]).max() <= 1e-11 * np.abs(res[0][1]).max()
        for q in range(6):
            assert np.abs(r[3][q] - res[0][3][q]).max() <= 1e-11 * max(np.abs(res[0][3][q]).max(), 1e-300)


def _fd_w(cfg, fields, part, pe, pb, nsteps):
    pair = Pair(cfg, psi=(pe, pb), fields=fields, part=part)
    P.pic_step(pair.h, nsteps)
    w = P.pic_energy(pair.h)["w_perp"]
    P.pic_destroy(pair.h)
    return w


def test_adjoint_matches_central_differences_gamma130():
    # a relativistic beam (gamma = 130) on a 64 x 128 grid, 20 steps, checkpoints every 5
    nx, nz, nsteps, alpha = 64, 128, 20, 0.5
    cfg = make_cfg(nx=nx, nz=nz, dt=alpha, gamma=130.0, precision=1, ppc=4, u_th=1e-4, seed=9)
    st, pe, pb = O.rational_coeffs(0, alpha)
    o = O.Sim(ndim=2, nx=nx, nz=nz, dt=alpha)
    o.init_beam(ppc=4, gamma=130.0, u_th=1e-4, seed=9)
    part = dict(o.part)
    part["id"] = o.pid.copy()
    rng = np.random.default_rng(9)
    fields = {n: 1e-3 * rng.standard_normal((nz, 1, nx)) for n in FN}
    pair = Pair(cfg, psi=(pe, pb), fields=fields, part=part)
    w, ge, gb, gf = _gpu_grad(pair.h, cfg, nsteps, 5)
    h = 1e-4
    for n in range(5):
        d = np.zeros(5)
        d[n] = h
        fd = (_fd_w(cfg, fields, part, pe + d, pb, nsteps) - _fd_w(cfg, fields, part, pe - d, pb, nsteps)) / (2 * h)
        assert abs(ge[n] - fd) <= 1e-6 * np.abs(ge).max(), (n, ge[n], fd)
    for q, (kz, kx) in ((0, (3, 7)), (1, (60, 20)), (3, (100, 63)), (4, (0, 0)), (2, (17, 40)), (5, (90, 11))):
        fp = {k: v.copy() for k, v in fields.items()}
        fm = {k: v.copy() for k, v in fields.items()}
        fp[FN[q]][kz, 0, kx] += h
        fm[FN[q]][kz, 0, kx] -= h
        fd = (_fd_w(cfg, fp, part, pe, pb, nsteps) - _fd_w(cfg, fm, part, pe, pb, nsteps)) / (2 * h)
        assert abs(gf[q][kz, kx] - fd) <= 1e-6 * max(abs(fd), np.abs(gf[q]).max()), (q, gf[q][kz, kx], fd)


def test_state_after_backward_is_the_final_state():
    pair, pe, pb = _beam_pair(nx=32, nz=48)
    w = P.pic_adjoint_forward(pair.h, 9, 4)
    e0 = P.pic_energy(pair.h)
    P.pic_adjoint_backward(pair.h, 1.0)
    e1 = P.pic_energy(pair.h)
    assert e1["w_perp"] == w == e0["w_perp"]
    assert e1["np"] == e0["np"]
    assert abs(e1["k"] - e0["k"]) <= 1e-13 * abs(e0["k"])
    # a second backward on the same recording gives the same gradient
    g1 = P.pic_adjoint_backward(pair.h, 2.0)
    g2 = P.pic_adjoint_backward(pair.h, 1.0)
    assert np.abs(g1[0] - 2 * g2[0]).max() <= 1e-12 * np.abs(g1[0]).max()


def test_autograd_function():
    from paper_1401_0838_gb300.autograd import WPerp
    pair, pe, pb = _beam_pair(nx=16, nz=32)
    cfg = pair.cfg
    f0 = [torch.tensor(pair.o.f[n][:, 0, :].reshape(-1), device="cuda", requires_grad=True) for n in FN]
    a_e = torch.tensor(pe, requires_grad=True)
    a_b = torch.tensor(pb, requires_grad=True)
    # the handle holds the initial particles; WPerp sets the coefficients and the fields
    w = WPerp.apply(pair.h, 6, 3, a_e, a_b, *f0)
    (3.0 * w).backward()
    wo, ge_o, gb_o, gf_o = _oracle_grad(pair, pe, pb, 6)
    assert abs(w.item() - wo) <= 1e-10 * wo
    assert np.abs(a_e.grad.numpy() - 3.0 * ge_o).max() <= 1e-9 * 3.0 * np.abs(ge_o).max()
    assert np.abs(a_b.grad.numpy() - 3.0 * gb_o).max() <= 1e-9 * 3.0 * np.abs(gb_o).max()
    for q in range(6):
        g = f0[q].grad.cpu().numpy().reshape(cfg.nz, cfg.nx)
        assert np.abs(g - 3.0 * gf_o[q]).max() <= 1e-9 * 3.0 * max(np.abs(gf_o[q]).max(), 1e-12 * wo)


def test_adjoint_errors():
    cfg = make_cfg(nx=16, nz=16, precision=1, init_beam=1, track_ids=0)
    h = P.pic_create(cfg)
    with pytest.raises(P.PicError) as e:
        P.pic_adjoint_forward(h, 2, 1)
    assert e.value.code == P.PIC_E_STATE
    P.pic_destroy(h)
    h = P.pic_create(make_cfg(nx=16, nz=16, precision=1, init_beam=1, track_ids=1))
    with pytest.raises(P.PicError) as e:
        P.pic_adjoint_backward(h)
    assert e.value.code == P.PIC_E_STATE
    P.pic_adjoint_forward(h, 3, 2)
    P.pic_step(h, 1)  # the state moved on: the recording no longer applies
    with pytest.raises(P.PicError) as e:
        P.pic_adjoint_backward(h)
    assert e.value.code == P.PIC_E_STATE
    with pytest.raises(P.PicError) as e:
        P.pic_adjoint_forward(h, 3, 0)
    assert e.value.code == P.PIC_E_ARG
    P.pic_adjoint_release(h)
    P.pic_destroy(h)
    h3 = P.pic_create(make_cfg(ndim=3, nx=8, ny=8, nz=8, precision=1, init_beam=1, track_ids=1, ppc=1))
    with pytest.raises(P.PicError) as e:
        P.pic_adjoint_forward(h3, 1, 1)
    assert e.value.code == P.PIC_E_ARG
    P.pic_destroy(h3)


def _config5(precision):
    # 2D 256 x 512, 8 particles/cell/species, gamma = 130, c dt/dz = 0.5, Galerkin, correction on,
    # filter (1, 1, a = 3) on J and on the gather copies; the seeded beam, E = B = 0 at t = 0
    return P.pic_config_default(nx=256, nz=512, dt=0.5, gamma=130.0, precision=precision, ppc_per_species=8,
                                init_beam=1, track_ids=1, seed=5)


def _w_after(precision, pe, pb, nsteps):
    h = P.pic_create(_config5(precision))
    P.pic_set_correction_stencil(h, pe, pb)
    P.pic_step(h, nsteps)
    w = P.pic_energy(h)["w_perp"]
    P.pic_destroy(h)
    return w


def test_adjoint_256x512_100_steps():
    # FP64: the adjoint against central differences (h = 1e-3) of the FP64 forward, <= 1e-5 relative.
    # FP32: the adjoint of the FP32 run differs from the FP64 gradient by no more than the FP32 run's
    # own W_perp differs from the FP64 one (the forward's precision bounds it, not the adjoint).
    pe, pb = P.pic_compute_correction_coeffs(P.PIC_GALERKIN, 0.5)
    res = {}
    for prec in (P.PIC_FP64, P.PIC_FP32):
        h = P.pic_create(_config5(prec))
        P.pic_set_correction_stencil(h, pe, pb)
        w = P.pic_adjoint_forward(h, 100, 10)
        ge, gb = P.pic_adjoint_backward(h, 1.0)
        res[prec] = (w, ge, gb)
        P.pic_destroy(h)
    w64, ge64, gb64 = res[P.PIC_FP64]
    hh = 1e-3
    fd = np.zeros(5)
    for n in (0, 2, 4):
        d = np.zeros(5)
        d[n] = hh
        fd[n] = (_w_after(P.PIC_FP64, pe + d, pb, 100) - _w_after(P.PIC_FP64, pe - d, pb, 100)) / (2 * hh)
        assert abs(ge64[n] - fd[n]) <= 1e-5 * np.abs(ge64).max(), (n, ge64[n], fd[n])
    w32, ge32, gb32 = res[P.PIC_FP32]
    fwd = abs(w32 - w64) / w64
    assert fwd < 2e-2
    assert np.abs(ge32 - ge64).max() <= max(3 * fwd, 1e-4) * np.abs(ge64).max()
    assert np.abs(gb32 - gb64).max() <= max(3 * fwd, 1e-4) * np.abs(gb64).max()


def test_gradient_step_lowers_late_time_energy():
    # the use the gradient is for: a small step of the Psi_E coefficients against dW_perp/da lowers
    # W_perp(T) of the same seeded run (gamma = 130 beam, 40 steps)
    cfg = P.pic_config_default(nx=64, nz=128, dt=0.5, gamma=130.0, precision=P.PIC_FP64, ppc_per_species=4,
                               init_beam=1, track_ids=1, seed=21)
    pe, pb = P.pic_compute_correction_coeffs(P.PIC_GALERKIN, 0.5)
    h = P.pic_create(cfg)
    P.pic_set_correction_stencil(h, pe, pb)
    w0 = P.pic_adjoint_forward(h, 40, 10)
    ge, _ = P.pic_adjoint_backward(h, 1.0)
    P.pic_destroy(h)
    step = 1e-2 * np.linalg.norm(pe) / np.linalg.norm(ge)
    h = P.pic_create(cfg)
    P.pic_set_correction_stencil(h, pe - step * ge, pb)
    P.pic_step(h, 40)
    w1 = P.pic_energy(h)["w_perp"]
    P.pic_destroy(h)
    predicted = -step * float(ge @ ge)
    assert w1 < w0
    assert abs((w1 - w0) - predicted) <= 0.1 * abs(predicted)  # first-order prediction holds
