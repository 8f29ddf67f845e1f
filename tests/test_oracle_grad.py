"""Pins of the oracle-side gradient (oracle/torch_step.py).

* Forward: the PyTorch restatement advances a beam exactly like orc_step (C, FP64) to roundoff,
  for both gather schemes, with the correction and both filters on.
* Gradient: torch.autograd through the restatement agrees with central finite differences of the
  C oracle (which shares no code with it) for the Psi_E / Psi_B coefficients (Sec. 2) and for
  sampled entries of the initial fields.
* Without particles W_perp(T) is a quadratic form in the initial fields, so <grad, F0> = 2 W_perp.
"""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import torch_step as TS

FNAMES = ("ex", "ey", "ez", "bx", "by", "bz")


def _sim(scheme=O.GALERKIN, nx=12, nz=20, alpha=0.5, gamma=3.0, ppc=4, seed=3, field_amp=2e-2, f_targets=3,
         corr=True):
    st, pe, pb = O.rational_coeffs(scheme, alpha)
    assert st == 0
    if not corr:
        pe = pb = np.array([1.0, 0, 0, 0, 0])
    sim = O.Sim(ndim=2, nx=nx, nz=nz, dt=alpha, scheme=scheme, psi_e=pe, psi_b=pb, f_nbin=1, f_ncomp=1,
                f_targets=f_targets)
    sim.init_beam(ppc=ppc, gamma=gamma, u_th=5e-2, seed=seed)
    rng = np.random.default_rng(seed)
    for n in FNAMES:
        sim.f[n][...] = field_amp * rng.standard_normal(sim.shape)
    return sim, np.asarray(pe, dtype=np.float64), np.asarray(pb, dtype=np.float64)


def _oracle_w_perp(sim, pe, pb, nsteps, fields=None):
    s = sim.copy()
    s.set_correction(pe, pb)
    if fields is not None:
        for n, f in zip(FNAMES, fields):
            s.f[n][:, 0, :] = f
    s.step(nsteps)
    return s.energy()[2]


@pytest.mark.parametrize("scheme", [O.GALERKIN, O.UNIFORM])
def test_forward_matches_c_oracle(scheme):
    sim, pe, pb = _sim(scheme=scheme)
    g, F, P = TS.from_sim(sim)
    te, tb = TS.psi_taps(torch.tensor(pe)), TS.psi_taps(torch.tensor(pb))
    assert np.allclose(te.numpy(), O.psi_taps(pe), rtol=0, atol=1e-15)
    ref = sim.copy()
    for _ in range(4):
        F, P = TS.step(g, te, tb, F, P)
    ref.step(4)
    for n, f in zip(FNAMES, F):
        r = ref.f[n][:, 0, :]
        assert np.abs(f.numpy() - r).max() <= 1e-12 * np.abs(r).max(), n
    for k in ("x", "z", "ux", "uy", "uz"):
        assert np.abs(P[k].numpy() - ref.part[k]).max() <= 1e-12 * max(1.0, np.abs(ref.part[k]).max()), k
    assert abs(TS.w_perp(g, F).item() - ref.energy()[2]) <= 1e-12 * ref.energy()[2]


@pytest.mark.parametrize("scheme", [O.GALERKIN, O.UNIFORM])
def test_coefficient_gradient_matches_oracle_differences(scheme):
    nsteps = 6
    sim, pe, pb = _sim(scheme=scheme)
    g, F, P = TS.from_sim(sim)
    a_e = torch.tensor(pe, requires_grad=True)
    a_b = torch.tensor(pb, requires_grad=True)
    w = TS.run_w_perp(g, a_e, a_b, F, P, nsteps)
    w.backward()
    assert abs(w.item() - _oracle_w_perp(sim, pe, pb, nsteps)) <= 1e-12 * w.item()
    h = 1e-4
    for which, grad in ((0, a_e.grad.numpy()), (1, a_b.grad.numpy())):
        fd = np.zeros(5)
        for n in range(5):
            dp = np.zeros(5)
            dp[n] = h
            if which == 0:
                wp = _oracle_w_perp(sim, pe + dp, pb, nsteps)
                wm = _oracle_w_perp(sim, pe - dp, pb, nsteps)
            else:
                wp = _oracle_w_perp(sim, pe, pb + dp, nsteps)
                wm = _oracle_w_perp(sim, pe, pb - dp, nsteps)
            fd[n] = (wp - wm) / (2 * h)
        scale = np.abs(fd).max()
        assert scale > 1e-9 * w.item()  # the coefficients do matter
        assert np.abs(grad - fd).max() <= 1e-5 * scale, (which, grad, fd)


def test_field_gradient_matches_oracle_differences():
    nsteps = 5
    sim, pe, pb = _sim()
    g, F, P = TS.from_sim(sim)
    F = [f.clone().requires_grad_(True) for f in F]
    w = TS.run_w_perp(g, torch.tensor(pe), torch.tensor(pb), F, P, nsteps)
    w.backward()
    rng = np.random.default_rng(11)
    h = 1e-5
    base = [f.detach().numpy().copy() for f in F]
    for _ in range(8):
        c = int(rng.integers(0, 6))
        kz, kx = int(rng.integers(0, g.nz)), int(rng.integers(0, g.nx))
        fp = [b.copy() for b in base]
        fm = [b.copy() for b in base]
        fp[c][kz, kx] += h
        fm[c][kz, kx] -= h
        fd = (_oracle_w_perp(sim, pe, pb, nsteps, fp) - _oracle_w_perp(sim, pe, pb, nsteps, fm)) / (2 * h)
        ad = F[c].grad[kz, kx].item()
        assert abs(ad - fd) <= 1e-6 * max(abs(fd), 1e-3 * w.item()), (c, kz, kx, ad, fd)


def test_field_gradient_homogeneity_without_particles():
    # W_perp(T) of a vacuum run is a quadratic form in the initial fields: <grad, F0> = 2 W_perp(T).
    sim, pe, pb = _sim()
    g, F, _ = TS.from_sim(sim)
    P = {k: torch.zeros(0, dtype=torch.float64) for k in ("x", "z", "ux", "uy", "uz", "w", "q")}
    F = [f.clone().requires_grad_(True) for f in F]
    w = TS.run_w_perp(g, torch.tensor(pe), torch.tensor(pb), F, P, 7)
    w.backward()
    dot = sum((f.grad * f.detach()).sum().item() for f in F)
    assert abs(dot - 2 * w.item()) <= 1e-12 * w.item()
    # and the correction coefficients have no effect on the fields of a vacuum run
    a = torch.tensor(pe, requires_grad=True)
    TS.run_w_perp(g, a, torch.tensor(pb), [f.detach() for f in F], P, 3).backward()
    assert a.grad is None or float(a.grad.abs().max()) == 0.0
