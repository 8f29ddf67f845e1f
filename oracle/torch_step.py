"""Differentiable FP64 restatement of the 2D step, for the oracle-side gradient.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only ``tests/`` and the benchmark's CPU legs may
import it. It shares nothing with the CUDA library.

The step is the same algorithm as ``orc_step`` in ``oracle.c`` (pinned there against the paper and
FDTD theory), written with plain PyTorch CPU ops on whole arrays, so that ``torch.autograd`` gives
the exact derivative (almost everywhere: the shapes are piecewise linear) of the final transverse
field energy with respect to the Psi_E / Psi_B polynomial coefficients (Sec. 2) and the initial
fields. ``tests/test_oracle_grad.py`` pins this module to ``orc_step`` (forward, to roundoff) and its
gradients to central finite differences of ``orc_step``.

Passes are applied one at a time in the paper's loop order (no fusion, no tiles):
  1. gather copies: Psi_E(D_z) on Ex, Ey, Psi_B(D_z) on Ez, Bx, By, Bz (Sec. 2, last paragraph),
     then the gather-side filter (Sec. 3, Eq. 6);
  2. field gather with linear shapes, Galerkin (order 0 along half-staggered directions) or Uniform
     (Sec. 2, Eq. 3-4);
  3. relativistic Boris push (standard; the paper does not state its pusher);
  4. move, x += dt u / gamma;
  5. Esirkepov deposition of J (Esirkepov 2001, cited in Sec. 2), the shape change formed from the
     displacement on a linear piece of S1;
  6. current filter (Sec. 3, Eq. 6);
  7. Yee: B half step, E full step with J, B half step.
2D x-z only (the y-invariant case ny = 1).
"""
from __future__ import annotations

import torch

# stagger of Ex, Ey, Ez, Bx, By, Bz along (x, y, z)
STAG = ((1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 1, 1), (1, 0, 1), (1, 1, 0))
FILTER_J, FILTER_GATHER = 1, 2
GALERKIN, UNIFORM = 0, 1
WIN = 6  # deposit window: nodes -2..3 relative to the start cell


class Grid:
    """Parameters of a 2D run (grid units, c = 1)."""

    def __init__(self, nx, nz, dx=1.0, dz=1.0, dt=0.5, scheme=GALERKIN, f_nbin=1, f_ncomp=1, f_alpha=3.0,
                 f_targets=FILTER_J | FILTER_GATHER):
        self.nx, self.nz, self.dx, self.dz, self.dt = nx, nz, dx, dz, dt
        self.scheme = scheme
        self.f_nbin, self.f_ncomp, self.f_alpha, self.f_targets = f_nbin, f_ncomp, f_alpha, f_targets

    @property
    def dv(self):
        return self.dx * self.dz


def psi_taps(a: torch.Tensor) -> torch.Tensor:
    """Sec. 2: the 9 taps (offsets -4..4) of Psi(D) = sum_n a_n D^n with D = -(1, -2, 1)/4.
    Linear in a, so the taps carry the gradient back to the coefficients."""
    d = (-0.25, 0.5, -0.25)
    pw = [0.0] * 9
    pw[4] = 1.0
    taps = a[0] * torch.tensor(pw, dtype=torch.float64)
    for n in range(1, 5):
        nxt = [0.0] * 9
        for m in range(9):
            for t in (-1, 0, 1):
                if 0 <= m + t < 9:
                    nxt[m + t] += pw[m] * d[t + 1]
        pw = nxt
        taps = taps + a[n] * torch.tensor(pw, dtype=torch.float64)
    return taps


def conv(f: torch.Tensor, taps, dim: int) -> torch.Tensor:
    """Periodic convolution along one array dimension: out[i] = sum_m taps[m + h] f[i + m]."""
    h = (len(taps) - 1) // 2
    out = torch.zeros_like(f)
    for m in range(-h, h + 1):
        out = out + taps[m + h] * torch.roll(f, shifts=-m, dims=dim)
    return out


def filt(g: Grid, f: torch.Tensor) -> torch.Tensor:
    """Sec. 3, Eq. 6: f_nbin bilinear passes (1/4, 1/2, 1/4) and f_ncomp compensation passes
    (-(a-1)/2, a, -(a-1)/2) along x, then along z."""
    bil = (0.25, 0.5, 0.25)
    cmp_ = (-(g.f_alpha - 1.0) / 2.0, g.f_alpha, -(g.f_alpha - 1.0) / 2.0)
    for dim in (1, 0):  # x is the last array dimension, z the first
        for _ in range(g.f_nbin):
            f = conv(f, bil, dim)
        for _ in range(g.f_ncomp):
            f = conv(f, cmp_, dim)
    return f


def gather_copies(g: Grid, F, te: torch.Tensor, tb: torch.Tensor):
    out = []
    for c in range(6):
        h = conv(F[c], te if c < 2 else tb, 0)
        if g.f_targets & FILTER_GATHER:
            h = filt(g, h)
        out.append(h)
    return out


def S1(t: torch.Tensor) -> torch.Tensor:
    """Linear spline max(0, 1 - |t|)."""
    return torch.clamp(1.0 - torch.abs(t), min=0.0)


def gather(g: Grid, G, x: torch.Tensor, z: torch.Tensor):
    """Sec. 2: six components at the particle positions (grid units, shape (N,))."""
    out = []
    for c in range(6):
        wts, idx = [], []
        for pos, st, n in ((x, STAG[c][0], g.nx), (z, STAG[c][2], g.nz)):
            xs = pos - 0.5 * st
            order = 1 - st if g.scheme == GALERKIN else 1
            if order == 1:
                fl = torch.floor(xs).detach()
                wts.append([S1(xs - fl), S1(xs - (fl + 1.0))])
                b = fl.long()
                idx.append([torch.remainder(b, n), torch.remainder(b + 1, n)])
            else:
                b = torch.floor(xs + 0.5).detach().long()
                wts.append([torch.ones_like(xs)])
                idx.append([torch.remainder(b, n)])
        acc = torch.zeros_like(x)
        for kz, wz in zip(idx[1], wts[1]):
            for kx, wx in zip(idx[0], wts[0]):
                acc = acc + wx * wz * G[c][kz, kx]
        out.append(acc)
    return out


def boris(q: torch.Tensor, dt: float, E, B, u):
    h = 0.5 * q * dt
    um = [u[a] + h * E[a] for a in range(3)]
    gam = torch.sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2])
    t = [h * B[a] / gam for a in range(3)]
    tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2]
    s = [2.0 * t[a] / (1.0 + tt) for a in range(3)]
    up = [um[0] + (um[1] * t[2] - um[2] * t[1]), um[1] + (um[2] * t[0] - um[0] * t[2]),
          um[2] + (um[0] * t[1] - um[1] * t[0])]
    upl = [um[0] + (up[1] * s[2] - up[2] * s[1]), um[1] + (up[2] * s[0] - up[0] * s[2]),
           um[2] + (up[0] * s[1] - up[1] * s[0])]
    return [upl[a] + h * E[a] for a in range(3)]


def _piece(a: torch.Tensor) -> torch.Tensor:
    """Linear piece of S1 holding a: 0 (a <= -1), 1 (-1 < a <= 0), 2 (0 < a < 1), 3 (a >= 1)."""
    return (a > -1.0).long() + (a > 0.0).long() + (a >= 1.0).long()


def shape_window(r0: torch.Tensor, dr: torch.Tensor):
    """S0 and dS on nodes -2..3 relative to the start cell floor(r0), shape (N, WIN); dS from the
    displacement where both shape arguments lie on one linear piece, else the plain difference."""
    c = torch.floor(r0).detach()
    o = r0 - c
    node = torch.arange(-2, WIN - 2, dtype=torch.float64)
    a0 = node[None, :] - o[:, None]
    a1 = a0 - dr[:, None]
    p0, p1 = _piece(a0.detach()), _piece(a1.detach())
    slope = torch.where(p0 == 1, 1.0, torch.where(p0 == 2, -1.0, 0.0)).to(torch.float64)
    ds = torch.where(p0 == p1, slope * (-dr[:, None]), S1(a1) - S1(a0))
    return c.long() - 2, S1(a0), ds


def deposit(g: Grid, x0, z0, ddx, ddz, vy, qw):
    """Esirkepov 2D3V current J^{n+1/2} of all particles (Jx, Jy, Jz arrays of shape (nz, nx))."""
    ncell = g.nx * g.nz
    dV = g.dv
    ia, S0x, dSx = shape_window(x0, ddx)
    ka, S0z, dSz = shape_window(z0, ddz)
    cx = -qw * g.dx / (dV * g.dt)
    cz = -qw * g.dz / (dV * g.dt)
    cy = qw * vy / dV
    ar = torch.arange(WIN)
    ix = torch.remainder(ia[:, None] + ar[None, :], g.nx)  # (N, WIN)
    iz = torch.remainder(ka[:, None] + ar[None, :], g.nz)
    flat = iz[:, :, None] * g.nx + ix[:, None, :]  # (N, b, a)
    # Jx(i+1/2, k): running sum over the x window of dSx (S0z + dSz/2)
    wx = dSx[:, None, :] * (S0z + 0.5 * dSz)[:, :, None]
    jx = cx[:, None, None] * torch.cumsum(wx, dim=2)
    # Jz(i, k+1/2): running sum over the z window of dSz (S0x + dSx/2)
    wz = dSz[:, :, None] * (S0x + 0.5 * dSx)[:, None, :]
    jz = cz[:, None, None] * torch.cumsum(wz, dim=1)
    # Jy(i, k): out-of-plane weight
    wy = (S0x[:, None, :] * S0z[:, :, None] + 0.5 * dSx[:, None, :] * S0z[:, :, None] +
          0.5 * S0x[:, None, :] * dSz[:, :, None] + dSx[:, None, :] * dSz[:, :, None] / 3.0)
    jy = cy[:, None, None] * wy
    out = []
    for jj in (jx, jy, jz):
        out.append(torch.zeros(ncell, dtype=torch.float64).index_add(0, flat.reshape(-1), jj.reshape(-1))
                   .reshape(g.nz, g.nx))
    return out


def curl_e(g: Grid, E):
    """curl E at the B locations (forward differences; y-invariant)."""
    ex, ey, ez = E
    dzp = lambda f: (torch.roll(f, -1, 0) - f) / g.dz
    dxp = lambda f: (torch.roll(f, -1, 1) - f) / g.dx
    return [-dzp(ey), dzp(ex) - dxp(ez), dxp(ey)]


def curl_b(g: Grid, B):
    """curl B at the E locations (backward differences; y-invariant)."""
    bx, by, bz = B
    dzm = lambda f: (f - torch.roll(f, 1, 0)) / g.dz
    dxm = lambda f: (f - torch.roll(f, 1, 1)) / g.dx
    return [-dzm(by), dzm(bx) - dxm(bz), dxm(by)]


def step(g: Grid, te, tb, F, P):
    """One step. F: list of six (nz, nx) tensors (Ex, Ey, Ez, Bx, By, Bz); P: dict with x, z, ux, uy,
    uz, w, q (shape (N,), positions in grid units). Returns the new (F, P)."""
    G = gather_copies(g, F, te, tb)
    x0, z0 = P["x"], P["z"]
    f = gather(g, G, x0, z0)
    u = boris(P["q"], g.dt, f[:3], f[3:], [P["ux"], P["uy"], P["uz"]])
    gam = torch.sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2])
    ddx = g.dt * u[0] / gam / g.dx
    ddz = g.dt * u[2] / gam / g.dz
    J = deposit(g, x0, z0, ddx, ddz, u[1] / gam, P["q"] * P["w"])
    if g.f_targets & FILTER_J:
        J = [filt(g, j) for j in J]
    E, B = list(F[:3]), list(F[3:])
    h = 0.5 * g.dt
    B = [b - h * c for b, c in zip(B, curl_e(g, E))]
    cb = curl_b(g, B)
    E = [e + g.dt * (c - j) for e, c, j in zip(E, cb, J)]
    B = [b - h * c for b, c in zip(B, curl_e(g, E))]
    x1 = x0 + ddx
    z1 = z0 + ddz
    Pn = dict(P)
    Pn["x"] = x1 - g.nx * torch.floor(x1 / g.nx).detach()
    Pn["z"] = z1 - g.nz * torch.floor(z1 / g.nz).detach()
    Pn["ux"], Pn["uy"], Pn["uz"] = u
    return E + B, Pn


def w_perp(g: Grid, F) -> torch.Tensor:
    """Transverse field energy 1/2 sum (Ex^2 + Ey^2 + Bx^2 + By^2) dV (Sec. 4 diagnostics)."""
    return 0.5 * g.dv * (F[0].pow(2).sum() + F[1].pow(2).sum() + F[3].pow(2).sum() + F[4].pow(2).sum())


def run_w_perp(g: Grid, psi_e: torch.Tensor, psi_b: torch.Tensor, F0, P0, nsteps: int) -> torch.Tensor:
    """W_perp after nsteps from (F0, P0); differentiable in psi_e, psi_b and F0."""
    te, tb = psi_taps(psi_e), psi_taps(psi_b)
    F, P = list(F0), dict(P0)
    for _ in range(nsteps):
        F, P = step(g, te, tb, F, P)
    return w_perp(g, F)


def from_sim(sim):
    """(Grid, fields, particles) as FP64 tensors from an ``oracle.Sim`` (2D)."""
    p = sim.p
    assert p.ndim == 2
    g = Grid(p.nx, p.nz, p.dx, p.dz, p.dt, p.scheme, p.f_nbin, p.f_ncomp, p.f_alpha, p.f_targets)
    F = [torch.tensor(sim.f[n][:, 0, :].copy()) for n in ("ex", "ey", "ez", "bx", "by", "bz")]
    P = {k: torch.tensor(sim.part[k].copy()) for k in ("x", "z", "ux", "uy", "uz", "w", "q")}
    return g, F, P
