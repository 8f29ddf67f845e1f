"""Pins of the oracle's higher-order shapes (Sec. 3 runs with cubic interpolation) and of the
momentum-conserving gather (the scheme Eq. 5 belongs to): B-spline identities, gather partition of
unity, exact linear reproduction and a brute-force sum over the whole grid, Esirkepov continuity
and total current with cubic shapes (including moves of 1e-9 cell), and Gauss's law over whole
steps."""
import numpy as np
import pytest

import oracle as O

STAG = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 1, 1), (1, 0, 1), (1, 1, 0)]
MOMENTUM = O.MOMENTUM


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_bspline_moments(n):
    # partition of unity, first moment t (n >= 1), and for n >= 2 (splines reproducing quadratics) the
    # second moment (n+1)/12, the variance of a sum of n+1 independent uniform variables on [-1/2, 1/2)
    rng = np.random.default_rng(n)
    for t in rng.uniform(-3, 3, 50):
        ks = np.arange(int(np.floor(t)) - 4, int(np.floor(t)) + 5)
        w = np.array([O.bspline(n, t - k) for k in ks])
        assert abs(w.sum() - 1.0) < 1e-14
        if n >= 1:
            assert abs((w * ks).sum() - t) < 1e-13
        if n >= 2:
            assert abs((w * (ks - t) ** 2).sum() - (n + 1) / 12.0) < 1e-13


@pytest.mark.parametrize("n", [1, 2, 3])
def test_bspline_is_box_convolution(n):
    # S_n(t) = integral over s in [-1/2, 1/2) of S_{n-1}(t - s), by a midpoint rule on m points: first
    # order in 1/m for the discontinuous box (n = 1), second order for the continuous S1, S2
    m = 10000 if n == 1 else 5000
    s = (np.arange(m) + 0.5) / m - 0.5
    tol = 2.0 / m if n == 1 else 2e-6
    for t in np.linspace(-2.3, 2.3, 23):
        v = np.mean([O.bspline(n - 1, t - si) for si in s])
        assert abs(v - O.bspline(n, t)) < tol


def _rand_pos(rng, sim, n, margin=0.0):
    nz, ny, nx = sim.shape
    x = rng.uniform(margin, nx - margin, n)
    y = rng.uniform(margin, ny - margin, n) if sim.ndim == 3 else np.zeros(n)
    z = rng.uniform(margin, nz - margin, n)
    return x, y, z


SCHEMES = [(O.GALERKIN, 3), (O.UNIFORM, 3), (MOMENTUM, 3), (MOMENTUM, 1)]


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("scheme,order", SCHEMES)
def test_gather_partition_and_linear_reproduction(ndim, scheme, order):
    # every scheme of order >= 1 along every direction reproduces a linear field exactly: S1, S2, S3
    # all have first moment t, and the momentum scheme's average of a linear field to the node is the
    # field at the node
    rng = np.random.default_rng(11)
    sim = O.Sim(ndim=ndim, nx=12, ny=9, nz=14, scheme=scheme, order=order)
    nz, ny, nx = sim.shape
    G = [np.full(sim.shape, 1.5 + c) for c in range(6)]
    x, y, z = _rand_pos(rng, sim, 100)
    out = sim.gather(G, x, y, z)
    for c in range(6):
        np.testing.assert_allclose(out[c], 1.5 + c, rtol=0, atol=1e-14)
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ay = 0.4 if ndim == 3 else 0.0
    G = [0.3 * c + 0.7 * (i + 0.5 * STAG[c][0]) + ay * (j + 0.5 * STAG[c][1]) - 0.9 * (k + 0.5 * STAG[c][2])
         for c in range(6)]
    x, y, z = _rand_pos(rng, sim, 200, margin=3.0)
    out = sim.gather(G, x, y, z)
    for c in range(6):
        np.testing.assert_allclose(out[c], 0.3 * c + 0.7 * x + ay * y - 0.9 * z, atol=1e-12)


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("scheme,order", SCHEMES)
def test_gather_brute_force(ndim, scheme, order):
    # sum over every node of the periodic grid of B-spline products times the field value; the
    # momentum scheme first averages the component to the nodes
    rng = np.random.default_rng(12)
    sim = O.Sim(ndim=ndim, nx=6, ny=5, nz=7, scheme=scheme, order=order)
    nz, ny, nx = sim.shape
    G = [rng.normal(size=sim.shape) for _ in range(6)]
    npart = 12
    x, y, z = _rand_pos(rng, sim, npart)
    out = sim.gather(G, x, y, z)
    for c in range(6):
        st = STAG[c]
        Gc = G[c]
        if scheme == MOMENTUM:  # average to the nodes over the half-staggered directions
            for ax, arr_ax in ((0, 2), (1, 1), (2, 0)):
                if st[ax] and not (ax == 1 and ndim == 2):
                    Gc = 0.5 * (Gc + np.roll(Gc, 1, axis=arr_ax))
        for p in range(npart):
            acc = 0.0
            for kk in range(nz):
                for jj in range(ny):
                    for ii in range(nx):
                        w = 1.0
                        for ax, (pos, node, n) in enumerate(((x[p], ii, nx), (y[p], jj, ny), (z[p], kk, nz))):
                            if ax == 1 and ndim == 2:
                                continue
                            if scheme == MOMENTUM:
                                loc, o = node, order
                            else:
                                loc = node + 0.5 * st[ax]
                                o = order - st[ax] if scheme == O.GALERKIN else order
                            d = (loc - pos + n / 2) % n - n / 2  # nearest periodic image
                            w *= O.bspline(o, d)
                        acc += w * Gc[kk, jj, ii]
            assert abs(out[c][p] - acc) < 1e-12, (c, p)


def _moves(rng, sim, n, dmax=0.95):
    x0, y0, z0 = _rand_pos(rng, sim, n)
    d = rng.uniform(-dmax, dmax, size=(n, 3))
    if sim.ndim == 2:
        d[:, 1] = 0
    return x0, y0, z0, x0 + d[:, 0], y0 + d[:, 1], z0 + d[:, 2]


@pytest.mark.parametrize("ndim", [2, 3])
def test_cubic_esirkepov_continuity(ndim):
    # (rho1 - rho0)/dt + div J = 0 at every node, rho with cubic shapes, moves crossing cells and the wrap
    rng = np.random.default_rng(13)
    dt = 0.6
    kw = dict(ndim=ndim, nx=9, ny=7, nz=11, dx=1.1, dy=0.9, dz=1.3, order=3)
    sim = O.Sim(dt=dt, **kw)
    n = 40
    x0, y0, z0, x1, y1, z1 = _moves(rng, sim, n)
    qw = rng.normal(size=n)
    for p in range(n):
        sim.deposit(x0[p], z0[p], x1[p], z1[p], 0.0, qw[p], y0=y0[p], y1=y1[p])
    nz, ny, nx = sim.shape

    def rho(x, y, z):
        s = O.Sim(**kw)
        s.set_particles(x % nx, y % ny if ndim == 3 else None, z % nz, np.zeros(n), np.zeros(n), np.zeros(n),
                        np.abs(qw), np.sign(qw))
        return s.rho()

    r0, r1 = rho(x0, y0, z0), rho(x1, y1, z1)
    J = sim.f
    div = (J["jx"] - np.roll(J["jx"], 1, axis=2)) / 1.1 + (J["jz"] - np.roll(J["jz"], 1, axis=0)) / 1.3
    if ndim == 3:
        div = div + (J["jy"] - np.roll(J["jy"], 1, axis=1)) / 0.9
    res = (r1 - r0) / dt + div
    assert np.abs(res).max() < 1e-13 * np.abs(r0).max() / dt


@pytest.mark.parametrize("d", [0.7, -0.4, 1e-3, -1e-6, 1e-9])
def test_cubic_total_current_and_small_moves(d):
    # sum J dV = q w (x1 - x0) / dt along each moved axis, to 1e-12 relative even for a 1e-9-cell move
    # (the shape change is formed from the displacement on each polynomial piece of the cubic)
    rng = np.random.default_rng(14)
    dt = 0.5
    sim = O.Sim(ndim=2, nx=10, nz=10, dt=dt, order=3)
    x0, z0 = rng.uniform(2, 8, 2)
    qw, vy = 0.7, 0.3
    sim.deposit_move(x0, z0, d, -0.5 * d, vy, qw)
    assert abs(sim.f["jx"].sum() - qw * d / dt) <= 1e-12 * abs(qw * d / dt)
    assert abs(sim.f["jz"].sum() + qw * 0.5 * d / dt) <= 1e-12 * abs(qw * 0.5 * d / dt)
    assert abs(sim.f["jy"].sum() - qw * vy) < 1e-13


@pytest.mark.parametrize("scheme,order", SCHEMES)
def test_gauss_law_whole_steps(scheme, order):
    # div(F J) = F div J: div E - F rho stays constant step after step with any shape and gather
    st, pe, pb = O.rational_coeffs(scheme, 0.5)
    sim = O.Sim(ndim=2, nx=12, nz=20, dt=0.5, scheme=scheme, order=order, psi_e=pe, psi_b=pb)
    sim.init_beam(ppc=4, u_th=1e-2, seed=3)
    rng = np.random.default_rng(15)
    for n in ("ex", "ey", "ez", "bx", "by", "bz"):
        sim.f[n][...] = 1e-2 * rng.standard_normal(sim.shape)
    g0 = sim.div_e() - sim.filter(sim.rho())
    scale = np.abs(sim.part["w"]).max()
    for _ in range(5):
        sim.step(1)
    g = sim.div_e() - sim.filter(sim.rho())
    assert np.abs(g - g0).max() < 1e-12 * max(scale, np.abs(g0).max())
