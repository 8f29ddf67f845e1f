"""Pins of the oracle's particle operators: gather (partition of unity, exact linear reproduction,
brute-force sum over the whole grid), relativistic Boris push (exact gyration, exact E kick) and
Esirkepov deposition (continuity to roundoff, total current, brute-force node-by-node W)."""
import math

import numpy as np
import pytest

import oracle as O

# stagger of Ex, Ey, Ez, Bx, By, Bz along x, y, z (standard Yee mesh)
STAG = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (0, 1, 1), (1, 0, 1), (1, 1, 0)]


def _rand_pos(rng, sim, n, margin=0.0):
    nz, ny, nx = sim.shape
    x = rng.uniform(margin, nx - margin, n)
    y = rng.uniform(margin, ny - margin, n) if sim.ndim == 3 else np.zeros(n)
    z = rng.uniform(margin, nz - margin, n)
    return x, y, z


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("scheme", [O.GALERKIN, O.UNIFORM])
def test_gather_partition_of_unity(ndim, scheme):
    rng = np.random.default_rng(0)
    sim = O.Sim(ndim=ndim, nx=8, ny=6, nz=10, scheme=scheme)
    G = [np.full(sim.shape, 1.5 + c) for c in range(6)]
    x, y, z = _rand_pos(rng, sim, 200)
    out = sim.gather(G, x, y, z)
    for c in range(6):
        np.testing.assert_allclose(out[c], 1.5 + c, rtol=0, atol=1e-14)


def _linear_field(sim, c, a0, ax, ay, az):
    nz, ny, nx = sim.shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    st = STAG[c]
    return a0 + ax * (i + 0.5 * st[0]) + ay * (j + 0.5 * st[1]) + az * (k + 0.5 * st[2])


@pytest.mark.parametrize("ndim", [2, 3])
def test_gather_linear_reproduction(ndim):
    # Uniform (S1 everywhere) reproduces a linear field exactly; Galerkin replaces the coordinate along
    # each half-staggered direction by the cell centre floor(x) + 1/2 (its S0 box).
    rng = np.random.default_rng(1)
    sim_u = O.Sim(ndim=ndim, nx=12, ny=9, nz=14, scheme=O.UNIFORM)
    sim_g = O.Sim(ndim=ndim, nx=12, ny=9, nz=14, scheme=O.GALERKIN)
    ay = 0.4 if ndim == 3 else 0.0
    G = [_linear_field(sim_u, c, 0.3 * c, 0.7, ay, -0.9) for c in range(6)]
    x, y, z = _rand_pos(rng, sim_u, 300, margin=1.0)
    ou = sim_u.gather(G, x, y, z)
    og = sim_g.gather(G, x, y, z)
    for c in range(6):
        np.testing.assert_allclose(ou[c], 0.3 * c + 0.7 * x + ay * y - 0.9 * z, atol=1e-12)
        st = STAG[c]
        gx = np.floor(x) + 0.5 if st[0] else x
        gy = (np.floor(y) + 0.5 if st[1] else y) if ndim == 3 else 0
        gz = np.floor(z) + 0.5 if st[2] else z
        np.testing.assert_allclose(og[c], 0.3 * c + 0.7 * gx + ay * gy - 0.9 * gz, atol=1e-12)


def _S1(d):
    return np.maximum(0.0, 1.0 - np.abs(d))


def _S0(d):
    return ((d >= -0.5) & (d < 0.5)).astype(float)


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("scheme", [O.GALERKIN, O.UNIFORM])
def test_gather_brute_force(ndim, scheme):
    # sum over every node of the (periodic) grid of shape products times the field value
    rng = np.random.default_rng(2)
    sim = O.Sim(ndim=ndim, nx=6, ny=5, nz=7, scheme=scheme)
    nz, ny, nx = sim.shape
    G = [rng.normal(size=sim.shape) for _ in range(6)]
    x, y, z = _rand_pos(rng, sim, 40)
    out = sim.gather(G, x, y, z)
    for c in range(6):
        st = STAG[c]
        for p in range(40):
            acc = 0.0
            for k in range(nz):
                for j in range(ny):
                    for i in range(nx):
                        w = 1.0
                        for ax, (pos, node, n) in enumerate(((x[p], i, nx), (y[p], j, ny), (z[p], k, nz))):
                            if ax == 1 and ndim == 2:
                                continue
                            loc = node + 0.5 * st[ax]
                            # nearest periodic image of the node
                            d = (loc - pos + n / 2) % n - n / 2
                            if scheme == O.GALERKIN and st[ax]:
                                w *= _S0(d)
                            else:
                                w *= _S1(d)
                        acc += w * G[c][k, j, i]
            assert abs(out[c][p] - acc) < 1e-12


def test_boris_uniform_b_gyration():
    # E = 0, uniform B: |u| is conserved and the rotation per step is 2 atan(q B dt / (2 gamma)).
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = rng.choice([-1.0, 1.0])
        B = rng.normal(size=3)
        u = rng.normal(size=3) * 5
        dt = rng.uniform(0.1, 1.0)
        g = math.sqrt(1 + u @ u)
        u1 = O.boris(q, dt, [0, 0, 0], B, u)
        assert abs(np.linalg.norm(u1) - np.linalg.norm(u)) < 1e-13 * np.linalg.norm(u)
        bh = B / np.linalg.norm(B)
        up0 = u - (u @ bh) * bh
        up1 = u1 - (u1 @ bh) * bh
        assert abs(u1 @ bh - u @ bh) < 1e-12
        ang = math.atan2(np.cross(up0, up1) @ bh, up0 @ up1)
        expect = -2 * math.atan(q * np.linalg.norm(B) * dt / (2 * g))
        assert abs(ang - expect) < 1e-12


def test_boris_uniform_e_kick():
    # B = 0: u gains exactly q E dt (two half kicks).
    rng = np.random.default_rng(4)
    for _ in range(10):
        q = rng.choice([-1.0, 1.0])
        E = rng.normal(size=3)
        u = rng.normal(size=3)
        dt = 0.37
        u1 = O.boris(q, dt, E, [0, 0, 0], u)
        np.testing.assert_allclose(u1, u + q * E * dt, atol=1e-14)


def test_boris_ultra_relativistic_parallel_b():
    # u parallel to B is unchanged by any B.
    u = np.array([0.0, 0.0, 129.996])
    u1 = O.boris(-1.0, 0.5, [0, 0, 0], [0, 0, 3.0], u)
    np.testing.assert_allclose(u1, u, atol=1e-13)


def _moves(rng, sim, n):
    x0, y0, z0 = _rand_pos(rng, sim, n)
    d = rng.uniform(-0.95, 0.95, size=(n, 3))
    if sim.ndim == 2:
        d[:, 1] = 0
    return x0, y0, z0, x0 + d[:, 0], y0 + d[:, 1], z0 + d[:, 2]


@pytest.mark.parametrize("ndim", [2, 3])
def test_esirkepov_continuity(ndim):
    # (rho1 - rho0)/dt + div J = 0 at every node to roundoff, for moves crossing cells and the wrap.
    rng = np.random.default_rng(5)
    dt = 0.6
    sim = O.Sim(ndim=ndim, nx=7, ny=5, nz=9, dt=dt, dx=1.1, dy=0.9, dz=1.3)
    n = 60
    x0, y0, z0, x1, y1, z1 = _moves(rng, sim, n)
    qw = rng.normal(size=n)
    for p in range(n):
        sim.deposit(x0[p], z0[p], x1[p], z1[p], 0.0, qw[p], y0=y0[p], y1=y1[p])
    nz, ny, nx = sim.shape

    def rho(x, y, z):
        s = O.Sim(ndim=ndim, nx=nx, ny=ny, nz=nz, dx=1.1, dy=0.9, dz=1.3)
        s.set_particles(x % nx, y % ny if ndim == 3 else None, z % nz, np.zeros(n), np.zeros(n), np.zeros(n),
                        np.abs(qw), np.sign(qw))
        return s.rho()

    r0, r1 = rho(x0, y0, z0), rho(x1, y1, z1)
    J = sim.f
    div = ((J["jx"] - np.roll(J["jx"], 1, axis=2)) / 1.1 + (J["jz"] - np.roll(J["jz"], 1, axis=0)) / 1.3)
    if ndim == 3:
        div = div + (J["jy"] - np.roll(J["jy"], 1, axis=1)) / 0.9
    res = (r1 - r0) / dt + div
    scale = np.abs(r0).max() / dt
    assert np.abs(res).max() < 1e-13 * scale


@pytest.mark.parametrize("ndim", [2, 3])
def test_esirkepov_total_current(ndim):
    # sum J dV = q w (x1 - x0) d / dt along each moved axis; in 2D, sum Jy dV = q w vy.
    rng = np.random.default_rng(6)
    dt = 0.5
    sim = O.Sim(ndim=ndim, nx=8, ny=6, nz=8, dt=dt)
    x0, y0, z0, x1, y1, z1 = _moves(rng, sim, 1)
    qw, vy = 0.7, 0.3
    sim.deposit(x0[0], z0[0], x1[0], z1[0], vy, qw, y0=y0[0], y1=y1[0])
    assert abs(sim.f["jx"].sum() - qw * (x1[0] - x0[0]) / dt) < 1e-13
    assert abs(sim.f["jz"].sum() - qw * (z1[0] - z0[0]) / dt) < 1e-13
    if ndim == 2:
        assert abs(sim.f["jy"].sum() - qw * vy) < 1e-13
    else:
        assert abs(sim.f["jy"].sum() - qw * (y1[0] - y0[0]) / dt) < 1e-13


def test_esirkepov_brute_force_2d():
    # Whole-grid W computed by hand for a few particles away from the wrap; J from a cumulative sum
    # starting at the first node of the grid (where J = 0 for these particles), compared node by node.
    rng = np.random.default_rng(7)
    nx, nz, dt, dx, dz = 9, 10, 0.4, 1.0, 1.0
    sim = O.Sim(ndim=2, nx=nx, nz=nz, dt=dt)
    jx = np.zeros((nz, nx))
    jy = np.zeros((nz, nx))
    jz = np.zeros((nz, nx))
    ii = np.arange(nx)
    kk = np.arange(nz)
    for _ in range(5):
        x0, z0 = rng.uniform(2, nx - 3), rng.uniform(2, nz - 3)
        x1, z1 = x0 + rng.uniform(-0.9, 0.9), z0 + rng.uniform(-0.9, 0.9)
        qw, vy = rng.normal(), rng.normal() * 0.2
        sim.deposit(x0, z0, x1, z1, vy, qw)
        S0x, S1x = _S1(ii - x0), _S1(ii - x1)
        S0z, S1z = _S1(kk - z0), _S1(kk - z1)
        dSx, dSz = S1x - S0x, S1z - S0z
        Wx = np.outer(S0z + 0.5 * dSz, dSx)
        Wz = np.outer(dSz, S0x + 0.5 * dSx)
        Wy = (np.outer(S0z, S0x) + 0.5 * np.outer(S0z, dSx) + 0.5 * np.outer(dSz, S0x) + np.outer(dSz, dSx) / 3)
        jx += -qw * dx / (dx * dz * dt) * np.cumsum(Wx, axis=1)
        jz += -qw * dz / (dx * dz * dt) * np.cumsum(Wz, axis=0)
        jy += qw * vy / (dx * dz) * Wy
    np.testing.assert_allclose(sim.f["jx"][:, 0, :], jx, atol=1e-14)
    np.testing.assert_allclose(sim.f["jz"][:, 0, :], jz, atol=1e-14)
    np.testing.assert_allclose(sim.f["jy"][:, 0, :], jy, atol=1e-14)


def test_esirkepov_brute_force_3d():
    rng = np.random.default_rng(8)
    n = 8
    dt = 0.4
    sim = O.Sim(ndim=3, nx=n, ny=n, nz=n, dt=dt)
    J = [np.zeros((n, n, n)) for _ in range(3)]
    nodes = np.arange(n)
    for _ in range(4):
        r0 = rng.uniform(2, n - 3, 3)
        r1 = r0 + rng.uniform(-0.9, 0.9, 3)
        qw = rng.normal()
        sim.deposit(r0[0], r0[2], r1[0], r1[2], 0.0, qw, y0=r0[1], y1=r1[1])
        S0 = [_S1(nodes - r0[a]) for a in range(3)]
        dS = [_S1(nodes - r1[a]) - S0[a] for a in range(3)]
        for a in range(3):
            b1, b2 = (a + 1) % 3, (a + 2) % 3
            tr = (np.outer(S0[b1], S0[b2]) + 0.5 * np.outer(dS[b1], S0[b2]) + 0.5 * np.outer(S0[b1], dS[b2])
                  + np.outer(dS[b1], dS[b2]) / 3)
            W = np.einsum("a,bc->abc", dS[a], tr)  # axes (a, b1, b2)
            Jl = -qw / dt * np.cumsum(W, axis=0)
            # move axes to (z, y, x) storage order
            order = {a: 0, b1: 1, b2: 2}
            Jl = np.transpose(Jl, (order[2], order[1], order[0]))
            J[a] += Jl
    for a, nm in enumerate(("jx", "jy", "jz")):
        np.testing.assert_allclose(sim.f[nm], J[a], atol=1e-14)


@pytest.mark.parametrize("ndim", [2, 3])
def test_esirkepov_tiny_move_precision(ndim):
    # A transverse move of 1e-9 cells far from the origin (the drift of a cold gamma = 130 beam is
    # ~4e-7 cells per step): the current is linear in the displacement, so J / d must match the
    # small-move limit to FP64 precision, not to 1e-16 / 1e-9.
    dt, qw = 0.5, 0.8
    sim = O.Sim(ndim=ndim, nx=300, ny=8, nz=300, dt=dt)
    x0, y0, z0 = 201.3, 3.6, 123.7
    d = 1e-9
    sim.deposit_move(x0, z0, d, 0.0, 0.0, qw, y0=y0, ddy=0.0)
    jx = sim.f["jx"]
    assert abs(jx.sum() - qw * d / dt) < 1e-12 * qw * d / dt
    # node values: Jx(i+1/2) = (qw/dt) d * S1(z) (S1(y)): the particle's cell column only
    i, k = 201, 123
    wz = [1 - 0.7, 0.7]
    for b in range(2):
        v = jx[k + b, 3 if ndim == 3 else 0, i] if ndim == 3 else jx[k + b, 0, i]
        wy = (1 - 0.6) if ndim == 3 else 1.0
        assert abs(v - qw / dt * d * wz[b] * wy) < 1e-12 * qw / dt * d
