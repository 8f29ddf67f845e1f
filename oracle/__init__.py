"""FP64 CPU oracle for the stabilised FDTD-Esirkepov PIC step (Godfrey & Vay, arXiv 1401.0838).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library shares no code with it and never calls it.

The arithmetic lives in ``oracle.c`` (plain C, FP64, ``-ffp-contract=off``); this module compiles it
with gcc into ``oracle/_build/liboracle.so`` on first use and wraps it with numpy arrays. ``fit.py``
holds the growth-rate fit and ``torch_step.py`` a plain PyTorch-CPU restatement of the step used for
the oracle-side gradient.

Parity pins: ``tests/test_oracle_*.py``. Every oracle function is pinned there against a closed form,
an invariant, a special case or brute force; none is marked "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

GALERKIN, UNIFORM, MOMENTUM = 0, 1, 2
FILTER_J, FILTER_GATHER = 1, 2
YEE, CK = 0, 1  # field solvers: Yee, Cole-Karkkainen (2D) in the B update


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library with gcc (FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


class Params(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double), ("dt", ctypes.c_double),
                ("scheme", ctypes.c_int), ("psi_e", ctypes.c_double * 9), ("psi_b", ctypes.c_double * 9),
                ("f_nbin", ctypes.c_int), ("f_ncomp", ctypes.c_int), ("f_alpha", ctypes.c_double),
                ("f_targets", ctypes.c_int), ("order", ctypes.c_int), ("corr_mode", ctypes.c_int),
                ("psi_b_coef", ctypes.c_double * 5), ("solver", ctypes.c_int), ("ck_beta_x", ctypes.c_double),
                ("ck_beta_z", ctypes.c_double)]


_DP = ctypes.POINTER(ctypes.c_double)


class _Fields(ctypes.Structure):
    _fields_ = [(n, _DP) for n in ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz")]


class _Particles(ctypes.Structure):
    _fields_ = [("n", ctypes.c_long)] + [(n, _DP) for n in ("x", "y", "z", "ux", "uy", "uz", "w", "q")]


class _Beam(ctypes.Structure):
    _fields_ = [("ppc", ctypes.c_int), ("gamma", ctypes.c_double), ("omega_p_dz", ctypes.c_double),
                ("jitter", ctypes.c_double), ("u_th", ctypes.c_double), ("sigma_perp", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


def _declare(L):
    P = ctypes.POINTER
    L.orc_multiplier.restype = ctypes.c_double
    L.orc_multiplier.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
    L.orc_rational_coeffs.restype = ctypes.c_int
    L.orc_rational_coeffs.argtypes = [ctypes.c_int, ctypes.c_double, _DP, _DP]
    L.orc_psi_taps.argtypes = [_DP, _DP]
    L.orc_bspline.restype = ctypes.c_double
    L.orc_bspline.argtypes = [ctypes.c_int, ctypes.c_double]
    L.orc_conv_axis.argtypes = [P(Params), _DP, ctypes.c_int, _DP, ctypes.c_int]
    L.orc_filter.argtypes = [P(Params), _DP]
    L.orc_gather_copies.argtypes = [P(Params), P(_Fields), _DP * 6]
    L.orc_inverse_psi_z.argtypes = [P(Params), _DP]
    L.orc_yee_b.argtypes = [P(Params), P(_Fields), ctypes.c_double]
    L.orc_yee_e.argtypes = [P(Params), P(_Fields), ctypes.c_double]
    L.orc_gather.argtypes = [P(Params), _DP * 6, _DP, _DP, _DP, ctypes.c_long, _DP * 6]
    L.orc_boris.argtypes = [ctypes.c_double, ctypes.c_double, _DP, _DP, _DP]
    L.orc_deposit_2d.argtypes = [P(Params), P(_Fields)] + [ctypes.c_double] * 6
    L.orc_deposit_3d.argtypes = [P(Params), P(_Fields), _DP, _DP, ctypes.c_double]
    L.orc_rho.argtypes = [P(Params), P(_Particles), _DP]
    L.orc_step.argtypes = [P(Params), P(_Fields), P(_Particles)]
    L.orc_run.argtypes = [P(Params), P(_Fields), P(_Particles), ctypes.c_int]
    L.orc_energy.argtypes = [P(Params), P(_Fields), P(_Particles), _DP]
    L.orc_div_e.argtypes = [P(Params), P(_Fields), _DP]
    L.orc_div_b.argtypes = [P(Params), P(_Fields), _DP]
    L.orc_philox4x32_10.argtypes = [P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)]
    L.orc_lattice_dims.argtypes = [ctypes.c_int, ctypes.c_int, P(ctypes.c_int)]
    L.orc_init_beam.argtypes = [P(Params), P(_Beam), P(_Particles)]


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


# ---------------------------------------------------------------------------------------------
# Scalar / small helpers
# ---------------------------------------------------------------------------------------------
def multiplier(scheme: int, alpha: float, s: float) -> float:
    """Eq. 3 (Galerkin), Eq. 4 (Uniform) or Eq. 5 (momentum-conserving) at s = k_z dz / 2."""
    return lib().orc_multiplier(scheme, alpha, s)


def rational_coeffs(scheme: int, alpha: float):
    """(4,4) rational interpolation of the multiplier (Sec. 2). Returns (status, psi_e[5], psi_b[5])."""
    pe = np.zeros(5)
    pb = np.zeros(5)
    st = lib().orc_rational_coeffs(scheme, alpha, _ptr(pe), _ptr(pb))
    return st, pe, pb


def bspline(n: int, t: float) -> float:
    """Centred cardinal B-spline of order n (0..3) at t (particle shapes, Sec. 3 uses n = 3)."""
    return lib().orc_bspline(int(n), float(t))


def psi_taps(a) -> np.ndarray:
    """9-tap z-stencil of Psi(D) = sum a_n D^n, D = -(1,-2,1)/4 (Sec. 2)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    t = np.zeros(9)
    lib().orc_psi_taps(_ptr(a), _ptr(t))
    return t


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def lattice_dims(ndim: int, ppc: int):
    o = (ctypes.c_int * 3)()
    lib().orc_lattice_dims(ndim, ppc, o)
    return tuple(o)


def boris(q: float, dt: float, E, B, u):
    E = np.ascontiguousarray(E, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    u = np.array(u, dtype=np.float64)
    lib().orc_boris(q, dt, _ptr(E), _ptr(B), _ptr(u))
    return u


# ---------------------------------------------------------------------------------------------
# Simulation state
# ---------------------------------------------------------------------------------------------
FIELD_NAMES = ("ex", "ey", "ez", "bx", "by", "bz", "jx", "jy", "jz")
PART_NAMES = ("x", "y", "z", "ux", "uy", "uz", "w", "q")


class Sim:
    """numpy-backed oracle state. Fields have shape (nz, ny, nx) (ny = 1 in 2D); particle arrays are 1D.

    psi_e / psi_b are the 5 polynomial coefficients (powers of xi, constant first) or None for
    Psi = 1 (correction off).
    """

    def __init__(self, ndim=2, nx=16, ny=1, nz=16, dx=1.0, dy=1.0, dz=1.0, dt=0.5, scheme=GALERKIN,
                 psi_e=None, psi_b=None, f_nbin=1, f_ncomp=1, f_alpha=3.0, f_targets=FILTER_J | FILTER_GATHER,
                 order=1, corr_mode=0, solver=YEE, ck_beta=(0.125, 0.125)):
        if ndim == 2:
            ny, dy = 1, 1.0
        if solver == CK and ndim != 2:
            raise ValueError("the Cole-Karkkainen solver is defined here for 2D x-z runs only")
        self.p = Params()
        self.p.ndim, self.p.nx, self.p.ny, self.p.nz = ndim, nx, ny, nz
        self.p.dx, self.p.dy, self.p.dz, self.p.dt = dx, dy, dz, dt
        self.p.scheme = scheme
        self.p.f_nbin, self.p.f_ncomp, self.p.f_alpha, self.p.f_targets = f_nbin, f_ncomp, f_alpha, f_targets
        self.p.order = order
        self.p.corr_mode = corr_mode
        self.p.solver = solver
        self.p.ck_beta_x, self.p.ck_beta_z = float(ck_beta[0]), float(ck_beta[1])
        self.set_correction(psi_e, psi_b)
        self.shape = (nz, ny, nx)
        self.f = {n: np.zeros(self.shape) for n in FIELD_NAMES}
        self.part = {n: np.zeros(0) for n in PART_NAMES}
        self.pid = np.zeros(0, dtype=np.int64)

    # -- configuration --------------------------------------------------------------------------
    def set_correction(self, psi_e, psi_b):
        one = np.array([1.0, 0, 0, 0, 0])
        te = psi_taps(one if psi_e is None else psi_e)
        tb = psi_taps(one if psi_b is None else psi_b)
        for m in range(9):
            self.p.psi_e[m] = te[m]
            self.p.psi_b[m] = tb[m]
        cb = one if psi_b is None else np.asarray(psi_b, dtype=np.float64)
        for m in range(5):
            self.p.psi_b_coef[m] = float(cb[m])

    @property
    def ndim(self):
        return self.p.ndim

    @property
    def n(self):
        return len(self.part["x"])

    # -- ctypes views ---------------------------------------------------------------------------
    def _fields(self) -> _Fields:
        F = _Fields()
        for n in FIELD_NAMES:
            a = self.f[n]
            assert a.shape == self.shape and a.dtype == np.float64 and a.flags.c_contiguous
            setattr(F, n, _ptr(a))
        return F

    def _particles(self) -> _Particles:
        P = _Particles()
        n = self.n
        P.n = n
        for k in PART_NAMES:
            a = self.part[k]
            assert a.shape == (n,) and a.dtype == np.float64 and a.flags.c_contiguous, k
            setattr(P, k, _ptr(a))
        return P

    # -- state ------------------------------------------------------------------------------------
    def set_particles(self, x, y, z, ux, uy, uz, w, q, pid=None):
        n = len(x)
        arrs = dict(x=x, y=y if y is not None else np.zeros(n), z=z, ux=ux, uy=uy, uz=uz, w=w, q=q)
        self.part = {k: np.ascontiguousarray(v, dtype=np.float64).copy() for k, v in arrs.items()}
        self.pid = np.arange(n, dtype=np.int64) if pid is None else np.asarray(pid, dtype=np.int64).copy()

    def init_beam(self, ppc, gamma=130.0, omega_p_dz=0.3868, jitter=0.1, u_th=1e-4, sigma_perp=0.0, seed=1):
        """Seeded beam state (Philox4x32-10); particle i has id i."""
        ncell = self.shape[0] * self.shape[1] * self.shape[2]
        n = ncell * ppc * 2
        self.part = {k: np.zeros(n) for k in PART_NAMES}
        b = _Beam(ppc, gamma, omega_p_dz, jitter, u_th, sigma_perp, seed)
        P = self._particles()
        lib().orc_init_beam(ctypes.byref(self.p), ctypes.byref(b), ctypes.byref(P))
        self.pid = np.arange(n, dtype=np.int64)

    # -- stages -------------------------------------------------------------------------------------
    def gather_copies(self):
        out = [np.zeros(self.shape) for _ in range(6)]
        F = self._fields()
        arr = (_DP * 6)(*[_ptr(a) for a in out])
        lib().orc_gather_copies(ctypes.byref(self.p), ctypes.byref(F), arr)
        return out

    def conv_axis(self, f, axis, taps):
        f = np.ascontiguousarray(f, dtype=np.float64).copy()
        taps = np.ascontiguousarray(taps, dtype=np.float64)
        lib().orc_conv_axis(ctypes.byref(self.p), _ptr(f), axis, _ptr(taps), (len(taps) - 1) // 2)
        return f

    def inverse_psi_z(self, f):
        """Psi_B(D_z)^-1 applied to a field (exact circulant inverse along z)."""
        f = np.ascontiguousarray(f, dtype=np.float64).copy()
        lib().orc_inverse_psi_z(ctypes.byref(self.p), _ptr(f))
        return f

    def filter(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).copy()
        lib().orc_filter(ctypes.byref(self.p), _ptr(f))
        return f

    def gather(self, G, x, y, z):
        n = len(x)
        G = [np.ascontiguousarray(g, dtype=np.float64) for g in G]
        x, z = (np.ascontiguousarray(v, dtype=np.float64) for v in (x, z))
        y = np.ascontiguousarray(y if y is not None else np.zeros(n), dtype=np.float64)
        out = [np.zeros(n) for _ in range(6)]
        lib().orc_gather(ctypes.byref(self.p), (_DP * 6)(*[_ptr(g) for g in G]), _ptr(x), _ptr(y), _ptr(z), n,
                         (_DP * 6)(*[_ptr(o) for o in out]))
        return out

    def yee_b(self, h):
        F = self._fields()
        lib().orc_yee_b(ctypes.byref(self.p), ctypes.byref(F), h)

    def yee_e(self, h):
        F = self._fields()
        lib().orc_yee_e(ctypes.byref(self.p), ctypes.byref(F), h)

    def deposit(self, x0, z0, x1, z1, vy, qw, y0=None, y1=None):
        """Esirkepov deposit of one particle moving from (x0, y0, z0) to (x1, y1, z1), unwrapped grid
        units, into self.f['jx','jy','jz'] (accumulating)."""
        F = self._fields()
        if self.ndim == 2:
            lib().orc_deposit_2d(ctypes.byref(self.p), ctypes.byref(F), x0, z0, x1 - x0, z1 - z0, vy, qw)
        else:
            r0 = np.array([x0, y0, z0], dtype=np.float64)
            dr = np.array([x1 - x0, y1 - y0, z1 - z0], dtype=np.float64)
            lib().orc_deposit_3d(ctypes.byref(self.p), ctypes.byref(F), _ptr(r0), _ptr(dr), qw)

    def deposit_move(self, x0, z0, ddx, ddz, vy, qw, y0=0.0, ddy=0.0):
        """Esirkepov deposit of one particle given its start position and its displacement (grid units)."""
        F = self._fields()
        if self.ndim == 2:
            lib().orc_deposit_2d(ctypes.byref(self.p), ctypes.byref(F), x0, z0, ddx, ddz, vy, qw)
        else:
            r0 = np.array([x0, y0, z0], dtype=np.float64)
            dr = np.array([ddx, ddy, ddz], dtype=np.float64)
            lib().orc_deposit_3d(ctypes.byref(self.p), ctypes.byref(F), _ptr(r0), _ptr(dr), qw)

    def rho(self):
        out = np.zeros(self.shape)
        P = self._particles()
        lib().orc_rho(ctypes.byref(self.p), ctypes.byref(P), _ptr(out))
        return out

    def div_e(self):
        out = np.zeros(self.shape)
        F = self._fields()
        lib().orc_div_e(ctypes.byref(self.p), ctypes.byref(F), _ptr(out))
        return out

    def div_b(self):
        out = np.zeros(self.shape)
        F = self._fields()
        lib().orc_div_b(ctypes.byref(self.p), ctypes.byref(F), _ptr(out))
        return out

    def step(self, nsteps=1):
        F = self._fields()
        P = self._particles()
        lib().orc_run(ctypes.byref(self.p), ctypes.byref(F), ctypes.byref(P), int(nsteps))

    def energy(self):
        """(W_E, W_B, W_perp, K, W_E + W_B + K), FP64."""
        out = np.zeros(5)
        F = self._fields()
        P = self._particles()
        lib().orc_energy(ctypes.byref(self.p), ctypes.byref(F), ctypes.byref(P), _ptr(out))
        return out

    def copy(self) -> "Sim":
        s = Sim.__new__(Sim)
        s.p = Params()
        ctypes.pointer(s.p)[0] = self.p
        s.shape = self.shape
        s.f = {k: v.copy() for k, v in self.f.items()}
        s.part = {k: v.copy() for k, v in self.part.items()}
        s.pid = self.pid.copy()
        return s
