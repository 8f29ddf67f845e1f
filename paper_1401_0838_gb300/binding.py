"""Thin Python binding of the C ABI in include/pic.h (argument marshalling only).

Every function keeps the C name. Arrays are passed as raw pointers: numpy arrays (host) or torch
tensors (device or pinned host). No step of the PIC method runs here; if the CUDA library is not
built the import fails loudly (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpic_gb300.so")

PIC_OK = 0
PIC_E_ARG, PIC_E_CFL, PIC_E_SINGULAR, PIC_E_OOM, PIC_E_CUDA = -1, -2, -3, -4, -5
PIC_E_TIMEOUT, PIC_E_NONFINITE, PIC_E_OVERFLOW, PIC_E_STATE = -6, -7, -8, -9
PIC_GALERKIN, PIC_UNIFORM, PIC_MOMENTUM = 0, 1, 2
PIC_FP32, PIC_FP64 = 0, 1
PIC_FILTER_J, PIC_FILTER_GATHER = 1, 2
PIC_HOST, PIC_DEVICE = 0, 1
PIC_CORR_SPLIT, PIC_CORR_RATIONAL = 0, 1
PIC_YEE, PIC_CK = 0, 1  # field solvers: Yee, Cole-Karkkainen (2D)

# every symbol the header declares
EXPORTS = ("pic_config_default", "pic_compute_correction_coeffs", "pic_create", "pic_set_stream",
           "pic_set_correction_stencil", "pic_step", "pic_sync", "pic_energy", "pic_num_particles",
           "pic_get_state", "pic_set_state", "pic_debug_gather_copies", "pic_debug_current",
           "pic_fit_growth_rate", "pic_destroy", "pic_last_error", "pic_strerror", "pic_energy_history",
           "pic_enable_timing", "pic_kernel_times", "pic_launch_count", "pic_field_energy_noalloc",
           "pic_batch_create", "pic_batch_size", "pic_batch_run", "pic_batch_set_correction_stencil",
           "pic_batch_set_stream", "pic_batch_step", "pic_batch_sync", "pic_batch_energy_history",
           "pic_batch_autotune", "pic_batch_destroy", "pic_batch_last_error", "pic_adjoint_forward",
           "pic_adjoint_backward", "pic_adjoint_release", "pic_charge_residual", "pic_bin_stats")
PIC_NKERNEL = 8
KERNEL_CLASSES = ("copies", "push", "filter", "yee", "diag", "other", "migrate", "spill")


class pic_config(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double), ("dt", ctypes.c_double),
                ("gamma", ctypes.c_double), ("scheme", ctypes.c_int), ("shape_order", ctypes.c_int),
                ("precision", ctypes.c_int), ("ppc_per_species", ctypes.c_int), ("omega_p_dz", ctypes.c_double),
                ("jitter", ctypes.c_double), ("u_th", ctypes.c_double), ("sigma_perp", ctypes.c_double),
                ("filter_nbin", ctypes.c_int), ("filter_ncomp", ctypes.c_int), ("filter_comp_alpha", ctypes.c_double),
                ("filter_targets", ctypes.c_int), ("seed", ctypes.c_ulonglong), ("init_beam", ctypes.c_int),
                ("bin_capacity", ctypes.c_int), ("track_ids", ctypes.c_int), ("diag_every", ctypes.c_int),
                ("diag_capacity", ctypes.c_int), ("correction_mode", ctypes.c_int),
                ("field_solver", ctypes.c_int), ("ck_beta_x", ctypes.c_double), ("ck_beta_z", ctypes.c_double)]


class pic_energy_t(ctypes.Structure):
    _fields_ = [("w_e", ctypes.c_double), ("w_b", ctypes.c_double), ("w_perp", ctypes.c_double),
                ("k", ctypes.c_double), ("total", ctypes.c_double), ("np", ctypes.c_longlong)]


class pic_state(ctypes.Structure):
    _fields_ = [("where", ctypes.c_int)] + [(n, ctypes.c_void_p) for n in ("ex", "ey", "ez", "bx", "by", "bz")] + \
               [("np", ctypes.c_longlong), ("cell", ctypes.c_void_p), ("species", ctypes.c_void_p)] + \
               [(n, ctypes.c_void_p) for n in ("ox", "oy", "oz", "dux", "duy", "duz", "w", "id")] + \
               [("u_drift", ctypes.c_double)]


class PicError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """Load libpic_gb300.so (built in-tree); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run `python -m paper_1401_0838_gb300.build` "
                               "(no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        P, V, I, D = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        DP = P(ctypes.c_double)
        L.pic_config_default.argtypes = [P(pic_config)]
        L.pic_config_default.restype = None
        L.pic_compute_correction_coeffs.argtypes = [I, D, DP, DP]
        L.pic_create.argtypes = [P(pic_config), P(V)]
        L.pic_set_stream.argtypes = [V, V]
        L.pic_set_correction_stencil.argtypes = [V, DP, DP]
        L.pic_step.argtypes = [V, I]
        L.pic_sync.argtypes = [V]
        L.pic_energy.argtypes = [V, P(pic_energy_t)]
        L.pic_num_particles.argtypes = [V, P(ctypes.c_longlong)]
        L.pic_bin_stats.argtypes = [V, P(I), P(ctypes.c_longlong)]
        L.pic_get_state.argtypes = [V, P(pic_state)]
        L.pic_set_state.argtypes = [V, P(pic_state)]
        L.pic_debug_gather_copies.argtypes = [V, I, P(V)]
        L.pic_debug_current.argtypes = [V, I, P(V)]
        L.pic_fit_growth_rate.argtypes = [DP, DP, I, DP, P(I), P(I)]
        L.pic_charge_residual.argtypes = [V, DP]
        L.pic_destroy.argtypes = [V]
        L.pic_destroy.restype = None
        L.pic_last_error.argtypes = [V]
        L.pic_last_error.restype = ctypes.c_char_p
        L.pic_energy_history.argtypes = [V, P(pic_energy_t), I, P(I)]
        L.pic_enable_timing.argtypes = [V, I]
        L.pic_kernel_times.argtypes = [V, DP, P(ctypes.c_longlong)]
        L.pic_launch_count.argtypes = [V, P(ctypes.c_longlong)]
        L.pic_field_energy_noalloc.argtypes = [P(V), ctypes.c_longlong, I, D, DP, V]
        L.pic_batch_create.argtypes = [P(pic_config), I, P(V)]
        L.pic_batch_size.argtypes = [V]
        L.pic_batch_run.argtypes = [V, I]
        L.pic_batch_run.restype = V
        L.pic_batch_set_correction_stencil.argtypes = [V, I, DP, DP]
        L.pic_batch_set_stream.argtypes = [V, V]
        L.pic_batch_step.argtypes = [V, I]
        L.pic_batch_sync.argtypes = [V]
        L.pic_batch_energy_history.argtypes = [V, I, P(pic_energy_t), I, P(I)]
        L.pic_batch_autotune.argtypes = [V, I, P(I)]
        L.pic_batch_destroy.argtypes = [V]
        L.pic_batch_destroy.restype = None
        L.pic_batch_last_error.argtypes = [V]
        L.pic_batch_last_error.restype = ctypes.c_char_p
        L.pic_adjoint_forward.argtypes = [V, I, I, DP]
        L.pic_adjoint_backward.argtypes = [V, D, DP, DP, P(V)]
        L.pic_adjoint_release.argtypes = [V]
        L.pic_adjoint_release.restype = None
        L.pic_strerror.argtypes = [I]
        L.pic_strerror.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name not in ("pic_config_default", "pic_destroy", "pic_last_error", "pic_strerror", "pic_batch_run",
                            "pic_batch_destroy", "pic_batch_last_error", "pic_adjoint_release"):
                getattr(L, name).restype = I
        _lib = L
    return _lib


def _check(rc, h=None):
    if rc != PIC_OK:
        msg = lib().pic_strerror(rc).decode()
        if h is not None:
            detail = lib().pic_last_error(h).decode()
            if detail:
                msg = f"{msg}: {detail}"
        raise PicError(rc, msg)


def _ptr(a):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


# ------------------------------------------------------------------------------------------------
# C ABI, same names
# ------------------------------------------------------------------------------------------------
def pic_config_default(**overrides) -> pic_config:
    """Default pic_config (2D 64x128 FP64 Galerkin beam at gamma = 130, c dt/dz = 0.5) with keyword overrides set
    on the struct."""
    c = pic_config()
    lib().pic_config_default(ctypes.byref(c))
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def pic_compute_correction_coeffs(scheme: int, alpha: float):
    """Psi_E, Psi_B coefficients (powers of xi, constant first) of the (4,4) rational interpolant of Sec. 2 for the
    gather scheme at alpha = c dt/dz; raises PicError (PIC_E_SINGULAR) when no interpolant exists."""
    pe = (ctypes.c_double * 5)()
    pb = (ctypes.c_double * 5)()
    _check(lib().pic_compute_correction_coeffs(scheme, alpha, pe, pb))
    return np.array(pe[:]), np.array(pb[:])


def pic_create(cfg: pic_config):
    """Validates cfg, allocates the run on the current device and returns its opaque handle (the seeded beam when
    cfg.init_beam)."""
    h = ctypes.c_void_p()
    rc = lib().pic_create(ctypes.byref(cfg), ctypes.byref(h))
    if rc != PIC_OK:
        raise PicError(rc, f"{lib().pic_strerror(rc).decode()}: {lib().pic_last_error(None).decode()}")
    return h


def pic_set_stream(h, stream_ptr: int | None):
    """Queues the handle's later work on the cudaStream_t address stream_ptr (None: the handle's own stream)."""
    _check(lib().pic_set_stream(h, stream_ptr), h)


def pic_set_correction_stencil(h, psi_e=None, psi_b=None):
    """Sets the Psi_E / Psi_B coefficients (Sec. 2) of the gather correction; both None turns it off."""
    pe = None if psi_e is None else (ctypes.c_double * 5)(*[float(v) for v in psi_e])
    pb = None if psi_b is None else (ctypes.c_double * 5)(*[float(v) for v in psi_b])
    _check(lib().pic_set_correction_stencil(h, pe, pb), h)


def pic_step(h, nsteps: int = 1):
    """Advances nsteps time steps, asynchronously on the handle's stream."""
    _check(lib().pic_step(h, int(nsteps)), h)


def pic_sync(h):
    """Waits for the handle's stream and raises PicError on any kernel error of the queued steps."""
    _check(lib().pic_sync(h), h)


def pic_energy(h) -> dict:
    """FP64 energies of the current state: W_E, W_B, W_perp (the transverse field energy of Sec. 4), kinetic, total,
    particle count."""
    e = pic_energy_t()
    _check(lib().pic_energy(h, ctypes.byref(e)), h)
    return {"w_e": e.w_e, "w_b": e.w_b, "w_perp": e.w_perp, "k": e.k, "total": e.total, "np": e.np}


def pic_num_particles(h) -> int:
    """Current number of particles (synchronises)."""
    n = ctypes.c_longlong()
    _check(lib().pic_num_particles(h, ctypes.byref(n)), h)
    return n.value


def pic_bin_stats(h) -> tuple[int, int]:
    """(slots per cell and species of the bins, which grow as cells fill; insertions since creation
    that found their bin full and went to the spill list). Synchronises."""
    cap, spilled = ctypes.c_int(), ctypes.c_longlong()
    _check(lib().pic_bin_stats(h, ctypes.byref(cap), ctypes.byref(spilled)), h)
    return cap.value, spilled.value


def _itemsize(a) -> int:
    """Bytes per element of a numpy array or torch tensor."""
    return a.itemsize if isinstance(a, np.ndarray) else a.element_size()


def make_state(where: int, fields=None, particles=None) -> pic_state:
    """pic_state from dicts of arrays: fields {ex..bz}, particles {cell, species, ox, oy, oz, dux, duy, duz, w, id}."""
    s = pic_state()
    s.where = where
    for n in ("ex", "ey", "ez", "bx", "by", "bz"):
        setattr(s, n, _ptr((fields or {}).get(n)))
    p = particles or {}
    s.np = len(p["cell"]) if "cell" in p else 0
    # the library reads np elements of every particle array it is given: refuse shorter ones here
    for n, a in p.items():
        if a is not None and len(a) != s.np:
            raise ValueError(f"particle array {n!r} has {len(a)} elements, cell has {s.np}")
    for n in ("cell", "species", "id"):
        a = p.get(n)
        if a is not None and _itemsize(a) != 4:
            raise ValueError(f"particle array {n!r} must hold 4-byte integers")
    for n in ("cell", "species", "ox", "oy", "oz", "dux", "duy", "duz", "w", "id"):
        setattr(s, n, _ptr(p.get(n)))
    return s


def pic_set_state(h, state: pic_state):
    """Replaces the non-NULL fields and the particles of the run (state.np = -1 keeps the particles)."""
    _check(lib().pic_set_state(h, ctypes.byref(state)), h)


def pic_get_state(h, state: pic_state) -> pic_state:
    """Copies the state out into the arrays state points at (state.np in: their capacity) and returns state."""
    _check(lib().pic_get_state(h, ctypes.byref(state)), h)
    return state


def pic_debug_gather_copies(h, where: int, outs):
    """Test hook: copies the six field copies the particles gathered from in the last step into outs (Ex Ey Ez Bx By
    Bz)."""
    arr = (ctypes.c_void_p * 6)(*[_ptr(o) for o in outs])
    _check(lib().pic_debug_gather_copies(h, where, arr), h)


def pic_debug_current(h, where: int, outs):
    """Test hook: copies the filtered current J^{n+1/2} of the last step into outs (Jx Jy Jz)."""
    arr = (ctypes.c_void_p * 3)(*[_ptr(o) for o in outs])
    _check(lib().pic_debug_current(h, where, arr), h)


def pic_charge_residual(h) -> dict:
    """Gauss-law residual of the current state (FP64, on the device): max and RMS of div E - F rho over
    the nodes, and max |F rho| as the scale."""
    out = (ctypes.c_double * 3)()
    _check(lib().pic_charge_residual(h, out), h)
    return {"max": out[0], "rms": out[1], "rho_max": out[2]}


def pic_fit_growth_rate(t, w):
    """Growth rate Gamma = 1/2 d ln W / dt fitted over the exponential window of the series (t, w); returns (Gamma,
    first, last sample index of the window)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    if t.shape != w.shape or t.ndim != 1:
        raise ValueError(f"t and w must be 1-D arrays of one length (got {t.shape} and {w.shape})")
    g = ctypes.c_double()
    i0 = ctypes.c_int()
    i1 = ctypes.c_int()
    DP = ctypes.POINTER(ctypes.c_double)
    _check(lib().pic_fit_growth_rate(t.ctypes.data_as(DP), w.ctypes.data_as(DP), len(t), ctypes.byref(g),
                                     ctypes.byref(i0), ctypes.byref(i1)))
    return g.value, i0.value, i1.value


def pic_destroy(h):
    """Frees the handle and everything it owns (None is a no-op)."""
    if h is not None:
        lib().pic_destroy(h)


def pic_last_error(h) -> str:
    """Text of the last error on the handle (None: the last failed pic_create on this thread)."""
    return lib().pic_last_error(h).decode()


def pic_strerror(code: int) -> str:
    """Name of a PIC_E_* status code."""
    return lib().pic_strerror(code).decode()


def pic_energy_history(h, max_samples: int = 4096):
    """Energies recorded on the device every cfg.diag_every steps, oldest first, at most max_samples dicts as
    pic_energy returns."""
    buf = (pic_energy_t * max(max_samples, 1))()
    n = ctypes.c_int()
    _check(lib().pic_energy_history(h, buf, max_samples, ctypes.byref(n)), h)
    return [{"w_e": e.w_e, "w_b": e.w_b, "w_perp": e.w_perp, "k": e.k, "total": e.total, "np": e.np}
            for e in buf[:n.value]]


def pic_enable_timing(h, on: bool = True):
    """Turns per-kernel-class CUDA-event timing of the handle's launches on (resetting the totals) or off."""
    _check(lib().pic_enable_timing(h, 1 if on else 0), h)


def pic_kernel_times(h):
    """Device milliseconds and launch counts per kernel class since timing was enabled: {class: (ms, launches)}."""
    ms = (ctypes.c_double * PIC_NKERNEL)()
    cnt = (ctypes.c_longlong * PIC_NKERNEL)()
    _check(lib().pic_kernel_times(h, ms, cnt), h)
    return {KERNEL_CLASSES[i]: (ms[i], cnt[i]) for i in range(PIC_NKERNEL)}


def pic_launch_count(h) -> int:
    """Number of kernel launches the handle has made since it was created."""
    n = ctypes.c_longlong()
    _check(lib().pic_launch_count(h, ctypes.byref(n)), h)
    return n.value


def pic_field_energy_noalloc(fields, ncell: int, precision: int, dv: float, stream_ptr=None):
    """W_E, W_B, W_perp of six device arrays, computed without allocating (see include/pic.h)."""
    arr = (ctypes.c_void_p * 6)(*[_ptr(f) if not isinstance(f, int) else f for f in fields])
    out = (ctypes.c_double * 3)()
    _check(lib().pic_field_energy_noalloc(arr, int(ncell), int(precision), float(dv), out, stream_ptr))
    return out[0], out[1], out[2]


# ------------------------------------------------------------------------------------------------
# adjoint
# ------------------------------------------------------------------------------------------------
def pic_adjoint_forward(h, nsteps: int, checkpoint_every: int = 10) -> float:
    """Runs nsteps recording checkpoints; returns W_perp after them."""
    w = ctypes.c_double()
    _check(lib().pic_adjoint_forward(h, int(nsteps), int(checkpoint_every), ctypes.byref(w)), h)
    return w.value


def pic_adjoint_backward(h, dw: float = 1.0, grad_fields=None):
    """Gradient of dw * W_perp(T): returns (dPsi_E coefficients, dPsi_B coefficients) as numpy arrays
    and writes dE0, dB0 into grad_fields (six device tensors or addresses; None skips)."""
    ge = (ctypes.c_double * 5)()
    gb = (ctypes.c_double * 5)()
    gf = None
    if grad_fields is not None:
        gf = (ctypes.c_void_p * 6)(*[f if isinstance(f, int) or f is None else _ptr(f) for f in grad_fields])
    _check(lib().pic_adjoint_backward(h, float(dw), ge, gb, gf), h)
    return np.array(ge[:]), np.array(gb[:])


def pic_adjoint_release(h):
    """Frees the adjoint's checkpoints and work storage of the handle."""
    lib().pic_adjoint_release(h)


# ------------------------------------------------------------------------------------------------
# batched runs
# ------------------------------------------------------------------------------------------------
def _bcheck(rc, b):
    if rc != PIC_OK:
        msg = lib().pic_strerror(rc).decode()
        detail = lib().pic_batch_last_error(b).decode() if b is not None else ""
        raise PicError(rc, f"{msg}: {detail}" if detail else msg)


def pic_batch_create(cfgs):
    """Creates a batch of independent runs (a sequence of pic_config) advanced together by shared launches."""
    arr = (pic_config * len(cfgs))(*cfgs)
    b = ctypes.c_void_p()
    _check(lib().pic_batch_create(arr, len(cfgs), ctypes.byref(b)))
    return b


def pic_batch_size(b) -> int:
    """Number of runs in the batch."""
    return lib().pic_batch_size(b)


def pic_batch_run(b, run: int):
    """Handle of one run of the batch (owned by the batch) for state copies and energies between steps."""
    h = lib().pic_batch_run(b, run)
    if not h:
        raise PicError(PIC_E_ARG, "no such run")
    return ctypes.c_void_p(h)


def pic_batch_set_correction_stencil(b, run: int, psi_e=None, psi_b=None):
    """Sets the Psi_E / Psi_B coefficients of one run of the batch; both None turns its correction off."""
    pe = None if psi_e is None else (ctypes.c_double * 5)(*[float(v) for v in psi_e])
    pb = None if psi_b is None else (ctypes.c_double * 5)(*[float(v) for v in psi_b])
    _bcheck(lib().pic_batch_set_correction_stencil(b, run, pe, pb), b)


def pic_batch_set_stream(b, stream_ptr):
    """Queues the batch's later work on the cudaStream_t address stream_ptr (None: the batch's own stream)."""
    _bcheck(lib().pic_batch_set_stream(b, stream_ptr), b)


def pic_batch_step(b, nsteps: int = 1):
    """Advances every run of the batch nsteps time steps (a replayed CUDA graph per step)."""
    _bcheck(lib().pic_batch_step(b, int(nsteps)), b)


def pic_batch_sync(b):
    """Waits for the batch's stream and raises PicError on any kernel error."""
    _bcheck(lib().pic_batch_sync(b), b)


def pic_batch_energy_history(b, run: int, max_samples: int = 4096):
    """Energy samples of one run of the batch, oldest first, as pic_energy_history returns."""
    buf = (pic_energy_t * max(max_samples, 1))()
    n = ctypes.c_int()
    _bcheck(lib().pic_batch_energy_history(b, run, buf, max_samples, ctypes.byref(n)), b)
    return [{"w_e": e.w_e, "w_b": e.w_b, "w_perp": e.w_perp, "k": e.k, "total": e.total, "np": e.np}
            for e in buf[:n.value]]


def pic_batch_autotune(b, trial_steps: int = 3, ngroups: int = 8):
    """Times the lanes-per-cell and blocks-per-SM candidates of the persistent push for every group, keeps the
    fastest, resets every run to its seeded start; returns the chosen lanes per cell per group."""
    out = (ctypes.c_int * ngroups)()
    _bcheck(lib().pic_batch_autotune(b, int(trial_steps), out), b)
    return list(out)


def pic_batch_destroy(b):
    """Frees the batch and all its runs (None is a no-op)."""
    if b is not None:
        lib().pic_batch_destroy(b)
