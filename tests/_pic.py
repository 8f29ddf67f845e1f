"""Test helpers: build the same state in the oracle and in the CUDA handle, and compare them.

Only marshalling (absolute positions <-> cell index + offsets, full u <-> u - u0 z_hat) and
error norms live here.
"""
from __future__ import annotations

import math

import numpy as np

import oracle as O

try:
    import paper_1401_0838_gb300 as P
except Exception:  # the library may not be built on a CPU-only machine
    P = None


def make_cfg(ndim=2, nx=40, ny=1, nz=72, dt=0.5, gamma=130.0, scheme=0, precision=1, ppc=4, nbin=1, ncomp=1,
             calpha=3.0, targets=3, init_beam=0, track_ids=1, sigma_perp=0.0, seed=1, cap=0, dx=1.0, dy=1.0,
             dz=1.0, u_th=1e-4, order=1, corr_mode=0, solver=0, ck_beta=(0.125, 0.125)):
    return P.pic_config_default(ndim=ndim, nx=nx, ny=ny if ndim == 3 else 1, nz=nz, dt=dt, gamma=gamma,
                                scheme=scheme, precision=precision, ppc_per_species=ppc, filter_nbin=nbin,
                                filter_ncomp=ncomp, filter_comp_alpha=calpha, filter_targets=targets,
                                init_beam=init_beam, track_ids=track_ids, sigma_perp=sigma_perp, seed=seed,
                                bin_capacity=cap, dx=dx, dy=dy if ndim == 3 else 1.0, dz=dz, u_th=u_th,
                                shape_order=order, correction_mode=corr_mode, field_solver=solver,
                                ck_beta_x=ck_beta[0], ck_beta_z=ck_beta[1])


def oracle_for(cfg, psi_e=None, psi_b=None) -> O.Sim:
    return O.Sim(ndim=cfg.ndim, nx=cfg.nx, ny=cfg.ny, nz=cfg.nz, dx=cfg.dx, dy=cfg.dy, dz=cfg.dz, dt=cfg.dt,
                 scheme=cfg.scheme, psi_e=psi_e, psi_b=psi_b, f_nbin=cfg.filter_nbin, f_ncomp=cfg.filter_ncomp,
                 f_alpha=cfg.filter_comp_alpha, f_targets=cfg.filter_targets, order=cfg.shape_order,
                 corr_mode=cfg.correction_mode, solver=cfg.field_solver, ck_beta=(cfg.ck_beta_x, cfg.ck_beta_z))


def uniform_weight(cfg):
    wp = cfg.omega_p_dz / cfg.dz
    return wp * wp * cfg.dx * cfg.dy * cfg.dz / (2.0 * cfg.ppc_per_species)


def dtype_of(cfg):
    return np.float32 if cfg.precision == 0 else np.float64


def to_native(cfg, part: dict, u0: float) -> dict:
    """Absolute FP64 particles -> native arrays of the handle's precision."""
    T = dtype_of(cfg)
    nx, ny, nz = cfg.nx, cfg.ny, cfg.nz
    fx, fy, fz = np.floor(part["x"]), np.floor(part["y"]), np.floor(part["z"])
    i = fx.astype(np.int64) % nx
    j = (fy.astype(np.int64) % ny) if cfg.ndim == 3 else np.zeros_like(i)
    k = fz.astype(np.int64) % nz
    nat = {
        "cell": np.ascontiguousarray(((k * ny + j) * nx + i).astype(np.int32)),
        "species": np.ascontiguousarray((part["q"] > 0).astype(np.int32)),
        "ox": (part["x"] - fx).astype(T),
        "oy": (part["y"] - fy).astype(T) if cfg.ndim == 3 else None,
        "oz": (part["z"] - fz).astype(T),
        "dux": part["ux"].astype(T),
        "duy": part["uy"].astype(T),
        "duz": (part["uz"] - u0).astype(T),
        "w": part["w"].astype(T) if cfg.sigma_perp > 0 else None,
        "id": part["id"].astype(np.uint32),
    }
    return {k2: (np.ascontiguousarray(v) if v is not None else None) for k2, v in nat.items()}


def from_native(cfg, nat: dict, u0: float, w_const: float | None = None) -> dict:
    """Native arrays -> absolute FP64 particle dict (sorted by id)."""
    nx, ny = cfg.nx, cfg.ny
    cell = nat["cell"].astype(np.int64)
    i, j, k = cell % nx, (cell // nx) % ny, cell // (nx * ny)
    p = {
        "x": i + nat["ox"].astype(np.float64),
        "y": (j + nat["oy"].astype(np.float64)) if cfg.ndim == 3 else np.zeros(len(cell)),
        "z": k + nat["oz"].astype(np.float64),
        "ux": nat["dux"].astype(np.float64),
        "uy": nat["duy"].astype(np.float64),
        "uz": u0 + nat["duz"].astype(np.float64),
        "q": np.where(nat["species"] == 1, 1.0, -1.0),
        "id": nat["id"].astype(np.int64),
    }
    p["w"] = nat["w"].astype(np.float64) if nat.get("w") is not None else np.full(len(cell), w_const or 0.0)
    order = np.argsort(p["id"], kind="stable")
    return {k2: v[order] for k2, v in p.items()}


class Pair:
    """The same simulation in the oracle (FP64) and in a CUDA handle."""

    def __init__(self, cfg, psi=None, fields=None, part=None, handle=None):
        """handle: an existing handle (a run of a batch) whose correction stencil the caller has set;
        it is not destroyed by close()."""
        self.cfg = cfg
        self.T = dtype_of(cfg)
        self.u0 = math.sqrt(cfg.gamma ** 2 - 1.0)
        pe, pb = psi if psi is not None else (None, None)
        self.owns = handle is None
        self.h = P.pic_create(cfg) if handle is None else handle
        if pe is not None and self.owns:
            P.pic_set_correction_stencil(self.h, pe, pb)
        self.o = oracle_for(cfg, pe, pb)
        shape = self.o.shape
        if fields is None:
            fields = {n: np.zeros(shape) for n in ("ex", "ey", "ez", "bx", "by", "bz")}
        # round the shared initial state to the handle's precision once, and give the oracle the same values
        fn = {n: np.ascontiguousarray(fields[n].astype(self.T)) for n in ("ex", "ey", "ez", "bx", "by", "bz")}
        for n, a in fn.items():
            self.o.f[n] = np.ascontiguousarray(a.astype(np.float64).reshape(shape))
        if part is not None:
            part = dict(part)
            if cfg.sigma_perp <= 0:  # the handle's uniform beam weight
                part["w"] = np.full(len(part["x"]), uniform_weight(cfg))
            nat = to_native(cfg, part, self.u0)
            back = from_native(cfg, {k: v for k, v in nat.items()}, self.u0)
            if cfg.sigma_perp <= 0:
                back["w"] = part["w"][np.argsort(part["id"], kind="stable")].copy()
            self.o.set_particles(back["x"], back["y"] if cfg.ndim == 3 else None, back["z"], back["ux"], back["uy"],
                                 back["uz"], back["w"], back["q"], pid=back["id"])
            P.pic_set_state(self.h, P.make_state(P.PIC_HOST, fn, nat))
        else:
            P.pic_set_state(self.h, P.make_state(P.PIC_HOST, fn, None))
        self.npart = 0 if part is None else len(part["x"])

    def close(self):
        if self.owns:
            P.pic_destroy(self.h)
        self.h = None

    def step(self, n=1):
        P.pic_step(self.h, n)
        self.o.step(n)

    def gpu_state(self):
        cfg = self.cfg
        shape = self.o.shape
        f = {n: np.zeros(shape, dtype=self.T) for n in ("ex", "ey", "ez", "bx", "by", "bz")}
        n = max(P.pic_num_particles(self.h), 1)
        nat = {"cell": np.zeros(n, np.int32), "species": np.zeros(n, np.int32), "id": np.zeros(n, np.uint32)}
        for k in ("ox", "oy", "oz", "dux", "duy", "duz", "w"):
            nat[k] = np.zeros(n, dtype=self.T)
        s = P.make_state(P.PIC_HOST, f, nat)
        s.np = n
        P.pic_get_state(self.h, s)
        m = s.np
        nat = {k: v[:m] for k, v in nat.items()}
        w_const = None
        part = from_native(cfg, nat, self.u0, w_const)
        return {k: v.astype(np.float64) for k, v in f.items()}, part


def rel_l2(a, b, floor=0.0):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = max(np.linalg.norm(b), floor)
    return np.linalg.norm(a - b) / den if den > 0 else np.linalg.norm(a - b)


def periodic_diff(a, b, n):
    d = (np.asarray(a) - np.asarray(b) + n / 2) % n - n / 2
    return d
