#!/usr/bin/env python
"""Throughput of the stabilised FDTD-Esirkepov PIC step (Godfrey & Vay, arXiv 1401.0838) on GB300.

Workload (one step = one pass of the whole hot path): 2D x-z periodic 512 x 1024 grid,
16 particles per cell per species (16,777,216 particles), gamma = 130 beam along +z,
c dt / dz = 0.5, Galerkin gather, Psi_E / Psi_B correction (Sec. 2) and the 3-pass filter
(2 bilinear + 1 compensation pass, a = 2, per direction) on the current and on the field copies,
FP32, seeded Philox beam; energies recorded on the device every step. Per step:
copy stencil -> fused gather/Boris/move/Esirkepov/rebin -> current filter -> Yee (3) -> energy.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: the path does not shard (one independent replica per GPU, no collective on the data
path); value = particles of all ranks x K / max-over-ranks time. Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import threading
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (gather+push+deposit+filter) and % HBM roofline, FP32 vs FP64"
UNIT = "particle-steps/s"
NX, NZ, PPC, ALPHA, GAMMA = 512, 1024, 16, 0.5, 130.0
FILTER = dict(filter_nbin=2, filter_ncomp=1, filter_comp_alpha=2.0)
WORKLOAD = ("2D x-z 512x1024 periodic beam, 16 particles/cell/species (16.8M particles), gamma=130, "
            "c dt/dz=0.5, Galerkin gather, Psi correction + 3-pass binomial/compensation filter, FP32")
# algorithmic bytes of the fused particle kernel (2D), per particle-step: the cell index, 2 offsets and
# 3 momenta read and written (48 B in FP32, 88 B in FP64); the storage keeps the cell index implicit
# in the per-cell bins, so what the layout must move is 40 B (80 B). Per cell: 6 field copies read,
# 3 currents written.
PUSH_BYTES_PER_PARTICLE = {4: 48, 8: 88}
PUSH_LAYOUT_BYTES_PER_PARTICLE = {4: 40, 8: 80}
PUSH_BYTES_PER_CELL = {4: 36, 8: 72}
FALLBACK_HBM_GBS = 6800.0


def config_dict(n_gpus: int, order: int = 1, scheme: str = "galerkin", solver: str = "yee",
                correction: str = "split") -> dict:
    wl = WORKLOAD
    if order != 1 or scheme != "galerkin":
        wl = wl.replace("Galerkin gather", f"{scheme} gather, shape order {order}")
    if solver != "yee":
        wl += ", Cole-Karkkainen solver"
    if correction != "split":
        wl += ", exact rational multiplier on the transverse E copies"
    return {"workload": wl, "grid": [NX, NZ], "ppc_per_species": PPC, "particles": NX * NZ * PPC * 2,
            "alpha": ALPHA, "gamma": GAMMA, "scheme": scheme, "shape_order": order, "solver": solver,
            "correction": correction,
            "filter": "2 bilinear + 1 compensation (a=2) per direction on J and on the field copies",
            "l2": "inputs larger than L2: 671 MB of particle state read + written per step (L2 129 MB)",
            "parallelism": "replicas" if n_gpus > 1 else "single"}


# ------------------------------------------------------------------------------------------------
# distributed helpers (used with NCCL on GPUs, tested with gloo on CPU)
# ------------------------------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), ws


def reduce_max(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(device=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        if device is not None and device.type == "cuda":
            dist.barrier(device_ids=[device.index])
        else:
            dist.barrier()


def aggregate(ms_local: float, units_local: float, steps: int, device=None) -> dict:
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    ms = reduce_max(ms_local, device)
    units = reduce_sum(units_local, device)
    return {"ms": ms, "units": units, "value": units * steps / (ms / 1e3) if ms > 0 else 0.0}


# ------------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        """Start sampling every 50 ms and return once the first sample is in, so that the samples
        collected until stop() fall inside the timed region (the first one is not counted)."""
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        box = []
        reader = threading.Thread(target=lambda: box.append(self.proc.stdout.readline()), daemon=True)
        reader.start()
        reader.join(timeout=10.0)

    def sample(self) -> str:
        """One synchronous sample (a CSV line), or "" when nvidia-smi is unavailable."""
        try:
            r = subprocess.run(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits", "-i",
                                str(self.gpu)], capture_output=True, text=True, timeout=20)
            return r.stdout.strip()
        except (OSError, subprocess.TimeoutExpired):
            return ""

    def stop(self, before: str = "", after: str = "") -> dict:
        """Samples of the stream, plus the synchronous `before` / `after` samples taken right around
        the timed region (a short region may hold no stream sample at all)."""
        if self.proc is None:
            out = ""
        else:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
        res = parse_clock_samples("\n".join(x for x in (before, out, after) if x))
        inside = parse_clock_samples(out)
        res["samples_inside"] = inside["samples"]
        res["sm_mhz_before"] = parse_clock_samples(before)["sm_mhz"]
        res["sm_mhz_after"] = parse_clock_samples(after)["sm_mhz"]
        if res["sm_mhz"] is None:
            res["reasons"] = res["reasons"] + ["nvidia-smi unavailable"]
        return res


def parse_clock_samples(text: str) -> dict:
    """Median SM clock, maximum clock and active throttle reasons from ClockSampler.QUERY CSV lines."""
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in text.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            mx = float(f[2])
        except ValueError:
            continue
        for nm, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
            "samples": len(sm)}


def profiled_traffic(prof=None, src=None):
    """DRAM bytes per launch of the push kernel from the committed ncu summary, if that summary was
    taken on the current kernel source (else None). src: a file or a list of files, hashed as one
    byte string in order (the push: its kernel file, then the header that fixes its tile shape)."""
    import hashlib
    prof = prof or os.path.join(ROOT, "profiles", "k_push_2d_512x1024_fp32.md")
    csrc = os.path.join(ROOT, "paper_1401_0838_gb300", "csrc")
    src = src or [os.path.join(csrc, "k_particles.cu"), os.path.join(csrc, "common.cuh")]
    files = [src] if isinstance(src, str) else list(src)
    try:
        text = open(prof).read()
        digest = hashlib.sha256(b"".join(open(f, "rb").read() for f in files)).hexdigest()
    except OSError:
        return None
    sha, traffic = None, None
    for line in text.splitlines():
        if line.startswith("source_sha256:"):
            sha = line.split(":", 1)[1].strip()
        if line.startswith("dram_bytes_per_launch:"):
            traffic = float(line.split(":", 1)[1].strip())
    return traffic if sha == digest else None


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
SCHEMES = {"galerkin": 0, "uniform": 1, "momentum": 2}


def make_handle(P, precision: int, seed: int, stream_ptr, order: int = 1, scheme: str = "galerkin",
                solver: str = "yee", correction: str = "split"):
    sc = SCHEMES[scheme]
    cfg = P.pic_config_default(nx=NX, nz=NZ, dt=ALPHA, gamma=GAMMA, scheme=sc, precision=precision,
                               ppc_per_species=PPC, seed=seed, init_beam=1, diag_every=1, shape_order=order,
                               field_solver=P.PIC_CK if solver == "ck" else P.PIC_YEE,
                               correction_mode=P.PIC_CORR_RATIONAL if correction == "rational" else P.PIC_CORR_SPLIT,
                               **FILTER)
    h = P.pic_create(cfg)
    pe, pb = P.pic_compute_correction_coeffs(sc, ALPHA)
    P.pic_set_correction_stencil(h, pe, pb)
    P.pic_set_stream(h, stream_ptr)
    return h, cfg


def timed_steps(P, torch, h, stream, steps: int, device):
    """Device time of `steps` whole steps run by one pic_step call (CUDA events on the launching
    stream; the library replays its captured step graph), then per-kernel times from a second,
    separately timed pass of `steps` single steps with event-bracketed launches: per kernel class,
    the median over the steps of its time in one step (so one stray slow launch does not move it),
    returned as (median x steps, launches)."""
    l0 = P.pic_launch_count(h)
    barrier(device)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    P.pic_step(h, steps)
    e1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    barrier(device)
    ms = e0.elapsed_time(e1)
    launches = P.pic_launch_count(h) - l0
    P.pic_sync(h)
    per_step = []
    for _ in range(steps):
        P.pic_enable_timing(h, True)  # resets the totals
        P.pic_step(h, 1)
        P.pic_sync(h)
        per_step.append(P.pic_kernel_times(h))
    P.pic_enable_timing(h, False)
    kt = median_kernel_times(per_step)
    return ms, kt, launches


def warm_up(P, h, n: int):
    """n untimed steps (at least 4) in one pic_step call: besides warming up, it captures the step
    graph that the timed call then replays (a call of fewer than two graphs' worth of steps runs
    single steps, and a timed call would otherwise capture the graph inside its timed region)."""
    P.pic_step(h, max(n, 4))


def bin_stats(P, h) -> dict:
    """Slots per cell and species, and particles sent through the spill list so far (full bins)."""
    cap, spilled = P.pic_bin_stats(h)
    return {"capacity": cap, "spilled": spilled}


def median_kernel_times(per_step: list) -> dict:
    """{class: (median over steps of the class's ms in a step x steps, launches over all steps)}."""
    out = {}
    for k in per_step[0]:
        ms = sorted(t[k][0] for t in per_step)
        n = len(ms)
        med = ms[n // 2] if n % 2 else 0.5 * (ms[n // 2 - 1] + ms[n // 2])
        out[k] = (med * n, sum(t[k][1] for t in per_step))
    return out


def push_time_in_step(kt: dict, step_ms: float):
    """The push kernel's time inside the graph-replayed step: the step's time less the event-timed
    times of every other kernel of a step (gaps between launches count against the push)."""
    ms, cnt = kt["push"]
    if not cnt or step_ms is None:
        return None
    others = sum(v[0] for k, v in kt.items() if k != "push") / cnt  # one push per step in the timed pass
    t = step_ms - others
    return t if t > 0 else None


def roofline(kt: dict, np_: int, ncell: int, es: int, peak: float, peak_kind: str, traffic=None,
             step_ms=None) -> dict:
    ms, cnt = kt["push"]
    ev_s = ms / 1e3 / max(cnt, 1)
    in_step = push_time_in_step(kt, step_ms)
    per_launch_s = in_step / 1e3 if in_step else ev_s
    bytes_per_launch = np_ * PUSH_BYTES_PER_PARTICLE[es] + ncell * PUSH_BYTES_PER_CELL[es]
    layout_bytes = np_ * PUSH_LAYOUT_BYTES_PER_PARTICLE[es] + ncell * PUSH_BYTES_PER_CELL[es]
    achieved = bytes_per_launch / per_launch_s / 1e9 if per_launch_s > 0 else 0.0
    achieved_layout = layout_bytes / per_launch_s / 1e9 if per_launch_s > 0 else 0.0
    return {"kernel": "k_push (fused gather + Boris + move + Esirkepov + rebin)", "bound": "hbm",
            "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "peak_source": f"{peak_kind} hbm_gbs", "traffic": traffic, "algorithmic_bytes_per_launch": bytes_per_launch,
            "bytes_basis": f"{PUSH_BYTES_PER_PARTICLE[es]} B/particle (cell index + offsets + momenta, each way) + "
                           f"{PUSH_BYTES_PER_CELL[es]} B/cell (6 field copies read, 3 currents written)",
            "frac_layout_bytes": round(achieved_layout / peak, 4),
            "layout_bytes_per_launch": layout_bytes,
            "launch_ms": round(per_launch_s * 1e3, 4), "launch_ms_events": round(ev_s * 1e3, 4),
            "time_basis": ("graph-replayed step time less the event-timed other kernels of a step" if in_step
                           else "event-bracketed launches")}


def e2e_measure(P, torch, h, cfg, stream, steps: int):
    """Same metric through the C ABI with host buffers: per step, the full state goes host -> device
    from pinned memory (pic_set_state), one step runs, and the step's energy sample comes back."""
    import numpy as np
    ncell = cfg.nx * cfg.ny * cfg.nz
    n = P.pic_num_particles(h)
    pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True)
    f = {k: pin((ncell,), torch.float32) for k in ("ex", "ey", "ez", "bx", "by", "bz")}
    part = {"cell": pin((n,), torch.int32), "species": pin((n,), torch.int32)}
    for k in ("ox", "oz", "dux", "duy", "duz"):
        part[k] = pin((n,), torch.float32)
    s = P.make_state(P.PIC_HOST, f, part)
    s.np = n
    P.pic_get_state(h, s)
    state_in = P.make_state(P.PIC_HOST, f, part)
    state_in.np = n
    h2d = 6 * ncell * 4 + n * (4 + 4 + 5 * 4)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        P.pic_set_state(h, state_in)
        P.pic_step(h, 1)
        hist = P.pic_energy_history(h, 1)
        times.append(time.perf_counter() - t0)
        assert hist and hist[-1]["np"] == n
    t = statistics.median(times)
    return {"value": n / t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 48,
            "ms_per_step": round(t * 1e3, 3), "how": "pic_set_state (pinned host) + pic_step(1) + "
                                                      "pic_energy_history(1), median of steps"}


# ------------------------------------------------------------------------------------------------
# oracle (CPU baseline and reference arm)
# ------------------------------------------------------------------------------------------------
SAMPLE_NZ = 64  # the CPU sample is a 512 x 64 slab of the same beam (1/16 of the box)


def oracle_sample(nz: int = SAMPLE_NZ, seed: int = 2):
    import oracle as O
    st, pe, pb = O.rational_coeffs(O.GALERKIN, ALPHA)
    sim = O.Sim(ndim=2, nx=NX, nz=nz, dt=ALPHA, scheme=O.GALERKIN, psi_e=pe, psi_b=pb,
                f_nbin=FILTER["filter_nbin"], f_ncomp=FILTER["filter_ncomp"], f_alpha=FILTER["filter_comp_alpha"],
                f_targets=3)
    sim.init_beam(ppc=PPC, gamma=GAMMA, seed=seed)
    return sim


def host_threads() -> int:
    """Cores this process may run on: its CPU affinity, capped by a cgroup v2 CPU quota if one is set."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    try:
        with open("/sys/fs/cgroup/cpu.max") as f:
            cap = cgroup_cpu_limit(f.read())
    except OSError:
        cap = None
    return min(n, cap) if cap else n


def cgroup_cpu_limit(text: str):
    """Whole cores allowed by a cgroup v2 cpu.max line ("quota period"; "max" = no limit), else None."""
    parts = text.split()
    if len(parts) < 2 or parts[0] == "max":
        return None
    try:
        return max(1, int(parts[0]) // int(parts[1]))
    except ValueError:
        return None


def oracle_sample_3d(nz: int = 8, seed: int = 3):
    """A 128 x 128 x nz slab of the 3D workload: 8 particles/cell/species, transverse Gaussian weights
    (sigma 20 cells), gamma 130, c dt/dz 0.5, Galerkin, correction + filter (1, 1, a = 3)."""
    import oracle as O
    st, pe, pb = O.rational_coeffs(O.GALERKIN, 0.5)
    sim = O.Sim(ndim=3, nx=128, ny=128, nz=nz, dt=0.5, scheme=O.GALERKIN, psi_e=pe, psi_b=pb, f_nbin=1,
                f_ncomp=1, f_alpha=3.0, f_targets=3)
    sim.init_beam(ppc=8, gamma=130.0, sigma_perp=20.0, seed=seed)
    return sim


def oracle_time(steps: int, warmup: int, nz: int = SAMPLE_NZ, threads: int = 1, sample=None):
    """Wall time of each of `steps` oracle steps (+ energies) of `threads` independent slabs of the beam
    (seeds 2, 3, ...; `sample(nz, seed)` builds one, default the 2D workload's), one slab per host
    thread; the oracle is one C call per step and releases the GIL, so the slabs run concurrently.
    Returns (particles over all slabs, per-step seconds)."""
    from concurrent.futures import ThreadPoolExecutor

    sample = sample or oracle_sample

    def one(sim):
        sim.step(1)
        sim.energy()

    with ThreadPoolExecutor(max_workers=threads) as ex:
        sims = list(ex.map(lambda k: sample(nz, seed=2 + k), range(threads)))
        for _ in range(warmup):
            list(ex.map(one, sims))
        times = []
        for _ in range(steps):
            t0 = time.perf_counter()
            list(ex.map(one, sims))
            times.append(time.perf_counter() - t0)
    return sum(s.n for s in sims), times


def cpu_baseline(steps: int = 8, threads: int = 0) -> dict:
    threads = threads if threads > 0 else host_threads()
    n1, t1 = oracle_time(steps, 1)
    one = n1 / (sum(t1) / len(t1))
    n, times = oracle_time(steps, 1, threads=threads) if threads > 1 else (n1, t1)
    value = n / (sum(times) / len(times))
    return {"value": value, "unit": UNIT, "cores": threads, "host_cores": os.cpu_count(), "kind": "oracle",
            "one_thread": one,
            "sample": f"FP64 C oracle on {threads} host threads, each its own 512x{SAMPLE_NZ} slab of the same beam "
                      f"(seeds 2..{1 + threads}; {n1} particles a slab, same density, gamma, alpha, correction and "
                      f"filter): {steps} steps + energies each, all slabs concurrently; one_thread = one slab alone"}


def run_reference(args):
    rank, _, ws = dist_env()
    if rank != 0:
        return
    steps, warmup = max(args.steps, 1), max(args.warmup, 0)
    threads = args.cpu_threads if args.cpu_threads > 0 else host_threads()
    # one oracle step of a 512 x 64 slab takes about 0.5 s (every thread its own slab, concurrently):
    # past 400 steps the slabs shrink so that the whole run stays near two minutes (the unit is per
    # particle-step either way)
    nz = SAMPLE_NZ if steps + warmup <= 400 else max(8, SAMPLE_NZ * 400 // (steps + warmup) // 8 * 8)
    n, times = oracle_time(steps, warmup, nz, threads=threads)
    total = sum(times)
    value = n * steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warmup, "ms_per_step": total / steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "host_cores": os.cpu_count(),
                             "kind": "oracle",
                             "sample": f"each step: one FP64 oracle step + energies of {threads} independent "
                                       f"512x{nz} slabs of the workload ({n} particles in all), one per host "
                                       f"thread, concurrently"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_1401_0838_gb300 as P

    rank, local, ws = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group("nccl", device_id=device)
    P.lib()
    stream = torch.cuda.Stream(device=device)
    peak, peak_kind = measured_hbm_peak()

    # FP32: the headline
    h, cfg = make_handle(P, P.PIC_FP32, seed=2 + rank, stream_ptr=stream.cuda_stream, order=args.order,
                         scheme=args.scheme, solver=args.solver, correction=args.correction)
    ncell = cfg.nx * cfg.ny * cfg.nz
    np_ = P.pic_num_particles(h)
    with torch.cuda.stream(stream):
        warm_up(P, h, args.warmup)
    P.pic_sync(h)
    clocks = ClockSampler(local)
    before = clocks.sample()
    clocks.start()
    ms, kt, launches = timed_steps(P, torch, h, stream, args.steps, device)
    clk = clocks.stop(before, clocks.sample())
    hist = P.pic_energy_history(h, 1)
    assert hist and hist[-1]["np"] == np_, "particle count changed"
    bins = bin_stats(P, h)
    agg = aggregate(ms, np_, args.steps, device)
    cells = aggregate(ms, ncell, args.steps, device)
    launches_all = int(reduce_sum(launches, device))
    traffic = args.traffic if args.traffic is not None else (
        profiled_traffic() if args.order == 1 and args.scheme == "galerkin" else None)
    rf = roofline(kt, np_, ncell, 4, peak, peak_kind, traffic=traffic, step_ms=ms / args.steps)
    kernel_ms = {k: round(v[0] / max(v[1], 1), 4) for k, v in kt.items() if v[1]}

    e2e = None
    if not args.no_e2e:
        e2e = e2e_measure(P, torch, h, cfg, stream, args.e2e_steps)
        e2e_all = aggregate(e2e["ms_per_step"] * args.e2e_steps, np_, args.e2e_steps, device)
        e2e["value"] = e2e_all["value"]
    P.pic_destroy(h)

    # FP64 on the same workload (the metric compares the two precisions)
    fp64 = None
    if args.fp64_steps > 0:
        h64, _ = make_handle(P, P.PIC_FP64, seed=2 + rank, stream_ptr=stream.cuda_stream, order=args.order,
                             scheme=args.scheme, solver=args.solver, correction=args.correction)
        warm_up(P, h64, 2)
        P.pic_sync(h64)
        ms64, kt64, _ = timed_steps(P, torch, h64, stream, args.fp64_steps, device)
        a64 = aggregate(ms64, np_, args.fp64_steps, device)
        fp64 = {"value": a64["value"], "unit": UNIT, "ms_per_step": a64["ms"] / args.fp64_steps,
                "roofline": roofline(kt64, np_, ncell, 8, peak, peak_kind, step_ms=ms64 / args.fp64_steps)}
        P.pic_destroy(h64)

    line = {"metric": METRIC, "value": agg["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": agg["ms"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_dict(ws, args.order, args.scheme, args.solver, args.correction), "roofline": rf, "kernel_ms_per_launch": kernel_ms,
            "cell_updates_per_s": cells["value"], "fp64": fp64, "e2e": e2e, "gpu_launches": launches_all,
            "bins": bins,
            "clocks": clk}
    if rank == 0 and ws == 1 and not args.no_extras:
        # the other workloads, each measured here so that every one has a record from the same run
        line["config1"] = measure_config1(P, torch, 200, 5)
        line["config3d"] = measure_3d(P, torch, 10, 3, peak, peak_kind)
        line["sweep"] = measure_sweep(P, torch, 64, 20, 10)
        line["adjoint"] = measure_adjoint(P, torch, 100, 1, fd=True)
    if rank == 0 and ws == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(args.cpu_steps, args.cpu_threads)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist.is_initialized():
        barrier(device)
        dist.destroy_process_group()


# ------------------------------------------------------------------------------------------------
# batched sweep (64 independent 2D runs; not the default workload)
# ------------------------------------------------------------------------------------------------
def sweep_configs(P, nruns=64, seed=4):
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nruns):
        nx = int(rng.choice([64, 128, 256]))
        nz = int(rng.choice([128, 256, 512, 1024]))
        ppc = int(rng.choice([4, 8, 16]))
        alpha = float(rng.uniform(0.1, 0.7))
        gamma = float(rng.choice([10.0, 50.0, 130.0]))
        corr = bool(rng.integers(0, 2))
        c = P.pic_config_default(nx=nx, nz=nz, dt=alpha, gamma=gamma, scheme=P.PIC_GALERKIN, precision=P.PIC_FP32,
                                 ppc_per_species=ppc, seed=100 + i, init_beam=1, diag_every=10, **FILTER)
        out.append((c, corr))
    return out


def measure_sweep(P, torch, nruns: int, steps: int, seq_steps: int, autotune: bool = True) -> dict:
    """The batched sweep (one persistent push launch per lanes-per-cell group per step, replayed from a
    CUDA graph) against the same runs stepped one after another with plain per-step launches."""
    import numpy as np
    stream = torch.cuda.Stream()
    runs = sweep_configs(P, nruns)
    cfgs = [c for c, _ in runs]
    particles = sum(c.nx * c.nz * c.ppc_per_species * 2 for c in cfgs)
    b = P.pic_batch_create(cfgs)
    P.pic_batch_set_stream(b, stream.cuda_stream)
    skipped = 0
    for i, (c, corr) in enumerate(runs):
        if corr:
            try:  # inside a breakdown window of the interpolation the run goes uncorrected
                coeffs = P.pic_compute_correction_coeffs(P.PIC_GALERKIN, c.dt)
            except P.PicError:
                runs[i] = (c, False)
                skipped += 1
                continue
            P.pic_batch_set_correction_stencil(b, i, *coeffs)
    lpcs = P.pic_batch_autotune(b, trial_steps=2) if autotune else None
    P.pic_batch_step(b, 10)  # warm-up (includes the graph capture)
    P.pic_batch_sync(b)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    P.pic_batch_step(b, steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1)
    P.pic_batch_sync(b)
    rates = []
    for i, c in enumerate(cfgs):
        w = [e["w_perp"] for e in P.pic_batch_energy_history(b, i)]
        t = np.arange(1, len(w) + 1) * 10 * c.dt
        try:
            rates.append(P.pic_fit_growth_rate(t, w)[0])
        except P.PicError:
            rates.append(float("nan"))
    P.pic_batch_destroy(b)
    # the same runs one after another, each with plain per-step launches
    handles = []
    for c, corr in runs:
        h = P.pic_create(c)
        P.pic_set_stream(h, stream.cuda_stream)
        if corr:
            P.pic_set_correction_stencil(h, *P.pic_compute_correction_coeffs(P.PIC_GALERKIN, c.dt))
        P.pic_step(h, 1)
        handles.append(h)
    torch.cuda.synchronize()
    e0.record(stream)
    for h in handles:
        for _ in range(seq_steps):
            P.pic_step(h, 1)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    for h in handles:
        P.pic_destroy(h)
    vb = particles * steps / (ms_b / 1e3)
    vs = particles * seq_steps / (ms_s / 1e3)
    finite = [r for r in rates if r == r]
    return {"value": vb, "unit": UNIT, "steps": steps, "ms_per_step": ms_b / steps, "runs": len(runs),
            "particles": particles,
            "workload": f"batched sweep: {len(runs)} independent 2D runs, grids 64-256 x 128-1024 (seeded mix), "
                        "4-16 particles/cell/species, c dt/dz U[0.1,0.7), gamma in {10,50,130}, correction on/off, "
                        "FP32, one persistent push launch per lanes-per-cell group per step, CUDA graph",
            "sequential": {"value": vs, "unit": UNIT, "steps": seq_steps, "ms_per_step": ms_s / seq_steps,
                           "how": "each run alone, pic_step(1) per step (plain launches), runs one after another"},
            "speedup_vs_sequential": vb / vs, "autotune_lanes_per_cell": lpcs,
            "corrections_skipped_in_breakdown_windows": skipped,
            "growth_rates": {"min": float(min(finite)), "median": float(np.median(finite)),
                             "max": float(max(finite))} if finite else None}


def run_sweep(args):
    import torch

    import paper_1401_0838_gb300 as P
    torch.cuda.set_device(0)
    m = measure_sweep(P, torch, args.sweep_runs, args.steps, max(2, min(args.steps, args.sweep_seq_steps)))
    line = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": 10,
            "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": m["workload"], "runs": m["runs"], "particles": m["particles"]},
            "sequential": m["sequential"], "speedup_vs_sequential": m["speedup_vs_sequential"],
            "autotune_lanes_per_cell": m["autotune_lanes_per_cell"],
            "corrections_skipped_in_breakdown_windows": m["corrections_skipped_in_breakdown_windows"],
            "growth_rates": m["growth_rates"]}
    print(json.dumps(line), flush=True)


def measure_adjoint(P, torch, nsteps: int = 100, reps: int = 1, fd: bool = True) -> dict:
    """Adjoint of the 2D step on 256 x 512, 8 particles/cell/species, gamma 130, `nsteps` steps with a
    checkpoint every 10: the time of the forward run with checkpoints and of the backward pass
    against the plain forward run, and the Psi_E gradient against central differences (h = 1e-3) of
    the FP64 forward run."""
    import numpy as np
    every, alpha = 10, 0.5
    pe, pb = P.pic_compute_correction_coeffs(P.PIC_GALERKIN, alpha)

    def cfg(prec):
        return P.pic_config_default(nx=256, nz=512, dt=alpha, gamma=130.0, precision=prec, ppc_per_species=8,
                                    init_beam=1, track_ids=1, seed=5)

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    def w_after(prec, a_e):
        h = P.pic_create(cfg(prec))
        P.pic_set_correction_stencil(h, a_e, pb)
        P.pic_step(h, nsteps)
        w = P.pic_energy(h)["w_perp"]
        P.pic_destroy(h)
        return w

    res = {}
    for prec, name in ((P.PIC_FP32, "f32"), (P.PIC_FP64, "f64")):
        rs = []
        for _ in range(max(1, reps)):
            h = P.pic_create(cfg(prec))
            P.pic_set_correction_stencil(h, pe, pb)
            P.pic_sync(h)  # the library's stream is synchronised by every call that returns data
            w, t_f = timed(lambda: P.pic_adjoint_forward(h, nsteps, every))
            (ge, gb), t_b = timed(lambda: P.pic_adjoint_backward(h, 1.0))
            P.pic_destroy(h)
            h = P.pic_create(cfg(prec))
            P.pic_set_correction_stencil(h, pe, pb)
            P.pic_sync(h)
            _, t_p = timed(lambda: (P.pic_step(h, nsteps), P.pic_sync(h)))
            P.pic_destroy(h)
            rs.append((t_f, t_b, t_p))
        t_f, t_b, t_p = (float(np.median([r[i] for r in rs])) for i in range(3))
        res[name] = {"w_perp": w, "grad_psi_e": ge.tolist(), "grad_psi_b": gb.tolist(), "ms_forward_checkpointed": t_f,
                     "ms_backward": t_b, "ms_plain_forward": t_p, "adjoint_over_forward": (t_f + t_b) / t_p}
    fdv = None
    if fd:
        fdv = []
        for n in range(5):
            d = np.zeros(5)
            d[n] = 1e-3
            fdv.append((w_after(P.PIC_FP64, pe + d) - w_after(P.PIC_FP64, pe - d)) / 2e-3)
        fdv = np.array(fdv)
        for name in ("f32", "f64"):
            ge = np.array(res[name]["grad_psi_e"])
            res[name]["max_rel_err_vs_central_differences"] = float(np.abs(ge - fdv).max() / np.abs(fdv).max())
    np_ = 256 * 512 * 8 * 2
    r32 = res["f32"]
    return {"value": np_ * nsteps / ((r32["ms_forward_checkpointed"] + r32["ms_backward"]) / 1e3),
            "unit": "particle-steps/s through forward + adjoint", "steps": nsteps, "particles": np_,
            "workload": "adjoint: 2D 256x512, 8 particles/cell/species (2,097,152 particles), gamma 130, c dt/dz "
                        f"0.5, Galerkin, correction + filter (1,1,a=3), {nsteps} steps, checkpoint every 10; "
                        "gradient of W_perp(T) w.r.t. Psi_E, Psi_B and E0/B0",
            "central_differences": None if fdv is None else
            {"h": 1e-3, "forward": "FP64 library run", "grad_psi_e": fdv.tolist()},
            "f32": r32, "f64": res["f64"]}


def run_adjoint(args):
    import torch

    import paper_1401_0838_gb300 as P
    torch.cuda.set_device(0)
    m = measure_adjoint(P, torch, args.adjoint_steps, args.adjoint_reps, fd=not args.no_fd)
    r32 = m["f32"]
    line = {"metric": "particle-steps/s through forward + adjoint (gradient of W_perp(T))", "value": m["value"],
            "unit": "particle-steps/s", "n_gpus": 1, "steps": m["steps"], "warmup": 0,
            "ms_per_step": (r32["ms_forward_checkpointed"] + r32["ms_backward"]) / m["steps"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": m["workload"], "central_differences": m["central_differences"]},
            "f32": r32, "f64": m["f64"]}
    print(json.dumps(line), flush=True)


# 3D bytes per particle-step: cell index, 3 offsets, 3 momenta and the weight, each way (survey's 64 B);
# the per-cell bins keep the cell index implicit (56 B)
PUSH3D_BYTES_PER_PARTICLE, PUSH3D_LAYOUT_BYTES_PER_PARTICLE = 64, 56


def measure_3d(P, torch, steps: int, warmup: int, peak: float, peak_kind: str, nz: int = 512,
               nxy: int = 128) -> dict:
    """The 3D workload: 128 x 128 x 512, 8 particles/cell/species (134,217,728 particles), transverse
    Gaussian weights (sigma 20 cells), gamma 130, c dt/dz 0.5, Galerkin, correction + filter
    (1, 1, a = 3), FP32. Same timing as the default line; roofline with the 3D bytes per particle."""
    device = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream()
    cfg = P.pic_config_default(ndim=3, nx=nxy, ny=nxy, nz=nz, dt=0.5, gamma=130.0, scheme=P.PIC_GALERKIN,
                               precision=P.PIC_FP32, ppc_per_species=8, sigma_perp=20.0, seed=3, init_beam=1,
                               diag_every=1)
    h = P.pic_create(cfg)
    P.pic_set_stream(h, stream.cuda_stream)
    P.pic_set_correction_stencil(h, *P.pic_compute_correction_coeffs(P.PIC_GALERKIN, 0.5))
    ncell = cfg.nx * cfg.ny * cfg.nz
    np_ = P.pic_num_particles(h)
    with torch.cuda.stream(stream):
        warm_up(P, h, warmup)
    P.pic_sync(h)
    clocks = ClockSampler(device.index)
    before = clocks.sample()
    clocks.start()
    ms, kt, launches = timed_steps(P, torch, h, stream, steps, device)
    clk = clocks.stop(before, clocks.sample())
    hist = P.pic_energy_history(h, 1)
    assert hist and hist[-1]["np"] == np_, "particle count changed"
    bins = bin_stats(P, h)
    P.pic_destroy(h)
    ev_s = kt["push"][0] / 1e3 / max(kt["push"][1], 1)
    in_step = push_time_in_step(kt, ms / steps)
    per_launch_s = in_step / 1e3 if in_step else ev_s
    bytes_per_launch = np_ * PUSH3D_BYTES_PER_PARTICLE + ncell * 36
    layout_bytes = np_ * PUSH3D_LAYOUT_BYTES_PER_PARTICLE + ncell * 36
    achieved = bytes_per_launch / per_launch_s / 1e9
    return {"value": np_ * steps / (ms / 1e3), "unit": UNIT, "steps": steps, "warmup": warmup,
            "ms_per_step": ms / steps, "particles": np_,
            "workload": f"3D {nxy}x{nxy}x{nz}, 8 particles/cell/species ({np_} particles), Gaussian transverse weights "
                        "sigma 20 cells, gamma 130, c dt/dz 0.5, Galerkin, correction + filter (1,1,a=3), FP32",
            "roofline": {"kernel": "k_push", "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                         "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": f"{peak_kind} hbm_gbs",
                         "algorithmic_bytes_per_launch": bytes_per_launch,
                         "frac_layout_bytes": round(layout_bytes / per_launch_s / 1e9 / peak, 4),
                         "launch_ms": round(per_launch_s * 1e3, 4), "launch_ms_events": round(ev_s * 1e3, 4)},
            "bins": bins,
            "kernel_ms_per_launch": {k: round(v[0] / max(v[1], 1), 4) for k, v in kt.items() if v[1]},
            "cell_updates_per_s": ncell * steps / (ms / 1e3), "gpu_launches": launches, "clocks": clk}


def run_3d(args):
    import torch

    import paper_1401_0838_gb300 as P
    torch.cuda.set_device(0)
    peak, peak_kind = measured_hbm_peak()
    m = measure_3d(P, torch, args.steps, args.warmup, peak, peak_kind, nz=args.config3d_nz, nxy=args.config3d_nxy)
    line = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": m["workload"], "particles": m["particles"]}, "roofline": m["roofline"],
            "kernel_ms_per_launch": m["kernel_ms_per_launch"], "cell_updates_per_s": m["cell_updates_per_s"],
            "gpu_launches": m["gpu_launches"], "bins": m["bins"], "clocks": m["clocks"]}
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline_3d(args.cpu_steps_3d, args.cpu_threads)
    print(json.dumps(line), flush=True)


def measure_config1(P, torch, steps: int, warmup: int) -> dict:
    """The small 2D workload: 64 x 128, 4 particles/cell/species (65,536 particles), gamma 130,
    c dt/dz 0.5, Galerkin, correction + filter (1, 1, a = 3), FP64, energies every step, the steps
    replayed from the step graph. Its 7 MB stay in L2, so it is bound by launch latency: microseconds
    and launches per step, not an HBM roofline."""
    device = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream()
    cfg = P.pic_config_default(nx=64, nz=128, dt=0.5, gamma=130.0, scheme=P.PIC_GALERKIN, precision=P.PIC_FP64,
                               ppc_per_species=4, seed=1, init_beam=1, diag_every=1)
    h = P.pic_create(cfg)
    P.pic_set_stream(h, stream.cuda_stream)
    P.pic_set_correction_stencil(h, *P.pic_compute_correction_coeffs(P.PIC_GALERKIN, 0.5))
    np_ = P.pic_num_particles(h)
    with torch.cuda.stream(stream):
        warm_up(P, h, warmup)
    P.pic_sync(h)
    clocks = ClockSampler(device.index)
    before = clocks.sample()
    clocks.start()
    ms, kt, launches = timed_steps(P, torch, h, stream, steps, device)
    clk = clocks.stop(before, clocks.sample())
    P.pic_destroy(h)
    return {"value": np_ * steps / (ms / 1e3), "unit": UNIT, "steps": steps, "warmup": warmup,
            "ms_per_step": ms / steps, "particles": np_,
            "workload": "2D 64x128, 4 particles/cell/species (65,536 particles), gamma 130, c dt/dz 0.5, Galerkin, "
                        "correction + filter (1,1,a=3), FP64, energies every step",
            "l2": "L2 resident (7 MB): bound by launch latency, no flush",
            "us_per_step": 1e3 * ms / steps, "launches_per_step": launches / steps,
            "kernel_ms_per_launch": {k: round(v[0] / max(v[1], 1), 4) for k, v in kt.items() if v[1]},
            "cell_updates_per_s": 64 * 128 * steps / (ms / 1e3), "gpu_launches": launches, "clocks": clk}


def run_config1(args):
    """The small 64 x 128 FP64 workload alone, beside the oracle running the whole workload."""
    import torch

    import paper_1401_0838_gb300 as P
    torch.cuda.set_device(0)
    m = measure_config1(P, torch, args.steps, args.warmup)
    line = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": m["workload"], "particles": m["particles"], "l2": m["l2"]},
            "us_per_step": m["us_per_step"], "launches_per_step": m["launches_per_step"],
            "kernel_ms_per_launch": m["kernel_ms_per_launch"], "cell_updates_per_s": m["cell_updates_per_s"],
            "gpu_launches": m["gpu_launches"], "clocks": m["clocks"]}
    if not args.no_cpu:
        line["cpu_baseline"] = oracle_config1(args.cpu_steps_c1)
    print(json.dumps(line), flush=True)


def oracle_config1(steps: int = 200) -> dict:
    """The oracle running the whole 64 x 128 FP64 workload of run_config1 for `steps` steps (+ energies
    each step) on one thread: a single run does not split over threads."""
    import oracle as O
    st, pe, pb = O.rational_coeffs(O.GALERKIN, 0.5)
    sim = O.Sim(ndim=2, nx=64, nz=128, dt=0.5, scheme=O.GALERKIN, psi_e=pe, psi_b=pb, f_nbin=1, f_ncomp=1,
                f_alpha=3.0, f_targets=3)
    sim.init_beam(ppc=4, gamma=130.0, seed=1)
    t0 = time.perf_counter()
    for _ in range(steps):
        sim.step(1)
        sim.energy()
    t = time.perf_counter() - t0
    return {"value": sim.n * steps / t, "unit": UNIT, "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": f"the whole workload ({sim.n} particles), {steps} steps + energies each, one thread"}


def cpu_baseline_3d(steps: int = 3, threads: int = 0, nz: int = 8) -> dict:
    """The oracle on a few steps of thin slabs of the 3D workload, every host core one slab."""
    threads = threads if threads > 0 else host_threads()
    n, times = oracle_time(steps, 0, nz=nz, threads=threads, sample=oracle_sample_3d)
    return {"value": n / (sum(times) / len(times)), "unit": UNIT, "cores": threads, "host_cores": os.cpu_count(),
            "kind": "oracle",
            "sample": f"FP64 C oracle on {threads} host threads, each its own 128x128x{nz} slab of the 3D workload "
                      f"({n // threads} particles a slab, 1/{512 // nz} of the box; same density, weights, gamma, "
                      f"alpha, correction and filter): {steps} steps + energies each, concurrently; a short "
                      f"sample of the workload, per particle-step"}


def run_gamma_sweep(args):
    """Growth against c dt/dz at gamma 3 and 130 with the correction and the filter (cubic shapes,
    128 x 128 mesh, the setting of Sec. 3): the peak fitted growth rate of W_perp per gamma and the
    ratio of the peaks, against the paper's rough gamma^(-1/2) scaling."""
    import numpy as np
    import torch

    import paper_1401_0838_gb300 as P
    torch.cuda.set_device(0)
    tmax, every = args.gamma_time, 10  # the same physical time c t / dz for every c dt / dz
    solver = P.PIC_CK if args.solver == "ck" else P.PIC_YEE
    alphas = [0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7]
    if solver == P.PIC_CK:  # past Yee's 2D limit 1/sqrt(2); 0.771-0.783 is a Galerkin breakdown window
        alphas += [0.75, 0.8, 0.85, 0.9, 0.95]
    table = {}
    t0 = time.perf_counter()
    for scheme_name, scheme in (("galerkin", 0), ("uniform", 1)):
        for gamma in (3.0, 130.0):
            rates = []
            for alpha in alphas:
                cfg = P.pic_config_default(nx=128, nz=128, dt=alpha, gamma=gamma, scheme=scheme, precision=P.PIC_FP32,
                                           ppc_per_species=4, shape_order=3, init_beam=1, seed=11,
                                           diag_every=every, bin_capacity=96, field_solver=solver)
                h = P.pic_create(cfg)
                P.pic_set_correction_stencil(h, *P.pic_compute_correction_coeffs(scheme, alpha))
                steps = int(round(tmax / alpha / every)) * every
                P.pic_step(h, steps)
                w = [e["w_perp"] for e in P.pic_energy_history(h, 4096)]
                P.pic_destroy(h)
                t = np.arange(1, len(w) + 1) * every * alpha
                rates.append(float(P.pic_fit_growth_rate(t, w)[0]))
            table[f"{scheme_name}_gamma{int(gamma)}"] = rates
    out = {"alphas": alphas, "growth_rates": table, "unit": "1 / (dz/c)", "omega_p_dz": 0.3868}
    for scheme_name in ("galerkin", "uniform"):
        p3 = max(table[f"{scheme_name}_gamma3"])
        p130 = max(table[f"{scheme_name}_gamma130"])
        out[f"{scheme_name}_peak_ratio_gamma3_over_gamma130"] = p3 / p130
    out["gamma_minus_half_ratio"] = (130.0 / 3.0) ** 0.5
    for scheme_name in ("galerkin", "uniform"):
        out[f"{scheme_name}_ratio_per_alpha"] = [a / b for a, b in zip(table[f"{scheme_name}_gamma3"],
                                                                        table[f"{scheme_name}_gamma130"])]
    line = {"metric": "peak growth rate of W_perp against c dt/dz, gamma 3 vs 130 (corrected, filtered)",
            "value": out["galerkin_peak_ratio_gamma3_over_gamma130"], "unit": "ratio", "n_gpus": 1,
            "steps": int(round(tmax / alphas[0])), "warmup": 0, "higher_is_better": False, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "2D 128x128 beam, 4 particles/cell/species, cubic shapes, Psi correction + "
                                   f"filter (1,1,a=3), gamma in {{3, 130}}, c dt/dz {alphas[0]}..{alphas[-1]}, "
                                   f"{args.solver.upper()} solver, c t/dz = {tmax} each",
                       "wall_s":
                       round(time.perf_counter() - t0, 1)},
            "sweep": out}
    print(json.dumps(line), flush=True)


def run_variants(args):
    """Sec. 3's sensitivity variants of the corrected, filtered run (cubic Galerkin, 128 x 128, gamma
    130): the fitted growth rate of W_perp at several c dt/dz for the baseline (Psi_E on E, Psi_B on
    the other copies, filter (1,1,a=3) on J and the copies), (1) no digital filter apart from Psi_B,
    (2) the rational multiplier Psi_E / Psi_B on E only, (3) no compensation pass, and (0) no
    correction at all."""
    import numpy as np
    import torch

    import paper_1401_0838_gb300 as P
    torch.cuda.set_device(0)
    every, tmax = 10, args.gamma_time
    solver = P.PIC_CK if args.solver == "ck" else P.PIC_YEE
    alphas = [0.3, 0.5, 0.6, 0.7] if solver == P.PIC_YEE else [0.3, 0.5, 0.7, 0.8, 0.9, 0.95]
    variants = {
        "baseline": dict(),
        "no_filter": dict(filter_targets=0),
        "rational_on_E_only": dict(correction_mode=1),
        "no_compensation": dict(filter_ncomp=0),
        "no_correction": dict(_corr=False),
    }
    table = {}
    t0 = time.perf_counter()
    for name, kw in variants.items():
        kw = dict(kw)
        corr = kw.pop("_corr", True)
        rates = []
        for alpha in alphas:
            cfg = P.pic_config_default(nx=128, nz=128, dt=alpha, gamma=130.0, scheme=0, precision=P.PIC_FP32,
                                       ppc_per_species=4, shape_order=3, init_beam=1, seed=13, diag_every=every,
                                       bin_capacity=96, field_solver=solver, **kw)
            h = P.pic_create(cfg)
            if corr:
                P.pic_set_correction_stencil(h, *P.pic_compute_correction_coeffs(0, alpha))
            steps = int(round(tmax / alpha / every)) * every
            P.pic_step(h, steps)
            w = [e["w_perp"] for e in P.pic_energy_history(h, 4096)]
            P.pic_destroy(h)
            t = np.arange(1, len(w) + 1) * every * alpha
            rates.append(float(P.pic_fit_growth_rate(t, w)[0]))
        table[name] = rates
    line = {"metric": "fitted growth rate of W_perp per variant of the correction (Sec. 3)", "value": None,
            "unit": "1 / (dz/c)", "n_gpus": 1, "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"2D 128x128 beam, 4 particles/cell/species, cubic Galerkin, gamma 130, "
                                   f"{args.solver.upper()} solver, c t/dz = {tmax} per run", "alphas": alphas,
                       "wall_s": round(time.perf_counter() - t0, 1)},
            "growth_rates": table}
    print(json.dumps(line), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-steps", type=int, default=8)
    ap.add_argument("--cpu-threads", type=int, default=0, help="oracle threads (0: every host core)")
    ap.add_argument("--cpu-steps-3d", type=int, default=3, help="oracle steps of the --config3d CPU baseline")
    ap.add_argument("--cpu-steps-c1", type=int, default=200, help="oracle steps of the --config1 CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the config1 / config3d / sweep / adjoint keys of the default line")
    ap.add_argument("--sweep", action="store_true", help="time the batched 64-run sweep instead")
    ap.add_argument("--sweep-runs", type=int, default=64)
    ap.add_argument("--sweep-seq-steps", type=int, default=40)
    ap.add_argument("--adjoint", action="store_true", help="time the adjoint (256x512, 100 steps) instead")
    ap.add_argument("--adjoint-reps", type=int, default=3)
    ap.add_argument("--adjoint-steps", type=int, default=100)
    ap.add_argument("--no-fd", action="store_true", help="--adjoint without the central differences")
    ap.add_argument("--config3d", action="store_true", help="time the 3D 128x128x512 workload instead")
    ap.add_argument("--config3d-nz", type=int, default=512, help="z cells of the --config3d grid (profiling: fewer)")
    ap.add_argument("--config3d-nxy", type=int, default=128,
                    help="x and y cells of the --config3d grid (profiling: fewer)")
    ap.add_argument("--config1", action="store_true", help="time the small 64x128 FP64 workload instead")
    ap.add_argument("--order", type=int, default=1, choices=(1, 3), help="particle shape order of the workload")
    ap.add_argument("--gamma-sweep", action="store_true", help="growth against c dt/dz at gamma 3 and 130 instead")
    ap.add_argument("--gamma-time", type=float, default=2000.0,
                    help="c t / dz of each --gamma-sweep / --variants run")
    ap.add_argument("--variants", action="store_true", help="growth of the Sec. 3 correction variants instead")
    ap.add_argument("--solver", default="yee", choices=("yee", "ck"),
                    help="field solver (ck: Cole-Karkkainen; --gamma-sweep / --variants then run c dt/dz up to 0.95)")
    ap.add_argument("--correction", default="split", choices=("split", "rational"),
                    help="Psi_E / Psi_B on the copies (split) or the exact rational multiplier on E (rational)")
    ap.add_argument("--scheme", default="galerkin", choices=("galerkin", "uniform", "momentum"))
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per push launch from an ncu capture of this kernel (reported as is)")
    args = ap.parse_args(argv)
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.sweep:
        run_sweep(args)
    elif args.adjoint:
        run_adjoint(args)
    elif args.config3d:
        run_3d(args)
    elif args.config1:
        run_config1(args)
    elif args.gamma_sweep:
        run_gamma_sweep(args)
    elif args.variants:
        run_variants(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
