"""Benchmark of the fused coupled LB step on GB300 (one JSON line on rank 0).

Workload: the 512 x 512 sessile-droplet freezing case (Sec. 4.3 shape:
droplet R = 100 on a cold solid layer, seeded contact angle and Stefan
number), all three lattices, FP32 populations.  One bench step is one full
time step of the coupled update (enthalpy inversion, order parameter,
stencils, three collisions, streaming with walls, lag store and the fused
FP64 diagnostics) over the whole grid.  The FP32 working set (~70 MB) fits in the
129 MB L2, so the L2 is flushed (256 MB written, then read) before every timed step and
each step is timed alone with CUDA events on the launching stream: the
number is the HBM-bound one.  Under torchrun every rank advances its own
replica (weak scaling, no collective on the data path).

``--impl reference`` times the FP64 CPU oracle on the same workload instead
(a bounded sample of steps per bench step), on the host cores.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "coupled MLUPS"  # node updates of all enabled lattices per second / 1e6
WORKLOAD = "sessile droplet freezing 512x512 (R=100, cold solid layer), 3 lattices, seed 0"
L2_FLUSH_BYTES = 256 << 20


class L2Flush:
    """Evicts the L2 before a timed step: a write of L2_FLUSH_BYTES and, in
    the "clean" mode, a read of the same buffer after it, so that the lines
    the timed kernel then evicts are clean (with a write alone the kernel
    also pays for writing the flush buffer's dirty lines back to HBM)."""

    def __init__(self, mode):
        import torch
        self.clean = mode == "clean"
        self.buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        self.acc = torch.zeros((), dtype=torch.float32, device="cuda")

    def __call__(self):
        import torch
        self.buf.zero_()
        if self.clean:
            torch.sum(self.buf, 0, out=self.acc)

    @property
    def describe(self):
        mb = L2_FLUSH_BYTES >> 20
        return (f"flushed before every timed step ({mb} MB written, then read: no dirty lines "
                f"left in L2)" if self.clean else f"flushed before every timed step ({mb} MB write)")


def _droplet512(seed):
    from paper_2510_18688_gb300 import workloads as W
    return [W.sessile_droplet(512, seed=seed)]


def _droplet1024(seed):
    from paper_2510_18688_gb300 import workloads as W
    return [W.sessile_droplet(1024, seed=seed, radius=200.0)]


def _porous(seed):
    from paper_2510_18688_gb300 import workloads as W
    return [W.porous(seed=seed)]


def _neumann(seed):
    from paper_2510_18688_gb300 import workloads as W
    return [W.neumann()]


def _stefan(seed):
    from paper_2510_18688_gb300 import workloads as W
    return [W.stefan()]


def _batch64(seed):
    """64 droplets on cold cylinders, sides drawn from {128, 256, 384, 512}."""
    from paper_2510_18688_gb300 import workloads as W
    r = W.rng(1000 + seed)
    sides = r.choice([128, 256, 384, 512], size=64)
    return [W.cylinder_droplet(int(sd), seed=64 * seed + i) for i, sd in enumerate(sides)]


WORKLOADS = {
    "droplet512": (_droplet512, "sessile droplet freezing 512x512 (R=100, cold solid layer), 3 lattices"),
    "droplet1024": (_droplet1024, "sessile droplet freezing 1024x1024 (R=200, cold solid layer), 3 lattices"),
    "porous2048x1024": (_porous, "freezing in a porous medium 2048x1024 (porosity 0.6, saturation 0.5), 3 lattices"),
    "neumann400x4": (_neumann, "conduction-induced freezing column 400x4 (flow + enthalpy lattices)"),
    "stefan512x8": (_stefan, "three-phase Stefan column 512x8, 3 lattices"),
    "batch64": (_batch64, "64 droplets on cold cylinders, sides in {128,256,384,512}, one persistent launch per step"),
}


# three-dimensional (D3Q19) context lines: run by fracture_line
WORKLOADS3 = {
    "fracture256x128x30": "freezing in a rough fracture 256x128x30 (Sec. 4.5 shape: self-affine "
                          "aperture, liquid column with three bubbles, cold wall at x = 0), "
                          "D3Q19, 3 lattices",
}


def algorithmic_bytes_per_node3(esize: int) -> int:
    """D3Q19: 57 populations read and written, 7 lag fields read and
    written, phi0 read."""
    return 2 * 57 * esize + 2 * 7 * esize + esize


def algorithmic_bytes_per_node(esize: int, has_mask: bool, pop_bytes: int = 0,
                               nlag: int = 6) -> int:
    """27 populations read and written, the lag fields read and written (6;
    7 for float arithmetic, whose well-balanced storage also keeps the
    previous temperature), phi0 read, mask byte read."""
    return 2 * 27 * (pop_bytes or esize) + 2 * nlag * esize + esize + (1 if has_mask else 0)


def lag_planes(precision: str) -> int:
    return 7 if precision in ("fp32", "fp16s") else 6


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the sources the step kernels are compiled from (host API and probes excluded)
KERNEL_SOURCES = ("lbm_kernels.cuh", "lbm_dual.cuh", "lbm_step.cuh", "lbm_split.cuh",
                  "lbm_tile.cuh", "lbm_tma.cuh", "lbm_launch.h", "lbm_f32.cu", "lbm_f64.cu",
                  "lbm_f16.cu", "lbm_tan.cu")


# the sources of the 3-D step kernels
KERNEL_SOURCES3 = ("lbm3d.cu", "lbm_kernels.cuh", "lbm_dual.cuh", "lbm_host.h")


def kernel_source_hash(sources=KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2510_18688_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_name(workload: str, precision: str) -> str:
    kind = "batch" if workload.startswith("batch") else "step"
    tag = {"fp32": "f32", "fp64": "f64", "fp16s": "f16s", "tangent": "tan"}[precision]
    return f"lbm_{kind}_{tag}_{workload}.md"


def profiled_value(workload: str, precision: str, key: str):
    """A per-launch figure (e.g. "dram bytes per launch") from the committed
    ncu summary of this workload, if it was taken on the current kernel
    source; else None."""
    if workload in WORKLOADS3:
        path = os.path.join(ROOT, "profiles", f"lbm3_collide_{ {'fp32': 'f32', 'fp64': 'f64'}[precision] }_{workload}.md")
        if not os.path.exists(path):
            return None
        txt = open(path).read()
        m = re.search(r"kernel source hash:\s*([0-9a-f]+)", txt)
        t = re.search(re.escape(key) + r":\s*([0-9.eE+]+)", txt)
        if not m or not t or m.group(1) != kernel_source_hash(KERNEL_SOURCES3):
            return None
        return float(t.group(1))
    path = os.path.join(ROOT, "profiles", profile_name(workload, precision))
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"kernel source hash:\s*([0-9a-f]+)", txt)
    t = re.search(re.escape(key) + r":\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != kernel_source_hash():
        return None
    return float(t.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
            # nvidia-smi takes a moment to start: wait for its first sample so
            # that the window covers what follows
            t0 = time.perf_counter()
            while not self.samples and time.perf_counter() - t0 < 3.0:
                time.sleep(0.01)
        except (FileNotFoundError, OSError):
            self._proc = None
        return self

    def mark(self):
        """Index of the next sample (to split warm-up from the timed region)."""
        return len(self.samples)

    def _read(self):
        for line in self._proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *exc):
        if self._proc:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._proc.kill()

    def summary(self, start: int = 0, window: str = ""):
        """Median SM clock, maximum clock and throttle reasons of the samples
        from index `start` on."""
        samples = self.samples[start:]
        if not samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in samples for k in range(4)
                          if s[3 + k].lower() == "active"})
        out = {"sm_mhz": float(np.median(sm)) if sm else None,
               "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
               "samples": len(samples)}
        if window:
            out["window"] = window
        return out


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(value: float, pg) -> float:
    """Largest value over all ranks (the timed region is the slowest rank's)."""
    if pg is None:
        return value
    import torch
    dev = "cuda" if pg.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank: int, world: int, steps: int, t_max_ms: float) -> float:
    """Weak scaling: every rank advances its own replica, so the job updates
    world * nodes * steps nodes in the slowest rank's time."""
    return world * nodes_per_rank * steps / (t_max_ms * 1e-3) / 1e6


def reference_arm(args, rank, world, budget_s: float = 150.0):
    """The FP64 CPU oracle timed on the host cores.  Each step is one full
    time step of the sessile-droplet workload; when K + W full 512^2 steps
    would take longer than budget_s, every step is a bounded sample: the
    same workload on a smaller square grid (droplet radius and solid layer
    scaled with it), stated in the line."""
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2510_18688_gb300 import workloads as W
    cores = O.set_threads(0)
    side = 512
    o = O.from_workload(W.sessile_droplet(side, seed=0))
    t0 = time.perf_counter()
    o.step(1)
    t_full = time.perf_counter() - t0
    total = max(1, args.steps + args.warmup)
    if total * t_full > budget_s:
        side = int(512 * math.sqrt(budget_s / (total * t_full))) // 32 * 32
        side = max(64, side)
        k = side / 512
        o = O.from_workload(W.sessile_droplet(side, seed=0, radius=100.0 * k,
                                              hs=max(4.0, 12.0 * k)))
    n = side * side
    for _ in range(args.warmup):
        o.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(1)
    dt = time.perf_counter() - t0
    mlups = n * args.steps / dt / 1e6
    sample = (f"{args.steps} full time steps of the {side}x{side} droplet workload"
              + ("" if side == 512 else f" (bounded sample of the 512x512 case, whose steps take "
                                         f"{t_full * 1e3:.0f} ms each here)"))
    line = {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [side, side], "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def back_to_back_line(args, rank, world):
    """Launch-overhead context for small grids: K steps in one lbm_step call
    (whole periods replayed from a captured CUDA graph) against K calls of
    one step each, both timed with CUDA events around the whole run.  The
    grid stays in L2 (no flush): this measures launch cost, not HBM."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    from paper_2510_18688_gb300 import build, lbm
    build.build()
    lbm.load()
    make, workload_name = WORKLOADS[args.workload]
    (cfg, arr), = make(rank)
    n = cfg["nx"] * cfg["ny"]
    stream = torch.cuda.current_stream()
    sptr = ctypes.c_void_p(stream.cuda_stream)
    s = lbm.Solver(cfg, precision=args.precision, diag_every=args.diag_every).set_geometry(arr)
    K = args.steps

    def timed(fn):
        fn(args.warmup)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn(K)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / K  # ms per step

    t_graph = timed(lambda k: lbm.lbm_step(s.ctx, k, sptr))
    t_single = timed(lambda k: [lbm.lbm_step(s.ctx, 1, sptr) for _ in range(k)])
    s.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": n / (t_graph * 1e-3) / 1e6, "unit": "MLUPS", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": t_graph,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp16s": "f32 (f16 storage)",
                  "tangent": "f64 (value and derivative)"}[args.precision],
        "data": "synthetic",
        "config": {"workload": workload_name, "grid": [cfg["nx"], cfg["ny"]],
                   "l2": "not flushed: back-to-back steps of a grid far smaller than L2 "
                         "(a launch-overhead context line, not an HBM measurement)",
                   "diag_every": args.diag_every},
        "single_step_calls_ms_per_step": t_single,
        "graph_speedup": t_single / t_graph,
    }
    print(json.dumps(line), flush=True)


def adjoint_line(args, rank, world, every: int = 64):
    """Reverse sweep against K forward steps of the same context (FP64).
    freezing: the frozen fraction of the 512^2 droplet with the phase field
    and the enthalpy lattice coupled and its gradient w.r.t. (T_wall, L,
    theta, sigma).
    heat: frozen fraction of a conduction-freezing column (Sec. 4.1 shape,
    2048 x 256, enthalpy lattice alone) and its gradient w.r.t. the wall
    temperatures and L.  phase: the tip height of a 512^2 sessile droplet
    (phase-field lattice alone) and its gradient w.r.t. theta and sigma."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    from paper_2510_18688_gb300 import build, lbm, workloads as W
    build.build()
    lbm.load()
    if args.adjoint == "phase":
        cfg, arr = W.sessile_droplet(512, seed=0)
        cfg = dict(cfg, lattices=W.PHASE)
    elif args.adjoint == "freezing":
        # the droplet cooled through its solid layer from the cold wall below
        # (no cold mask); phase field and enthalpy lattices
        cfg, arr = W.sessile_droplet(512, seed=0)
        cfg = dict(cfg, lattices=W.PHASE | W.HEAT)
        arr = {k: v for k, v in arr.items() if k != "mask"}
    elif args.adjoint == "coupled":
        # the headline workload itself: all three lattices, cold substrate
        cfg, arr = W.sessile_droplet(512, seed=0)
    else:
        cfg, arr = W.neumann(nx=2048, ny=256)
        cfg = dict(cfg, lattices=W.HEAT)
    n = cfg["nx"] * cfg["ny"]
    stream = torch.cuda.current_stream()
    sptr = ctypes.c_void_p(stream.cuda_stream)
    K = args.steps
    s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
    s.step(args.warmup)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm.lbm_step(s.ctx, K, sptr)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    s.set_geometry(arr)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if args.adjoint == "phase":
        ff, grad = lbm.lbm_adjoint_crossing(s.ctx, K, every, 1, cfg["nx"] // 2, sptr)
    elif args.adjoint == "freezing":
        ff, grad = lbm.lbm_adjoint_freezing(s.ctx, K, every, 0, 0, 0, sptr)
    elif args.adjoint == "coupled":
        ff, grad = lbm.lbm_adjoint_coupled(s.ctx, K, every, 0, 0, 0, None, sptr)
    else:
        ff, grad = lbm.lbm_adjoint_frozen_fraction(s.ctx, K, every, sptr)
    t_adj = time.perf_counter() - t0
    s.close()
    if rank != 0:
        return
    line = {
        "metric": METRIC + " (forward + reverse sweep)", "value": n * K / t_adj / 1e6,
        "unit": "MLUPS", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": t_adj / K * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": ("sessile droplet 512x512, phase-field lattice alone, tip height "
                                "and its gradient w.r.t. contact angle and surface tension"
                                if args.adjoint == "phase" else
                                "sessile droplet 512x512 cooled through its solid layer, phase "
                                "field + enthalpy lattices, frozen fraction and its gradient "
                                "w.r.t. wall temperatures, latent heat, contact angle and surface "
                                "tension" if args.adjoint == "freezing" else
                                "sessile droplet freezing 512x512 on its cold substrate (the "
                                "headline workload), frozen fraction and its gradient w.r.t. "
                                "wall temperatures, latent heat, contact angle, surface tension, "
                                "body force and substrate temperature" if args.adjoint == "coupled" else
                                "conduction-freezing column 2048x256 (Sec. 4.1 shape), enthalpy "
                                "lattice alone, frozen fraction and its gradient w.r.t. wall "
                                "temperatures and latent heat"), "checkpoint_every": every},
        "adjoint_forward_ratio": t_adj / t_fwd,
        "forward_ms_per_step": t_fwd / K * 1e3,
        **({"tip": ff, "grad": {"theta_deg": grad[0], "sigma": grad[1]}}
           if args.adjoint == "phase" else
           {"ff": ff, "grad": {"T_wall": grad[:4], "latent": grad[4], "theta_deg": grad[5],
                               "sigma": grad[6]}}
           if args.adjoint == "freezing" else
           {"ff": ff, "grad": {"T_wall": grad[:4], "latent": grad[4], "theta_deg": grad[5],
                               "sigma": grad[6], "gx": grad[7], "gy": grad[8],
                               "T_cold": grad[9]}}
           if args.adjoint == "coupled" else
           {"ff": ff, "grad": {"T_wall": grad[:4], "latent": grad[4]}}),
        "note": "host wall-clock around whole calls (synchronised); both include launch overheads",
    }
    print(json.dumps(line), flush=True)


def fracture_line(args, rank, world):
    """The D3Q19 step on the 256 x 128 x 30 rough fracture (FP32 or FP64).
    Each step is two kernels (local state; stencils, collisions and
    streaming); the state (57 planes, 224 MB in FP32 per buffer) is larger
    than L2, so no flush is needed between steps.  The roofline is taken
    over the whole step (both kernels) with the single-pass state traffic."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    from paper_2510_18688_gb300 import build, lbm, workloads as W
    build.build()
    lbm.load()
    if args.precision not in ("fp32", "fp64"):
        raise SystemExit("the 3-D workload takes --precision fp32 or fp64")
    cfg, arr = W.rough_fracture(seed=rank)
    n = cfg["nx"] * cfg["ny"] * cfg["nz"]
    stream = torch.cuda.current_stream()
    sptr = ctypes.c_void_p(stream.cuda_stream)
    s = lbm.Solver3(cfg, args.precision).set_geometry(arr)
    s.step(args.warmup)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        for k in range(args.steps):
            starts[k].record(stream)
            lbm.lbm3_step(s.ctx, 1, sptr)
            ends[k].record(stream)
        torch.cuda.synchronize()
    times = np.array([a.elapsed_time(b) for a, b in zip(starts, ends)])
    t_step = float(times.mean())
    diag = s.diagnostics()

    # end to end through the C ABI with host buffers: geometry upload from
    # pinned memory, K steps, phi/fl/T download to pinned memory
    def pinned(a, dtype):
        t = torch.empty(a.shape, dtype=dtype, pin_memory=True)
        t.numpy()[...] = a
        return t

    ht = {k: pinned(arr[k], torch.float64) for k in ("phi0", "phi", "T", "fl")}
    ot = {k: torch.empty(arr["phi"].shape, dtype=torch.float64, pin_memory=True)
          for k in ("phi", "fl", "T")}
    fmask = sum(1 << lbm.FIELDS3.index(k) for k in ot)
    ptrs = [ot[k].numpy().ctypes.data if k in ot else None for k in lbm.FIELDS3]
    h = {k: v.numpy() for k, v in ht.items()}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm.lbm3_set_geometry(s.ctx, h["phi0"].ctypes.data, None, h["phi"].ctypes.data,
                          h["T"].ctypes.data, h["fl"].ctypes.data, lbm.LBM_HOST, sptr)
    lbm.lbm3_step(s.ctx, args.steps, sptr)
    lbm.lbm3_read_fields(s.ctx, fmask, ptrs, lbm.LBM_HOST, sptr)
    e2e_s = time.perf_counter() - t0
    s.close()
    if rank != 0:
        return
    esize = 8 if args.precision == "fp64" else 4
    bpn = algorithmic_bytes_per_node3(esize)
    peak, peak_src = measured_peak()
    achieved = bpn * n / (t_step * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": n / (t_step * 1e-3) / 1e6 * world, "unit": "MLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64"}[args.precision], "data": "synthetic",
        "config": {"workload": WORKLOADS3["fracture256x128x30"] + f", seed {rank}",
                   "grid": [cfg["nx"], cfg["ny"], cfg["nz"]], "precision": args.precision,
                   "l2": "not flushed: the state (57 population planes) is larger than L2",
                   "parallelism": f"replicas x{world}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": profiled_value(args.workload, args.precision, "dram bytes per step"),
                     "peak_source": peak_src, "bytes_per_node": bpn,
                     "scope": "whole step (local-state and collide kernels together)"},
        "gpu_launches": 2 * args.steps,
        "e2e": {"value": n * args.steps / e2e_s / 1e6, "unit": "MLUPS",
                "h2d_bytes_per_step": 4 * n * 8 / args.steps,
                "d2h_bytes_per_step": 3 * n * 8 / args.steps},
        "diag_last": {k: diag[k] for k in ("material_mass", "frozen_volume", "nonfinite", "step")},
        "clocks": clk.summary(),
    }
    if not args.no_cpu_baseline:
        from oracle import oracle3d as O3
        cores = int(os.cpu_count() or 1)
        o = O3.from_workload((cfg, arr))
        o.step(1)
        t0 = time.perf_counter()
        k = 0
        while time.perf_counter() - t0 < 12.0:
            o.step(1)
            k += 1
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": n * k / dt / 1e6, "unit": "MLUPS", "cores": cores,
                                "kind": "oracle",
                                "sample": f"{k} full steps of the same 3-D workload (about 12 s)"}
    print(json.dumps(line), flush=True)


def fp64_record(lbm, wl, flush, stream, sptr, args, t32_ms):
    """The FP64 step on the same workload: MLUPS, its HBM fraction and its
    fraction of the FP64 FMA rate measured now (the FP64 pipe, not HBM,
    bounds this step on GB300), each step timed alone after an L2 flush."""
    import torch
    cfg, arr = wl
    n = cfg["nx"] * cfg["ny"]
    s = lbm.Solver(cfg, precision="fp64", diag_every=args.diag_every).set_geometry(arr)
    # the autotuner's kernel form for this grid, as for the FP32 line
    form = None
    if not args.no_autotune:
        us, chosen = s.autotune(16)
        form = chosen // 2
    k = max(10, min(args.steps, 40))
    for _ in range(3):
        flush()
        lbm.lbm_step(s.ctx, 1, sptr)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(k)]
    for j in range(k):
        flush()
        starts[j].record(stream)
        lbm.lbm_step(s.ctx, 1, sptr)
        ends[j].record(stream)
    torch.cuda.synchronize()
    t = float(np.mean([a.elapsed_time(b) for a, b in zip(starts, ends)]))
    s.close()
    fma = lbm.lbm_probe_fma_rate("fp64", sptr) / 1e12
    bpn = algorithmic_bytes_per_node(8, "mask" in arr)
    peak, peak_src = measured_peak()
    hbm = bpn * n / (t * 1e-3) / 1e9
    fpn = profiled_value(args.workload, "fp64", "fp64 flops per node")
    ach = fpn * n / (t * 1e-3) / 1e12 if fpn else None
    return {"value": n / (t * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": t, "steps": k,
            "kernel_form": form, "fp32_over_fp64": t / t32_ms,
            "fp64_pipe": {"achieved": ach, "peak": fma, "unit": "TFLOP/s",
                          "frac": ach / fma if ach else None, "flops_per_node": fpn,
                          "peak_source": "FP64 FMA rate measured in this run"},
            "hbm": {"achieved": hbm, "peak": peak, "unit": "GB/s", "frac": hbm / peak,
                    "bytes_per_node": bpn, "peak_source": peak_src}}


def adjoint_record(lbm, wl, sptr, t32_ms, steps: int = 256, every: int = 16):
    """Reverse sweep of the whole coupled step (FP64, checkpointed recompute):
    the frozen fraction of the same workload after `steps` steps and its
    gradient w.r.t. (T_wall, L, theta, sigma, g, T_cold), timed against the
    FP64 forward run of the same steps (host clock around synchronised
    calls)."""
    import torch
    cfg, arr = wl
    s = lbm.Solver(cfg, precision="fp64").set_geometry(arr)
    lbm.lbm_step(s.ctx, 3, sptr)
    s.set_geometry(arr)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm.lbm_step(s.ctx, steps, sptr)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    s.set_geometry(arr)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ff, grad = lbm.lbm_adjoint_coupled(s.ctx, steps, every, 0, 0, 0, None, sptr)
    torch.cuda.synchronize()
    t_adj = time.perf_counter() - t0
    s.close()
    return {"adjoint_forward_ratio": t_adj / t_fwd,
            "adjoint_over_fp32_forward": (t_adj / steps * 1e3) / t32_ms,
            "steps": steps, "checkpoint_every": every,
            "forward_ms_per_step": t_fwd / steps * 1e3,
            "adjoint_ms_per_step": t_adj / steps * 1e3,
            "observable": "frozen fraction", "ff": ff,
            "grad": {"T_wall": grad[:4], "latent": grad[4], "theta_deg": grad[5],
                     "sigma": grad[6], "gx": grad[7], "gy": grad[8], "T_cold": grad[9]},
            "note": "forward + reverse sweep over the FP64 forward run of the same steps "
                    "(adjoint_forward_ratio); adjoint_over_fp32_forward divides by the timed "
                    "FP32 step of this line"}


def cpu_baseline_sample(target_s: float = 12.0):
    """Time the oracle on the same workload for about target_s seconds."""
    from oracle import oracle as O
    from paper_2510_18688_gb300 import workloads as W
    wl = W.sessile_droplet(512, seed=0)
    o = O.from_workload(wl)
    cores = O.set_threads(0)
    n = wl[0]["nx"] * wl[0]["ny"]
    t0 = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t0
    k = max(2, min(200, int(target_s / max(one, 1e-3))))
    t0 = time.perf_counter()
    o.step(k)
    dt = time.perf_counter() - t0
    return {"value": n * k / dt / 1e6, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{k} time steps of the 512x512 droplet workload (FP64 oracle)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp16s", "tangent"],
                    help="fp16s: FP16 population storage, FP32 arithmetic; tangent: FP64 "
                         "step with its derivative along the wall temperature")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--l2-flush", default="clean", choices=["clean", "write"],
                    help="L2 eviction before each timed step: clean (write then read a "
                         "256 MB buffer) or write (the write alone, which leaves dirty lines "
                         "that the timed kernel must write back)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="step with the library's default kernel form (no lbm_autotune)")
    ap.add_argument("--no-sub-records", action="store_true",
                    help="skip the FP64 and adjoint sub-records of the default FP32 line")
    ap.add_argument("--diag-every", type=int, default=1,
                    help="steps between fused FP64 diagnostic reductions (0: none)")
    ap.add_argument("--back-to-back", action="store_true",
                    help="context line for small grids: one call of K steps (captured CUDA "
                         "graphs), no L2 flush, against K single-step calls")
    ap.add_argument("--adjoint", nargs="?", const="heat", choices=("heat", "phase", "freezing", "coupled"),
                    help="time a reverse-mode gradient against its forward run (FP64): heat, the "
                         "frozen fraction of the conduction column 2048 x 256 (enthalpy lattice "
                         "alone); phase, the tip height of the 512^2 droplet (phase field alone); "
                         "freezing, the frozen fraction of the 512^2 droplet (phase field and "
                         "enthalpy coupled); coupled, the same with all three lattices")
    ap.add_argument("--workload", default="droplet512",
                    choices=sorted(WORKLOADS) + sorted(WORKLOADS3),
                    help="droplet512 is the headline; the others are context lines")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()

    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if args.adjoint:
        adjoint_line(args, rank, world)
        return
    if args.back_to_back:
        back_to_back_line(args, rank, world)
        return
    if args.workload in WORKLOADS3:
        fracture_line(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    from paper_2510_18688_gb300 import build, lbm, workloads as W
    build.build()
    L = lbm.load()

    make, workload_name = WORKLOADS[args.workload]
    wls = make(rank)
    n = sum(c["nx"] * c["ny"] for c, _ in wls)
    stream = torch.cuda.current_stream()
    sptr = ctypes.c_void_p(stream.cuda_stream)
    # tangent: derivative along the wall temperature (cold substrate and walls)
    tan = {"T_cold": 1.0, "T_wall": [1.0, 1.0, 1.0, 1.0]} if args.precision == "tangent" else None
    solvers = [lbm.Solver(c, precision=args.precision, diag_every=args.diag_every,
                          tangent=tan).set_geometry(a) for c, a in wls]
    batch = lbm.Batch(solvers) if len(solvers) > 1 else None
    # the library's autotuner picks the kernel form and graph period for this
    # grid (state unchanged); batches use the batch kernel
    tune = None
    if batch is None and not args.no_autotune:
        us, chosen = solvers[0].autotune(64)
        tune = {"chosen": chosen, "us_per_step": us,
                "variants": "kernel form v//2 (0 one CTA per 32x8 tile; 1 float TMA-staged "
                            "one stage / fp64 two-kernel split; 2 TMA-staged two stages "
                            "2 CTAs/SM; 3 TMA-staged one stage 3 CTAs/SM; 4 one CTA per "
                            "32x4 tile; 5 one CTA per 32x16 tile; -1: not available) x "
                            "captured period (v even 32, odd 256); timed back to back "
                            "without L2 flush"}

    def step(k):
        if batch is not None:
            lbm.lbm_batch_step(batch.handle, k, sptr)
        else:
            lbm.lbm_step(solvers[0].ctx, k, sptr)

    flush = L2Flush(args.l2_flush)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    # the clock sampler runs from before the warm-up to after the timed
    # region; a short timed region (tens of steps, about a millisecond) falls
    # between two nvidia-smi samples, so the warm-up ends with a sustained
    # untimed load of the same kernel (at least 0.3 s) whose clocks are
    # recorded with it
    with ClockSampler(local) as clk:
        for _ in range(args.warmup):
            flush()
            step(1)
        torch.cuda.synchronize()
        t_load = time.perf_counter()
        while time.perf_counter() - t_load < 0.3:
            step(64)
            torch.cuda.synchronize()
        for _ in range(3):
            flush()
            step(1)
        if pg:
            pg.barrier()
        torch.cuda.synchronize()
        timed_mark = clk.mark()
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush()
            starts[k].record(stream)
            step(1)
            ends[k].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        time.sleep(0.05)  # one more sample after the timed region
    if pg:
        pg.barrier()
    times = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])  # ms
    t_step = float(times.mean())
    t_tot = max_over_ranks(float(times.sum()), pg)
    # the fused reduction of the last diagnosed step, or one on request
    diag = solvers[0].diagnostics(compute=args.diag_every == 0)

    # end to end through the C ABI with host buffers: geometry upload,
    # the same K steps, fields (phi, fl, T) read back to host memory
    def pinned(a, dtype):
        t = torch.empty(a.shape, dtype=dtype, pin_memory=True)
        t.numpy()[...] = a
        return t

    keep = []
    uploads, downloads = [], []
    fmask = lbm.FIELD_BIT["phi"] | lbm.FIELD_BIT["fl"] | lbm.FIELD_BIT["T"]
    h2d = d2h = 0
    for (c, a), sv in zip(wls, solvers):
        ht = {k: pinned(a[k], torch.float64) for k in ("phi0", "phi", "T", "fl")}
        hm = pinned(a["mask"], torch.uint8) if "mask" in a else None
        ot = {k: torch.empty((c["ny"], c["nx"]), dtype=torch.float64, pin_memory=True)
              for k in ("phi", "fl", "T")}
        keep += [ht, hm, ot]
        h = {k: v.numpy() for k, v in ht.items()}
        uploads.append((sv.ctx, h["phi0"].ctypes.data, hm.numpy().ctypes.data if hm is not None else None,
                        h["phi"].ctypes.data, h["T"].ctypes.data, h["fl"].ctypes.data))
        ptrs = [ot[k].numpy().ctypes.data if k in ot else None for k in lbm.FIELDS]
        downloads.append((sv.ctx, ptrs))
        h2d += 4 * c["nx"] * c["ny"] * 8 + (c["nx"] * c["ny"] if hm is not None else 0)
        d2h += 3 * c["nx"] * c["ny"] * 8
    # a job of at least 2000 steps, so that the upload does not dominate
    k_e2e = max(args.steps, 2000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for u in uploads:
        lbm.lbm_set_geometry(*u, lbm.LBM_HOST, sptr)
    step(k_e2e)
    for ctx, ptrs in downloads:
        lbm.lbm_read_fields(ctx, fmask, ptrs, lbm.LBM_HOST, sptr)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": n * k_e2e / e2e_s / 1e6, "unit": "MLUPS", "steps": k_e2e,
           "h2d_bytes_per_step": h2d / k_e2e, "d2h_bytes_per_step": d2h / k_e2e,
           "note": (f"one job of {k_e2e} steps through the C ABI: pinned-host geometry upload, "
                    "the steps back to back (no L2 flush between them, unlike the per-step "
                    "timing of value), phi/fl/T download to pinned host memory; host clock "
                    "around the synchronised job")}

    # steady state without flushes (context only, not the value)
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    step(args.steps)
    g1.record(stream)
    torch.cuda.synchronize()
    l2_ms = g0.elapsed_time(g1) / args.steps

    if rank != 0:
        if pg:
            pg.destroy_process_group()
        return
    esize = {"fp64": 8, "tangent": 16}.get(args.precision, 4)
    pop_bytes = 2 if args.precision == "fp16s" else esize
    # node-weighted bytes per node (grids with a cold mask read one more byte)
    bpn = sum(algorithmic_bytes_per_node(esize, "mask" in a, pop_bytes,
                                         lag_planes(args.precision)) * c["nx"] * c["ny"]
              for c, a in wls) / n
    peak, peak_src = measured_peak()
    achieved = bpn * n / (t_step * 1e-3) / 1e9
    traffic = profiled_value(args.workload, args.precision, "dram bytes per launch")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": peak_src, "bytes_per_node": bpn}
    if args.precision in ("fp64", "tangent"):
        # the FP64 pipe, not HBM, bounds the double-precision step on this
        # part: compare its executed FP64 flops with the FMA rate measured now
        fma = lbm.lbm_probe_fma_rate("fp64", sptr)
        fpn = profiled_value(args.workload, args.precision, "fp64 flops per node")
        ach = fpn * n / (t_step * 1e-3) / 1e12 if fpn else None
        roofline = {"bound": "alu", "achieved": ach, "peak": fma / 1e12, "unit": "TFLOP/s",
                    "frac": ach / (fma / 1e12) if ach else None, "traffic": traffic,
                    "peak_source": "FP64 FMA rate measured in this run (lbm_probe_fma_rate)",
                    "flops_per_node": fpn,
                    "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "bytes_per_node": bpn}}
    value = whole_job_mlups(n, world, args.steps, t_tot)
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "fp16s": "f32 (f16 storage)",
                  "tangent": "f64 (value and derivative)"}[args.precision],
        "data": "synthetic",
        "config": {"workload": workload_name + f", seed {rank}",
                   "grid": ([wls[0][0]["nx"], wls[0][0]["ny"]] if len(wls) == 1
                            else f"{len(wls)} grids, {n} nodes"),
                   "precision": args.precision,
                   "l2": flush.describe,
                   "diag_every": args.diag_every,
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "autotune": tune,
        "gpu_launches": args.steps,
        "e2e": e2e,
        "l2_resident_mlups": n / (l2_ms * 1e-3) / 1e6,
        "diag_last": {k: diag[k] for k in ("material_mass", "frozen_volume", "nonfinite", "step")},
        "clocks": clk.summary(timed_mark, "timed region"),
        "clocks_window": clk.summary(0, "warm-up (with at least 0.3 s of sustained untimed steps) "
                                        "through the timed region"),
        "wall_s_timed_region": wall,
    }
    if args.precision == "fp32" and len(wls) == 1 and not args.no_sub_records:
        # the other two parts of the metric on the same workload: the FP64
        # step, and the reverse sweep of the coupled step against its forward
        line["fp64"] = fp64_record(lbm, wls[0], flush, stream, sptr, args, t_step)
        line["adjoint"] = adjoint_record(lbm, wls[0], sptr, t_step)
    line["build"] = {"source_hash": lbm.lbm_source_hash()}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample()
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
