"""Throughput of the fused ternary colour-gradient LBM step (D2Q9) on GB300.

Workload: the 2048x2048 periodic compound double droplet (fluid-3 core radius
200 inside a fluid-2 shell radius 400 in a fluid-1 matrix, tau = (0.6, 0.7,
0.9) for viscosity ratio 1:2:4, sigma_12/13/23 = 0.01/0.012/0.005,
beta^0 = 0.7), FP32 arithmetic.  A "step" is one lattice time step of the
whole grid (one launch of the fused kernel).  The metric is MLUPS (million
lattice-node updates per second), reported with the HBM roofline fraction.
Two forms of the state are timed: the chosen form, the reduced state (phi_k,
f^dagger_i and V_k per node; 144 algorithmic bytes per node update), which is
the headline, and the plain FP32 form (27 populations; 216 bytes); both give
bit-identical states, so they are compared at equal error.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torchrun as independent replicas, one per GPU (the method
has no exchange step on one grid per GPU; weak scaling).  --impl reference
times the FP64 CPU oracle on the host cores on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_NODE = 216            # 27 pops x 4 B read + 27 x 4 B written
BYTES_PER_NODE_REDUCED = 144    # 18 values (phi_k, f^dagger_i, V_k) x 4 B read + written
FALLBACK_HBM_GBS = 6800.0
WORKLOAD = ("compound double droplet 2048x2048 periodic, fluid-3 core r=200 in fluid-2 shell r=400, "
            "tau=(0.6,0.7,0.9), sigma12/13/23=0.01/0.012/0.005, beta0=0.7, FP32 arithmetic")
STEP_KERNEL = "fused_step_kernel"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("lbm3_step.cu", "lbm3_internal.h"):
        with open(os.path.join(ROOT, "paper_1808_08555_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(form: str = "fp32"):
    """Per-launch DRAM bytes of the step kernel in the given form from the
    committed ncu summary, if it was taken on the current kernel source (else
    None)."""
    name = "fused_step_compound_2048_traffic.json" if form == "fp32" else f"fused_step_{form}_compound_2048_traffic.json"
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as fh:
            d = json.load(fh)
        if d.get("source_hash") == kernel_source_hash():
            return float(d["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running, each
    stamped with the host time it arrived, so that the samples taken inside
    the timed region can be told from those just before and after it."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def wait_first(self, timeout: float = 2.0):
        """Return once the first sample has arrived (nvidia-smi is running)."""
        t0 = time.time()
        while self.proc is not None and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.01)

    def stop(self, region=None):
        """Median SM clock and the throttle reasons seen; region = (t0, t1)
        host times of the timed region: its samples are used when there are
        any, else every sample (a region shorter than the sampling interval)."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for t_recv, ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm_v, mx_v = float(parts[0]), float(parts[1])
            except ValueError:
                continue
            rows.append((t_recv, sm_v, mx_v, {nm for nm, v in zip(names, parts[4:8]) if v.lower().startswith("active")}))
        if not rows:
            return None
        # a sample's line arrives just after it was taken: within the region
        # when received between its start and its end plus one interval
        inside = [r for r in rows if region is not None and region[0] <= r[0] <= region[1] + 0.1]
        use = inside or rows
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": max(r[2] for r in rows),
                "reasons": sorted(set().union(*(r[3] for r in use))), "samples": len(rows),
                "samples_in_timed_region": len(inside)}


def reduce_max(x: float, ws: int, device) -> float:
    """Maximum of x over all ranks (the slowest rank's time)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(ws: int, nodes: int, steps: int, seconds: float) -> float:
    """Whole-job throughput: node updates of all ranks over the slowest time."""
    return ws * nodes * steps / seconds / 1e6


def make_case(size: int = 2048):
    from paper_1808_08555_gb300 import workloads as W
    return W.case_compound_2048() if size == 2048 else W.case_compound_scaled(size)


def workload_name(size: int) -> str:
    if size == 2048:
        return WORKLOAD
    return (f"compound double droplet {size}x{size} periodic (the 2048^2 workload with radii scaled by "
            f"{size}/2048), tau=(0.6,0.7,0.9), sigma12/13/23=0.01/0.012/0.005, beta0=0.7, FP32 arithmetic")


def run_ours(args, ws, rank, local):
    """The compound-droplet workload in the chosen form (reduced state) and the
    plain FP32 form; `value` is the chosen form's throughput (both give
    bit-identical states, so the error is equal by construction), the plain
    form is reported beside it.  --storage restricts the run to one form."""
    import torch

    from paper_1808_08555_gb300 import build as B
    if rank == 0 or ws == 1:
        B.build()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    from paper_1808_08555_gb300 import lbm3 as L

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    case = make_case(args.size or 2048)
    nodes = case.nx * case.ny
    forms = {"reduced": L.REDUCED, "fp32": L.FP32}
    order = ["reduced", "fp32"] if args.storage == "both" else [args.storage]

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    def max_over_ranks(x: float) -> float:
        return reduce_max(x, ws, dev)

    peak, peak_kind = hbm_peak()
    res = {}
    for name in order:
        p = L.Params(case.nx, case.ny, tau=case.tau, sigma=case.sigma, beta0=case.beta0, storage=forms[name])
        sim = L.Simulation(p, device=dev)
        stream = sim.stream
        sim.init(case.rho)
        sim.step(args.warmup)
        sim.sync()
        # ---------------- device-resident throughput (inputs already in HBM)
        clocks = ClockSampler(local)
        barrier()
        clocks.start()
        clocks.wait_first()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t_region = time.time()
        e0.record(stream)
        sim.step(args.steps)
        e1.record(stream)
        e1.synchronize()
        region = (t_region, time.time())
        ms = e0.elapsed_time(e1)
        clk = clocks.stop(region)
        sim.sync()
        barrier()
        ms = max_over_ranks(ms)
        m, mom = sim.mass()
        # ---------------- end to end through the C ABI with host buffers
        host_rho = torch.from_numpy(case.rho).pin_memory()
        outs = {k: torch.empty(sh, dtype=torch.float64).pin_memory() for k, sh in
                (("rho", (3, case.ny, case.nx)), ("ux", (case.ny, case.nx)), ("uy", (case.ny, case.nx)),
                 ("p", (case.ny, case.nx)))}
        barrier()
        t0 = time.perf_counter()
        L.lbm3_init(sim.ctx, host_rho)
        L.lbm3_step(sim.ctx, args.steps)
        L.lbm3_fields(sim.ctx, outs["rho"], outs["ux"], outs["uy"], outs["p"])
        e2e_s = time.perf_counter() - t0
        barrier()
        e2e_s = max_over_ranks(e2e_s)
        sim.close()
        bpn = BYTES_PER_NODE_REDUCED if name == "reduced" else BYTES_PER_NODE
        per_launch_s = ms / 1e3 / args.steps
        achieved = bpn * nodes / per_launch_s / 1e9
        res[name] = {
            "value": aggregate_mlups(ws, nodes, args.steps, ms / 1e3), "ms": ms, "clocks": clk,
            "mass": [float(x) for x in m], "momentum": [float(x) for x in mom],
            "e2e": ws * nodes * args.steps / e2e_s / 1e6,
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4),
                         "traffic": recorded_traffic(name) if case.nx == 2048 else None,
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                         else "fallback 6.8 TB/s", "bytes_per_node": bpn,
                         "kernel": f"{STEP_KERNEL}<{'reduced state' if name == 'reduced' else 'FP32 populations'}>"},
        }

    if rank != 0:
        return None
    head = order[0]
    h = res[head]
    total_updates = ws * nodes * args.steps
    line = {
        "metric": "ternary D2Q9 MLUPS (fused colour-gradient step, 2048^2 compound droplet)",
        "value": round(h["value"], 2),
        "unit": "MLUPS",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(h["ms"] / args.steps, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seedless analytic droplet fields, Eq. 21 tanh edges)",
        "config": {"workload": workload_name(case.nx), "nx": case.nx, "ny": case.ny, "nodes_per_step": nodes,
                   "form": head, "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": (f"inputs larger than L2: two {h['roofline']['bytes_per_node'] / 2 * case.ny * (case.nx + 8) / 1e6:.0f} MB "
                          "state buffers vs 129 MB L2") if case.nx >= 1024 else
                         "inputs smaller than L2 (small profiling case)"},
        "roofline": h["roofline"],
        "e2e": {"value": round(h["e2e"], 2), "unit": "MLUPS",
                "h2d_bytes_per_step": round(3 * nodes * 8 / args.steps, 1),
                "d2h_bytes_per_step": round(6 * nodes * 8 / args.steps, 1),
                "note": "lbm3_init from pinned host rho, K steps, lbm3_fields to pinned host; bytes amortised over K"},
        "gpu_launches": args.steps,
        "clocks": h["clocks"],
        "checks": {"mass": h["mass"], "momentum": h["momentum"]},
    }
    if len(order) > 1:
        line["forms"] = {n: {"MLUPS": round(r["value"], 2), "ms_per_step": round(r["ms"] / args.steps, 5),
                             "e2e_MLUPS": round(r["e2e"], 2), "roofline": r["roofline"], "clocks": r["clocks"]}
                         for n, r in res.items()}
        line["forms"]["equal_error"] = ("the reduced state rebuilds every population with the FP32 form's own "
                                        "operations: states and masses are bit-identical "
                                        f"(masses equal here: {res['reduced']['mass'] == res['fp32']['mass']})")
        line["speedup_vs_plain_fp32"] = round(res["reduced"]["value"] / res["fp32"]["value"], 4)
    if not args.no_cpu_baseline and ws == 1:
        line["cpu_baseline"] = cpu_baseline(case, args.cpu_steps)
    return line


def run_sweep(args):
    """Morphology sweep: 64 independent instances (grid edges drawn from
    {128,192,256,384,512} with seed 0, two touching droplets of radius N/6,
    sigma_12/sigma_23 and sigma_13/sigma_23 on an 8x8 grid of
    {0.2,...,2.0}), advanced together by one launch per step replayed from a
    CUDA graph, in the reduced state (headline) and with FP32 populations
    (bit-identical); the tile height is first the makespan model's, then the
    empirical tuner's.  Compared with the same instances stepped one after
    another with the single-grid kernel (FP32 populations)."""
    import torch

    from paper_1808_08555_gb300 import build as B
    B.build()
    from paper_1808_08555_gb300 import lbm3 as L
    from paper_1808_08555_gb300 import workloads as W

    cases = W.sweep_instances(seed=0)
    nodes = sum(c.nx * c.ny for c in cases)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(batch):
        s = batch.stream
        torch.cuda.synchronize()
        e0.record(s)
        batch.step(args.steps)
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1)

    forms = {}
    for name, storage in (("reduced", L.REDUCED), ("fp32", L.FP32)):
        if getattr(args, "storage", "both") not in ("both", name):
            continue
        params = [L.Params(c.nx, c.ny, tau=c.tau, sigma=c.sigma, beta0=c.beta0, storage=storage) for c in cases]
        batch = L.Batch(params)
        items_model = batch.work_items
        for i, c in enumerate(cases):
            batch.init(i, W.touching_droplets(c.nx))
        batch.step(args.warmup)
        batch.sync()
        ms_model = timed(batch)
        tune = batch.autotune(candidates=5, steps=20)
        batch.step(2)
        ms = timed(batch)
        forms[name] = {"MLUPS": nodes * args.steps / (ms / 1e3) / 1e6, "ms": ms, "work_items": batch.work_items,
                       "model": {"work_items": items_model,
                                 "MLUPS": round(nodes * args.steps / (ms_model / 1e3) / 1e6, 2)},
                       "autotuned": {"rows": tune["rows"], "candidates_ms_per_step": tune["candidates"]},
                       "mass_instance0": [float(v) for v in batch.mass(0)[0]]}
        batch.close()
    # the same instances one after another with the single-grid kernel
    sims = []
    for c in cases:
        sim = L.Simulation(L.Params(c.nx, c.ny, tau=c.tau, sigma=c.sigma, beta0=c.beta0))
        sim.init(W.touching_droplets(c.nx))
        sim.step(args.warmup)
        sims.append(sim)
    s = sims[0].stream
    torch.cuda.synchronize()
    e0.record(s)
    for sim in sims:
        sim.step(args.steps)
    e1.record(s)
    e1.synchronize()
    ms_seq = e0.elapsed_time(e1)
    for sim in sims:
        sim.close()
    peak, peak_kind = hbm_peak()
    out = {}
    for name, f in forms.items():
        bpn = BYTES_PER_NODE_REDUCED if name == "reduced" else BYTES_PER_NODE
        ach = bpn * nodes / (f["ms"] / 1e3 / args.steps) / 1e9
        out[name] = {"MLUPS": round(f["MLUPS"], 2), "ms_per_step": round(f["ms"] / args.steps, 5),
                     "work_items": f["work_items"], "tile_height": {"model": f["model"], "autotuned": f["autotuned"]},
                     "roofline": {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                                  "frac": round(ach / peak, 4), "traffic": None, "bytes_per_node": bpn,
                                  "kernel": f"fused_batch_param_kernel<{name}>", "peak_source": peak_kind}}
    head = "reduced" if "reduced" in out else "fp32"
    h = out[head]
    return {"metric": "ternary D2Q9 MLUPS, batched morphology sweep (64 instances)", "value": h["MLUPS"],
            "unit": "MLUPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": h["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sweep of 64 instances, edges {128..512} seed 0, touching droplets R=N/6",
                       "nodes_per_step": nodes,
                       "form": "reduced (headline); fp32 beside it" if len(out) == 2 else head},
            "forms": out,
            "equal_error": (forms["reduced"]["mass_instance0"] == forms["fp32"]["mass_instance0"]
                            if len(forms) == 2 else None),
            "sequential_single_instance": {"value": round(nodes * args.steps / (ms_seq / 1e3) / 1e6, 2),
                                           "unit": "MLUPS", "ms_per_step": round(ms_seq / args.steps, 5)},
            "roofline": h["roofline"],
            "gpu_launches": args.steps}


def run_janus(args):
    """Storage forms on the 4096^2 Janus droplet (fluid 2 left and fluid 3
    right half of one circle of radius 600, sigma = 0.010/0.008/0.012, a
    Neumann triangle): FP32 populations, FP16 and BF16 deviations and the
    reduced state; MLUPS and HBM fraction of each (216 B/node-update for FP32,
    132 B for the 16-bit forms, 144 B for the reduced state), and the FP64
    device diagnostics after the run (contact angles, bulk pressures) against
    the FP32 form's."""
    import torch

    from paper_1808_08555_gb300 import build as B
    B.build()
    from paper_1808_08555_gb300 import lbm3 as L
    from paper_1808_08555_gb300 import workloads as W

    n = args.size or 4096
    R = 600.0 * n / 4096
    rho = W.janus_droplet(n, R)
    peak, _ = hbm_peak()
    out = {}
    for st, name, bpn in ((0, "fp32", 216), (1, "fp16_dev", 132), (2, "bf16_dev", 132), (3, "reduced", 144)):
        sim = L.Simulation(L.Params(n, n, tau=(1.0, 1.0, 1.0), sigma=(0.010, 0.008, 0.012), storage=st))
        sim.init(rho)
        sim.step(args.warmup)
        sim.sync()
        s = sim.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        sim.step(args.steps)
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        m, _ = sim.mass()
        d = sim.interfaces()
        sim.close()
        mlups = n * n / ms / 1e3
        out[name] = {"MLUPS": round(mlups, 1), "ms_per_step": round(ms, 5), "bytes_per_node": bpn,
                     "hbm_frac": round(bpn * mlups * 1e6 / (peak * 1e9), 4), "mass": [float(v) for v in m],
                     "varphi_deg": [round(v, 4) for v in d["varphi"]], "p_bulk": d["p_bulk"]}
    for name in ("fp16_dev", "bf16_dev", "reduced"):
        out[name]["varphi_minus_fp32_deg"] = [round(a - b, 4) for a, b in
                                              zip(out[name]["varphi_deg"], out["fp32"]["varphi_deg"])]
    head = out["reduced"]
    return {"metric": "ternary D2Q9 MLUPS by state storage (Janus droplet)", "value": head["MLUPS"],
            "unit": "MLUPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"Janus droplet {n}x{n}, R={R:g}, sigma=0.010/0.008/0.012, tau=1",
                       "form": "reduced (headline); every storage in 'storages'",
                       "state_after": f"{args.warmup + args.steps} steps from the straight split (a transient)"},
            "storages": out,
            "roofline": {"bound": "hbm", "achieved": round(144 * head["MLUPS"] / 1e3, 1),
                         "peak": peak, "unit": "GB/s", "frac": head["hbm_frac"], "traffic": None,
                         "bytes_per_node": 144, "kernel": "fused_step_kernel<reduced state>"},
            "gpu_launches": args.steps}


def run_nphase(args):
    """N fluids (three kernels per step): four fluids in a nested droplet on
    an n x n grid (default 2048^2; radii 3n/8, n/4, n/8), tensions 0.01 /
    0.008 / 0.006 between neighbouring layers and 0.012 otherwise, tau =
    (1.0, 0.8, 0.9, 1.2), in the reduced state (the headline) and with FP32
    populations (bit-identical trajectories); --storage restricts the run to
    one form.  Algorithmic bytes per node update are the state's: 2 x 9N x 4 =
    288 B for the populations, 2 x (3N + 9) x 4 = 168 B for the reduced state
    at N = 4; the three kernels also move their intermediates through HBM
    (written once, read by the next kernel; the stencil reads from L2)."""
    import torch

    from paper_1808_08555_gb300 import build as B
    B.build()
    from paper_1808_08555_gb300 import lbm3 as L
    from paper_1808_08555_gb300 import workloads as W

    n = args.size or 2048
    y, x = np.mgrid[0:n, 0:n].astype(float)
    r = np.hypot(x - n / 2, y - n / 2)
    disc = [0.5 + 0.5 * np.tanh((R - r) / W.XI) for R in (3 * n / 8, n / 4, n / 8)]
    rho = np.stack([np.clip(1 - disc[0], 0, None), np.clip(disc[0] - disc[1], 0, None),
                    np.clip(disc[1] - disc[2], 0, None), disc[2]])
    sig = np.full((4, 4), 0.012)
    np.fill_diagonal(sig, 0.0)
    for (k, l, v) in ((0, 1, 0.01), (1, 2, 0.008), (2, 3, 0.006)):
        sig[k, l] = sig[l, k] = v
    storage = getattr(args, "storage", "both")
    order = ["reduced", "fp32"] if storage == "both" else [storage]
    peak, peak_kind = hbm_peak()
    forms, masses = {}, {}
    for name in order:
        sim = L.NSimulation(n, n, sig, tau=(1.0, 0.8, 0.9, 1.2), storage=L.REDUCED if name == "reduced" else L.FP32)
        sim.init(rho)
        sim.step(args.warmup)
        s = sim.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        sim.step(args.steps)
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        masses[name] = [float(v) for v in sim.mass()[0]]
        sim.close()
        mlups = n * n / ms / 1e3
        bpn = 2 * (3 * 4 + 9) * 4 if name == "reduced" else 2 * 9 * 4 * 4
        forms[name] = {"MLUPS": round(mlups, 1), "ms_per_step": round(ms, 5), "bytes_per_node": bpn,
                       "achieved_GBs": round(bpn * mlups / 1e3, 1),
                       "frac": round(bpn * mlups * 1e6 / (peak * 1e9), 4)}
    head = forms[order[0]]
    checks = {"mass": masses[order[0]]}
    if len(masses) == 2:
        checks["same_masses_both_forms"] = masses["reduced"] == masses["fp32"]
    return {"metric": "D2Q9 MLUPS, four fluids (N-fluid path)", "value": head["MLUPS"], "unit": "MLUPS",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"four-fluid nested droplet {n}x{n}, radii {3 * n // 8}/{n // 4}/{n // 8}",
                       "form": order[0] + (" (headline); fp32 populations in 'forms'" if len(order) == 2 else "")},
            "roofline": {"bound": "hbm", "achieved": head["achieved_GBs"], "peak": peak, "unit": "GB/s",
                         "frac": head["frac"], "traffic": None, "bytes_per_node": head["bytes_per_node"],
                         "kernel": "n_density + n_tension + n_collide kernels (N = 4)", "peak_source": peak_kind},
            "forms": forms, "checks": checks, "gpu_launches": 3 * args.steps * len(order)}


def run_d3q19(args):
    """Three fluids on the D3Q19 lattice (three kernels per step): two spheres,
    fluid 2 (R = 3n/16 at x = n/4) and fluid 3 (R = 5n/32 at x = 3n/4), in
    fluid 1 on an n^3 grid (default 256^3), sigma_12 / 13 / 23 = 0.01 / 0.013
    / 0.007, tau = (0.6, 0.9, 1.3), in the reduced state (the headline) and
    with FP32 populations (bit-identical trajectories); --storage restricts
    the run to one form.  Algorithmic bytes per node update are the state's:
    2 x 19N x 4 = 456 B for the populations, 2 x (19 + 4N) x 4 = 248 B for
    the reduced state at N = 3; the kernels also move their intermediates
    through HBM."""
    import torch

    from paper_1808_08555_gb300 import build as B
    B.build()
    from paper_1808_08555_gb300 import lbm3 as L
    from paper_1808_08555_gb300 import workloads as W

    n = args.size or 256
    rho = W.spheres_3d(n, n, n, [(1, (n / 4, n / 2, n / 2), 3 * n / 16), (2, (3 * n / 4, n / 2, n / 2), 5 * n / 32)])
    sig = np.array([[0.0, 0.01, 0.013], [0.01, 0.0, 0.007], [0.013, 0.007, 0.0]])
    storage = getattr(args, "storage", "both")
    order = ["reduced", "fp32"] if storage == "both" else [storage]
    peak, peak_kind = hbm_peak()
    forms, masses = {}, {}
    for name in order:
        sim = L.D3Q19Simulation(n, n, n, sig, tau=(0.6, 0.9, 1.3),
                                storage=L.REDUCED if name == "reduced" else L.FP32)
        sim.init(rho)
        sim.step(args.warmup)
        s = sim.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        sim.step(args.steps)
        e1.record(s)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        masses[name] = [float(v) for v in sim.mass()[0]]
        sim.close()
        torch.cuda.empty_cache()
        mlups = n ** 3 / ms / 1e3
        bpn = 2 * (19 + 4 * 3) * 4 if name == "reduced" else 2 * 19 * 3 * 4
        forms[name] = {"MLUPS": round(mlups, 1), "ms_per_step": round(ms, 5), "bytes_per_node": bpn,
                       "achieved_GBs": round(bpn * mlups / 1e3, 1),
                       "frac": round(bpn * mlups * 1e6 / (peak * 1e9), 4)}
    del rho
    head = forms[order[0]]
    checks = {"mass": masses[order[0]]}
    if len(masses) == 2:
        checks["same_masses_both_forms"] = masses["reduced"] == masses["fp32"]
    return {"metric": "D3Q19 MLUPS, three fluids (3D path)", "value": head["MLUPS"], "unit": "MLUPS",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"two spheres of fluids 2 and 3 in fluid 1, {n}^3, R {3 * n // 16}/{5 * n // 32}",
                       "form": order[0] + (" (headline); fp32 populations in 'forms'" if len(order) == 2 else "")},
            "roofline": {"bound": "hbm", "achieved": head["achieved_GBs"], "peak": peak, "unit": "GB/s",
                         "frac": head["frac"], "traffic": None, "bytes_per_node": head["bytes_per_node"],
                         "kernel": "d_density + d_tension + d_collide kernels (N = 3)", "peak_source": peak_kind},
            "forms": forms, "checks": checks, "gpu_launches": 3 * args.steps * len(order)}


def run_adjoint(args):
    """Reverse mode on the gradient workload: 256^2 touching discs (sigma =
    0.01 each, tau = 1), J = sum (phi - phi_target)^2 after 2000 steps, the
    gradient dJ/drho0 (all nodes) and dJ/dsigma by lbm3_tape_forward +
    lbm3_tape_backward.  One timed step = one full gradient evaluation
    (forward run recorded + reverse run), with every state kept
    (checkpoint_every = 1: 2000 x 7 MB fit easily in HBM) and, beside it, with
    checkpoints every 100 steps (segments recomputed).  MLUPS counts the
    2000 x N node updates of the forward run per evaluation."""
    import torch

    from paper_1808_08555_gb300 import build as B
    B.build()
    from paper_1808_08555_gb300 import lbm3 as L
    from paper_1808_08555_gb300 import workloads as W

    n = args.size or 256
    horizon = args.horizon
    rho0, tgt = W.case_adjoint(n)
    phit = torch.tensor(tgt / tgt.sum(axis=0), device="cuda")
    sim = L.Simulation(L.Params(n, n, sigma=(0.01, 0.01, 0.01)))
    rho_d = torch.tensor(rho0, device="cuda")
    phi = torch.empty_like(rho_d)
    drho = torch.empty_like(rho_d)
    s = sim.stream
    res = {}
    for every in (1, 100):
        def evaluate():
            L.lbm3_init(sim.ctx, rho_d)
            L.lbm3_tape_forward(sim.ctx, horizon, every)
            L.lbm3_phi(sim.ctx, phi)
            return L.lbm3_tape_backward(sim.ctx, 2 * (phi - phit), None, drho)
        for _ in range(args.warmup):
            ds = evaluate()
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        fwd = 0.0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e[0].record(s)
            L.lbm3_init(sim.ctx, rho_d)
            L.lbm3_tape_forward(sim.ctx, horizon, every)
            L.lbm3_phi(sim.ctx, phi)
            e[1].record(s)
            ds = L.lbm3_tape_backward(sim.ctx, 2 * (phi - phit), None, drho)
            e[2].record(s)
            e[2].synchronize()
            fwd += e[0].elapsed_time(e[1])
        ms = (time.perf_counter() - t0) * 1e3 / args.steps
        J = float(((phi - phit) ** 2).sum())
        res[every] = {"ms_per_gradient": round(ms, 3), "ms_forward_recorded": round(fwd / args.steps, 3),
                      "ms_reverse": round(ms - fwd / args.steps, 3),
                      "MLUPS": round(n * n * horizon / (ms / 1e3) / 1e6, 1), "loss": J,
                      "dJ_dsigma": [float(v) for v in ds]}
    sim.close()
    golden = os.path.join(ROOT, "tests", "golden", f"adjoint_fd_{n}.json")
    check = None
    if os.path.exists(golden):
        g = json.load(open(golden))
        if g["steps"] == horizon:
            check = {"max_rel_err_dJ_dsigma_vs_oracle_differences":
                     float(max(abs(a / b - 1) for a, b in zip(res[1]["dJ_dsigma"], g["dJ_dsigma"])))}
    best = res[1]
    peak, peak_kind = hbm_peak()
    # algorithmic bytes per node-step of one evaluation with every state kept:
    # 216 forward + 616 reverse (272 node VJP, 236 tension VJP + densities,
    # 108 gradient VJP + grad phi and T of the next state)
    achieved = 832 * best["MLUPS"] / 1e3
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None, "bytes_per_node": 832,
                "kernel": "one gradient evaluation (fused step + three adjoint kernels per step)",
                "peak_source": peak_kind}
    return {"metric": "ternary D2Q9 gradient evaluations: forward-run MLUPS through reverse mode",
            "value": best["MLUPS"], "unit": "MLUPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": best["ms_per_gradient"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (gradient sums f64)", "data": "synthetic",
            "config": {"workload": f"gradient workload {n}x{n}: touching discs R=n/6, sigma=0.01, tau=1, "
                                   f"J = sum (phi - phi_target)^2 after {horizon} steps, dJ/drho0 and dJ/dsigma",
                       "horizon_steps": horizon, "step": "one full gradient evaluation (recorded forward + reverse)",
                       "l2": "state 7 MB per step: L2-resident at this size"},
            "checkpoint_every": {str(k): v for k, v in res.items()}, "checks": check, "roofline": roofline,
            "gpu_launches": args.steps * (1 + horizon + 1 + 3 + 6 * horizon + 1)}


def cpu_baseline(case, steps: int):
    """The FP64 oracle as it stands on a bounded sample of the same workload
    (`steps` steps of the full grid), on all host cores (its node loops run
    under OpenMP; the results do not depend on the thread count) and on one
    core.  The all-cores figure is the baseline; the one-core figure is
    reported beside it."""
    import oracle as O
    op = O.Params(case.nx, case.ny, tau=case.tau, sigma=case.sigma, beta0=case.beta0)
    f = O.init(op, case.rho)
    out = {}
    for cores in (os.cpu_count() or 1, 1):
        used = O.threads(cores)
        t0 = time.perf_counter()
        O.step(op, f, steps)
        dt = time.perf_counter() - t0
        out[cores] = (used, dt)
    O.threads(os.cpu_count() or 1)
    (used, dt), (_, dt1) = out[os.cpu_count() or 1], out[1]
    rate = lambda t: round(case.nx * case.ny * steps / t / 1e6, 4)
    return {"value": rate(dt), "unit": "MLUPS", "cores": used, "kind": "oracle",
            "sample": f"{steps} steps of the full {case.nx}x{case.ny} grid ({dt:.1f} s on {used} threads)",
            "single_core": {"value": rate(dt1), "cores": 1, "seconds": round(dt1, 1)}}


def run_reference(args, ws, rank):
    """The FP64 oracle as it stands, on all host cores (OpenMP over its node
    loops).  Each timed step is one lattice step of an n x n window cut from
    the centre of the same workload (through the droplet's interfaces), with
    n chosen from a short probe of the oracle's speed so that the K timed
    steps take about --ref-seconds (default two minutes) whatever K is (the
    full grid when that fits)."""
    if rank != 0:
        return None
    case = make_case(args.size or 2048)
    import oracle as O
    O.build()
    cores = O.threads(os.cpu_count() or 1)

    def window(n):
        y0, x0 = (case.ny - n) // 2, (case.nx - n) // 2
        rho = np.ascontiguousarray(case.rho[:, y0:y0 + n, x0:x0 + n])
        op = O.Params(n, n, tau=case.tau, sigma=case.sigma, beta0=case.beta0)
        return op, O.init(op, rho)

    # size the window from the oracle's speed, then re-measure at that size
    # (small windows pay the threads' start-up per loop; at most one thread
    # per 16384 nodes)
    def use_threads(n):
        return O.threads(max(1, min(cores, n * n // 16384)))

    n = min(256, case.nx, case.ny)
    for _ in range(3):
        used = use_threads(n)
        op, f = window(n)
        t0 = time.perf_counter()
        O.step(op, f, 2)
        rate = 2 * n * n / (time.perf_counter() - t0)          # node updates per second
        n_new = int(math.sqrt(args.ref_seconds * rate / max(1, args.steps))) // 4 * 4
        n_new = max(16, min(n_new, case.nx, case.ny))
        if abs(n_new - n) <= max(4, n // 8):
            n = n_new
            break
        n = n_new
    used = use_threads(n)
    op, f = window(n)
    for _ in range(min(args.warmup, 1)):
        f = O.step(op, f, 1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        f = O.step(op, f, 1)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n * n * len(times) / total / 1e6
    sample = f"each step = one lattice step of the central {n}x{n} window of the {case.nx}x{case.ny} workload"
    return {
        "impl": "reference",
        "metric": "ternary D2Q9 MLUPS (fused colour-gradient step, 2048^2 compound droplet)",
        "value": round(value, 4), "unit": "MLUPS", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total / args.steps * 1e3, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(case.nx), "nx": case.nx, "ny": case.ny, "sample_window": n},
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": used, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def other_workloads(args):
    """The other configurations, shortened so that together they add about a
    minute: the batched sweep, the storage forms on the 4096^2 Janus droplet,
    gradient evaluations, four fluids on D2Q9 and three on D3Q19.  Each entry
    is that workload's own line without its bulky fields, or its error."""
    import copy

    import torch

    plan = [("sweep", run_sweep, 500, 20), ("janus", run_janus, 300, 10), ("adjoint", run_adjoint, 3, 1),
            ("nphase", run_nphase, 200, 10), ("d3q19", run_d3q19, 50, 3)]
    out = {}
    for name, fn, steps, warmup in plan:
        a = copy.copy(args)
        a.steps, a.warmup, a.size, a.workload = steps, warmup, None, name
        try:
            d = fn(a)
            keep = ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "config", "roofline", "forms",
                    "storages", "sequential_single_instance", "equal_error", "checks", "gpu_launches")
            out[name] = {k: d[k] for k in keep if k in d}
        except Exception as e:  # reported, never fatal to the headline
            out[name] = {"error": f"{type(e).__name__}: {e}"[:300]}
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--ref-seconds", type=float, default=120.0,
                    help="--impl reference: time budget of the timed steps (sets the sampled window)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="default run: skip the shortened runs of the other configurations (sweep, Janus storage "
                         "forms, gradient, N fluids, D3Q19) that are added to the line under other_workloads")
    ap.add_argument("--workload", default="compound", choices=["compound", "sweep", "janus", "adjoint", "nphase", "d3q19"],
                    help="compound: the 2048^2 compound droplet (default); sweep: the 64-instance batch; "
                         "janus: the 4096^2 Janus droplet with FP32 / FP16 / BF16 storage; "
                         "adjoint: gradient evaluations of the 256^2 gradient workload; nphase: four fluids, "
                         "2048^2; d3q19: three fluids on the D3Q19 lattice, 256^3")
    ap.add_argument("--horizon", type=int, default=2000,
                    help="adjoint workload: steps of the differentiated run (2000 is the workload; fewer for profiling)")
    ap.add_argument("--storage", default="both", choices=["both", "fp32", "reduced"],
                    help="compound, sweep, nphase and d3q19 workloads: state storage (both: the reduced form as the headline and the "
                         "plain FP32 form beside it; fp32: 27 populations only; reduced: phi_k, f^dagger_i, V_k only)")
    ap.add_argument("--size", type=int, default=None,
                    help="grid edge (default: 2048 compound, 4096 janus, 256 adjoint); other edges scale the "
                         "droplet radii (profiling and larger cases only)")
    args = ap.parse_args()
    # default K / W per workload: a step of the adjoint workload is a whole
    # gradient evaluation (~60-80 ms), of the others one lattice step
    dflt = {"compound": (5000, 50), "sweep": (2000, 20), "janus": (1000, 20), "adjoint": (10, 3),
            "nphase": (500, 10), "d3q19": (200, 5)}[args.workload]
    if args.steps is None:
        args.steps = 3 if args.impl == "reference" else dflt[0]
    if args.warmup is None:
        args.warmup = 3 if args.impl == "reference" else dflt[1]
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        if backend == "nccl":
            import torch
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            line = run_reference(args, ws, rank)
        elif args.workload == "sweep":
            line = run_sweep(args) if rank == 0 else None
        elif args.workload == "janus":
            line = run_janus(args) if rank == 0 else None
        elif args.workload == "adjoint":
            line = run_adjoint(args) if rank == 0 else None
        elif args.workload == "nphase":
            line = run_nphase(args) if rank == 0 else None
        elif args.workload == "d3q19":
            line = run_d3q19(args) if rank == 0 else None
        else:
            line = run_ours(args, ws, rank, local)
            # one GPU, the default workload: the other configurations as well,
            # after the timed headline
            if line is not None and ws == 1 and args.size is None and not args.no_other_workloads:
                line["other_workloads"] = other_workloads(args)
        if line is not None:
            print(json.dumps(line), flush=True)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
