#!/usr/bin/env python
"""Throughput benchmark of the GB300 lattice Boltzmann hot path.

Metric: GLUPS (10^9 lattice-node updates per second) of the fused
collide-and-stream step, next to the HBM roofline of its algorithmic traffic
(2 Q s bytes per node update: every population read once and written once).

Default workload: periodic 3D Taylor-Green vortex, 512^3 nodes, D3Q19, FP32
populations, Re = 1600, u0 = 0.04 (tau = 0.506112), BGK.  One benchmark step
is ``inner`` lattice steps followed by the FP64 reduction (mass, momentum,
kinetic energy) read back to the host, as a run that samples its kinetic
energy does; the reduction is fused into the last step
(``lbm_step_reduce``).  Inputs (two population arrays of 10.2 GB each) are far larger
than L2, so no flush is needed between steps.

Also reported: ``e2e`` (each step uploads the initial fields from pinned host
memory through the C ABI, runs the lattice steps and reads the reduction
back), FP16/BF16-shifted and other workload variants with their error against
the FP64 run, SM clocks sampled during the timed region, and the CPU oracle
timed on the host cores.

Launch: ``python bench.py [--gpus N --steps K --warmup W]``; for N > 1 under
torchrun every rank runs an independent replica (the path has no exchange
step on one lattice per GPU), timing is the max over ranks, and the value is
the sum over ranks.  ``--impl reference`` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

METRIC = "GLUPS per GB300 vs HBM roofline; FP32 vs FP16-shifted storage at stated error"
UNIT = "GLUPS"
SIZE = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2, "f16s": 2}


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------
def tgv_tau(n: int, u0: float, re: float) -> float:
    """tau for a Taylor-Green vortex whose reference length is n / (2 pi)."""
    return 0.5 + 3.0 * u0 * (n / (2.0 * math.pi)) / re


_FIELDS = {}


def tgv_fields(n: int):
    """The 3D Taylor-Green initial fields, generated once per size."""
    import lbm_inputs as inp
    if n not in _FIELDS:
        _FIELDS.clear()
        _FIELDS[n] = inp.tgv3d(n, 0.04)
    return _FIELDS[n]


CLOSURES = ("bgk", "smagorinsky", "mlp")


def make_workload(name: str, dtype: str, closure: str = "bgk", pattern: str = "ab"):
    """Returns (lattice, fields, description) with the lattice initialised.
    closure "mlp" installs seeded random network weights: the cost of the
    learned closure does not depend on the weight values.  pattern "aa"
    streams in place in one population array."""
    import numpy as np
    import lbm_inputs as inp
    from paper_2506_09242_gb300 import lbm

    m = re.fullmatch(r"(tgv|cavity|porous)(\d+)_d3q(19|27)", name)
    if not m:
        raise SystemExit(f"unknown workload {name}")
    kind, n, Q = m.group(1), int(m.group(2)), int(m.group(3))
    lat = lbm.Lattice(n, n, n, Q, dtype, pattern=pattern)
    ckind = {"bgk": lbm.CLOSURE_BGK, "smagorinsky": lbm.CLOSURE_SMAGORINSKY, "mlp": lbm.CLOSURE_MLP}[closure]
    if closure == "mlp":
        norm = np.concatenate([np.zeros(6), [1.0], np.full(6, 1e-3), [0.01], [1e-4, 0.0]])
        lat.set_closure_weights(inp.mlp_init(0).astype(np.float32), norm.astype(np.float32))
    if kind == "tgv":
        tau = tgv_tau(n, 0.04, 1600.0)
        lat.set_params(tau, closure=ckind, cs_smag=0.1)
        rho, u = tgv_fields(n)
        desc = {"workload": f"tgv3d_{n}_d3q{Q}_{dtype}", "problem": "periodic 3D Taylor-Green vortex",
                "u0": 0.04, "Re": 1600, "tau": tau}
    elif kind == "porous":
        centres, radii = inp.sphere_list((n, n, n), seed=2506, rmin=4.0, rmax=10.0, count=100_000)
        _, por = lat.geometry_spheres(centres, radii, 0.2, lbm.TAG_FORCED)
        lat.set_params(1.0, force=(1e-6, 0.0, 0.0), closure=ckind, cs_smag=0.1)
        rho, u = None, None
        desc = {"workload": f"porous_{n}_d3q{Q}_{dtype}", "problem": "random-sphere porous medium, body force",
                "porosity": por, "g": 1e-6, "tau": 1.0}
    else:
        tau = 0.5 + 3.0 * 0.1 * n / 1000.0
        lat.set_tags(inp.cavity_tags(n))
        lat.set_params(tau, wall_u=[(0.1, 0.0, 0.0)], closure=ckind, cs_smag=0.1)
        rho, u = None, None
        desc = {"workload": f"cavity_{n}_d3q{Q}_{dtype}", "problem": "lid-driven cavity, Ladd lid",
                "u_lid": 0.1, "Re": 1000, "tau": tau}
    lat.init_equilibrium(rho, u)
    census = lat.census()
    desc.update({"lattice": f"D3Q{Q}", "storage": dtype, "nx": n, "ny": n, "nz": n, "closure": closure,
                 "fluid_nodes": int(census[lbm.TAG_FLUID] + census[lbm.TAG_FORCED])})
    if closure != "bgk":
        desc["workload"] += f"_{closure}"
    if pattern != "ab":
        desc["workload"] += f"_{pattern}"
        desc["pattern"] = pattern
    return lat, (rho, u), desc


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            self.out = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                 "-lms", "200"], stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:  # no nvidia-smi: no clock record
            self.proc = None
            if self.path:
                self.out.close()
                os.unlink(self.path)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        with open(self.path) as fh:
            summary = parse_clock_samples(fh)
        os.unlink(self.path)
        return summary


def parse_clock_samples(lines):
    """Summary of nvidia-smi rows in ClockSampler.FIELDS order: the median SM
    clock, the largest maximum clock, and the slowdown reasons seen Active in
    any row; None when no row parses."""
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm = float(parts[1].split()[0])
            smax = float(parts[2].split()[0])
        except (ValueError, IndexError):
            continue
        rows.append((sm, smax, parts[5:9]))
    if not rows:
        return None
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[k] for _, _, flags in rows for k, f in enumerate(flags) if f.lower() == "active"})
    return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
            "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# Timing helpers
# ---------------------------------------------------------------------------
def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for name in ("lbm_kernels.cuh", "lbm_internal.cuh"):
        h.update((ROOT / "paper_2506_09242_gb300" / "csrc" / name).read_bytes())
    return h.hexdigest()[:16]


def recorded_traffic(workload: str):
    """DRAM bytes per collide-stream launch from the committed ncu summary, if
    it was taken on the current kernel source."""
    for p in (ROOT / "profiles").glob("*.md"):
        text = p.read_text()
        if f"workload: {workload}" not in text:
            continue
        m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
        s = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
        if m and s and s.group(1) == kernel_source_hash():
            return float(m.group(1))
    return None


def recorded_fp64_ops(workload: str):
    """FP64 instructions per node update of the collide-stream kernel (DFMA,
    DADD and DMUL counted by ncu), if recorded on the current kernel source."""
    for p in (ROOT / "profiles").glob("*.md"):
        text = p.read_text()
        if f"workload: {workload}" not in text:
            continue
        m = re.search(r"fp64_inst_per_node:\s*([0-9.eE+]+)", text)
        s = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
        if m and s and s.group(1) == kernel_source_hash():
            return float(m.group(1))
    return None


def measured_peak_hbm():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        try:
            return float(json.loads(p.read_text())["hbm_gbs"]), "measured"
        except (KeyError, ValueError):
            pass
    return 6800.0, "fallback"


def time_lattice(lat, steps: int, warmup: int, inner: int, sync_all=None):
    """Times ``steps`` benchmark steps (inner lattice steps + reduction).

    Returns (total_ms, mean collide-stream launch ms, reductions, per-step ms)."""
    import torch
    for _ in range(warmup):
        lat.step(inner - 1)
        lat.step_reduce(1)
    torch.cuda.synchronize()
    if sync_all:
        sync_all()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    reds = []
    t0.record()
    for k in range(steps):
        ev[k][0].record()
        lat.step(inner - 1)
        ev[k][1].record()
        reds.append(lat.step_reduce(1))  # last step fused with the FP64 reduction
    t1.record()
    torch.cuda.synchronize()
    if sync_all:
        sync_all()
    total = t0.elapsed_time(t1)
    kernel = sum(a.elapsed_time(b) for a, b in ev) / (steps * (inner - 1))
    marks = [e[0] for e in ev] + [t1]
    per_step = [marks[k].elapsed_time(marks[k + 1]) for k in range(steps)]
    return total, kernel, reds, per_step


def d2d_copy_gbs(nbytes: int = 1 << 32, reps: int = 5) -> float:
    """Bandwidth of a plain device-to-device copy (bytes read + written per
    second), for context next to the measured peak; torch's copy kernel."""
    import torch
    a = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    b = torch.empty_like(a)
    b.copy_(a)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        b.copy_(a)
    e1.record()
    torch.cuda.synchronize()
    gbs = 2 * nbytes * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9
    del a, b
    torch.cuda.empty_cache()
    return gbs


def time_e2e(lat, fields, steps: int, inner: int):
    """Each step: upload rho and u from pinned host memory, run ``inner``
    lattice steps, read the reduction back (all through the C ABI)."""
    import numpy as np
    import torch
    rho, u = fields
    if rho is None:  # cavity: start from rest with uniform density
        rho = np.ones((lat.nz, lat.ny, lat.nx))
        u = np.zeros((3, lat.nz, lat.ny, lat.nx))
    rho_h = torch.from_numpy(np.ascontiguousarray(rho)).pin_memory()
    u_h = torch.from_numpy(np.ascontiguousarray(u)).pin_memory()
    lat.init_equilibrium(rho_h, u_h)  # warm-up of the staging buffers
    lat.step_reduce(inner)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(steps):
        lat.init_equilibrium(rho_h, u_h)
        lat.step_reduce(inner)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t) * 1e3
    h2d = rho_h.numel() * 8 + u_h.numel() * 8
    d2h = 12 * 8  # the reduction struct
    return ms, h2d, d2h


def replica_throughput(local_ms: float, local_updates: int, dist=None, device: str = "cpu"):
    """Whole-job throughput of independent replicas (one lattice per rank, no
    exchange): node updates summed over ranks divided by the slowest rank's
    time.  Returns (GLUPS, max ms)."""
    if dist is None:
        return local_updates / (local_ms * 1e-3) / 1e9, local_ms
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_updates)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms = float(t.item())
    return float(u.item()) / (ms * 1e-3) / 1e9, ms


def host_info() -> dict:
    """Core count, CPU model and architecture of the host."""
    import platform
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if not model.isdigit():
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and Path("/proc/cpuinfo").exists():
        for line in Path("/proc/cpuinfo").read_text().splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    return {"nproc": os.cpu_count(), "cpu_model": model, "arch": platform.machine()}


# (Q, n, threads, warm-up steps, timed steps, repeats); threads 0 = every host core
CPU_PLANS = {
    # bounded: about a minute of CPU work inside the default bench run
    "bounded": [(19, 128, 0, 2, 10, 3), (27, 128, 0, 2, 10, 3), (19, 256, 0, 2, 10, 3), (27, 256, 0, 2, 10, 3),
                (19, 128, 1, 1, 3, 3), (27, 128, 1, 1, 3, 3)],
    # the full measurement plan: single thread and all cores, 128^3 and 256^3,
    # D3Q19 and D3Q27, 10 steps after 2 warm-up steps, 3 repeats
    "full": [(q, n, t, 2, 10, 3) for t in (0, 1) for n in (128, 256) for q in (19, 27)],
    # its single-thread half (one core; can run beside other work)
    "single": [(q, n, 1, 2, 10, 3) for n in (128, 256) for q in (19, 27)],
}


def oracle_timing(Q: int, n: int, threads: int, warmup: int, steps: int, repeats: int) -> dict:
    """FP64 CPU oracle on the host: periodic 3D TGV n^3 (u0 = 0.04, Re = 1600),
    OpenMP over the z planes with the given number of threads.  Returns the
    mean MLUPS over the repeats, each repeat timing ``steps`` steps."""
    import lbm_inputs as inp
    import oracle
    cores = oracle.set_threads(threads if threads > 0 else (os.cpu_count() or 1))
    rho, u = inp.tgv3d(n, 0.04)
    prob = oracle.Problem(Q, n, n, n, tau=tgv_tau(n, 0.04, 1600.0), openmp=True)
    f = prob.step(prob.init_equilibrium(rho, u), warmup)
    rates = []
    for _ in range(repeats):
        t = time.perf_counter()
        f = prob.step(f, steps)
        rates.append(n ** 3 * steps / (time.perf_counter() - t) / 1e6)
    return {"lattice": f"D3Q{Q}", "n": n, "threads": cores, "mlups": statistics.mean(rates),
            "mlups_per_core": statistics.mean(rates) / cores, "spread": [min(rates), max(rates)],
            "steps": steps, "warmup": warmup, "repeats": repeats}


def cpu_baseline(plan: str = "bounded") -> dict:
    """The oracle timed on the host cores (the ``cpu_baseline`` object): the
    headline value is D3Q19 256^3 on every core, in GLUPS."""
    rows = [oracle_timing(*cfg) for cfg in CPU_PLANS[plan]]
    head = next(r for r in rows if r["lattice"] == "D3Q19" and r["n"] == 256 and r["threads"] > 1) \
        if any(r["threads"] > 1 for r in rows) else rows[0]
    return {"value": head["mlups"] / 1e3, "unit": UNIT, "cores": head["threads"],
            "per_core": head["mlups_per_core"] / 1e3, "kind": "oracle",
            "sample": (f"periodic 3D TGV {head['n']}^3 {head['lattice']} FP64 oracle, {head['steps']} steps after "
                       f"{head['warmup']} warm-up, mean of {head['repeats']} repeats, {head['threads']} threads "
                       f"(OpenMP over z planes)"),
            "host": host_info(), "plan": plan, "table": rows}


# ---------------------------------------------------------------------------
# Arms
# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import lbm_inputs as inp
    import oracle
    n = args.ref_n
    cores = oracle.set_threads(os.cpu_count() or 1)
    rho, u = inp.tgv3d(n, 0.04)
    prob = oracle.Problem(19, n, n, n, tau=tgv_tau(n, 0.04, 1600.0), openmp=True)
    f = prob.init_equilibrium(rho, u)
    for _ in range(args.warmup):
        f = prob.step(f, 1)
    t = time.perf_counter()
    for _ in range(args.steps):
        f = prob.step(f, 1)
    dt = time.perf_counter() - t
    glups = n ** 3 * args.steps / dt / 1e9
    sample = (f"periodic 3D TGV {n}^3 (bounded sample of the 512^3 workload), D3Q19 FP64 oracle, "
              f"{cores} threads (OpenMP over z planes)")
    line = {
        "impl": "reference", "metric": METRIC, "value": glups, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "tgv3d_512_d3q19_f32", "sample_n": n, "inner_steps": 1},
        "cpu_baseline": {"value": glups, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                         "host": host_info()},
        "e2e": {"value": glups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_cpu_baseline_only(args):
    """Only the oracle timing (no GPU): the ``cpu_baseline`` object as one
    JSON line."""
    print(json.dumps({"cpu_baseline": cpu_baseline(args.cpu_plan)}), flush=True)
    return 0


def error_vs_f64(dtypes=("f32", "f16", "bf16", "f16s"), n=64, steps=400):
    """Velocity relative L2 error of each storage type against the FP64 run of
    the same lattice (periodic 3D TGV n^3, D3Q19, u0 = 0.04, Re = 1600 at n)."""
    import numpy as np
    import lbm_inputs as inp
    from paper_2506_09242_gb300 import lbm
    rho, u = inp.tgv3d(n, 0.04)
    tau = tgv_tau(n, 0.04, 1600.0)
    res = {}
    ref = None
    for dt in ("f64",) + tuple(dtypes):
        with lbm.Lattice(n, n, n, 19, dt) as lat:
            lat.set_params(tau)
            lat.init_equilibrium(rho, u)
            lat.step(steps)
            _, uu = lat.moments()
        if dt == "f64":
            ref = uu
        else:
            res[dt] = float(np.linalg.norm(uu - ref) / np.linalg.norm(ref))
    return {"case": f"periodic 3D TGV {n}^3 D3Q19 Re=1600, {steps} steps, velocity rel. L2 vs the FP64 run",
            **res}


def run_ours(args):
    import torch
    from paper_2506_09242_gb300 import _build
    _build.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def sync_all():
        if dist is not None:
            dist.barrier()

    lat, fields, desc = make_workload(args.workload, args.dtype, args.closure, args.pattern)
    Q = int(desc["lattice"][3:])
    cells = lat.N
    sampler = ClockSampler(local)
    sampler.start()
    total_ms, kernel_ms, reds, per_step = time_lattice(lat, args.steps, args.warmup, args.inner, sync_all)
    clocks = sampler.stop()
    glups, total_ms = replica_throughput(total_ms, cells * args.inner * args.steps, dist, "cuda")

    # roofline of the dominant kernel (collide-stream), timed on its stream
    alg_bytes = 2 * Q * SIZE[args.dtype] * cells
    achieved = alg_bytes / (kernel_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak_hbm()
    traffic = recorded_traffic(desc["workload"])

    e2e_steps = max(2, args.steps // 2)
    e2e_ms, h2d, d2h = time_e2e(lat, fields, e2e_steps, args.inner)
    e2e_glups, _ = replica_throughput(e2e_ms, cells * args.inner * e2e_steps, dist, "cuda")
    lat.close()
    del lat
    torch.cuda.empty_cache()

    variants = {}
    errors = None
    cpu = None
    d2d = d2d_copy_gbs() if rank == 0 else None
    if rank == 0 and not args.no_extras:
        for wl, dt, cl, pat in (("tgv512_d3q19", "f16", "bgk", "ab"), ("tgv512_d3q19", "bf16", "bgk", "ab"),
                                ("cavity256_d3q19", "f32", "bgk", "ab"), ("tgv512_d3q27", "f32", "bgk", "ab"),
                                ("tgv512_d3q27", "f16", "bgk", "ab"), ("tgv512_d3q19", "f32", "smagorinsky", "ab"),
                                ("tgv512_d3q19", "f32", "mlp", "ab"), ("tgv128_d3q19", "f32", "bgk", "ab"),
                                ("tgv128_d3q19", "f32", "mlp", "ab"), ("porous400_d3q19", "f32", "bgk", "ab"),
                                ("porous400_d3q19", "f16", "bgk", "ab"), ("tgv512_d3q19", "f32", "bgk", "aa"),
                                ("tgv512_d3q19", "f16", "bgk", "aa"), ("cavity256_d3q19", "f32", "bgk", "aa"),
                                ("porous400_d3q19", "f32", "bgk", "aa"), ("tgv512_d3q19", "f16s", "bgk", "ab"),
                                ("tgv512_d3q27", "f16s", "bgk", "ab"), ("tgv512_d3q19", "f64", "bgk", "ab")):
            if (wl, dt, cl, pat) == (args.workload, args.dtype, args.closure, args.pattern):
                continue
            v, _, d = make_workload(wl, dt, cl, pat)
            tms, kms, _, _ = time_lattice(v, 5, 3, args.inner)
            q = int(d["lattice"][3:])
            ach = 2 * q * SIZE[dt] * v.N / (kms * 1e-3) / 1e9
            variants[d["workload"]] = {"glups": v.N * args.inner * 5 / (tms * 1e-3) / 1e9,
                                       "glups_fluid": d["fluid_nodes"] * args.inner * 5 / (tms * 1e-3) / 1e9,
                                       "kernel_gbs_fluid": 2 * q * SIZE[dt] * d["fluid_nodes"] / (kms * 1e-3) / 1e9}
            variants[d["workload"]]["frac_of_peak"] = variants[d["workload"]]["kernel_gbs_fluid"] / peak
            if dt == "f64":
                # FP64 storage collides in FP64: its roof is the FP64 pipe
                # (DFMA, DADD, DMUL each one instruction), measured live.
                from paper_2506_09242_gb300 import lbm as _lbm
                rate = _lbm.fp64_fma_rate()
                ops = recorded_fp64_ops(f"tgv3d_128_d3q{q}_f64")
                glups_k = d["fluid_nodes"] / (kms * 1e-3) / 1e9
                variants[d["workload"]]["alu"] = {
                    "bound": "fp64", "fp64_flops_measured": rate, "fp64_inst_per_node": ops,
                    "peak_inst_per_s": rate / 2.0,
                    "frac": (glups_k * 1e9 * ops / (rate / 2.0)) if ops else None}
            v.close()
            del v
            torch.cuda.empty_cache()
        errors = error_vs_f64()
        if world == 1:
            cpu = cpu_baseline(args.cpu_plan)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0
    line = {
        "metric": METRIC, "value": glups, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
        "config": {**desc, "inner_steps": args.inner, "parallelism": f"replicas{world}",
                   "l2": f"inputs larger than L2 ({alg_bytes / 1e9:.1f} GB moved per lattice step)",
                   "step": f"{args.inner} lattice steps, the last fused with the FP64 reduction, read back"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "kernel": "k_collide_stream", "kernel_ms": kernel_ms,
                     "algorithmic_bytes_per_launch": alg_bytes},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_glups, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "step": "upload rho,u (FP64, pinned host) + inner lattice steps + reduction read back"},
        "gpu_launches": args.steps * (args.inner + 2),
        "ms_per_step_spread": {"min": min(per_step), "median": sorted(per_step)[len(per_step) // 2],
                               "max": max(per_step)},
        "d2d_copy_gbs": d2d,
        "clocks": clocks,
        "mass_drift": abs(reds[-1]["mass"] - reds[0]["mass"]) / reds[0]["mass"] if reds else None,
        "variants": variants,
        "errors_vs_f64": errors,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="tgv512_d3q19")
    ap.add_argument("--dtype", default="f32", choices=sorted(SIZE))
    ap.add_argument("--closure", default="bgk", choices=CLOSURES)
    ap.add_argument("--pattern", default="ab", choices=("ab", "aa"),
                    help="streaming pattern: two arrays (ab) or one array updated in place (aa)")
    ap.add_argument("--inner", type=int, default=20, help="lattice steps per benchmark step (>= 2)")
    ap.add_argument("--ref-n", type=int, default=128, help="lattice size of the oracle sample (reference arm)")
    ap.add_argument("--cpu-plan", default="bounded", choices=sorted(CPU_PLANS),
                    help="oracle timing plan of the CPU baseline")
    ap.add_argument("--cpu-baseline-only", action="store_true",
                    help="only time the oracle on the host cores (no GPU) and print the cpu_baseline object")
    ap.add_argument("--no-extras", action="store_true", help="skip variants, error table and CPU baseline")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.inner < 2:
        raise SystemExit("--inner must be >= 2")
    if args.cpu_baseline_only:
        return run_cpu_baseline_only(args)
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
