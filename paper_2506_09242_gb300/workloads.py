"""The reference workloads as library call sequences (no numerics in Python).

- ``porous``: pore-scale flow through a random-sphere medium (the stand-in for
  the Berea sandstone of Sec. 3.3): body force on pore nodes, bounce-back on
  solids, run to steady state. Reports the permeability k = u_mean nu / g
  (u_mean over all nodes, solid = 0) and GLUPS over fluid nodes only.
- ``cavity``: lid-driven cavity of Sec. 3.2 (SOLID walls, Ladd lid).
- ``tgv_precision``: the 3D Taylor-Green vortex of Sec. 3.1 with FP64, FP32,
  FP16- and BF16-shifted storage. Records kinetic energy and enstrophy curves
  and the velocity error against the FP64 run at chosen times.
- ``size_sweep``: GLUPS against the lattice's share of device memory (the
  performance-versus-domain-size study of Sec. 4.1).

torch is used for device buffers, for differences of fields when evaluating
errors and for time averages of velocity fields.
"""
from __future__ import annotations

import json
import math
import sys
import time

import numpy as np

from . import lbm


def _sync():
    import torch
    torch.cuda.synchronize()


def porous(n: int = 400, *, seed: int = 2506, rmin: float = 4.0, rmax: float = 10.0, target: float = 0.2,
           g: float = 1e-6, tau: float = 1.0, max_steps: int = 50_000, check_every: int = 1000, tol: float = 1e-6,
           dtype: str = "f32", closure: str = "bgk", trt_magic: float = 3.0 / 16.0) -> dict:
    """Permeability of the random-sphere medium (the stand-in for the Berea
    sample of Sec. 3.3): body-force-driven flow until the mean velocity
    changes by less than tol (relative) over check_every steps, or max_steps.
    closure "trt" uses two relaxation times with the given magic parameter.
    The history holds (steps, mean velocity, permeability) at every check,
    the convergence record of the permeability."""
    import lbm_inputs as inp
    kind = {"bgk": lbm.CLOSURE_BGK, "trt": lbm.CLOSURE_TRT}[closure]
    centres, radii = inp.sphere_list((n, n, n), seed=seed, rmin=rmin, rmax=rmax, count=100_000)
    nu = (tau - 0.5) / 3.0
    with lbm.Lattice(n, n, n, lbm.D3Q19, dtype) as lat:
        used, por = lat.geometry_spheres(centres, radii, target, lbm.TAG_FORCED)
        lat.set_params(tau, force=(g, 0.0, 0.0), closure=kind, trt_magic=trt_magic)
        lat.init_equilibrium()
        n_fluid = int(lat.census()[lbm.TAG_FORCED])
        hist, steps, t_step, prev = [], 0, 0.0, None
        converged = False
        while steps < max_steps:
            _sync()
            t0 = time.perf_counter()
            lat.step(check_every)
            _sync()
            t_step += time.perf_counter() - t0
            steps += check_every
            red = lat.reduce()
            u_mean = red["vel"][0] / n ** 3
            hist.append((steps, u_mean, u_mean * nu / g))
            if prev is not None and abs(u_mean - prev) <= tol * abs(u_mean):
                converged = True
                break
            prev = u_mean
    k = u_mean * nu / g
    return {"n": n, "spheres": used, "porosity": por, "fluid_nodes": n_fluid, "tau": tau, "g": g,
            "closure": closure, "dtype": dtype, "steps": steps, "converged": converged, "tol": tol,
            "check_every": check_every, "u_mean": u_mean, "permeability_voxel2": k,
            "glups_fluid": n_fluid * steps / t_step / 1e9, "glups_all_nodes": n ** 3 * steps / t_step / 1e9,
            "history": hist}


def porous_tau_study(n: int = 200, *, taus=(0.6, 1.0, 1.5), closures=("bgk", "trt"), g: float = 1e-6,
                     max_steps: int = 60_000, check_every: int = 2000, tol: float = 1e-5, seed: int = 2506) -> dict:
    """Permeability of one random-sphere medium versus tau for BGK and TRT
    (Lambda = 3/16): with TRT the halfway wall does not move with tau, so the
    permeability should not change."""
    import lbm_inputs as inp
    centres, radii = inp.sphere_list((n, n, n), seed=seed, rmin=4.0, rmax=10.0, count=100_000)
    out = {"n": n, "g": g, "runs": []}
    for cl in closures:
        kind = {"bgk": lbm.CLOSURE_BGK, "trt": lbm.CLOSURE_TRT}[cl]
        for tau in taus:
            with lbm.Lattice(n, n, n, lbm.D3Q19, "f32") as lat:
                used, por = lat.geometry_spheres(centres, radii, 0.2, lbm.TAG_FORCED)
                lat.set_params(tau, force=(g, 0.0, 0.0), closure=kind)
                lat.init_equilibrium()
                nu = (tau - 0.5) / 3.0
                steps, prev, conv = 0, None, False
                while steps < max_steps:
                    lat.step(check_every)
                    steps += check_every
                    u_mean = lat.reduce()["vel"][0] / n ** 3
                    if prev is not None and abs(u_mean - prev) <= tol * abs(u_mean):
                        conv = True
                        break
                    prev = u_mean
            out["runs"].append({"closure": cl, "tau": tau, "steps": steps, "converged": conv, "porosity": por,
                                "permeability_voxel2": u_mean * nu / g})
    return out


def cavity(n: int = 256, *, re: float = 1000.0, u_lid: float = 0.1, steps: int = 10_000, dtype: str = "f32") -> dict:
    import lbm_inputs as inp
    tau = 0.5 + 3.0 * u_lid * n / re
    with lbm.Lattice(n, n, n, lbm.D3Q19, dtype) as lat:
        lat.set_tags(inp.cavity_tags(n))
        lat.set_params(tau, wall_u=[(u_lid, 0.0, 0.0)])
        lat.init_equilibrium()
        n_fluid = int(lat.census()[lbm.TAG_FLUID])
        _sync()
        t0 = time.perf_counter()
        lat.step(steps)
        _sync()
        dt = time.perf_counter() - t0
        red = lat.reduce()
        rho, u = lat.moments()
    mid = n // 2
    return {"n": n, "re": re, "tau": tau, "steps": steps, "t_c": steps * u_lid / n,
            "glups_all_nodes": n ** 3 * steps / dt / 1e9, "glups_fluid": n_fluid * steps / dt / 1e9,
            "ke_per_fluid_node": red["ke"] / red["n_fluid"], "umax": red["umax"],
            "ux_centreline_z": u[0, :, mid, mid][:: max(1, n // 16)].tolist()}


def _cavity_profiles(u, n: int, u_lid: float):
    """Centreline profiles of the cavity velocity u[3][nz][ny][nx] (numpy):
    u_x along the vertical centreline and u_z along the horizontal one, over
    the fluid nodes 1 .. n-2, with positions xi = (k - 0.5) / (n - 2) between
    the halfway walls."""
    import numpy as np
    m = n // 2
    k = np.arange(1, n - 1)
    xi = (k - 0.5) / (n - 2)
    if n % 2:  # odd n: the centreline is a node line
        ux = u[0, 1:n - 1, m, m]
        uz = u[2, m, m, 1:n - 1]
    else:      # even n: average the two node lines around the centre plane
        ux = 0.25 * (u[0, 1:n - 1, m - 1, m - 1] + u[0, 1:n - 1, m, m - 1] + u[0, 1:n - 1, m - 1, m] + u[0, 1:n - 1, m, m])
        uz = 0.25 * (u[2, m - 1, m - 1, 1:n - 1] + u[2, m, m - 1, 1:n - 1] + u[2, m - 1, m, 1:n - 1] + u[2, m, m, 1:n - 1])
    return xi, ux / u_lid, uz / u_lid


def cavity_steady(n: int = 256, *, re: float = 1000.0, u_lid: float = 0.1, t_max: float = 80.0,
                  check_tc: float = 0.5, tol: float = 1e-6, averages=(), dtype: str = "f32") -> dict:
    """The lid-driven cavity of Sec. 3.2 run for long times.

    The walls are halfway between the SOLID (or lid) nodes and the fluid, so
    the cavity side is L = n - 2 and nu = u_lid L / Re.  The kinetic energy
    per fluid node is checked every check_tc convective times t_c = L / u_lid;
    the run counts as steady once it changes by less than tol (relative) over
    one t_c.  For each window (t0, t1) in averages the velocity field is also
    averaged over samples taken every check_tc in [t0, t1] (for unsteady
    Reynolds numbers; the run then goes on to the last window's end);
    the centreline profiles of the final and averaged fields are returned.
    """
    import numpy as np
    import torch
    import lbm_inputs as inp
    L = n - 2
    tau = 0.5 + 3.0 * u_lid * L / re
    tc = L / u_lid
    hist, t_step, steps, converged = [], 0.0, 0, False
    means = [[None, 0] for _ in averages]
    with lbm.Lattice(n, n, n, lbm.D3Q19, dtype) as lat:
        lat.set_tags(inp.cavity_tags(n))
        lat.set_params(tau, wall_u=[(u_lid, 0.0, 0.0)])
        lat.init_equilibrium()
        n_fluid = int(lat.census()[lbm.TAG_FLUID])
        uu = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
        per_check = max(1, int(round(check_tc * tc)))
        per_tc = int(round(1.0 / check_tc))
        while steps < t_max * tc:
            _sync()
            t0 = time.perf_counter()
            lat.step(per_check)
            _sync()
            t_step += time.perf_counter() - t0
            steps += per_check
            ke = lat.reduce()["ke"] / n_fluid
            hist.append((steps / tc, ke))
            t = steps / tc
            inside = [k for k, w in enumerate(averages) if w[0] <= t <= w[1] + 1e-9]
            if inside:
                lat.moments(None, uu)
                for k in inside:
                    means[k][0] = uu.clone() if means[k][0] is None else means[k][0].add_(uu)
                    means[k][1] += 1
            if not averages and len(hist) > per_tc:
                prev = hist[-1 - per_tc][1]
                if abs(ke - prev) <= tol * abs(ke):
                    converged = True
                    break
        lat.moments(None, uu)
        final = uu.cpu().numpy()
        avgs = [(m / c).cpu().numpy() if c else None for m, c in means]
        del uu, means
    torch.cuda.empty_cache()
    xi, ux, uz = _cavity_profiles(final, n, u_lid)
    out = {"n": n, "re": re, "u_lid": u_lid, "tau": tau, "L": L, "t_c_steps": tc, "steps": steps,
           "t_end_tc": steps / tc, "converged": converged, "tol_per_tc": tol,
           "glups_fluid": n_fluid * steps / t_step / 1e9, "glups_all_nodes": n ** 3 * steps / t_step / 1e9,
           "ke_history": hist[:: max(1, len(hist) // 40)] + hist[-3:],
           "profile": {"xi": xi.tolist(), "ux_vertical": ux.tolist(), "uz_horizontal": uz.tolist()}}
    out["averages"] = []
    for w, avg in zip(averages, avgs):
        if avg is None:
            continue
        _, ua, za = _cavity_profiles(avg, n, u_lid)
        out["averages"].append({"window_tc": list(w), "ux_vertical": ua.tolist(), "uz_horizontal": za.tolist()})
    return out


def cavity_study(sizes=(128, 256), *, re: float = 1000.0, t_max: float = 80.0, re_unsteady: float = 3200.0,
                 n_unsteady: int = 256, windows=((20.0, 30.0), (30.0, 40.0))) -> dict:
    """Steady Re = 1000 on two grids (grid convergence of the centreline
    profiles, coarse positions, the fine profile interpolated), and two
    time-averaging windows of the unsteady Re = 3200 flow (statistical
    self-consistency of the averaged profiles)."""
    import numpy as np
    runs = {n: cavity_steady(n, re=re, t_max=t_max) for n in sizes}
    a, b = runs[sizes[0]]["profile"], runs[sizes[-1]]["profile"]
    dux = np.max(np.abs(np.interp(a["xi"], b["xi"], b["ux_vertical"]) - np.array(a["ux_vertical"])))
    duz = np.max(np.abs(np.interp(a["xi"], b["xi"], b["uz_horizontal"]) - np.array(a["uz_horizontal"])))
    out = {"steady": {str(n): {k: v for k, v in r.items() if k != "profile"} for n, r in runs.items()},
           "profiles": {str(n): r["profile"] for n, r in runs.items()},
           "grid_difference_max_over_u_lid": {"ux_vertical": float(dux), "uz_horizontal": float(duz)}}
    if re_unsteady:
        r = cavity_steady(n_unsteady, re=re_unsteady, t_max=max(w[1] for w in windows), averages=windows)
        a0, a1 = r["averages"][0], r["averages"][1]
        d1 = np.max(np.abs(np.array(a0["ux_vertical"]) - np.array(a1["ux_vertical"])))
        d2 = np.max(np.abs(np.array(a0["uz_horizontal"]) - np.array(a1["uz_horizontal"])))
        out["unsteady"] = {"re": re_unsteady, "n": n_unsteady, "windows_tc": [list(w) for w in windows],
                           "window_difference_max_over_u_lid": {"ux_vertical": float(d1), "uz_horizontal": float(d2)},
                           "ke_history": r["ke_history"], "glups_fluid": r["glups_fluid"],
                           "averages": r["averages"], "xi": r["profile"]["xi"]}
    return out


STORAGE_BYTES = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2, "f16s": 2}


def sweep_plan(sizes, Q: int, dtype: str, pattern: str, device_bytes: int, free_bytes: int, *,
               headroom: float = 0.8):
    """The cubes of the size sweep that fit: (n, population bytes, fraction of
    the device memory) for every n whose population arrays (two with the A/B
    pattern, one with AA; rows padded to 32 nodes) take at most headroom of
    the free memory.  The memory fraction is the x-axis of the paper's
    performance-versus-memory-use figure (Sec. 4.1)."""
    arrays = 1 if pattern == "aa" else 2
    plan = []
    for n in sizes:
        px = (n + 31) // 32 * 32
        plane = (px * n * n + 255) // 256 * 256
        nbytes = arrays * Q * plane * STORAGE_BYTES[dtype]
        if nbytes <= headroom * free_bytes:
            plan.append((n, nbytes, nbytes / device_bytes))
    return plan


def size_sweep(sizes=(64, 96, 128, 192, 256, 320, 384, 512, 640, 768, 896, 1024), *, Q: int = 19,
               dtype: str = "f32", pattern: str = "ab", steps: int = 40, peak_gbs: float | None = None) -> dict:
    """GLUPS of the periodic BGK step against the lattice's share of device
    memory, the analogue of the paper's study of performance versus domain
    size (Sec. 4.1, which finds performance rising with memory use).  Each
    size is timed with CUDA events over `steps` steps after 4 warm-up steps;
    sizes whose arrays would not fit in 80% of the free memory are skipped."""
    import torch
    free, total = torch.cuda.mem_get_info()
    rows = []
    for n, nbytes, frac_mem in sweep_plan(sizes, Q, dtype, pattern, total, free):
        with lbm.Lattice(n, n, n, Q, dtype, pattern=pattern) as lat:
            lat.set_params(0.6)
            lat.init_equilibrium()
            lat.step(4)
            _sync()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record()
            lat.step(steps)
            t1.record()
            _sync()
            ms = t0.elapsed_time(t1) / steps
        torch.cuda.empty_cache()
        glups = n ** 3 / (ms * 1e-3) / 1e9
        gbs = 2 * Q * STORAGE_BYTES[dtype] * n ** 3 / (ms * 1e-3) / 1e9
        row = {"n": n, "memory_fraction": frac_mem, "population_gb": nbytes / 1e9, "ms_per_step": ms,
               "glups": glups, "gbs": gbs}
        if peak_gbs:
            row["frac_of_peak"] = gbs / peak_gbs
        rows.append(row)
    return {"Q": Q, "dtype": dtype, "pattern": pattern, "steps": steps, "device_bytes": total, "rows": rows}


def tgv_precision(n: int = 512, Q: int = 27, *, dtypes=("f64", "f32", "f16", "bf16", "f16s"), u0: float = 0.04,
                  re: float = 1600.0, t_end: float = 10.0, every: float = 0.5, error_at=(1.0, 5.0, 10.0)) -> dict:
    """Runs the TGV once per storage type (FP64 first) and compares each
    velocity field with the FP64 one at the times in error_at."""
    import torch
    import lbm_inputs as inp
    tau = 0.5 + 3.0 * u0 * (n / (2.0 * math.pi)) / re
    spt = n / (2.0 * math.pi * u0)
    rho, u = inp.tgv3d(n, u0)
    ref_fields = {}
    out = {"n": n, "Q": Q, "re": re, "u0": u0, "tau": tau, "steps_per_tc": spt, "runs": {}}
    marks = sorted(set([round(j * every, 6) for j in range(int(round(t_end / every)) + 1)] + list(error_at)))
    for dt in dtypes:
        curves, errs = [], {}
        t_step = 0.0
        with lbm.Lattice(n, n, n, Q, dt) as lat:
            lat.set_params(tau)
            lat.init_equilibrium(rho, u)
            uu = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
            done = 0
            for t in marks:
                target = int(round(t * spt))
                if target > done:
                    _sync()
                    t0 = time.perf_counter()
                    lat.step(target - done)
                    _sync()
                    t_step += time.perf_counter() - t0
                    done = target
                try:
                    red = lat.reduce()
                except lbm.UnstableError:
                    curves.append((t, None, None))
                    break
                curves.append((t, red["ke"] / n ** 3, lat.enstrophy()))
                if t in error_at:
                    lat.moments(None, uu)
                    if dt == dtypes[0]:
                        ref_fields[t] = uu.clone()
                    else:
                        r = ref_fields[t]
                        errs[str(t)] = float(torch.linalg.vector_norm(uu - r) / torch.linalg.vector_norm(r))
            del uu
        out["runs"][dt] = {"glups": n ** 3 * done / t_step / 1e9, "curve_t_k_eps": curves, "vel_rel_l2_vs_first": errs}
        torch.cuda.empty_cache()
    return out


def main(argv=None):  # pragma: no cover - GPU workflow entry point
    import argparse
    ap = argparse.ArgumentParser(description="reference workloads")
    ap.add_argument("which", choices=["porous", "porous_tau", "cavity", "cavity_study", "tgv_precision",
                                      "size_sweep"])
    ap.add_argument("--dtype", default="f32", choices=sorted(STORAGE_BYTES))
    ap.add_argument("--pattern", default="ab", choices=("ab", "aa"))
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--Q", type=int, default=None, choices=(19, 27),
                    help="velocity set (tgv_precision: 27, size_sweep: 19 when not given)")
    ap.add_argument("--t-end", type=float, default=10.0)
    ap.add_argument("--closure", default="bgk", choices=("bgk", "trt"), help="porous: collision model")
    ap.add_argument("--max-steps", type=int, default=50_000, help="porous: step cap")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    if a.which == "porous":
        res = porous(a.n or 400, closure=a.closure, max_steps=a.max_steps, dtype=a.dtype)
    elif a.which == "porous_tau":
        res = porous_tau_study(a.n or 200)
    elif a.which == "cavity":
        res = cavity(a.n or 256)
    elif a.which == "cavity_study":
        res = cavity_study()
    elif a.which == "size_sweep":
        res = size_sweep(Q=a.Q or 19, dtype=a.dtype, pattern=a.pattern)
    else:
        res = tgv_precision(a.n or 512, a.Q or 27, t_end=a.t_end)
    text = json.dumps(res, indent=1)
    print(text)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(text)
    return 0


if __name__ == "__main__":  # pragma: no cover
    sys.exit(main())
