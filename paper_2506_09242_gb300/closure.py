"""Learned-closure workflow on the 3D Taylor-Green vortex (orchestration only).

Every numerical step runs in the CUDA library through the C ABI:
- stepping the fine and coarse lattices;
- moments and box filtering (`lbm_box_filter`);
- training samples (`lbm_coarse_samples`);
- loss gradients (`lbm_mlp_loss_grad`) and Adam (`lbm_mlp_adam`);
- the closure inside the collide kernel;
- the FP64 reductions.

Python sequences the calls. torch holds device buffers, draws minibatch
indices and takes one mean outside the library: the kinetic energy of the
box-filtered velocity, 0.5 <|u_filtered|^2>, over the coarse grid's cells.

Workflow (no counterpart in the paper; the TGV set-up is Sec. 3.1's):
1. Fine runs at resolution n_f and Reynolds numbers Re (u0 = 0.04,
   tau = 1/2 + 3 u0 (n_f / 2 pi) / Re). Snapshots are box-filtered by a
   factor f into training samples for the coarse grid n_c = n_f / f. With
   convective scaling the coarse time step is f fine steps, velocities are
   unchanged, and time is measured in convective units t_c = n / (2 pi u0)
   steps.
2. The closure network is trained with Adam on minibatches of the samples.
3. A-posteriori calibration: one scale factor alpha on the network output
   (dtau) is chosen from {0, 1/8, 1/4, 1/2, 1, 2}. The chosen alpha gives
   the smallest mean dissipation error of coarse runs at the training
   Reynolds numbers; alpha = 0 is plain BGK.
4. Coarse runs at n_c use plain BGK, Smagorinsky (Cs = 0.1), the raw
   learned closure, or the calibrated one. Each is judged by the relative
   L2 error of its dissipation rate -dk/dt against that of the box-filtered
   fine run, where k = <|u|^2 / 2> (Sec. 3.1).
5. Optionally (a posteriori), a second training stage uses inputs taken from
   the coarse solver's own populations (lbm_closure_features), recorded
   with the calibrated network in the loop and paired with the filtered
   fine targets at the same times.
"""
from __future__ import annotations

import json
import math
import sys
import time
from dataclasses import dataclass, field

import numpy as np

from . import lbm

U0 = 0.04


def tgv_tau(n: int, re: float, u0: float = U0) -> float:
    return 0.5 + 3.0 * u0 * (n / (2.0 * math.pi)) / re


def steps_per_tc(n: int, u0: float = U0) -> float:
    return n / (2.0 * math.pi * u0)


@dataclass
class FineRun:
    re: float
    n: int
    factor: int
    times: np.ndarray          # convective times of the energy samples
    k_filtered: np.ndarray     # k of the box-filtered velocity
    k_full: np.ndarray = None  # k of the fine velocity itself (the DNS reference)
    X: object = None           # training features (torch, device)
    y: object = None           # training targets (torch, device)
    y_fields: list = field(default_factory=list)  # (t, full coarse target field) per sample time
    glups: float = 0.0
    diverged_at: float | None = None


def _tgv_fields(n):
    import lbm_inputs as inp
    return inp.tgv3d(n, U0)


def fine_run(n: int, re: float, factor: int, *, t_end: float = 10.0, k_every: float = 0.1,
             sample_every: float = 0.5, samples_per_snapshot: int = 200_000, seed: int = 0,
             dtype: str = "f32") -> FineRun:
    """Runs the fine TGV, records the filtered kinetic energy every k_every t_c
    and collects training samples every sample_every t_c."""
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    lat = lbm.Lattice(n, n, n, lbm.D3Q19, dtype)
    lat.set_params(tgv_tau(n, re))
    rho, u = _tgv_fields(n)
    lat.init_equilibrium(rho, u)
    del rho, u
    rho_d = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
    u_d = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
    tau_c = tgv_tau(n // factor, re)
    spt = steps_per_tc(n)
    n_k = int(round(t_end / k_every))
    every = max(1, int(round(sample_every / k_every)))
    times, ks, kf, Xs, ys, y_fields = [], [], [], [], [], []
    done, t_step = 0, 0.0
    diverged = None
    for j in range(n_k + 1):
        target = int(round(j * k_every * spt))
        if target > done:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lat.step(target - done)
            torch.cuda.synchronize()
            t_step += time.perf_counter() - t0
            done = target
        lat.moments(rho_d, u_d)
        if not torch.isfinite(u_d).all():
            diverged = j * k_every
            break
        ub = lbm.box_filter(u_d, factor)
        times.append(j * k_every)
        ks.append(0.5 * float((ub * ub).sum(dim=0).mean()))  # the filtered field's mean energy (torch)
        kf.append(lat.reduce()["ke"] / n ** 3)  # the library's FP64 reduction (every node is fluid)
        if j % every == 0 and j > 0:
            X, y = lbm.coarse_samples(rho_d, u_d, factor, tau_c)
            idx = torch.randint(0, X.shape[0], (min(samples_per_snapshot, X.shape[0]),), generator=gen,
                                device="cuda")
            Xs.append(X[idx])
            ys.append(y[idx])
            y_fields.append((j * k_every, y))
    lat.close()
    run = FineRun(re, n, factor, np.array(times), np.array(ks), k_full=np.array(kf), diverged_at=diverged)
    run.glups = n ** 3 * done / max(t_step, 1e-9) / 1e9
    run.y_fields = y_fields
    if Xs:
        run.X = torch.cat(Xs)
        run.y = torch.cat(ys)
    return run


@dataclass
class Trained:
    params: object
    norm: object
    losses: list = field(default_factory=list)


def train(X, y, *, steps: int = 2000, batch: int = 8192, lr: float = 2e-3, seed: int = 0,
          init: Trained | None = None) -> Trained:
    """Adam on minibatches; normalisation from the sample statistics and an
    output scale that makes y = 0 predict the mean target.  With init, the
    network continues from init's weights (normalisation recomputed)."""
    import torch
    import lbm_inputs as inp
    mean = X.mean(dim=0)
    std = X.std(dim=0).clamp_min(1e-12)
    scale = float(y.mean()) / math.log(2.0) if float(y.mean()) > 0 else 1e-6
    norm = torch.cat([mean, std, torch.tensor([scale, 0.0], device="cuda")]).float().contiguous()
    if init is not None:
        P = init.params.clone()
    else:
        P = torch.from_numpy(inp.mlp_init(seed).astype(np.float32)).cuda()
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed + 1)
    ws = torch.empty((lbm.load().lbm_mlp_workspace_bytes(batch) + 3) // 4, dtype=torch.float32, device="cuda")
    losses = []
    for t in range(1, steps + 1):
        idx = torch.randint(0, X.shape[0], (batch,), generator=gen, device="cuda")
        loss, grad = lbm.mlp_loss_grad(P, norm, X[idx].contiguous(), y[idx].contiguous(), ws)
        lbm.mlp_adam(P, m, v, grad, t, lr)
        if t % max(1, steps // 20) == 0 or t == 1:
            losses.append((t, float(loss.item())))
    return Trained(P, norm, losses)


@dataclass
class CoarseRun:
    closure: str
    times: np.ndarray
    k: np.ndarray
    glups: float
    diverged_at: float | None


def coarse_run(n: int, re: float, closure: str, trained: Trained | None = None, *, cs: float = 0.1,
               t_end: float = 10.0, k_every: float = 0.1, dtype: str = "f32") -> CoarseRun:
    import torch
    lat = lbm.Lattice(n, n, n, lbm.D3Q19, dtype)
    kind = {"bgk": lbm.CLOSURE_BGK, "smagorinsky": lbm.CLOSURE_SMAGORINSKY, "mlp": lbm.CLOSURE_MLP}[closure]
    lat.set_params(tgv_tau(n, re), closure=kind, cs_smag=cs)
    if kind == lbm.CLOSURE_MLP:
        lat.set_closure_weights(trained.params, trained.norm)
    rho, u = _tgv_fields(n)
    lat.init_equilibrium(rho, u)
    spt = steps_per_tc(n)
    times, ks = [], []
    done, t_step, diverged = 0, 0.0, None
    for j in range(int(round(t_end / k_every)) + 1):
        target = int(round(j * k_every * spt))
        if target > done:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lat.step(target - done)
            torch.cuda.synchronize()
            t_step += time.perf_counter() - t0
            done = target
        try:
            red = lat.reduce()
        except lbm.UnstableError:
            diverged = j * k_every
            break
        times.append(j * k_every)
        ks.append(red["ke"] / red["n_fluid"])
    lat.close()
    return CoarseRun(closure, np.array(times), np.array(ks), n ** 3 * done / max(t_step, 1e-9) / 1e9, diverged)


def solver_samples(n: int, re: float, fine: FineRun, closure: str, trained: Trained | None = None, *,
                   samples_per_snapshot: int = 200_000, seed: int = 0, cs: float = 0.1):
    """A-posteriori training pairs: a coarse run (closure in the loop, from
    the coarse TGV initial field) records its own closure inputs
    (lbm_closure_features) at the fine run's sample times; each is paired
    with the filtered fine run's target field at the same time.  Stops early
    if the coarse run turns unstable."""
    import torch
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    lat = lbm.Lattice(n, n, n, lbm.D3Q19, "f32")
    kind = {"bgk": lbm.CLOSURE_BGK, "smagorinsky": lbm.CLOSURE_SMAGORINSKY, "mlp": lbm.CLOSURE_MLP}[closure]
    lat.set_params(tgv_tau(n, re), closure=kind, cs_smag=cs)
    if kind == lbm.CLOSURE_MLP:
        lat.set_closure_weights(trained.params, trained.norm)
    rho, u = _tgv_fields(n)
    lat.init_equilibrium(rho, u)
    spt = steps_per_tc(n)
    Xs, ys, done = [], [], 0
    X = torch.empty((n ** 3, 7), dtype=torch.float32, device="cuda")
    for t, y in fine.y_fields:
        target = int(round(t * spt))
        if target > done:
            lat.step(target - done)
            done = target
        try:
            lat.reduce()
        except lbm.UnstableError:
            break
        lat.closure_features(X)
        idx = torch.randint(0, n ** 3, (min(samples_per_snapshot, n ** 3),), generator=gen, device="cuda")
        Xs.append(X[idx])
        ys.append(y[idx])
    lat.close()
    return torch.cat(Xs), torch.cat(ys)


def scaled(trained: Trained, alpha: float) -> Trained:
    """The same network with its output (dtau) multiplied by alpha."""
    norm = trained.norm.clone()
    norm[14] = norm[14] * alpha
    return Trained(trained.params, norm, trained.losses)


def calibrate(trained: Trained, n_c: int, fines: dict, train_re, *, alphas=(0.0, 0.125, 0.25, 0.5, 1.0, 2.0),
              t_end: float = 10.0):
    """A-posteriori scale of the closure output: the alpha whose coarse runs
    at the training Reynolds numbers have the smallest mean dissipation error
    against the filtered fine runs (alpha = 0 is plain BGK)."""
    table = {}
    for a in alphas:
        errs = [dissipation_error(fines[re], coarse_run(n_c, re, "mlp", scaled(trained, a), t_end=t_end))
                for re in train_re]
        table[a] = float(np.mean(errs))
    best = min(table, key=lambda a: table[a])
    return best, table


def dissipation_error(fine: FineRun, coarse: CoarseRun, reference: str = "filtered") -> float:
    """Relative L2 error of -dk/dt over the fine run's time grid (inf if the
    coarse run diverged before the end), against the box-filtered fine run
    or (reference "fine") the fine run itself."""
    if coarse.diverged_at is not None or len(coarse.times) < len(fine.times):
        return math.inf
    ef = -np.gradient(fine.k_filtered if reference == "filtered" else fine.k_full, fine.times)
    ec = -np.gradient(coarse.k[:len(fine.times)], coarse.times[:len(fine.times)])
    return float(np.linalg.norm(ec - ef) / np.linalg.norm(ef))


def experiment(n_fine: int, factor: int, train_re, test_re: float, *, t_end: float = 10.0, steps: int = 2000,
               batch: int = 8192, samples_per_snapshot: int = 200_000, seed: int = 0,
               a_posteriori: bool = False) -> dict:
    """Fine runs at train_re (and test_re), training, and the three coarse
    runs at test_re; returns a JSON-able summary.

    a_posteriori: a second training stage uses the coarse solver's own
    inputs.  The calibrated first-stage network runs in the loop of coarse
    runs at the training Reynolds numbers (solver_samples), the network
    continues from its first-stage weights on those pairs, is recalibrated,
    and is judged at test_re like the first stage."""
    import torch
    n_c = n_fine // factor
    fines = {}
    for re in sorted(set(list(train_re) + [test_re])):
        fines[re] = fine_run(n_fine, re, factor, t_end=t_end, samples_per_snapshot=samples_per_snapshot,
                             seed=seed + int(re))
    X = torch.cat([fines[re].X for re in train_re])
    y = torch.cat([fines[re].y for re in train_re])
    t0 = time.perf_counter()
    trained = train(X, y, steps=steps, batch=batch, seed=seed)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    runs = {c: coarse_run(n_c, test_re, c, trained, t_end=t_end) for c in ("bgk", "smagorinsky", "mlp")}
    alpha, table = calibrate(trained, n_c, fines, train_re, t_end=t_end)
    runs["mlp_calibrated"] = coarse_run(n_c, test_re, "mlp", scaled(trained, alpha), t_end=t_end)
    second = {}
    if a_posteriori:
        pairs = [solver_samples(n_c, re, fines[re], "mlp", scaled(trained, alpha),
                                samples_per_snapshot=samples_per_snapshot, seed=seed + 7 + int(re)) for re in train_re]
        Xa = torch.cat([p[0] for p in pairs])
        ya = torch.cat([p[1] for p in pairs])
        trained2 = train(Xa, ya, steps=steps, batch=batch, seed=seed + 3, init=trained)
        alpha2, table2 = calibrate(trained2, n_c, fines, train_re, t_end=t_end)
        runs["mlp_a_posteriori"] = coarse_run(n_c, test_re, "mlp", trained2, t_end=t_end)
        runs["mlp_a_posteriori_calibrated"] = coarse_run(n_c, test_re, "mlp", scaled(trained2, alpha2), t_end=t_end)
        second = {"a_posteriori": {"samples": int(Xa.shape[0]), "alpha": alpha2,
                                   "mean_train_error": {str(a): e for a, e in table2.items()},
                                   "loss_first_last": [trained2.losses[0][1], trained2.losses[-1][1]],
                                   "feature_std_ce": X.std(dim=0).tolist(), "feature_std_solver": Xa.std(dim=0).tolist()}}
    ref = fines[test_re]
    # Equal cost: with convective scaling a run of n^3 nodes to a fixed time
    # costs n^4 / GLUPS, so plain BGK gets the grid n_eq = n_c (GLUPS_bgk /
    # GLUPS_mlp)^(1/4) (even) for the learned closure's cost; both are judged
    # against the fine run's own dissipation rate (no box filter fits n_eq).
    g_mlp = runs["mlp_calibrated"].glups
    n_eq = 2 * int(round(0.5 * n_c * (runs["bgk"].glups / max(g_mlp, 1e-9)) ** 0.25))
    eq = coarse_run(n_eq, test_re, "bgk", t_end=t_end)
    equal_cost = {"n_bgk": n_eq, "glups_bgk": eq.glups, "glups_mlp": g_mlp,
                  "dissipation_rel_l2_vs_fine": {
                      f"bgk_{n_eq}": dissipation_error(ref, eq, "fine"),
                      f"bgk_{n_c}": dissipation_error(ref, runs["bgk"], "fine"),
                      f"smagorinsky_{n_c}": dissipation_error(ref, runs["smagorinsky"], "fine"),
                      f"mlp_calibrated_{n_c}": dissipation_error(ref, runs["mlp_calibrated"], "fine")},
                  "diverged_at_tc": {f"bgk_{n_eq}": eq.diverged_at}}
    if "mlp_a_posteriori_calibrated" in runs:
        equal_cost["dissipation_rel_l2_vs_fine"][f"mlp_a_posteriori_calibrated_{n_c}"] = dissipation_error(
            ref, runs["mlp_a_posteriori_calibrated"], "fine")
    return {
        "n_fine": n_fine, "n_coarse": n_c, "factor": factor, "train_re": list(train_re), "test_re": test_re,
        "t_end_tc": t_end, "train_samples": int(X.shape[0]), "train_steps": steps, "batch": batch,
        "train_seconds": t_train, "loss_first_last": [trained.losses[0][1], trained.losses[-1][1]],
        "target_mean": float(y.mean()),
        "fine_glups": {str(re): fines[re].glups for re in fines},
        "fine_diverged": {str(re): fines[re].diverged_at for re in fines},
        "calibration": {"alpha": alpha, "mean_train_error": {str(a): e for a, e in table.items()}},
        "coarse": {c: {"dissipation_rel_l2": dissipation_error(ref, r), "glups": r.glups,
                       "diverged_at_tc": r.diverged_at} for c, r in runs.items()},
        "equal_cost": equal_cost,
        **second,
    }


def main(argv=None):  # pragma: no cover - GPU workflow entry point
    import argparse
    ap = argparse.ArgumentParser(description="learned-closure experiment on the 3D Taylor-Green vortex")
    ap.add_argument("--n-fine", type=int, default=512)
    ap.add_argument("--factor", type=int, default=4)
    ap.add_argument("--t-end", type=float, default=10.0)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--held-out", action="store_true", help="train on Re 800 and 3200, test on 1600")
    ap.add_argument("--a-posteriori", action="store_true", help="second training stage on the coarse solver's own inputs")
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    train_re = (800.0, 3200.0) if a.held_out else (800.0, 1600.0, 3200.0)
    res = experiment(a.n_fine, a.factor, train_re, 1600.0, t_end=a.t_end, steps=a.steps, a_posteriori=a.a_posteriori)
    text = json.dumps(res, indent=1)
    print(text)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(text)
    return 0


if __name__ == "__main__":  # pragma: no cover
    sys.exit(main())
