"""Training and evaluation of the learned Green's-function factor on the GPU.

The factor m(|k| / k_Ny, a) = 1 + MLP multiplies the potential's Green's function
(library entry points pm_set_mlp ... pm_mlp_adam).  It is fitted so that a cheap run
(few steps, force mesh as fine as the CDM grid) lands where an expensive run of the
same initial conditions (many steps, a finer force mesh) does:

  loss    either the spectrum-matching loss L = mean_b (P_b / P_ref,b - 1)^2 of the
          total-matter spectrum of the cheap run against the expensive run's, both
          measured by the cheap context's estimator, over the bins up to k_max
          (gradient by pm_power_vjp), or the displacement loss
          L = sum_i m_i |x_i - y_i|^2 / sum_i m_i between the cheap run's final CDM
          particles x and the expensive run's y, pairing by id (pm_displacement_loss;
          neutrinos are left out: their thermal streaming depends on the step schedule
          through the drift factor, which no force correction can remove).  The
          displacement loss is dominated by orbits inside haloes that neither run
          resolves alike, so the spectrum loss is the default;
  grad    the hand-written adjoint: pm_step_vjp backwards over per-step checkpoints
          accumulates d L / d theta in the library (each force evaluation adds the
          network's backward pass over the |n|^2 bins of d <lambda_F, F> / d m);
  update  Adam on the device (pm_mlp_adam).

Every step of the loop runs in the library's kernels; this module only sequences the
calls and keeps the checkpoints (torch tensors on the device).
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from .pm import MLP_NPARAM, SPECIES_ALL, SPECIES_CDM, ParticleMesh, RunConfig


def run(pm: ParticleMesh, noise, steps, a0: float, k_fs: float = 0.0, checkpoints: bool = False):
    """Zel'dovich ICs from device white noise, then KDK steps.  Returns (state, checkpoints):
    the checkpoints hold (u, p, id, f) at the start of every step (f = F(x) at that a)."""
    st = pm.ic(noise, a0, k_fs=k_fs)
    pm.set_force_time(a0)
    st["f"].copy_(pm.force(st["u"], st["id"]))
    st["f_valid"] = 1
    ckpts = []
    if not checkpoints:  # chained steps in one pm_run (the same states as stepping)
        pm.run(st, steps)
        return st, ckpts
    for (a, ah, b) in steps:
        ckpts.append({k: st[k].clone() for k in ("u", "p", "id", "f")} | {"a": a, "f_valid": 1})
        pm.step(st, a, ah, b)
    return st, ckpts


def loss_and_grad(pm: ParticleMesh, noise, ref, steps, a0: float, k_fs: float = 0.0,
                  species: int = SPECIES_CDM) -> float:
    """Displacement loss of the learned run against ref ({"u", "id"} on the device) over the
    selected species; adds d L / d theta to the library's accumulator (pm.mlp_grad)."""
    import torch
    st, ckpts = run(pm, noise, steps, a0, k_fs, checkpoints=True)
    L, lam_x = pm.displacement_loss(st, ref, species)
    lam_p = torch.zeros_like(lam_x)
    for ck, (a, ah, b) in zip(reversed(ckpts), reversed(steps)):
        lam_x, lam_p = pm.step_vjp(ck, a, ah, b, lam_x, lam_p)
    return L


def spectrum_loss_and_grad(pm: ParticleMesh, noise, p_ref, bins, nbins: int, steps, a0: float,
                           k_fs: float = 0.0, weights=None) -> float:
    """Spectrum-matching loss sum_b w_b (P_b / P_ref,b - 1)^2 / sum_b w_b of the learned run
    against the target spectrum p_ref (same estimator and nbins) over the bin indices in
    bins (weights w_b, default 1); adds d L / d theta to the library's accumulator."""
    import torch
    st, ckpts = run(pm, noise, steps, a0, k_fs, checkpoints=True)
    _, P, _ = pm.power(st["u"], st["id"], SPECIES_ALL, SPECIES_ALL, nbins=nbins)
    sel = np.zeros(nbins, dtype=bool)
    sel[list(bins)] = True
    w = np.ones(sel.sum()) if weights is None else np.asarray(weights, dtype=np.float64)[sel]
    w = w / w.sum()
    r = P[sel] / p_ref[sel] - 1.0
    dL_dP = np.zeros(nbins)
    dL_dP[sel] = 2.0 * w * r / p_ref[sel]
    g = pm.power_vjp(st["u"], st["id"], dL_dP)
    lam_x = torch.empty_like(g)
    lam_x[:, st["id"].long()] = g                   # state order -> canonical id order
    lam_p = torch.zeros_like(lam_x)
    for ck, (a, ah, b) in zip(reversed(ckpts), reversed(steps)):
        lam_x, lam_p = pm.step_vjp(ck, a, ah, b, lam_x, lam_p)
    return float(np.sum(w * r ** 2))


def loss_bins(k, nmodes, k_max: float):
    """Indices of the non-empty bins with 0 < k <= k_max."""
    return [int(b) for b in np.nonzero((nmodes > 0) & (k > 0) & (k <= k_max))[0]]


def target_spectrum(pm: ParticleMesh, ref, nbins: int):
    """(k, P, n_modes) of a target run's final particles on the cheap context's estimator."""
    return pm.power(ref["u"], ref["id"], SPECIES_ALL, SPECIES_ALL, nbins=nbins)


@dataclasses.dataclass
class TrainLog:
    losses: list
    seconds: float
    iters: int


def train(pm: ParticleMesh, examples, steps, a0: float, iters: int, lr: float = 2e-3, k_fs: float = 0.0,
          t0: int = 0, verbose: bool = False, species: int = SPECIES_CDM, loss: str = "spectrum",
          nbins: int = 0, k_max: float = 1.0, mode_power: float = 0.0) -> TrainLog:
    """Adam on the mean loss over examples [(noise, ref), ...] (ref: the target run's final
    {"u", "id"}): one update per pass over all examples, iters passes.  loss = "spectrum"
    (bins of width k_F up to k_max, weighted by n_modes^mode_power; nbins = 0 picks N/2)
    or "displacement".  The factor must be on (pm.set_mlp)."""
    import torch
    losses = []
    start = time.perf_counter()
    if loss == "spectrum":
        nbins = nbins or pm.n // 2
        prepared = []
        for noise, ref in examples:
            k, P, nm = target_spectrum(pm, ref, nbins)
            prepared.append((noise, P, loss_bins(k, nm, k_max), np.maximum(nm, 1) ** mode_power))
    pm.mlp_grad(reset=True)                     # clear anything accumulated before
    for it in range(iters):
        tot = 0.0
        for i, (noise, ref) in enumerate(examples):
            if loss == "spectrum":
                _, P_ref, bins, wts = prepared[i]
                tot += spectrum_loss_and_grad(pm, noise, P_ref, bins, nbins, steps, a0, k_fs, wts)
            else:
                tot += loss_and_grad(pm, noise, ref, steps, a0, k_fs, species)
        g = pm.mlp_grad(reset=True)
        g.mul_(1.0 / len(examples))
        pm.mlp_adam(g, t0 + it + 1, lr=lr)
        losses.append(tot / len(examples))
        if verbose:
            print(f"iter {it:4d}  loss {losses[-1]:.6e}", flush=True)
    torch.cuda.synchronize()
    return TrainLog(losses, time.perf_counter() - start, iters)


def final_positions(pm: ParticleMesh, noise, steps, a0: float, k_fs: float = 0.0):
    st, _ = run(pm, noise, steps, a0, k_fs)
    return {"u": st["u"], "id": st["id"]}


def matter_power(meas: ParticleMesh, st, nbins: int):
    """P_m(k) of a run's final particles on the measuring context's mesh."""
    k, P, nm = meas.power(st["u"], st["id"], SPECIES_ALL, SPECIES_ALL, nbins=nbins)
    return k, P


def max_power_error(k, P, P_ref, k_max: float) -> float:
    """max over bins with 0 < k <= k_max of |P / P_ref - 1|."""
    sel = (k > 0) & (k <= k_max) & np.isfinite(P_ref) & (P_ref > 0)
    return float(np.max(np.abs(P[sel] / P_ref[sel] - 1.0)))


def boosted(cfg: RunConfig, boost: int) -> RunConfig:
    """The same run with a force mesh boost times the CDM grid per side."""
    return dataclasses.replace(cfg, nmesh=cfg.nc * boost)


def zero_factor(seed: int = 0) -> np.ndarray:
    """Initial parameters: random hidden layers, zero last layer (factor exactly 1)."""
    from .inputs import mlp_parameters
    th = mlp_parameters(seed)
    assert th.size == MLP_NPARAM
    return th


def train_shared(groups, steps, a0: float, iters: int, lr: float = 1e-2, k_max: float = 1.0,
                 nbins: int = 0, verbose: bool = False) -> TrainLog:
    """Spectrum-loss training of one parameter vector over several contexts (for instance one
    per neutrino mass): groups = [(pm, examples), ...].  The first context holds the
    parameters and the Adam state; before every pass the others receive its parameters, and
    after it their accumulated gradients are added to its own."""
    import torch
    primary = groups[0][0]
    prepared = []
    for pm, examples in groups:
        nb = nbins or pm.n // 2
        rows = []
        for noise, ref in examples:
            k, P, nm = target_spectrum(pm, ref, nb)
            rows.append((noise, P, loss_bins(k, nm, k_max)))
        prepared.append((pm, nb, rows))
    n_ex = sum(len(r) for _, _, r in prepared)
    theta = primary.get_mlp()
    for pm, _, _ in prepared:
        if pm is not primary:
            pm.set_mlp(theta)
        pm.mlp_grad(reset=True)
    losses = []
    start = time.perf_counter()
    for it in range(iters):
        theta = primary.get_mlp()
        tot = 0.0
        for pm, nb, rows in prepared:
            if pm is not primary:
                pm.set_mlp(theta)
            for noise, P_ref, bins in rows:
                tot += spectrum_loss_and_grad(pm, noise, P_ref, bins, nb, steps, a0)
        g = primary.mlp_grad(reset=True)
        for pm, _, _ in prepared:
            if pm is not primary:
                g += pm.mlp_grad(reset=True)
        g.mul_(1.0 / n_ex)
        primary.mlp_adam(g, it + 1, lr=lr)
        losses.append(tot / n_ex)
        if verbose:
            print(f"pass {it:4d}  loss {losses[-1]:.5e}  {time.perf_counter() - start:.1f} s", flush=True)
    torch.cuda.synchronize()
    return TrainLog(losses, time.perf_counter() - start, iters)


def experiment(nc_train: int = 128, nsites_train: int = 32, nc_eval: int = 256, nsites_eval: int = 64,
               spacing: float = 2.0, masses=(0.1, 0.3, 0.6), train_seeds=range(1000, 1064),
               eval_seeds=range(9001, 9005), boost_target: int = 4, iters: int = 100, lr: float = 1e-2,
               k_max: float = 1.0, verbose: bool = True, coarse_boost: int = 1,
               train_k_max: float = 0.0) -> dict:
    """The learned-correction workload: train on 10-step runs on a force mesh coarse_boost
    times the CDM grid (1, or the paper's 2) against 40-step boost_target runs (seeds cycling
    over the neutrino masses), evaluate on unseen seeds at a larger size against plain 10-,
    25- and 40-step runs on the same coarse mesh.  The loss covers the bins up to train_k_max
    (0: k_max), the evaluation those up to k_max.  Returns a dict of the per-mass errors
    max_{k <= k_max} |P_m / P_m,target - 1|, the median run times and the wall-time ratio of
    plain 25 steps to corrected 10."""
    import torch
    from . import workloads
    from .inputs import white_noise
    s10, s25, s40 = (workloads.schedule_paper(n) for n in (10, 25, 40))
    a0 = s10[0][0]

    def cfg_for(nc, nsites, m_total):
        return RunConfig(box=spacing * nc, nmesh=nc * coarse_boost, nc=nc, nsites=nsites, nshell=10, nfib=3,
                         m_nu=(m_total / 3,) * 3)

    def noise(nc, seed):
        return torch.from_numpy(white_noise(nc, seed=seed)).cuda()

    out = {"train": {}, "eval": {}, "coarse_boost": coarse_boost, "target_boost": boost_target,
           "iters": iters, "lr": lr, "train_k_max": train_k_max or k_max, "k_max": k_max}
    groups = []
    t0 = time.perf_counter()
    for j, m in enumerate(masses):
        cfg = cfg_for(nc_train, nsites_train, m)
        coarse = ParticleMesh(cfg)
        fine = ParticleMesh(boosted(cfg, boost_target))
        seeds = [s for i, s in enumerate(train_seeds) if i % len(masses) == j]
        examples = [(noise(nc_train, s), final_positions(fine, noise(nc_train, s), s40, a0)) for s in seeds]
        del fine
        groups.append((coarse, examples))
    groups[0][0].set_mlp(zero_factor(0))
    out["train"]["targets_s"] = time.perf_counter() - t0
    log = train_shared(groups, s10, a0, iters, lr=lr, k_max=train_k_max or k_max, verbose=verbose)
    out["train"].update({"losses": log.losses, "seconds": log.seconds, "passes": iters,
                         "examples": sum(len(e) for _, e in groups)})
    theta = groups[0][0].get_mlp()
    del groups
    nb = nc_eval
    for m in masses:
        cfg = cfg_for(nc_eval, nsites_eval, m)
        coarse = ParticleMesh(cfg)
        fine = ParticleMesh(boosted(cfg, boost_target))
        meas = ParticleMesh(boosted(cfg, 2)) if coarse_boost != 2 else coarse
        rows = {"corrected10": [], "plain10": [], "plain25": [], "plain40": []}
        times = {}
        for seed in eval_seeds:
            ev = noise(nc_eval, seed)
            k, P_ref = matter_power(meas, final_positions(fine, ev, s40, a0), nb)
            for name, sched, learned_on in (("corrected10", s10, True), ("plain10", s10, False),
                                            ("plain25", s25, False), ("plain40", s40, False)):
                coarse.set_mlp(theta if learned_on else None)
                torch.cuda.synchronize()
                t = time.perf_counter()
                st = final_positions(coarse, ev, sched, a0)
                torch.cuda.synchronize()
                times.setdefault(name, []).append(time.perf_counter() - t)
                _, P = matter_power(meas, st, nb)
                rows[name].append(max_power_error(k, P, P_ref, k_max))
        out["eval"][str(m)] = {name: float(np.max(v)) for name, v in rows.items()}
        out["eval"][str(m)]["run_seconds"] = {name: float(np.median(v)) for name, v in times.items()}
        out["eval"][str(m)]["plain25_over_corrected10_time"] = float(np.median(times["plain25"]) /
                                                                     np.median(times["corrected10"]))
        if verbose:
            print(m, out["eval"][str(m)], flush=True)
        del coarse, fine, meas
    return out


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="Train and evaluate the learned Green's-function factor")
    ap.add_argument("--nc-train", type=int, default=128)
    ap.add_argument("--nsites-train", type=int, default=32)
    ap.add_argument("--nc-eval", type=int, default=256)
    ap.add_argument("--nsites-eval", type=int, default=64)
    ap.add_argument("--train-seeds", type=int, default=64)
    ap.add_argument("--eval-seeds", type=int, default=4)
    ap.add_argument("--boost-target", type=int, default=4)
    ap.add_argument("--coarse-boost", type=int, default=1, help="force mesh of the cheap runs: 1 or 2 x the CDM grid")
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--lr", type=float, default=1e-2)
    ap.add_argument("--train-k-max", type=float, default=0.0, help="loss bins up to this k (0: 1 h/Mpc)")
    ap.add_argument("--out", default="")
    args = ap.parse_args()
    res = experiment(args.nc_train, args.nsites_train, args.nc_eval, args.nsites_eval,
                     train_seeds=range(1000, 1000 + args.train_seeds), eval_seeds=range(9001, 9001 + args.eval_seeds),
                     boost_target=args.boost_target, iters=args.iters, lr=args.lr, coarse_boost=args.coarse_boost,
                     train_k_max=args.train_k_max)
    text = json.dumps(res)
    print(text)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
