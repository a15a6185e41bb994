"""Training and evaluation of the learned Green's-function factor on the GPU.

The factor m(|k| / k_Ny, a) = 1 + MLP multiplies the potential's Green's function
(library entry points pm_set_mlp ... pm_mlp_adam).  It is fitted so that a cheap run
(few steps, force mesh as fine as the CDM grid) lands where an expensive run of the
same initial conditions (many steps, a finer force mesh) does:

  loss    L = sum_i m_i |x_i - y_i|^2 / sum_i m_i, the periodic displacement between
          the cheap run's final CDM particles x and the expensive run's y, pairing by id
          (pm_displacement_loss).  Neutrinos are left out of the loss by default: their
          thermal streaming over the whole run depends on the step schedule through the
          drift factor, a difference no force correction can remove, and it would
          swamp the CDM signal;
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
    for (a, ah, b) in steps:
        if checkpoints:
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


@dataclasses.dataclass
class TrainLog:
    losses: list
    seconds: float
    iters: int


def train(pm: ParticleMesh, examples, steps, a0: float, iters: int, lr: float = 2e-3, k_fs: float = 0.0,
          t0: int = 0, verbose: bool = False, species: int = SPECIES_CDM) -> TrainLog:
    """Adam on the mean displacement loss over examples [(noise, ref), ...]: one update per
    pass over all examples, iters passes.  The factor must be on (pm.set_mlp)."""
    import torch
    losses = []
    start = time.perf_counter()
    pm.mlp_grad(reset=True)                     # clear anything accumulated before
    for it in range(iters):
        tot = 0.0
        for noise, ref in examples:
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
