"""Differentiable forward model for reconstruction: white noise -> Zel'dovich ICs ->
KDK steps -> final CIC density, as a ``torch.autograd.Function``.

The forward pass keeps a checkpoint of the particle state (u, p, id, f = F(x)) at the
start of every step; the backward pass runs the library's hand-written adjoint kernels
(``pm_paint_vjp``, ``pm_step_vjp`` in reverse, ``pm_ic_vjp``).  Cotangents travel in
canonical particle-id order, so the tile reordering of each step needs no bookkeeping
here beyond one scatter by id after the paint VJP.
"""
from __future__ import annotations

import torch

from .pm import ParticleMesh


class FinalDensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, noise, pmctx: ParticleMesh, steps, a0: float, k_fs: float):
        st = pmctx.ic(noise.contiguous(), a0, k_fs=k_fs)
        pmctx.set_force_time(a0)
        st["f"].copy_(pmctx.force(st["u"], st["id"]))
        st["f_valid"] = 1
        ckpts = []
        for (a, ah, b) in steps:
            ckpts.append({k: st[k].clone() for k in ("u", "p", "id", "f")} | {"a": a, "f_valid": 1})
            pmctx.step(st, a, ah, b)
        rho = pmctx.paint(st["u"], st["id"])
        ctx.pmctx, ctx.steps, ctx.a0, ctx.k_fs = pmctx, list(steps), a0, k_fs
        ctx.ckpts = ckpts
        ctx.final = {"u": st["u"], "id": st["id"]}
        return rho

    @staticmethod
    def backward(ctx, grad_rho):
        pmctx = ctx.pmctx
        u, ids = ctx.final["u"], ctx.final["id"]
        g = pmctx.paint_vjp(u, ids, grad_rho.contiguous().float())
        lam_x = torch.empty_like(g)
        lam_x[:, ids.long()] = g                       # state order -> canonical id order
        lam_p = torch.zeros_like(lam_x)
        for ck, (a, ah, b) in zip(reversed(ctx.ckpts), reversed(ctx.steps)):
            lam_x, lam_p = pmctx.step_vjp(ck, a, ah, b, lam_x, lam_p)
        grad_noise = pmctx.ic_vjp(lam_x, lam_p, ctx.a0, k_fs=ctx.k_fs)
        return grad_noise, None, None, None, None


def final_density(noise, pmctx: ParticleMesh, steps, a0: float, k_fs: float = 0.0):
    """Final CIC density rho / rho_bar (N^3) of the run started from white noise."""
    return FinalDensity.apply(noise, pmctx, steps, a0, k_fs)


def density_mse(noise, target, pmctx: ParticleMesh, steps, a0: float, k_fs: float = 0.0):
    """Reconstruction loss mean((rho - target)^2) with gradients to the noise."""
    rho = final_density(noise, pmctx, steps, a0, k_fs)
    return ((rho - target) ** 2).mean()
