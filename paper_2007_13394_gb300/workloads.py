"""Synthetic workloads: run configurations and time-step schedules.

Sizes follow the paper's set-up (Table 1: mesh twice the CDM grid, N_shell = 10,
N_fib = 3 per site, 5 log-a steps from z = 99 to z = 19 then linear-a steps to
z = 0, §3).  The cosmology is Omega_m = 0.31, h = 0.68, n_s = 0.965,
sigma_8 = 0.81, T_cmb = 2.7255 K, N_eff = 3.046.
"""
from __future__ import annotations

import math

from .pm import RunConfig


def cfg1() -> RunConfig:
    """256 Mpc/h, 32^3 CDM + 8^3 x 70 neutrinos (M_nu = 0.2 eV, 3 degenerate), mesh 64^3."""
    return RunConfig(box=256.0, nmesh=64, nc=32, nsites=8, nshell=10, nfib=3, m_nu=(0.2 / 3,) * 3)


def cfg2() -> RunConfig:
    """512 Mpc/h, 256^3 CDM + 32^3 x 70 neutrinos (M_nu = 0.1 eV), mesh 512^3 (boost 2)."""
    return RunConfig(box=512.0, nmesh=512, nc=256, nsites=32, nshell=10, nfib=3, m_nu=(0.1 / 3,) * 3)


def cfg2_parity() -> RunConfig:
    """The cfg2 physics at 128^3 CDM + 16^3 x 70 neutrinos, mesh 256^3, 256 Mpc/h."""
    return RunConfig(box=256.0, nmesh=256, nc=128, nsites=16, nshell=10, nfib=3, m_nu=(0.1 / 3,) * 3)


def cfg3() -> RunConfig:
    """1024 Mpc/h, 1024^3 CDM + 128^3 x 70 neutrinos (one effective distribution for the
    normal-hierarchy masses summing to 0.6 eV), mesh 2048^3."""
    return RunConfig(box=1024.0, nmesh=2048, nc=1024, nsites=128, nshell=10, nfib=3,
                     m_nu=(0.19786, 0.19805, 0.20408))


def cfg_mid() -> RunConfig:
    """1024 Mpc/h, 512^3 CDM + 64^3 x 70 neutrinos (M_nu = 0.6 eV hierarchy), mesh 1024^3: the
    cfg3 density and boost at one eighth of the volume."""
    return RunConfig(box=1024.0, nmesh=1024, nc=512, nsites=64, nshell=10, nfib=3,
                     m_nu=(0.19786, 0.19805, 0.20408))


PRESETS = {"cfg1": cfg1, "cfg2": cfg2, "cfg2_parity": cfg2_parity, "cfg_mid": cfg_mid, "cfg3": cfg3}


def schedule_linear(a0: float, a1: float, n: int):
    """n steps linear in a; half points are arithmetic means."""
    edges = [a0 + (a1 - a0) * i / n for i in range(n + 1)]
    return [(edges[i], 0.5 * (edges[i] + edges[i + 1]), edges[i + 1]) for i in range(n)]


def schedule_paper(n_total: int, a_start: float = 0.01, a_switch: float = 0.05, a_end: float = 1.0,
                   n_log: int = 5):
    """n_log steps in log a to a_switch (geometric half points), the rest linear in a."""
    l0, l1 = math.log(a_start), math.log(a_switch)
    out = []
    for i in range(n_log):
        x0 = l0 + (l1 - l0) * i / n_log
        x1 = l0 + (l1 - l0) * (i + 1) / n_log
        a0 = a_start if i == 0 else math.exp(x0)
        a1 = a_switch if i == n_log - 1 else math.exp(x1)
        out.append((a0, math.exp(0.5 * (x0 + x1)), a1))
    if n_total > n_log:
        out += schedule_linear(a_switch, a_end, n_total - n_log)
    return out


def free_streaming_k(cfg: RunConfig, a: float) -> float:
    """k_fs(a) = 0.82 sqrt(Omega_L + Omega_m a^-3) a^2 (m_nu / 1 eV) h/Mpc for the mean eigenstate
    mass, Omega_L = 1 - Omega_m: the scale of the synthetic suppression of the initial neutrino
    field."""
    m = sum(cfg.m_nu) / max(1, len(cfg.m_nu))
    return 0.82 * math.sqrt((1.0 - cfg.omega_m) + cfg.omega_m / a ** 3) * a * a * m
