"""Validation experiments of the method on synthetic runs (no datasets), on the GPU.

* ``mass_ratio``: total-matter spectrum of a massive-neutrino run over the massless
  run from the same white noise (§3 Fig. MR analogue), for several numbers of
  linear-a steps; on scales above the neutrino free-streaming scale the ratio is
  compared with the 1 - 8 f_nu estimate of §1 (f_nu = Omega_nu0 / Omega_m0).
* ``neutrino_count_sensitivity``: the total-matter spectrum when N_sites or N_fib
  grows past the fiducial values (§3 Fig. gadget, right panel): the paper finds a
  change below 0.1 %.
* ``sampling_noise``: the neutrino spectrum of quasi-random sampling (shells x
  Fibonacci directions at each site) against pseudo-random sampling with about the
  same number of particles (§3 Fig. Pn_shotnoise): the pseudo-random spectrum
  flattens to the shot noise V / N_n, the quasi-random one stays below it except for
  spikes at the neutrino-grid wavenumbers k_n, sqrt(2) k_n, sqrt(3) k_n, 2 k_n.

All runs start at z = 99 with the paper's schedule (5 log-a steps to z = 19, then
linear-a steps to z = 0) from the library's Zel'dovich ICs; spectra come from
pm_power on the run's own force mesh.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import workloads
from .inputs import white_noise
from .pm import SPECIES_ALL, SPECIES_CDM, SPECIES_NU, ParticleMesh, RunConfig, cosmo_params


def _noise(nc: int, seed: int):
    import torch
    return torch.from_numpy(white_noise(nc, seed=seed)).cuda()


def run_spectra(cfg: RunConfig, n_lin: int, seed: int = 1, nbins: int = 0, k_fs: float = 0.0,
                species=((SPECIES_ALL, SPECIES_ALL),)):
    """Evolve cfg from z = 99 to z = 0 (5 log steps + n_lin linear steps) and return
    (k, {(a, b): P_ab}) at z = 0."""
    pm = ParticleMesh(cfg)
    steps = workloads.schedule_paper(5 + n_lin)
    a0 = steps[0][0]
    st = pm.ic(_noise(cfg.nc, seed), a0, k_fs=k_fs)
    pm.run(st, steps)
    nb = nbins or cfg.nmesh // 2
    out = {}
    k = None
    for sa, sb in species:
        k, P, _ = pm.power(st["u"], st["id"], sa, sb, nbins=nb)
        out[(sa, sb)] = P
    pm.close()
    return k, out


def f_nu(cfg: RunConfig) -> float:
    """Omega_nu0 / Omega_m0 of the configuration (Poisson source, §1)."""
    p = cosmo_params(cfg)
    return p["omega_nu"] / (p["omega_nu"] + p["omega_c"])


def mass_ratio(cfg_massive: RunConfig, n_lin_list=(10, 20, 40), seed: int = 1):
    """P_m(massive) / P_m(massless) at z = 0 for each number of linear steps."""
    cfg0 = dataclasses.replace(cfg_massive, nsites=0, m_nu=(0.0, 0.0, 0.0))
    res = {}
    k = None
    for n_lin in n_lin_list:
        k, Pm = run_spectra(cfg_massive, n_lin, seed)
        _, P0 = run_spectra(cfg0, n_lin, seed)
        res[n_lin] = Pm[(SPECIES_ALL, SPECIES_ALL)] / P0[(SPECIES_ALL, SPECIES_ALL)]
    return k, res, f_nu(cfg_massive)


def neutrino_count_sensitivity(cfg: RunConfig, n_lin: int = 20, seed: int = 1, factors=((2, 1), (1, 5 / 3))):
    """P_m of variants with nsites x fs and nfib x ff over the fiducial run, at z = 0."""
    k, P = run_spectra(cfg, n_lin, seed)
    base = P[(SPECIES_ALL, SPECIES_ALL)]
    out = {}
    for fs, ff in factors:
        v = dataclasses.replace(cfg, nsites=int(round(cfg.nsites * fs)), nfib=int(round(cfg.nfib * ff)))
        _, Pv = run_spectra(v, n_lin, seed)
        out[(v.nsites, v.nfib)] = Pv[(SPECIES_ALL, SPECIES_ALL)] / base
    return k, out


def sampling_noise(box: float = 256.0, nc: int = 128, nmesh: int = 256, m_total: float = 0.2,
                   quasi=(4, 10, 25), pseudo_sites: int = 32, n_lin: int = 20, seed: int = 1,
                   useed: int = 7):
    """Neutrino spectra at z = 0 of quasi-random sampling (nsites, nshell, nfib = quasi) and
    pseudo-random sampling (pseudo_sites^3 particles, one per site) from the same CDM and
    white noise.  Returns (k, P_nu quasi, P_nu pseudo, shot noise V / N_n pseudo, k_n)."""
    import torch
    from .inputs import uniform_values
    ns, nsh, nf = quasi
    cq = RunConfig(box=box, nmesh=nmesh, nc=nc, nsites=ns, nshell=nsh, nfib=nf, m_nu=(m_total / 3,) * 3)
    cp = RunConfig(box=box, nmesh=nmesh, nc=nc, nsites=pseudo_sites, nshell=1, nfib=0, m_nu=(m_total / 3,) * 3)
    steps = workloads.schedule_paper(5 + n_lin)
    a0 = steps[0][0]
    nb = nmesh // 2
    out = []
    for cfg, pseudo in ((cq, False), (cp, True)):
        pm = ParticleMesh(cfg)
        noise = _noise(nc, seed)
        if pseudo:
            uni = torch.from_numpy(uniform_values((3, pseudo_sites ** 3), useed)).cuda()
            st = pm.ic_pseudo(noise, uni, a0)
        else:
            st = pm.ic(noise, a0)
        pm.run(st, steps)
        k, P, _ = pm.power(st["u"], st["id"], SPECIES_NU, SPECIES_NU, nbins=nb)
        out.append(P)
        pm.close()
    return k, out[0], out[1], box ** 3 / pseudo_sites ** 3, 2 * np.pi * ns / box
