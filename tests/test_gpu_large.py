"""GPU force against the FP64 oracle at the large meshes, on sampled particles.

Inputs are the oracle's own Zel'dovich particles (CPU, seeded) taken at a = 1, where the
displacements of several Mpc/h cross shells and cluster the particles into dense tiles.
The GPU evaluates the force at every particle (pm_force); the oracle paints every particle
on the FP64 mesh, transforms it and reads the force out at 4096 sampled particles of both
species (oracle.pm.force_at).  Bar: relative RMS < 1e-5 (FP32 against FP64).

* 512^3 mesh: the 256^3 CDM + 32^3 x 70 neutrino density of the throughput workload.
* 1024^3 mesh: 512^3 CDM + 64^3 x 70 neutrinos in 1024 Mpc/h (the 2048^3 scale run's
  particle density and mesh boost at one eighth of its volume; 1024-point FFT lines).
  The oracle needs ~40 GB of host memory and a few minutes.

The 2048^3 mesh of the scale run is not compared with the oracle: its FP64 density and
half spectrum alone take 137 GB, and the out-of-place transforms a second copy, beyond
the 199 GB of host memory on the GPU machine.  There the force is checked against the
library's independent k-space path, and the FFT against a closed form.
"""
import numpy as np
import pytest

from oracle import background as obg
from oracle import ic as oic
from oracle import neutrinos as onu
from oracle import pm as opm
from paper_2007_13394_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def pm():
    import __graft_entry__ as g
    g.build()
    from paper_2007_13394_gb300 import pm as _pm
    return _pm


def oracle_particles(cfg, a, seed):
    """The oracle's Zel'dovich CDM and neutrino particles at scale factor a, canonical order,
    with their masses in units of the mean mass per mesh cell."""
    bg = obg.Background.physical(cfg.h, cfg.omega_m, nu_masses_ev=cfg.m_nu)
    noise = inputs.white_noise(cfg.nc, seed=seed).astype(np.float64)
    plin = oic.linear_power(cfg.omega_m, cfg.h, cfg.ns, cfg.sigma8)
    uc, _ = oic.cdm_particles(noise, cfg.box, plin, bg.D(a), bg.gp(a))
    _, q, m_shell = onu.shell_table(cfg.nshell, list(cfg.m_nu))
    un, _ = oic.neutrino_particles(noise, cfg.box, plin, bg.D(a), bg.gp(a), cfg.nsites, cfg.nshell, cfg.nfib,
                                   q, onu.thermal_momentum_scale(bg.kT_nu0, max(cfg.m_nu)),
                                   k_fs=oic.free_streaming_k(list(cfg.m_nu), 0.01, cfg.omega_m))
    del noise
    mc, mn = onu.species_masses(cfg.nmesh, cfg.nc, cfg.nsites, cfg.nshell, cfg.nfib, bg.omega_c,
                                bg.omega_nu_poisson, m_shell)
    mass = onu.particle_masses(uc.shape[1], un.shape[1], cfg.nshell, cfg.nfib, mc, mn)
    return np.hstack([uc, un]), mass, uc.shape[1], bg


def sampled_force_check(pm, cfg, seed, n_cdm_pick=3584, n_nu_pick=512):
    u, mass, ncdm, bg = oracle_particles(cfg, 1.0, seed)
    n = u.shape[1]
    ctx = pm.ParticleMesh(cfg)
    F = ctx.force(pm.as_u32_tensor(u))
    ctx.sync()
    rng = np.random.default_rng(seed)
    pick = np.concatenate([rng.choice(ncdm, n_cdm_pick, replace=False),
                           ncdm + rng.choice(n - ncdm, n_nu_pick, replace=False)])
    got = F[:, torch.from_numpy(pick).cuda()].double().cpu().numpy()
    ctx.close()
    del F
    torch.cuda.empty_cache()
    import os
    ref = opm.force_at(u, mass, cfg.nmesh, cfg.box, bg.omega_m0, pick, workers=os.cpu_count())
    rel = np.sqrt(((got - ref) ** 2).sum() / (ref ** 2).sum())
    rel_nu = np.sqrt(((got[:, n_cdm_pick:] - ref[:, n_cdm_pick:]) ** 2).sum() / (ref[:, n_cdm_pick:] ** 2).sum())
    print(f"\nmesh {cfg.nmesh}^3, {n} particles: force relative RMS {rel:.2e} (neutrinos {rel_nu:.2e})")
    assert rel < 1e-5 and rel_nu < 1e-5, (rel, rel_nu)


def test_force_at_512_mesh_matches_oracle_on_sampled_particles(pm):
    from paper_2007_13394_gb300 import workloads
    sampled_force_check(pm, workloads.cfg2(), seed=3)


def test_force_at_1024_mesh_matches_oracle_on_sampled_particles(pm):
    from paper_2007_13394_gb300 import workloads
    sampled_force_check(pm, workloads.cfg_mid(), seed=4)
