"""FP64 Zel'dovich initial conditions on synthetic Gaussian fields.

Test infrastructure only (see the package docstring).

The paper sets initial perturbations with the Zel'dovich approximation
x = q + D s (§2.2, §2.3) from REPS two-fluid transfer functions, which are not
available here.  The stand-in, used identically by the oracle and the GPU
path: a BBKS spectrum (Bardeen, Bond, Kaiser & Szalay 1986) normalised to
sigma_8 with a top-hat of 8 Mpc/h, P(k) = A k^n_s T_BBKS(k)^2 at z = 0, and
a seeded unit white-noise field omega on the N_c^3 Lagrangian lattice
(random numbers come in as an input array).

Discrete conventions: delta_k = FFT(omega) sqrt(P(k)/V) N_c^(3/2), so that
<|delta_k|^2> = P N_c^6 / V; k = 0 and every Nyquist plane are zeroed;
s_k = i k delta_k / k^2 (so delta = -div s); s(x) = IFFT(s_k) / N_c^3.
CDM particle at lattice node q = i Delta_c: x = q + D(a0) s(q),
p = g_p(a0) s(q).  Neutrino sites take the displacement of the same Fourier
series evaluated exactly at the site (a phase shift by the site offset), of
a field optionally suppressed by 1 / (1 + (k / k_fs)^2) (a declared synthetic
free-streaming suppression); each neutrino adds its shell offset
r_shell n_dir to x and its thermal momentum p_th n_dir to p.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate

from . import neutrinos, pm


def bbks_transfer(k, omega_m, h):
    """BBKS transfer function with q = k / (Omega_m h), k in h/Mpc."""
    k = np.asarray(k, dtype=np.float64)
    q = k / (omega_m * h)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (np.log(1.0 + 2.34 * q) / (2.34 * q)
             * (1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4) ** -0.25)
    return np.where(q > 0, t, 1.0)


def tophat_window(x):
    x = np.asarray(x, dtype=np.float64)
    return 3.0 * (np.sin(x) - x * np.cos(x)) / x ** 3


def sigma_r_squared(pk, radius):
    """sigma^2(R) = int k^2 P(k) W_TH(kR)^2 dk / (2 pi^2)."""
    f = lambda lnk: (math.exp(lnk) ** 3 * pk(math.exp(lnk))
                     * float(tophat_window(math.exp(lnk) * radius)) ** 2 / (2.0 * math.pi ** 2))
    v, _ = integrate.quad(f, math.log(1e-6), math.log(1e3), epsabs=0.0, epsrel=1e-11, limit=2000)
    return v


def linear_power(omega_m, h, n_s, sigma8):
    """P(k) at z = 0 (D(1) = 1), a callable of k in h/Mpc, in (Mpc/h)^3."""
    shape = lambda k: float(k) ** n_s * float(bbks_transfer(k, omega_m, h)) ** 2
    amp = sigma8 ** 2 / sigma_r_squared(shape, 8.0)

    def pk(k):
        k = np.asarray(k, dtype=np.float64)
        return amp * np.where(k > 0, k, 1.0) ** n_s * bbks_transfer(k, omega_m, h) ** 2
    pk.amplitude = amp
    return pk


def _kgrid(nc, box):
    kfull, khalf, nfull, nhalf = pm.wavenumbers(nc, box)
    KX = kfull[:, None, None]
    KY = kfull[None, :, None]
    KZ = khalf[None, None, :]
    nyq = ((nfull == -nc // 2)[:, None, None] | (nfull == -nc // 2)[None, :, None]
           | (nhalf == nc // 2)[None, None, :])
    return KX, KY, KZ, nyq


def delta_k(noise, box, pk):
    """delta_k = FFT(omega) sqrt(P/V) N_c^(3/2), k = 0 and Nyquist planes zeroed."""
    nc = noise.shape[0]
    KX, KY, KZ, nyq = _kgrid(nc, box)
    k = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    dk = np.fft.rfftn(np.asarray(noise, dtype=np.float64)) * np.sqrt(pk(k) / box ** 3) * nc ** 1.5
    dk[nyq] = 0.0
    dk[0, 0, 0] = 0.0
    return dk


def free_streaming_k(masses_ev, a, omega_m):
    """Free-streaming wavenumber of the synthetic neutrino suppression, h/Mpc:
    k_fs(a) = 0.82 sqrt(Omega_L + Omega_m a^-3) a^2 (m / 1 eV) with Omega_L = 1 - Omega_m
    (flat, radiation neglected) and m the mean eigenstate mass (the standard scaling of
    Lesgourgues & Pastor, the reading taken for the REPS neutrino transfer functions the
    paper's initial conditions use, §2.2)."""
    m = sum(masses_ev) / len(masses_ev)
    return 0.82 * math.sqrt((1.0 - omega_m) + omega_m / a ** 3) * a * a * m


def displacement(dk, box, shift=0.0, k_fs=0.0):
    """s(x_i + shift) on the lattice, shape (3, N_c, N_c, N_c); optional 1/(1+(k/k_fs)^2)."""
    nc = dk.shape[0]
    KX, KY, KZ, _ = _kgrid(nc, box)
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = np.where(k2 > 0, 1.0 / k2, 0.0)
    filt = 1.0 / (1.0 + k2 / k_fs ** 2) if k_fs > 0 else 1.0
    phase = np.exp(1j * (KX + KY + KZ) * shift) if shift != 0.0 else 1.0
    out = []
    for kj in (KX, KY, KZ):
        sk = 1j * kj * dk * inv * filt * phase
        out.append(np.fft.irfftn(sk, s=(nc, nc, nc), axes=(0, 1, 2)))
    return np.stack(out)


def cdm_particles(noise, box, pk, D0, gp0):
    """(u, p) of the N_c^3 CDM particles, lattice order i = (i_x N_c + i_y) N_c + i_z."""
    nc = noise.shape[0]
    s = displacement(delta_k(noise, box, pk), box).reshape(3, -1)
    ax = np.arange(nc) * (box / nc)
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    q = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    return pm.quantise(q + D0 * s, box), gp0 * s


def neutrino_site_offset(nc, n_sites):
    """(lattice stride r, first node j0, extra shift) locating the sites on the CDM lattice.

    Sites sit at (i + 1/2) Delta_site + 1/2 Delta_c = ((i + 1/2) r + 1/2) Delta_c.
    For even r this is node r i + r/2 shifted by Delta_c / 2; for odd r it is
    node r i + (r + 1)/2 with no shift.
    """
    r = nc // n_sites
    if r % 2 == 0:
        return r, r // 2, 0.5
    return r, (r + 1) // 2, 0.0


def neutrino_particles(noise, box, pk, D0, gp0, n_sites, n_shell, n_fib, q_shell,
                       p_scale, k_fs=0.0):
    """(u, p) of the neutrino particles in order (site, shell, direction)."""
    nc = noise.shape[0]
    dc = box / nc
    r, j0, sh = neutrino_site_offset(nc, n_sites)
    s = displacement(delta_k(noise, box, pk), box, shift=sh * dc, k_fs=k_fs)
    idx = (j0 + r * np.arange(n_sites)) % nc
    s_site = s[:, idx][:, :, idx][:, :, :, idx].reshape(3, -1)          # (3, n_sites^3)
    site = neutrinos.site_positions(n_sites, nc, box).T                  # (3, n_sites^3)
    dirs = neutrinos.fibonacci_directions(n_fib)                         # (ndir, 3)
    q_shell = np.asarray(q_shell)
    radius = 0.45 * (box / n_sites) * q_shell / q_shell.max()
    ndir = 2 * n_fib + 1
    nsite = n_sites ** 3
    # broadcast to (3, site, shell, dir)
    off = radius[None, None, :, None] * dirs.T[:, None, None, :]
    pth = (p_scale * q_shell)[None, None, :, None] * dirs.T[:, None, None, :]
    x = site[:, :, None, None] + D0 * s_site[:, :, None, None] + off
    p = gp0 * s_site[:, :, None, None] + pth
    x = np.broadcast_to(x, (3, nsite, n_shell, ndir)).reshape(3, -1)
    p = np.broadcast_to(p, (3, nsite, n_shell, ndir)).reshape(3, -1)
    return pm.quantise(x, box), p


def pseudo_neutrino_particles(noise, box, pk, D0, gp0, n_sites, uniforms, masses_ev, p_scale, k_fs=0.0):
    """Pseudo-random neutrino sampling (the comparison scheme of §3 Fig. Pn_shotnoise): one
    particle per site of the neutrino lattice, at the site plus the Zel'dovich displacement,
    with a thermal momentum of speed q = speed_quantile(u_0) and an isotropic direction
    cos(theta) = 2 u_1 - 1, phi = 2 pi u_2 (uniforms (3, n_sites^3) in (0, 1), drawn
    outside).  Returns (u, p) in site order."""
    nc = noise.shape[0]
    dc = box / nc
    r, j0, sh = neutrino_site_offset(nc, n_sites)
    s = displacement(delta_k(noise, box, pk), box, shift=sh * dc, k_fs=k_fs)
    idx = (j0 + r * np.arange(n_sites)) % nc
    s_site = s[:, idx][:, :, idx][:, :, :, idx].reshape(3, -1)
    site = neutrinos.site_positions(n_sites, nc, box).T
    uq, umu, uphi = (np.asarray(x, dtype=np.float64) for x in uniforms)
    q = np.array([neutrinos.speed_quantile(v, masses_ev) for v in uq])
    mu = 2.0 * umu - 1.0
    phi = 2.0 * np.pi * uphi
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    dirs = np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), mu])
    x = site + D0 * s_site
    p = gp0 * s_site + p_scale * q[None, :] * dirs
    return pm.quantise(x, box), p
