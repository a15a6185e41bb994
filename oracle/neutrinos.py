"""FP64 quasi-random Fermi-Dirac sampling of neutrino particles.

Test infrastructure only (see the package docstring).

Follows the paper's §2.1: the Fermi-Dirac distribution f(q) = 1/(e^q + 1)
(Eq. fd) with dn = q^2 f dq dOmega (Eq. dn); N_shell shells with equal area
under g(q) = q f(q) (Eq. N_shell, kernel choice stated right after it); per
shell the speed q_shell = sqrt(int q^4 f / int q^2 f) (Eq. q_shell) and the
mass fraction m_shell = int_shell q^2 f / int_0^qmax q^2 f (Eq. m_shell); the
effective distribution f~(q) = sum_j alpha_j^4 f(alpha_j q), alpha_j = m_j /
m_heaviest, for non-degenerate masses (Eq. FD_deg, Appendix A); 2 N_fib + 1
Fibonacci directions per shell; N_n = N_sites N_shell (2 N_fib + 1) (Eq. N_n);
a neutrino site grid staggered from the CDM grid, with particles placed on
spheres of radius proportional to their speed (§2.1, last paragraphs).

Readings where the paper is silent:
* q_max = 40 (the q^4 f tail beyond it is ~1e-12 of the total).
* Fibonacci lattice: for i = -N_fib..N_fib, sin(lat_i) = 2 i / (2 N_fib + 1),
  lon_i = 2 pi i / golden ratio; direction (cos lat cos lon, cos lat sin lon,
  sin lat); the same directions at every site.
* Particle order: CDM first, then neutrinos with index
  (site * N_shell + shell) * (2 N_fib + 1) + direction, sites x-major.
* Sites at (i + 1/2) Delta_site + 1/2 Delta_c per axis (CDM lattice at
  i Delta_c); shell radius 0.45 Delta_site q_shell / q_shell,max.
* Thermal momentum in the code's units (p = a^2 dx/dt / H0, Mpc/h):
  q_shell (k_B T_nu0 / m_heaviest) (c / H0), a-independent.
* Particle masses in units of the mean mass per mesh cell:
  CDM (Omega_c0 / Omega_m0) N^3 / N_c; neutrino
  (Omega_nu0 / Omega_m0) m_shell / (2 N_fib + 1) N^3 / N_sites.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize

Q_MAX = 40.0


def fd(q):
    """Eq. fd: f(q) = 1 / (e^q + 1)."""
    return 1.0 / (np.exp(q) + 1.0)


def effective_fd(q, alphas):
    """Eq. FD_deg: f~(q) = sum_j alpha_j^4 f(alpha_j q)."""
    return sum(a ** 4 * fd(a * q) for a in alphas)


def mass_ratios(masses_ev):
    """alpha_j = m_j / m_heaviest (Appendix A chooses mu = the heaviest mass)."""
    m1 = max(masses_ev)
    return [m / m1 for m in masses_ev]


def _quad(fun, a, b):
    v, _ = integrate.quad(fun, a, b, epsabs=0.0, epsrel=1e-13, limit=400)
    return v


def shell_table(n_shell, masses_ev, q_max=Q_MAX):
    """Shell edges, speeds q_shell and mass fractions m_shell (Eqs. N_shell, q_shell, m_shell).

    Returns (edges[n_shell + 1], q_shell[n_shell], m_shell[n_shell]).
    """
    alphas = mass_ratios(masses_ev)
    ft = lambda q: effective_fd(q, alphas)
    g = lambda q: q * ft(q)                       # kernel g(q) = q f(q)
    g_total = _quad(g, 0.0, q_max)
    edges = [0.0]
    for i in range(1, n_shell):
        target = i / n_shell * g_total
        lo = edges[-1]
        fun = lambda q: _quad(g, 0.0, q) - target
        edges.append(optimize.brentq(fun, lo, q_max, xtol=1e-15, rtol=4 * np.finfo(float).eps,
                                     maxiter=400))
    edges.append(q_max)
    z2 = _quad(lambda q: q * q * ft(q), 0.0, q_max)
    q_shell, m_shell = [], []
    for i in range(n_shell):
        lo, hi = edges[i], edges[i + 1]
        m2 = _quad(lambda q: q * q * ft(q), lo, hi)
        m4 = _quad(lambda q: q ** 4 * ft(q), lo, hi)
        q_shell.append(math.sqrt(m4 / m2))
        m_shell.append(m2 / z2)
    return np.array(edges), np.array(q_shell), np.array(m_shell)


def fibonacci_directions(n_fib):
    """2 N_fib + 1 unit vectors of the Fibonacci sphere lattice, shape (2 N_fib + 1, 3)."""
    golden = (1.0 + math.sqrt(5.0)) / 2.0
    npts = 2 * n_fib + 1
    out = np.empty((npts, 3))
    for k, i in enumerate(range(-n_fib, n_fib + 1)):
        lat = math.asin(2.0 * i / npts)
        lon = 2.0 * math.pi * i / golden
        out[k] = (math.cos(lat) * math.cos(lon), math.cos(lat) * math.sin(lon), math.sin(lat))
    return out


def neutrino_count(n_sites_side, n_shell, n_fib):
    """Eq. N_n: N_n = N_sites * N_shell * (2 N_fib + 1)."""
    return n_sites_side ** 3 * n_shell * (2 * n_fib + 1)


def site_positions(n_sites_side, n_c_side, box):
    """Neutrino site lattice, (n_sites^3, 3), staggered from the CDM lattice."""
    d_site = box / n_sites_side
    d_c = box / n_c_side
    ax = (np.arange(n_sites_side) + 0.5) * d_site + 0.5 * d_c
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1) % box


def thermal_momentum_scale(kT_nu0_ev, m_heaviest_ev, c_over_h0=2997.92458):
    """p per unit q in Mpc/h: (k_B T_nu0 / m c^2) (c / H0)."""
    return kT_nu0_ev / m_heaviest_ev * c_over_h0


def species_masses(n_mesh, n_c_side, n_sites_side, n_shell, n_fib, omega_c, omega_nu, m_shell):
    """Particle masses in units of the mean mass per mesh cell.

    Returns (m_cdm, m_nu[n_shell]).  Summed over all particles they give N^3,
    so the painted mesh holds rho / rho_bar with mean 1.
    """
    om = omega_c + omega_nu
    cells = float(n_mesh) ** 3
    m_cdm = omega_c / om * cells / float(n_c_side) ** 3 if n_c_side > 0 else 0.0
    if n_sites_side > 0:
        m_nu = omega_nu / om * np.asarray(m_shell) / (2 * n_fib + 1) * cells / float(n_sites_side) ** 3
    else:
        m_nu = np.zeros(0)
    return m_cdm, m_nu


def particle_masses(n_cdm, n_nu, n_shell, n_fib, m_cdm, m_nu):
    """Mass of every particle in the canonical order (CDM, then neutrinos by site/shell/dir)."""
    ndir = 2 * n_fib + 1
    out = np.empty(n_cdm + n_nu)
    out[:n_cdm] = m_cdm
    if n_nu:
        shell = (np.arange(n_nu) // ndir) % n_shell
        out[n_cdm:] = np.asarray(m_nu)[shell]
    return out


# ------------------------------------------------------------ pseudo-random sampling
def speed_cdf(q, masses_ev, q_max=Q_MAX):
    """Fraction of neutrinos with speed below q under the speed density q^2 f~(q) on
    [0, q_max] (the phase-space measure of the distribution of Eq. FD_deg)."""
    alphas = mass_ratios(masses_ev)
    dens = lambda x: x * x * effective_fd(x, alphas)  # noqa: E731
    total = _quad(dens, 0.0, q_max)
    return _quad(dens, 0.0, min(float(q), q_max)) / total


def speed_quantile(u, masses_ev, q_max=Q_MAX):
    """Inverse of :func:`speed_cdf`: the speed below which a fraction u of neutrinos lies
    (root of speed_cdf(q) = u by bisection-secant, to 1e-13)."""
    from scipy.optimize import brentq
    u = float(u)
    if u <= 0.0:
        return 0.0
    if u >= 1.0:
        return float(q_max)
    return brentq(lambda q: speed_cdf(q, masses_ev, q_max) - u, 0.0, q_max, xtol=1e-13, rtol=1e-13)
