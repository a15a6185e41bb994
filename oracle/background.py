"""FP64 background expansion, linear growth and FastPM step coefficients.

Test infrastructure only (see the package docstring).

Follows the paper's §2.3 ("Evolution"): the Hubble function (Eq. Hubble) with
photons, CDM, massive neutrinos through the Fermi-Dirac integral F(y), and a
cosmological constant; the growth ODE (Eq. growthDE) with matter-domination
initial conditions D = D' = a_ini at z_ini = 159; and §2.2 (Eq. Om_pois) for
the Poisson/growth source, in which neutrinos count as matter with
Omega_m0 = Omega_c0 + Omega_nu0.

Readings where the paper is silent or garbled:
* Eq. Om_pois prints Omega_m(a) = Omega_m0 a^-3 without 1/E^2.  With
  ' = d/d ln a, the growth ODE needs Omega_m(a) = Omega_m0 a^-3 / E(a)^2; this is
  the form used (it is the one that makes g_f = 1.5 Omega_m0 D).
* Gamma_nu = (4/11)^(1/3) (N_eff/3)^(1/4); Omega_gamma0 from T_cmb by the
  Stefan-Boltzmann law; Omega_nu0 (Poisson source) = M_nu / (93.14 h^2 eV)
  (§1); Omega_c0 = Omega_m - Omega_nu0; Omega_Lambda closes E(1) = 1 with the
  exact F(y) neutrino density.
* FastPM growth functions: g_p = a^3 E dD/da = a^2 E D', g_f = a^2 E dg_p/da
  = 1.5 Omega_m0 D.  Kick over [a_b, a_c] with the force at a_f:
  (g_p(a_c) - g_p(a_b)) / g_f(a_f); drift over [a_0, a_1] with momenta at a_h:
  (D(a_1) - D(a_0)) / g_p(a_h).  These reproduce x = q + D(a) s exactly when
  F = g_f(a) s (the Zel'dovich trajectory, §2.3 first paragraph).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate

# CODATA 2018 / SI exact values (restated; not shared with the CUDA path)
C_LIGHT = 299792458.0            # m / s
G_NEWTON = 6.67430e-11           # m^3 kg^-1 s^-2
SIGMA_SB = 5.670374419e-8        # W m^-2 K^-4
K_BOLTZMANN_EV = 8.617333262e-5  # eV / K
MPC_M = 3.0856775814913673e22    # m
C_OVER_H0_MPC_H = C_LIGHT / 1.0e5  # c / (100 km/s/Mpc) in Mpc/h = 2997.92458


def omega_gamma_h2(t_cmb: float) -> float:
    """Omega_gamma0 h^2 from the CMB temperature (Stefan-Boltzmann law)."""
    rho_gamma = 4.0 * SIGMA_SB * t_cmb ** 4 / C_LIGHT ** 3          # kg / m^3
    h100 = 1.0e5 / MPC_M                                           # 1 / s
    rho_crit_over_h2 = 3.0 * h100 ** 2 / (8.0 * math.pi * G_NEWTON)
    return rho_gamma / rho_crit_over_h2


def fd_F(y: float) -> float:
    """F(y) = int_0^inf x^2 sqrt(x^2 + y^2) / (1 + e^x) dx   (§2.3, F(y))."""
    f = lambda x: x * x * math.sqrt(x * x + y * y) / (1.0 + math.exp(x)) if x < 700 else 0.0
    val, _ = integrate.quad(f, 0.0, np.inf, epsabs=0.0, epsrel=1e-13, limit=400)
    return val


def fd_dF(y: float) -> float:
    """dF/dy = int_0^inf x^2 y / sqrt(x^2 + y^2) / (1 + e^x) dx."""
    if y == 0.0:
        return 0.0
    f = lambda x: x * x * y / math.sqrt(x * x + y * y) / (1.0 + math.exp(x)) if x < 700 else 0.0
    val, _ = integrate.quad(f, 0.0, np.inf, epsabs=0.0, epsrel=1e-13, limit=400)
    return val


class Background:
    """E(a), Omega_m(a) and the growth solution for one set of parameters.

    Either build it from physical parameters with :meth:`physical`, or give the
    density parameters explicitly (used by the EdS / LCDM pins).
    """

    def __init__(self, omega_gamma=0.0, omega_c=0.3, omega_lambda=0.7,
                 omega_nu_poisson=0.0, nu_masses_ev=(), gamma_nu=0.0,
                 kT_nu0_ev=1.0, a_ini=1.0 / 160.0):
        self.omega_gamma = float(omega_gamma)
        self.omega_c = float(omega_c)
        self.omega_lambda = float(omega_lambda)
        self.omega_nu_poisson = float(omega_nu_poisson)
        self.nu_masses = [float(m) for m in nu_masses_ev]
        self.gamma_nu = float(gamma_nu)
        self.kT_nu0 = float(kT_nu0_ev)
        self.omega_m0 = self.omega_c + self.omega_nu_poisson   # Eq. Om_pois
        self.a_ini = float(a_ini)
        self._sol = None
        self._D1 = None

    # -- construction from physical parameters ----------------------------
    @classmethod
    def physical(cls, h, omega_m, t_cmb=2.7255, n_eff=3.046, nu_masses_ev=(0.0, 0.0, 0.0),
                 a_ini=1.0 / 160.0):
        gamma_nu = (4.0 / 11.0) ** (1.0 / 3.0) * (n_eff / 3.0) ** 0.25
        og = omega_gamma_h2(t_cmb) / h ** 2
        m_tot = float(sum(nu_masses_ev))
        onu_p = m_tot / (93.14 * h ** 2)                 # §1, Omega_nu0 = M_nu / 93.14 h^2 eV
        oc = omega_m - onu_p
        kT = K_BOLTZMANN_EV * gamma_nu * t_cmb
        bg = cls(omega_gamma=og, omega_c=oc, omega_lambda=0.0, omega_nu_poisson=onu_p,
                 nu_masses_ev=nu_masses_ev, gamma_nu=gamma_nu, kT_nu0_ev=kT, a_ini=a_ini)
        # flatness closes Omega_Lambda with the exact neutrino density at a = 1
        bg.omega_lambda = 1.0 - og - oc - bg.omega_nu_E2(1.0)
        return bg

    # -- Eq. Hubble and its neutrino term -----------------------------------
    def omega_nu_E2(self, a: float) -> float:
        """Omega_nu(a) E^2(a) = (15/pi^4) Gamma^4 Omega_gamma a^-4 sum_j F(m_j a / kT)."""
        if not self.nu_masses:
            return 0.0
        s = sum(fd_F(m * a / self.kT_nu0) for m in self.nu_masses)
        return 15.0 / math.pi ** 4 * self.gamma_nu ** 4 * self.omega_gamma / a ** 4 * s

    def _d_omega_nu_E2_dlna(self, a: float) -> float:
        if not self.nu_masses:
            return 0.0
        s = 0.0
        for m in self.nu_masses:
            y = m * a / self.kT_nu0
            s += -4.0 * fd_F(y) + y * fd_dF(y)
        return 15.0 / math.pi ** 4 * self.gamma_nu ** 4 * self.omega_gamma / a ** 4 * s

    def E2(self, a: float) -> float:
        return (self.omega_gamma / a ** 4 + self.omega_c / a ** 3 + self.omega_nu_E2(a)
                + self.omega_lambda)

    def E(self, a: float) -> float:
        return math.sqrt(self.E2(a))

    def dlnE_dlna(self, a: float) -> float:
        dE2 = (-4.0 * self.omega_gamma / a ** 4 - 3.0 * self.omega_c / a ** 3
               + self._d_omega_nu_E2_dlna(a))
        return 0.5 * dE2 / self.E2(a)

    def omega_m(self, a: float) -> float:
        """Source term of Eq. growthDE: Omega_m0 a^-3 / E^2 (reading of Eq. Om_pois)."""
        return self.omega_m0 / a ** 3 / self.E2(a)

    # -- Eq. growthDE ---------------------------------------------------------
    def _rhs(self, lna, y):
        a = math.exp(lna)
        D, Dp = y
        return [Dp, -(2.0 + self.dlnE_dlna(a)) * Dp + 1.5 * self.omega_m(a) * D]

    def _solve(self):
        if self._sol is None:
            y0 = [self.a_ini, self.a_ini]            # D(a_ini) = D'(a_ini) = a_ini
            self._sol = integrate.solve_ivp(self._rhs, (math.log(self.a_ini), math.log(2.0)), y0,
                                            method="DOP853", rtol=1e-13, atol=1e-16,
                                            dense_output=True)
            assert self._sol.success
            self._D1 = self._sol.sol(0.0)[0]
        return self._sol

    def growth_unnormalised(self, a: float):
        """(D, dD/dln a) with the paper's initial conditions, not normalised."""
        s = self._solve()
        D, Dp = s.sol(math.log(a))
        return float(D), float(Dp)

    def D(self, a: float) -> float:
        """Linear growth factor normalised to D(1) = 1."""
        self._solve()
        return self.growth_unnormalised(a)[0] / self._D1

    def dD_dlna(self, a: float) -> float:
        self._solve()
        return self.growth_unnormalised(a)[1] / self._D1

    def gp(self, a: float) -> float:
        """g_p(a) = a^3 E dD/da = a^2 E dD/dln a."""
        return a * a * self.E(a) * self.dD_dlna(a)

    def gf(self, a: float) -> float:
        """g_f(a) = a^2 E dg_p/da, which the growth ODE makes equal to 1.5 Omega_m0 D."""
        return 1.5 * self.omega_m0 * self.D(a)


def step_coefficients(bg: Background, a0: float, ah: float, a1: float):
    """FastPM kick-drift-kick factors for one step a0 -> a1 with half point ah.

    Returns (K1, Delta, K2): first half kick with the force at a0, drift with
    momenta at ah, second half kick with the force at a1.
    """
    K1 = (bg.gp(ah) - bg.gp(a0)) / bg.gf(a0)
    Delta = (bg.D(a1) - bg.D(a0)) / bg.gp(ah)
    K2 = (bg.gp(a1) - bg.gp(ah)) / bg.gf(a1)
    return K1, Delta, K2


def schedule_linear(a_start: float, a_end: float, nsteps: int):
    """Steps linear in a; half points are arithmetic means."""
    a = np.linspace(a_start, a_end, nsteps + 1)
    return [(a[i], 0.5 * (a[i] + a[i + 1]), a[i + 1]) for i in range(nsteps)]


def schedule_paper(nsteps_total: int, a_start=0.01, a_switch=0.05, a_end=1.0, nlog=5):
    """5 steps in log a from z = 99 to z = 19, then linear in a to z = 0 (§3).

    Half points: geometric mean on the log-a segment, arithmetic mean on the
    linear segment (the paper does not state them; this is the reading used).
    """
    la = np.linspace(math.log(a_start), math.log(a_switch), nlog + 1)
    edges = [math.exp(x) for x in la]
    edges[0], edges[-1] = a_start, a_switch
    steps = [(edges[i], math.exp(0.5 * (la[i] + la[i + 1])), edges[i + 1]) for i in range(nlog)]
    nlin = nsteps_total - nlog
    if nlin > 0:
        steps += schedule_linear(a_switch, a_end, nlin)
    return steps
