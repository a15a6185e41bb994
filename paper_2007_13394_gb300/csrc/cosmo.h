// Host FP64 cosmology for the particle-mesh step: background E(a), linear growth,
// FastPM kick/drift factors, Fermi-Dirac shell tables and the synthetic initial
// spectrum normalisation.  Plain C++17, no CUDA.
#pragma once

#include <vector>

#include "../../include/pm.h"

namespace pmnu {

struct Cosmo {
  // background (§2.3 Eq. Hubble; §1 Omega_nu0 = M_nu / 93.14 h^2 eV; §2.2 Eq. Om_pois)
  double h = 0, omega_m0 = 0, omega_gamma = 0, omega_c = 0, omega_nu = 0, omega_lambda = 0;
  double gamma_nu = 0, kT_nu0 = 0;  // T_nu0 / T_gamma0, k_B T_nu0 in eV
  std::vector<double> masses;       // distinct eigenstate masses (eV)
  std::vector<int> mult;            // multiplicity of each distinct mass
  // growth table on a uniform grid in ln a
  double lna0 = 0, dlna = 0, D1 = 1;
  std::vector<double> tabD, tabDp, tabDpp;   // D, dD/dln a, d2D/dln a^2 at the grid nodes
  std::vector<double> tabE2, tabE2p;         // E^2 and dE^2/dln a at the grid nodes
  bool fast = false;                         // evaluate D, g_p, E from the tables

  int init(const pm_config& cfg);
  double E2(double a) const;
  double E(double a) const;
  double dlnE_dlna(double a) const;
  void growth(double a, double* D, double* dDdlna) const;  // normalised D(1) = 1
  double D(double a) const;
  double gp(double a) const;
  double gf(double a) const;
  void coeffs(double a0, double ah, double a1, double out[3]) const;

 private:
  double omega_nu_E2(double a) const;
  double d_omega_nu_E2_dlna(double a) const;
  void rhs(double lna, const double y[2], double dy[2]) const;
  void rk4(double lna, double h, double y[2]) const;
};

// k_B T and the Fermi-Dirac integral F(y) = int x^2 sqrt(x^2 + y^2) / (1 + e^x) dx and dF/dy
double fd_integral(double y);
double fd_integral_dy(double y);

// Shell table for n_shell shells of the effective distribution of the given masses (eV).
int nu_shell_table(int n_shell, const double* masses, int nmass, double q_max, double* edges,
                   double* q_shell, double* m_shell);

// CDF of the neutrino speed density q^2 f~(q) (Eq. FD_deg over the given masses, relative
// to the heaviest) on [0, q_max] at nnodes equally spaced q, normalised to F(q_max) = 1.
int nu_speed_cdf_table(const double* masses, int nmass, double q_max, int nnodes, double* F);

// BBKS transfer function T(k), k in h/Mpc
double bbks(double k, double omega_m, double h);
// amplitude A of P(k) = A k^ns T(k)^2 giving sigma_8 at z = 0
double power_amplitude(double omega_m, double h, double ns, double sigma8);

int validate_config(const pm_config& cfg);

}  // namespace pmnu
