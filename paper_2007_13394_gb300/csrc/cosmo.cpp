// Host FP64 cosmology: background, growth ODE, KDK factors, neutrino shells,
// synthetic spectrum normalisation.  Quadrature is composite Gauss-Legendre with
// nodes from Newton iteration on P_n; the ODE is fixed-step RK4 in ln a.
#include "cosmo.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace pmnu {

namespace {

constexpr double kPi = 3.14159265358979323846;
// SI constants (CODATA 2018 / exact SI)
constexpr double kC = 299792458.0;
constexpr double kG = 6.67430e-11;
constexpr double kSigmaSB = 5.670374419e-8;
constexpr double kBoltzEV = 8.617333262e-5;
constexpr double kMpc = 3.0856775814913673e22;

struct GL {
  std::vector<double> x, w;  // nodes/weights on [-1, 1]
  explicit GL(int n) : x(n), w(n) {
    for (int i = 0; i < n; ++i) {
      double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        double dp = n * (z * p1 - p0) / (z * z - 1.0);
        double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      x[i] = z;
      w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
  }
};

const GL& gl20() {
  static GL g(20);
  return g;
}

template <class F>
double integrate(F f, double a, double b, int intervals) {
  const GL& g = gl20();
  double s = 0.0, h = (b - a) / intervals;
  for (int i = 0; i < intervals; ++i) {
    double lo = a + i * h, c = lo + 0.5 * h;
    double acc = 0.0;
    for (size_t k = 0; k < g.x.size(); ++k) acc += g.w[k] * f(c + 0.5 * h * g.x[k]);
    s += 0.5 * h * acc;
  }
  return s;
}

double fermi(double x) { return x > 700.0 ? 0.0 : 1.0 / (std::exp(x) + 1.0); }

}  // namespace

// F(y) = int_0^inf x^2 sqrt(x^2 + y^2) / (1 + e^x) dx, truncated at x = 80 (tail < 1e-30)
double fd_integral(double y) {
  return integrate([y](double x) { return x * x * std::sqrt(x * x + y * y) * fermi(x); }, 0.0,
                   80.0, 32);
}

double fd_integral_dy(double y) {
  if (y == 0.0) return 0.0;
  return integrate([y](double x) { return x * x * y / std::sqrt(x * x + y * y) * fermi(x); }, 0.0,
                   80.0, 32);
}

int validate_config(const pm_config& c) {
  if (!(c.box > 0.0) || !std::isfinite(c.box)) return PM_EINVAL;
  if (c.nmesh < 32 || c.nmesh > 2048 || (c.nmesh & (c.nmesh - 1))) return PM_EINVAL;
  if (c.nc < 0 || c.nsites < 0 || c.nc > c.nmesh) return PM_EINVAL;
  if (c.nsites > 0 && (c.nshell < 1 || c.nfib < 0)) return PM_EINVAL;
  if (!(c.h > 0.0) || !(c.omega_m > 0.0)) return PM_EINVAL;
  if (c.n_nu < 0 || c.n_nu > 3) return PM_EINVAL;
  if (c.flags & ~(uint32_t)(PM_FLAG_TWO_MESH | PM_FLAG_SPECTRAL_KERNEL | PM_FLAG_MLP_TENSOR |
                           PM_FLAG_KSPACE_GRADIENT))
    return PM_EINVAL;
  if (c.mem_limit < 0) return PM_EINVAL;
  for (int i = 0; i < c.n_nu; ++i)
    if (!(c.m_nu[i] >= 0.0) || !std::isfinite(c.m_nu[i])) return PM_EINVAL;
  if (c.nsites > 0) {
    double mmax = 0.0;
    for (int i = 0; i < c.n_nu; ++i) mmax = std::max(mmax, c.m_nu[i]);
    if (!(mmax > 0.0)) return PM_EINVAL;  // neutrino particles need a massive eigenstate
  }
  if (c.n_max < 0) return PM_EINVAL;
  if (c.a_ini_ode < 0.0 || c.a_ini_ode >= 1.0) return PM_EINVAL;
  return PM_OK;
}

int Cosmo::init(const pm_config& c) {
  int st = validate_config(c);
  if (st != PM_OK) return st;
  const double tcmb = c.t_cmb > 0 ? c.t_cmb : 2.7255;
  const double neff = c.n_eff > 0 ? c.n_eff : 3.046;
  h = c.h;
  omega_m0 = c.omega_m;
  // Stefan-Boltzmann photon density over the critical density
  const double rho_g = 4.0 * kSigmaSB * std::pow(tcmb, 4) / (kC * kC * kC);
  const double h100 = 1.0e5 / kMpc;
  const double rho_c = 3.0 * h100 * h100 / (8.0 * kPi * kG);
  omega_gamma = rho_g / rho_c / (h * h);
  gamma_nu = std::cbrt(4.0 / 11.0) * std::pow(neff / 3.0, 0.25);
  kT_nu0 = kBoltzEV * gamma_nu * tcmb;
  double mtot = 0.0;
  masses.clear();
  mult.clear();
  for (int i = 0; i < c.n_nu; ++i) {
    mtot += c.m_nu[i];
    bool found = false;
    for (size_t j = 0; j < masses.size(); ++j)
      if (masses[j] == c.m_nu[i]) {
        ++mult[j];
        found = true;
      }
    if (!found) {
      masses.push_back(c.m_nu[i]);
      mult.push_back(1);
    }
  }
  omega_nu = mtot / (93.14 * h * h);
  omega_c = omega_m0 - omega_nu;
  if (!(omega_c >= 0.0)) return PM_EINVAL;
  omega_lambda = 0.0;
  omega_lambda = 1.0 - omega_gamma - omega_c - omega_nu_E2(1.0);

  // growth ODE (§2.3 Eq. growthDE) from a_ini with D = D' = a_ini, RK4 in ln a up to a = 2
  const double a_ini = c.a_ini_ode > 0 ? c.a_ini_ode : 1.0 / 160.0;
  lna0 = std::log(a_ini);
  const double lna_end = std::log(2.0);
  const int nsteps = 4096;
  dlna = (lna_end - lna0) / nsteps;
  tabD.assign(nsteps + 1, 0.0);
  tabDp.assign(nsteps + 1, 0.0);
  double y[2] = {a_ini, a_ini};
  tabD[0] = y[0];
  tabDp[0] = y[1];
  for (int i = 0; i < nsteps; ++i) {
    rk4(lna0 + i * dlna, dlna, y);
    tabD[i + 1] = y[0];
    tabDp[i + 1] = y[1];
  }
  D1 = 1.0;
  double d1, dp1;
  growth(1.0, &d1, &dp1);
  D1 = d1;
  // node tables for the fast path: second derivative from the ODE, E^2 and its slope
  tabDpp.assign(nsteps + 1, 0.0);
  tabE2.assign(nsteps + 1, 0.0);
  tabE2p.assign(nsteps + 1, 0.0);
  for (int i = 0; i <= nsteps; ++i) {
    const double lna = lna0 + i * dlna, a = std::exp(lna);
    double y2[2] = {tabD[i], tabDp[i]}, dy[2];
    rhs(lna, y2, dy);
    tabDpp[i] = dy[1];
    tabE2[i] = E2(a);
    tabE2p[i] = 2.0 * tabE2[i] * dlnE_dlna(a);
  }
  fast = true;
  return PM_OK;
}

namespace {
// cubic Hermite interpolation on [x0, x0 + h] from values and slopes at both ends
inline double hermite(double t, double h, double f0, double d0, double f1, double d1) {
  const double t2 = t * t, t3 = t2 * t;
  return (2 * t3 - 3 * t2 + 1) * f0 + (t3 - 2 * t2 + t) * h * d0 + (-2 * t3 + 3 * t2) * f1 +
         (t3 - t2) * h * d1;
}
}  // namespace

double Cosmo::omega_nu_E2(double a) const {
  double s = 0.0;
  for (size_t j = 0; j < masses.size(); ++j) s += mult[j] * fd_integral(masses[j] * a / kT_nu0);
  return 15.0 / std::pow(kPi, 4) * std::pow(gamma_nu, 4) * omega_gamma / std::pow(a, 4) * s;
}

double Cosmo::d_omega_nu_E2_dlna(double a) const {
  double s = 0.0;
  for (size_t j = 0; j < masses.size(); ++j) {
    double yv = masses[j] * a / kT_nu0;
    s += mult[j] * (-4.0 * fd_integral(yv) + yv * fd_integral_dy(yv));
  }
  return 15.0 / std::pow(kPi, 4) * std::pow(gamma_nu, 4) * omega_gamma / std::pow(a, 4) * s;
}

double Cosmo::E2(double a) const {
  return omega_gamma / std::pow(a, 4) + omega_c / (a * a * a) + omega_nu_E2(a) + omega_lambda;
}

double Cosmo::E(double a) const {
  if (fast) {
    const double x = std::log(a);
    const double fi = (x - lna0) / dlna;
    int i = (int)std::floor(fi);
    if (i >= 0 && i < (int)tabE2.size() - 1)
      return std::sqrt(hermite(fi - i, dlna, tabE2[i], tabE2p[i], tabE2[i + 1], tabE2p[i + 1]));
  }
  return std::sqrt(E2(a));
}

double Cosmo::dlnE_dlna(double a) const {
  double dE2 = -4.0 * omega_gamma / std::pow(a, 4) - 3.0 * omega_c / (a * a * a) +
               d_omega_nu_E2_dlna(a);
  return 0.5 * dE2 / E2(a);
}

void Cosmo::rhs(double lna, const double y[2], double dy[2]) const {
  double a = std::exp(lna);
  double e2 = E2(a);
  dy[0] = y[1];
  dy[1] = -(2.0 + dlnE_dlna(a)) * y[1] + 1.5 * omega_m0 / (a * a * a) / e2 * y[0];
}

void Cosmo::rk4(double lna, double hh, double y[2]) const {
  double k1[2], k2[2], k3[2], k4[2], t[2];
  rhs(lna, y, k1);
  for (int i = 0; i < 2; ++i) t[i] = y[i] + 0.5 * hh * k1[i];
  rhs(lna + 0.5 * hh, t, k2);
  for (int i = 0; i < 2; ++i) t[i] = y[i] + 0.5 * hh * k2[i];
  rhs(lna + 0.5 * hh, t, k3);
  for (int i = 0; i < 2; ++i) t[i] = y[i] + hh * k3[i];
  rhs(lna + hh, t, k4);
  for (int i = 0; i < 2; ++i) y[i] += hh / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

void Cosmo::growth(double a, double* Dv, double* Dp) const {
  double x = std::log(a);
  if (fast) {  // Hermite on the RK4 grid: D from (D, D'), D' from (D', D'')
    double fi = (x - lna0) / dlna;
    int i = (int)std::floor(fi);
    if (i < 0) i = 0;
    if (i >= (int)tabD.size() - 1) i = (int)tabD.size() - 2;
    const double t = fi - i;
    *Dv = hermite(t, dlna, tabD[i], tabDp[i], tabD[i + 1], tabDp[i + 1]) / D1;
    *Dp = hermite(t, dlna, tabDp[i], tabDpp[i], tabDp[i + 1], tabDpp[i + 1]) / D1;
    return;
  }
  double fi = (x - lna0) / dlna;
  int i = (int)std::floor(fi);
  if (i < 0) i = 0;
  if (i >= (int)tabD.size() - 1) i = (int)tabD.size() - 2;
  double y[2] = {tabD[i], tabDp[i]};
  double step = x - (lna0 + i * dlna);
  if (step != 0.0) rk4(lna0 + i * dlna, step, y);
  *Dv = y[0] / D1;
  *Dp = y[1] / D1;
}

double Cosmo::D(double a) const {
  double d, dp;
  growth(a, &d, &dp);
  return d;
}

double Cosmo::gp(double a) const {
  double d, dp;
  growth(a, &d, &dp);
  return a * a * E(a) * dp;
}

double Cosmo::gf(double a) const { return 1.5 * omega_m0 * D(a); }

void Cosmo::coeffs(double a0, double ah, double a1, double out[3]) const {
  out[0] = (gp(ah) - gp(a0)) / gf(a0);
  out[1] = (D(a1) - D(a0)) / gp(ah);
  out[2] = (gp(a1) - gp(ah)) / gf(a1);
}

// ---------------------------------------------------------------- neutrino speeds
int nu_speed_cdf_table(const double* masses, int nmass, double q_max, int nnodes, double* F) {
  if (nmass < 1 || nnodes < 2 || !(q_max > 0.0)) return PM_EINVAL;
  double mmax = 0.0;
  for (int i = 0; i < nmass; ++i) mmax = std::max(mmax, masses[i]);
  if (!(mmax > 0.0)) return PM_EINVAL;
  auto dens = [&](double q) {
    double s = 0.0;
    for (int i = 0; i < nmass; ++i) {
      const double al = masses[i] / mmax;
      s += al * al * al * al / (std::exp(al * q) + 1.0);
    }
    return q * q * s;
  };
  // composite Simpson with 16 panels per table interval (the density is smooth)
  const double h = q_max / (nnodes - 1);
  F[0] = 0.0;
  for (int i = 1; i < nnodes; ++i) {
    const double a = (i - 1) * h, b = i * h;
    const int m = 16;
    const double dh = (b - a) / m;
    double acc = dens(a) + dens(b);
    for (int j = 1; j < m; ++j) acc += (j % 2 ? 4.0 : 2.0) * dens(a + j * dh);
    F[i] = F[i - 1] + acc * dh / 3.0;
  }
  const double tot = F[nnodes - 1];
  for (int i = 0; i < nnodes; ++i) F[i] /= tot;
  return PM_OK;
}

// ---------------------------------------------------------------- neutrino shells
int nu_shell_table(int n_shell, const double* masses, int nmass, double q_max, double* edges,
                   double* q_shell, double* m_shell) {
  if (n_shell < 1 || nmass < 1) return PM_EINVAL;
  double mmax = 0.0;
  for (int i = 0; i < nmass; ++i) mmax = std::max(mmax, masses[i]);
  if (!(mmax > 0.0)) return PM_EINVAL;
  std::vector<double> alpha(nmass);
  for (int i = 0; i < nmass; ++i) alpha[i] = masses[i] / mmax;
  auto ft = [&](double q) {  // effective distribution, Eq. FD_deg
    double s = 0.0;
    for (double al : alpha) s += al * al * al * al * fermi(al * q);
    return s;
  };
  // integrals over [lo, hi] with enough Gauss-Legendre panels for 1e-15
  auto integ = [&](auto f, double lo, double hi) {
    int panels = std::max(4, (int)std::ceil((hi - lo) / 0.25));
    return integrate(f, lo, hi, panels);
  };
  auto g = [&](double q) { return q * ft(q); };  // kernel g(q) = q f(q)
  const double gtot = integ(g, 0.0, q_max);
  edges[0] = 0.0;
  double lo = 0.0, cum = 0.0;  // cumulative area up to lo
  for (int i = 1; i < n_shell; ++i) {
    double target = gtot * i / n_shell;
    double a = lo, b = q_max;
    for (int it = 0; it < 200; ++it) {  // bisection on the cumulative area
      double mid = 0.5 * (a + b);
      double v = cum + integ(g, lo, mid);
      if (v < target) a = mid; else b = mid;
      if (b - a < 1e-15 * std::max(1.0, b)) break;
    }
    double e = 0.5 * (a + b);
    cum += integ(g, lo, e);
    lo = e;
    edges[i] = e;
  }
  edges[n_shell] = q_max;
  auto q2 = [&](double q) { return q * q * ft(q); };
  auto q4 = [&](double q) { return q * q * q * q * ft(q); };
  double z2 = integ(q2, 0.0, q_max);
  for (int i = 0; i < n_shell; ++i) {
    double m2 = integ(q2, edges[i], edges[i + 1]);
    double m4 = integ(q4, edges[i], edges[i + 1]);
    q_shell[i] = std::sqrt(m4 / m2);
    m_shell[i] = m2 / z2;
  }
  return PM_OK;
}

// ------------------------------------------------------------ synthetic spectrum
double bbks(double k, double omega_m, double h) {
  double q = k / (omega_m * h);
  if (q <= 0.0) return 1.0;
  double poly = 1.0 + 3.89 * q + std::pow(16.1 * q, 2) + std::pow(5.46 * q, 3) + std::pow(6.71 * q, 4);
  return std::log(1.0 + 2.34 * q) / (2.34 * q) * std::pow(poly, -0.25);
}

double power_amplitude(double omega_m, double h, double ns, double sigma8) {
  const double R = 8.0;
  auto f = [&](double lnk) {
    double k = std::exp(lnk), x = k * R;
    double w = 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
    if (x < 1e-3) w = 1.0 - x * x / 10.0;
    double t = bbks(k, omega_m, h);
    return k * k * k * std::pow(k, ns) * t * t * w * w / (2.0 * kPi * kPi);
  };
  double s2 = integrate(f, std::log(1e-6), std::log(1e3), 6000);
  return sigma8 * sigma8 / s2;
}

}  // namespace pmnu
