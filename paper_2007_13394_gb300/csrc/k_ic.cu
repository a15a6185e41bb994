// Zel'dovich initial conditions on the GPU (stand-in for the paper's §2.2 set-up).
//
// omega (unit white noise on the nc^3 lattice) -> r2c FFT -> per displacement
// component j: s_k = i k_j delta_k / k^2 with delta_k = omega_k sqrt(P/V) nc^1.5
// (a host FP64 table indexed by the integer |n|^2), k = 0 and Nyquist planes
// zeroed -> c2r -> particles.  CDM sit at lattice nodes; neutrino sites take the
// same series evaluated at the site (a phase e^{i k . d}, d = half a lattice
// spacing when the site stride is even), optionally suppressed by
// 1 / (1 + (k / k_fs)^2), plus their shell offsets and thermal momenta (§2.1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "pm_internal.cuh"

namespace pmnu {

namespace {

__global__ void k_ic_za(const float2* __restrict__ wk, float2* __restrict__ sk, int nc, int pc,
                        const float* __restrict__ amp, int comp, int phase_shift) {
  const int x = blockIdx.x / nc, y = blockIdx.x % nc;
  const int nx = x < nc / 2 ? x : x - nc, ny = y < nc / 2 ? y : y - nc;
  for (int kz = threadIdx.x; kz <= nc / 2; kz += blockDim.x) {
    const size_t idx = ((size_t)x * nc + y) * pc + kz;
    const long long n2 = (long long)nx * nx + (long long)ny * ny + (long long)kz * kz;
    float2 out = make_float2(0.f, 0.f);
    const bool nyq = (x == nc / 2) || (y == nc / 2) || (kz == nc / 2);
    if (n2 > 0 && !nyq) {
      const int nj = comp == 0 ? nx : (comp == 1 ? ny : kz);
      // i k_j / k^2 in units where k = 2 pi n / L: the 2 pi / L is folded into amp
      const float f = __ldg(amp + n2) * (float)nj / (float)n2;
      const float2 w = wk[idx];
      out = make_float2(-f * w.y, f * w.x);
      if (phase_shift) {
        float sn, cs;
        sincospif((float)(nx + ny + kz) / (float)nc, &sn, &cs);
        out = cmul(out, make_float2(cs, sn));
      }
    }
    sk[idx] = out;
  }
}

__global__ void k_ic_cdm(const float* __restrict__ s, int nc, int rp, int comp, double cell,
                         double D0, double gp0, double to_fix, int64_t n_offset,
                         uint32_t* __restrict__ u, float* __restrict__ p, int64_t n_total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ncell = (int64_t)nc * nc * nc;
  if (i >= ncell) return;
  const int ix = (int)(i / ((int64_t)nc * nc)), iy = (int)((i / nc) % nc), iz = (int)(i % nc);
  const float sv = s[((size_t)ix * nc + iy) * rp + iz];
  const int q = comp == 0 ? ix : (comp == 1 ? iy : iz);
  const double x = q * cell + D0 * (double)sv;
  const long long v = __double2ll_rn(x * to_fix);
  u[comp * n_total + n_offset + i] = (uint32_t)(unsigned long long)v;
  p[comp * n_total + n_offset + i] = (float)(gp0 * (double)sv);
}

__global__ void k_ic_nu(const float* __restrict__ s, int nc, int rp, int comp, int nsites,
                        int stride, int j0, double site_dx, double site_off, double D0, double gp0,
                        double to_fix, int nshell, int ndir, const double* __restrict__ tab,
                        int64_t n_offset, int64_t n_nu, uint32_t* __restrict__ u,
                        float* __restrict__ p, int64_t n_total) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_nu) return;
  const int dir = (int)(k % ndir);
  const int shell = (int)((k / ndir) % nshell);
  const int64_t site = k / ((int64_t)ndir * nshell);
  const int sx = (int)(site / ((int64_t)nsites * nsites)), sy = (int)((site / nsites) % nsites),
            sz = (int)(site % nsites);
  // site lattice node (periodic: stride 1 puts the last site on node nc -> 0)
  const int ix = (j0 + stride * sx) % nc, iy = (j0 + stride * sy) % nc, iz = (j0 + stride * sz) % nc;
  const float sv = s[((size_t)ix * nc + iy) * rp + iz];
  const int sd = comp == 0 ? sx : (comp == 1 ? sy : sz);
  const double radius = tab[shell], pth = tab[nshell + shell];
  const double dcomp = tab[2 * nshell + dir * 3 + comp];
  const double x = (sd + 0.5) * site_dx + site_off + D0 * (double)sv + radius * dcomp;
  const long long v = __double2ll_rn(x * to_fix);
  u[comp * n_total + n_offset + k] = (uint32_t)(unsigned long long)v;
  p[comp * n_total + n_offset + k] = (float)(gp0 * (double)sv + pth * dcomp);
}

// Pseudo-random sampling: one particle per site, no shell offset, thermal momentum of
// speed q = F^-1(u_0) (F tabulated at nF equally spaced q; bisection, then linear
// interpolation inside the bracket) along cos(theta) = 2 u_1 - 1, phi = 2 pi u_2.
__global__ void k_ic_nu_pseudo(const float* __restrict__ s, int nc, int rp, int comp, int nsites,
                               int stride, int j0, double site_dx, double site_off, double D0,
                               double gp0, double to_fix, double pscale, const double* __restrict__ F,
                               int nF, double dq, const float* __restrict__ uni, int64_t n_offset,
                               int64_t n_nu, uint32_t* __restrict__ u, float* __restrict__ p,
                               int64_t n_total) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_nu) return;
  const int sx = (int)(k / ((int64_t)nsites * nsites)), sy = (int)((k / nsites) % nsites),
            sz = (int)(k % nsites);
  const int ix = (j0 + stride * sx) % nc, iy = (j0 + stride * sy) % nc, iz = (j0 + stride * sz) % nc;
  const float sv = s[((size_t)ix * nc + iy) * rp + iz];
  const int sd = comp == 0 ? sx : (comp == 1 ? sy : sz);
  const double uq = (double)uni[k], umu = (double)uni[n_nu + k], uphi = (double)uni[2 * n_nu + k];
  int lo = 0, hi = nF - 1;  // F[lo] <= uq <= F[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (F[mid] <= uq) lo = mid; else hi = mid;
  }
  const double span = F[hi] - F[lo];
  const double q = dq * (lo + (span > 0.0 ? (uq - F[lo]) / span : 0.0));
  const double mu = 2.0 * umu - 1.0, phi = 6.283185307179586 * uphi;
  const double st = sqrt(fmax(0.0, 1.0 - mu * mu));
  const double dcomp = comp == 0 ? st * cos(phi) : (comp == 1 ? st * sin(phi) : mu);
  const double x = (sd + 0.5) * site_dx + site_off + D0 * (double)sv;
  const long long v = __double2ll_rn(x * to_fix);
  u[comp * n_total + n_offset + k] = (uint32_t)(unsigned long long)v;
  p[comp * n_total + n_offset + k] = (float)(gp0 * (double)sv + pscale * q * dcomp);
}

__global__ void k_iota(uint32_t* __restrict__ id, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) id[i] = (uint32_t)i;
}

}  // namespace

int ic_build(pm_ctx* c, const float* noise, double a0, double k_fs, pm_state* st, cudaStream_t s,
             const float* uniforms) {
  const pm_config& cf = c->cfg;
  if (uniforms && (cf.nsites <= 0 || cf.nshell != 1 || cf.nfib != 0)) return PM_EINVAL;
  const int nc = cf.nc;
  if (nc < 32 || (nc & (nc - 1)) || nc > c->g.n) return PM_EINVAL;
  if (cf.nsites > 0 && (nc % cf.nsites != 0)) return PM_EINVAL;
  if (!(a0 > 0.0) || a0 > 2.0) return PM_EINVAL;
  const int64_t n_cdm = (int64_t)nc * nc * nc;
  const int ndir = 2 * cf.nfib + 1;
  const int64_t n_nu = cf.nsites > 0 ? (int64_t)cf.nsites * cf.nsites * cf.nsites * cf.nshell * ndir : 0;
  const int64_t n = n_cdm + n_nu;
  if (st->n != n) return PM_EINVAL;  // the caller's arrays hold exactly every particle
  Geom gi;
  gi.n = nc;
  gi.logn = 0;
  while ((1 << gi.logn) < nc) ++gi.logn;
  gi.pc = nc / 2 + 2;
  const double L = cf.box;
  const double PI = 3.14159265358979323846;
  // amplitude tables by |n|^2 (FP64 on the host)
  const long long len = 3LL * (nc / 2) * (nc / 2) + 1;
  if (len > c->ic_amp_len || k_fs != c->ic_kfs) {
    ctx_free(c, c->ic_amp);
    ctx_free(c, c->ic_amp_nu);
    c->ic_amp = c->ic_amp_nu = nullptr;
    c->ic_amp_len = 0;
    if (ctx_alloc_n(c, &c->ic_amp, (size_t)len) != PM_OK || ctx_alloc_n(c, &c->ic_amp_nu, (size_t)len) != PM_OK)
      return PM_ENOMEM;
    c->ic_amp_len = len;
    c->ic_kfs = k_fs;
    const double A = power_amplitude(cf.omega_m, cf.h, cf.ns, cf.sigma8);
    const double kF = 2.0 * PI / L;
    std::vector<float> hc(len), hn(len);
    for (long long n2 = 0; n2 < len; ++n2) {
      double k = std::sqrt((double)n2) * kF;
      double pk = n2 > 0 ? A * std::pow(k, cf.ns) * std::pow(bbks(k, cf.omega_m, cf.h), 2) : 0.0;
      // sqrt(P/V) nc^1.5 for delta_k, / kF for k_j / k^2 in integer units, / nc^3 for the
      // normalised inverse transform s(x) = IFFT(s_k) / nc^3
      double amp = std::sqrt(pk / (L * L * L)) / std::pow((double)nc, 1.5) / kF;
      hc[n2] = (float)amp;
      double filt = k_fs > 0 ? 1.0 / (1.0 + (k / k_fs) * (k / k_fs)) : 1.0;
      hn[n2] = (float)(amp * filt);
    }
    PM_CUDA_TRY(cudaMemcpy(c->ic_amp, hc.data(), sizeof(float) * len, cudaMemcpyHostToDevice));
    PM_CUDA_TRY(cudaMemcpy(c->ic_amp_nu, hn.data(), sizeof(float) * len, cudaMemcpyHostToDevice));
  }
  // neutrino table: radius[shell], p_th[shell], directions[ndir][3] (quasi-random), or the
  // speed CDF at kNF equally spaced q in [0, 40] (pseudo-random)
  constexpr int kNF = 8193;
  constexpr double kQmax = 40.0;
  double* tab = nullptr;
  std::vector<double> htab;
  double pscale_ps = 0.0;
  if (n_nu > 0 && uniforms) {
    double mmax = 0.0;
    for (int i = 0; i < cf.n_nu; ++i) mmax = std::max(mmax, cf.m_nu[i]);
    pscale_ps = c->cosmo.kT_nu0 / mmax * 2997.92458;
    htab.resize(kNF);
    if (nu_speed_cdf_table(cf.m_nu, cf.n_nu, kQmax, kNF, htab.data()) != PM_OK) return PM_EINVAL;
    PM_CUDA_TRY(cudaMallocAsync(&tab, sizeof(double) * htab.size(), s));
    PM_CUDA_TRY(cudaMemcpyAsync(tab, htab.data(), sizeof(double) * htab.size(), cudaMemcpyHostToDevice, s));
  } else if (n_nu > 0) {
    const double qmax = *std::max_element(c->q_shell.begin(), c->q_shell.end());
    double mmax = 0.0;
    for (int i = 0; i < cf.n_nu; ++i) mmax = std::max(mmax, cf.m_nu[i]);
    const double pscale = c->cosmo.kT_nu0 / mmax * 2997.92458;
    htab.resize(2 * cf.nshell + 3 * ndir);
    for (int i = 0; i < cf.nshell; ++i) {
      htab[i] = 0.45 * (L / cf.nsites) * c->q_shell[i] / qmax;
      htab[cf.nshell + i] = pscale * c->q_shell[i];
    }
    const double golden = (1.0 + std::sqrt(5.0)) / 2.0;
    for (int d = 0; d < ndir; ++d) {
      int i = d - cf.nfib;
      double lat = std::asin(2.0 * i / ndir), lon = 2.0 * PI * i / golden;
      htab[2 * cf.nshell + 3 * d + 0] = std::cos(lat) * std::cos(lon);
      htab[2 * cf.nshell + 3 * d + 1] = std::cos(lat) * std::sin(lon);
      htab[2 * cf.nshell + 3 * d + 2] = std::sin(lat);
    }
    PM_CUDA_TRY(cudaMallocAsync(&tab, sizeof(double) * htab.size(), s));
    PM_CUDA_TRY(cudaMemcpyAsync(tab, htab.data(), sizeof(double) * htab.size(),
                                cudaMemcpyHostToDevice, s));
  }
  const double D0 = c->cosmo.D(a0), gp0 = c->cosmo.gp(a0);
  const double to_fix = 4294967296.0 / L;
  float2* A = c->meshA;
  float2* B = c->meshB;
  repack_real(c, gi, noise, nc, reinterpret_cast<float*>(A), 2 * gi.pc, s);
  fft_forward(c, gi, A, A, 0, s);
  const int stride = cf.nsites > 0 ? nc / cf.nsites : 1;
  const bool even = (stride % 2) == 0;
  const int j0 = even ? stride / 2 : (stride + 1) / 2;
  for (int species = 0; species < 2; ++species) {
    if (species == 1 && n_nu == 0) break;
    for (int comp = 0; comp < 3; ++comp) {
      {
        LaunchScope Lz(c, s, K_IC_ZA);
        k_ic_za<<<(unsigned)(nc * nc), 128, 0, s>>>(A, B, nc, gi.pc,
                                                    species == 0 ? c->ic_amp : c->ic_amp_nu, comp,
                                                    species == 1 && even ? 1 : 0);
      }
      fft_inverse_plain(c, gi, B, s);
      const float* sr = reinterpret_cast<const float*>(B);
      LaunchScope La(c, s, K_IC_ASSEMBLE);
      if (species == 0) {
        k_ic_cdm<<<(unsigned)((n_cdm + 255) / 256), 256, 0, s>>>(
            sr, nc, 2 * gi.pc, comp, L / nc, D0, gp0, to_fix, 0, st->u, st->p, st->n);
      } else if (uniforms) {
        k_ic_nu_pseudo<<<(unsigned)((n_nu + 255) / 256), 256, 0, s>>>(
            sr, nc, 2 * gi.pc, comp, cf.nsites, stride, j0, L / cf.nsites, 0.5 * L / nc, D0, gp0,
            to_fix, pscale_ps, tab, kNF, kQmax / (kNF - 1), uniforms, n_cdm, n_nu, st->u, st->p, st->n);
      } else {
        k_ic_nu<<<(unsigned)((n_nu + 255) / 256), 256, 0, s>>>(
            sr, nc, 2 * gi.pc, comp, cf.nsites, stride, j0, L / cf.nsites, 0.5 * L / nc, D0, gp0,
            to_fix, cf.nshell, ndir, tab, n_cdm, n_nu, st->u, st->p, st->n);
      }
    }
  }
  {
    LaunchScope Li(c, s, K_IC_ASSEMBLE);
    k_iota<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(st->id, n);
  }
  if (tab) cudaFreeAsync(tab, s);
  if (cudaGetLastError() != cudaSuccess) return PM_ECUDA;
  st->a = a0;
  st->f_valid = 0;
  return PM_OK;
}

}  // namespace pmnu
