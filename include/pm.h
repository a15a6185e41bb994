/*
 * pm.h -- C-ABI of libpmnu: a GB300 (sm_103a) particle-mesh step for CDM and
 * quasi-randomly sampled massive-neutrino particles.
 *
 * Method: Bayer, Banerjee & Feng, "A fast particle-mesh simulation of
 * non-linear cosmological structure formation with massive neutrinos"
 * (arXiv 2007.13394).  The paper runs FastPM's particle-mesh solver with a
 * kick-drift-kick integrator (§2.1 "Kick-Drift-Kick"; §2.3) whose growth-based
 * kick and drift factors follow the Zel'dovich trajectory x = q + D(a) s;
 * D(a) solves the growth ODE (§2.3 Eq. growthDE) on the background of
 * Eq. Hubble; neutrinos are a second particle species that counts as matter
 * in the Poisson source (§2.2 Eq. Om_pois); the force mesh is twice the CDM
 * grid (§3, Table 1).  Neutrino particles come from N_shell Fermi-Dirac shells
 * (§2.1 Eqs. q_shell, m_shell, N_shell, FD_deg) times 2 N_fib + 1 Fibonacci
 * directions per site (Eq. N_n).
 *
 * Definitions the paper leaves to FastPM and that this library fixes:
 *   positions   uint32 fixed point per axis, x = u L / 2^32, periodic by
 *               integer wraparound;
 *   paint       cloud-in-cell (CIC) of rho / rho_bar (mean 1) on an N^3 mesh,
 *               deterministic (tile-local integer accumulation, no float atomics);
 *   potential   phi_k = -(3/2) Omega_m0 delta_k / N^3 / k^2, phi_0 = 0;
 *   force       F_j = IFFT[-i D(k_j) phi_k] with the 4-point finite-difference
 *               gradient D(k) = (8 sin kH - sin 2kH) / (6H) (0 on the Nyquist
 *               index), read out with the paint's CIC weights.  Computed by
 *               default as minus the 4-point stencil [8 (phi(x+H) - phi(x-H)) -
 *               (phi(x+2H) - phi(x-2H))] / (12 H) of the real potential at the CIC
 *               corners (its transfer function is i D(k)), so one inverse
 *               transform serves all three components.  No window
 *               deconvolution: with the mesh finer than the CDM lattice (the
 *               paper's mesh is twice the CDM grid) a deconvolved spectral
 *               kernel amplifies the lattice's alias modes and breaks linear
 *               growth.  Flags bit 1 selects that kernel anyway
 *               (phi_k / W(k)^2, W = prod_d sinc^2(pi n_d / N), gradient k_j);
 *   kick/drift  p += K F, u += rne(Delta p 2^32 / L) (int32 wraparound), with
 *               K1 = (g_p(a_h) - g_p(a_0)) / g_f(a_0),
 *               Delta = (D(a_1) - D(a_0)) / g_p(a_h),
 *               K2 = (g_p(a_1) - g_p(a_h)) / g_f(a_1),
 *               g_p = a^3 E dD/da, g_f = 1.5 Omega_m0 D  (FP64 on the host).
 *
 * Units: box L in Mpc/h, H0 = 1; momentum p = a^2 (dx/dt) / H0 in Mpc/h; the
 * mesh holds rho / rho_bar.  Particle masses follow from the particle id:
 * id < n_cdm is CDM with mass (Omega_c0/Omega_m0) N^3 / n_c^3; a neutrino id
 * n_cdm + (site * n_shell + shell) * (2 n_fib + 1) + dir has mass
 * (Omega_nu0/Omega_m0) m_shell / (2 n_fib + 1) N^3 / n_sites^3 (units of the
 * mean mass per mesh cell).
 *
 * Memory and ownership: every particle and output array passed in is owned
 * by the caller; a context owns its scratch (three padded complex meshes of
 * N * N * (N/2 + 2) float2 each -- two with flags bit 0 or nmesh 2048; the default
 * force path uses one -- plus sort buffers for n_max particles).
 * Arrays are structure-of-arrays: u[3 * n] holds the x plane, then y, then z.
 * "Device" pointers are CUDA device memory of the context's device; "host"
 * pointers are ordinary (preferably pinned) host memory.
 *
 * Streams and errors: calls taking a cudaStream_t (passed as void*, NULL =
 * legacy default stream) enqueue work on it and return without waiting,
 * except those documented as synchronous.  Every call returns an int status
 * (PM_OK or a negative PM_E* code) and never aborts.  A kernel that detects a
 * bad input (an out-of-range particle id, a bucket overflow) sets a device
 * error word; synchronous calls and pm_sync() report it as PM_EKERNEL, and it
 * stays set (sticky) until pm_sync() returns it.  A NaN or infinite momentum
 * or force met by the kick kernels is reported the same way as PM_ENONFINITE,
 * and a bounded wait that gave up (a tensor copy that never arrived) as
 * PM_ETIMEOUT; the context stays usable after each.  A context is not
 * thread-safe; use one per host thread.
 */
#ifndef PMNU_PM_H
#define PMNU_PM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PM_OK = 0,
  PM_EINVAL = -1,    /* bad argument (size, pointer, range, non power-of-two mesh) */
  PM_ENOMEM = -2,    /* device or host allocation failed */
  PM_ECUDA = -3,     /* a CUDA runtime call failed */
  PM_EKERNEL = -4,   /* a kernel flagged bad input through the device error word */
  PM_ETIMEOUT = -5,  /* a bounded device wait gave up */
  PM_ENOTINIT = -6,  /* null or destroyed context */
  PM_ENONFINITE = -7 /* a kernel met a NaN or infinite momentum or force */
};

/* Species selectors for pm_paint and pm_power. */
enum { PM_SPECIES_CDM = 1, PM_SPECIES_NU = 2, PM_SPECIES_ALL = 3 };

/* pm_config.flags bits. */
enum { PM_FLAG_TWO_MESH = 1, PM_FLAG_SPECTRAL_KERNEL = 2, PM_FLAG_MLP_TENSOR = 4, PM_FLAG_KSPACE_GRADIENT = 8 };

/* Run configuration.  Zero-initialise, then set the fields. */
typedef struct pm_config {
  double box;          /* L, Mpc/h, > 0 */
  int32_t nmesh;       /* N, power of two, 32 <= N <= 2048 (mesh twice the CDM grid in the paper) */
  int32_t nc;          /* CDM lattice points per side (0: no CDM); nc <= N, N % nc == 0 for pm_ic */
  int32_t nsites;      /* neutrino sites per side (0: no neutrinos); nc % nsites == 0 for pm_ic */
  int32_t nshell;      /* Fermi-Dirac shells, >= 1 when nsites > 0 */
  int32_t nfib;        /* Fibonacci parameter: 2 nfib + 1 directions per shell */
  double h;            /* H0 / (100 km/s/Mpc) */
  double omega_m;      /* total matter today, Omega_c0 + Omega_nu0 */
  double t_cmb;        /* K; 0 selects 2.7255 */
  double n_eff;        /* 0 selects 3.046 */
  int32_t n_nu;        /* neutrino mass eigenstates in the background, 0..3 */
  int32_t pad0;
  double m_nu[3];      /* eigenstate masses in eV (M_nu = sum); heaviest sets the shell speeds */
  double a_ini_ode;    /* start of the growth ODE; 0 selects 1/160 (z = 159, §2.3) */
  int64_t n_max;       /* capacity of the sort scratch (>= every n passed later) */
  double ns;           /* spectral index of the synthetic initial spectrum (pm_ic) */
  double sigma8;       /* normalisation of the synthetic initial spectrum (pm_ic) */
  uint32_t flags;      /* Default force path: one potential mesh phi (forward FFT, Green's
                          function, inverse FFT, all in place) and the 4-point gradient
                          applied in real space inside the readout, which equals the k-space
                          kernel D(k) exactly.  bit 3 (PM_FLAG_KSPACE_GRADIENT): multiply by
                          -i D(k_j) in k-space instead and run three inverse transforms (bit 0,
                          PM_FLAG_TWO_MESH: one component at a time in two meshes, always so
                          for nmesh = 2048); bit 1 (PM_FLAG_SPECTRAL_KERNEL): deconvolved
                          spectral kernel (k-space gradient k_j, W^-2), implies the k-space
                          path; bit 2 (PM_FLAG_MLP_TENSOR): the learned factor's table on the
                          tensor cores (BF16 operands, FP32 accumulation) instead of FP32;
                          other bits 0 */
  int32_t pad1;
  int64_t mem_limit;   /* bytes of device memory the context may hold (its scratch, and the
                          buffers later calls allocate on first use); 0: no limit.  An
                          allocation that would pass it fails with PM_ENOMEM without calling
                          cudaMalloc (pm_init then frees what it had allocated). */
} pm_config;

/* Particle state.  All arrays are caller-owned device memory of length 3n (u, p, f)
 * or n (id).  pm_step reorders every array in place into the library's tile order;
 * id keeps each particle's canonical index.  f caches the force at a. */
typedef struct pm_state {
  uint32_t* u;
  float* p;
  uint32_t* id;
  float* f;
  int64_t n;
  double a;
  int32_t f_valid;
  int32_t pad0;
} pm_state;

typedef struct pm_ctx pm_ctx;

/* Human-readable text of a status code (static storage). */
const char* pm_strerror(int status);

/* ---- host-only FP64 helpers (no GPU needed) ------------------------------- */

/* D(a) (normalised D(1) = 1), g_p(a), g_f(a), E(a) for the configured cosmology:
 * growth ODE §2.3 Eq. growthDE with Omega_m(a) = Omega_m0 a^-3 / E^2, initial
 * conditions D = dD/dln a = a_ini.  out[4] host.  Solves the ODE on every call. */
int pm_cosmo_growth(const pm_config* cfg, double a, double* out);

/* FastPM KDK factors for one step a0 -> a1 with half point ah: out[3] = {K1, Delta, K2}. */
int pm_cosmo_coeffs(const pm_config* cfg, double a0, double ah, double a1, double* out);

/* Fermi-Dirac shell table (§2.1 Eqs. N_shell, q_shell, m_shell with the effective
 * distribution Eq. FD_deg over the configured masses): edges[nshell + 1],
 * q_shell[nshell], m_shell[nshell], host arrays; q_max = 40. */
int pm_nu_shells(const pm_config* cfg, double* edges, double* q_shell, double* m_shell);

/* Background densities: out[5] = {Omega_gamma0, Omega_c0, Omega_nu0 (Poisson),
 * Omega_Lambda, k_B T_nu0 in eV}. */
int pm_cosmo_params(const pm_config* cfg, double* out);

/* ---- context ----------------------------------------------------------------- */

/* Validates cfg, builds the FP64 tables the step needs -- the growth factor D(a) of
 * the ODE of §2.3 Eq. growthDE on the background of Eq. Hubble (with Omega_m(a) of
 * §2.2 Eq. Om_pois read as Omega_m0 a^-3 / E^2), the FastPM kick and drift factors it
 * feeds (§2.3), and the Fermi-Dirac shell table of §2.1 (Eqs. N_shell, q_shell, m_shell,
 * FD_deg) that sets the neutrino particle masses -- and allocates the scratch on the
 * current CUDA device.  cfg: host, read only, not kept.  *out receives the context,
 * owned by the caller until pm_destroy.  PM_EINVAL for a bad configuration (see
 * pm_config), PM_ENOMEM when an allocation fails (nothing is left allocated). */
int pm_init(const pm_config* cfg, pm_ctx** out);
int pm_destroy(pm_ctx* ctx);

/* Waits for the given stream, then returns PM_EKERNEL / PM_ETIMEOUT if a kernel set
 * the device error word since the last pm_sync (and clears it), else PM_OK. */
int pm_sync(pm_ctx* ctx, void* stream);

/* Step coefficients from the context's tables: out[5] = {K1, Delta, K2, D(a0), D(a1)}. */
int pm_coeffs(pm_ctx* ctx, double a0, double ah, double a1, double* out);

/* ---- the particle-mesh path (device arrays, stream-ordered) ----------------- */

/* Stable counting sort of particles into 16^3-cell tiles of the mesh.  key(i) =
 * tile(i) * 8 + class(i): tile = (t_x (N/16) + t_y)(N/16) + t_z of the particle's
 * cell, class = 4 [l_x = 15] + 2 [l_y = 15] + [l_z = 15] for its in-tile
 * coordinates.  perm_out[k] = incoming index of the k-th particle in key order,
 * ties in incoming order; key_out[k] its key (either output may be NULL). */
int pm_sort(pm_ctx* ctx, const uint32_t* u, int64_t n, uint32_t* perm_out, uint32_t* key_out,
            void* stream);

/* CIC density rho / rho_bar of the selected species (PM_SPECIES_*) on the N^3 mesh:
 * the source of the Poisson equation, where neutrino particles count as matter beside
 * CDM (§2.2 Eq. Om_pois; per-particle masses from the shell fractions of §2.1 Eq.
 * m_shell).  u: device, 3n uint32 fixed-point positions; id: device, n canonical ids,
 * or NULL (particle i has id i); mesh_out: device, N^3 floats, x-major with z fastest,
 * caller-owned.  Deterministic (integer accumulation).  PM_EINVAL for n < 0, n > n_max
 * or a null pointer; an id beyond the configured particles sets the error word. */
int pm_paint(pm_ctx* ctx, const uint32_t* u, const uint32_t* id, int64_t n, int32_t species,
             float* mesh_out, void* stream);

/* PM force at every particle: F = -grad phi with the Poisson equation of §2.2
 * (nabla^2 phi = 1.5 Omega_m0 delta, Eq. Om_pois; both species as matter), on the
 * mesh twice the CDM grid of §3 Table 1, by the kernel defined at the top of this
 * header.  u, id as pm_paint; F_out: device, 3n floats in input order, caller-owned.
 * PM_EINVAL as pm_paint. */
int pm_force(pm_ctx* ctx, const uint32_t* u, const uint32_t* id, int64_t n, float* F_out,
             void* stream);

/* One kick-drift-kick step a0 -> a1 (§2.1 "Kick-Drift-Kick": FastPM's KDK scheme;
 * §2.3: kick and drift factors built from the growth factor so that the Zel'dovich
 * trajectory x = q + D(a) s is followed exactly; CDM and neutrinos alike).  ah <= 0
 * selects the arithmetic mean.  If st->f_valid is 0 the force at a0 is computed first.
 * st: host struct of caller-owned device arrays (see pm_state).  On return the state
 * holds (u, p, f) at a1 in tile order, st->a = a1, st->f_valid = 1.  PM_EINVAL
 * unless 0 < a0 <= ah <= a1 <= 2 with a0 < a1, or for n > n_max or null arrays. */
int pm_step(pm_ctx* ctx, pm_state* st, double a0, double ah, double a1, void* stream);

/* nsteps chained KDK steps: schedule (host) holds (a0, ah, a1) per step, each step's a0
 * equal to the previous a1 (PM_EINVAL otherwise; ah <= 0: arithmetic mean).  The result
 * equals nsteps calls of pm_step bit for bit; on the default force path the readout
 * that ends one step also applies the next step's first half kick and drift (FastPM's
 * KDK with the two half kicks of a step boundary in one pass over the particles), so
 * there is no separate kick/drift pass between steps and f is written by the last step
 * only.  On return: as pm_step after the last step.  Stream ordered, with one host
 * synchronisation per step (the sort's choice of method).  On an error status the
 * state is undefined (steps before the failing one have already applied the next
 * step's kick and drift). */
int pm_run(pm_ctx* ctx, pm_state* st, const double* schedule, int64_t nsteps, void* stream);

/* pm_step on HOST arrays (u[3n], p[3n], id[n], f[3n]): copies in, steps, copies out;
 * synchronous.  *f_valid is read and updated.  Device state storage is allocated on
 * first use and kept by the context. */
int pm_step_host(pm_ctx* ctx, uint32_t* u, float* p, uint32_t* id, float* f, int64_t n,
                 int32_t* f_valid, double a0, double ah, double a1, void* stream);

/* Binned (cross) power spectrum of the species a and b (PM_SPECIES_*): the P_cdm,
 * P_m, P_cdm,nu and P_nu the results of §3 compare (Figs. MR, Pn_shotnoise); the paper
 * measures them with nbodykit and prints no estimator, so this is the reading:
 * P_ab(k) = (V / N^6) Re(delta_a delta_b^*) / W(k)^2 with each species' mesh over its
 * own mean and W the CIC window, no shot-noise subtraction, linear bins of width
 * k_F = 2 pi / L from k_F / 2, mode-weighted mean |k|, r2c modes with
 * 0 < n_z < N/2 counted twice.  u, id as pm_paint; k_out, P_out, nmodes_out: host
 * arrays of length nbins (<= 2048).  Synchronous; PM_EINVAL for a bad species or
 * nbins. */
int pm_power(pm_ctx* ctx, const uint32_t* u, const uint32_t* id, int64_t n, int32_t species_a,
             int32_t species_b, int32_t nbins, double* k_out, double* P_out, int64_t* nmodes_out,
             void* stream);

/* Zel'dovich initial conditions (stand-in for the paper's §2.2 REPS set-up): a BBKS
 * spectrum normalised to cfg->sigma8 with index cfg->ns, from unit white noise
 * noise[nc^3] (device, x-major).  CDM at lattice nodes i L / nc; neutrino sites at
 * (i + 1/2) L / nsites + L / (2 nc), displaced by the same field (optionally
 * suppressed by 1 / (1 + (k / k_fs)^2); k_fs <= 0 disables) evaluated exactly at the
 * site, plus shell offsets 0.45 (L / nsites) q_shell / q_max,shell and thermal
 * momenta q_shell k_B T_nu0 / m_heaviest (c / H0) along the Fibonacci directions.
 * Writes st->u, st->p, st->id (canonical order), st->n, st->a = a0, st->f_valid = 0. */
int pm_ic(pm_ctx* ctx, const float* noise, double a0, double k_fs, pm_state* st, void* stream);

/* pm_ic with pseudo-random neutrinos (the comparison scheme of §3 Fig. Pn_shotnoise):
 * requires nshell = 1 and nfib = 0, so one particle per site, placed at the site plus the
 * Zel'dovich displacement (no shell offset), with a thermal momentum of speed
 * q = F^-1(u_0) (F: CDF of the speed density q^2 f~(q) of Eq. FD_deg, tabulated in FP64
 * at 8193 speeds in [0, 40] and inverted by linear interpolation) along the direction
 * cos(theta) = 2 u_1 - 1, phi = 2 pi u_2.  uniforms: device, 3 x nsites^3 floats in
 * [0, 1) (u_0 of every site, then u_1, then u_2), drawn by the caller.  PM_EINVAL if the
 * configuration is not one particle per site. */
int pm_ic_pseudo(pm_ctx* ctx, const float* noise, const float* uniforms, double a0, double k_fs,
                 pm_state* st, void* stream);

/* Checkpoint of a particle state (per-step checkpoints for resuming and for the
 * adjoint).  File: a 512-byte ASCII JSON header padded with spaces ({"format":
 * "pmnu-state-1", "n", "a", "f_valid", "nmesh", "box", "config_hash"}), then u[3n]
 * uint32, p[3n] float32, id[n] uint32, f[3n] float32, little-endian.  Synchronous.
 * pm_state_load checks format, n and the configuration hash (PM_EINVAL on a mismatch)
 * and fills the caller's device arrays (st->n must equal the file's n). */
int pm_state_save(pm_ctx* ctx, const pm_state* st, const char* path);
int pm_state_load(pm_ctx* ctx, pm_state* st, const char* path);

/* ---- adjoint (gradients of a final-field loss; no counterpart in the paper) ----- */

/* Transpose of the paint with respect to the particle weights: out[i] = sum_c W(x_i - c)
 * mesh(c) (the CIC readout; mesh N^3 contiguous).  Same as pm_readout. */
int pm_paint_T(pm_ctx* ctx, const uint32_t* u, int64_t n, const float* mesh, float* out, void* stream);
/* Transpose of the readout: the deterministic CIC paint of signed per-particle weights
 * w[n] (input order) onto mesh_out (N^3 contiguous). */
int pm_readout_T(pm_ctx* ctx, const uint32_t* u, int64_t n, const float* w, float* mesh_out,
                 void* stream);
/* VJP of the paint with respect to positions: grad[3n] (input order, Mpc/h^-1 units)
 * = m_i grad_x sum_c W(x_i - c) lam_mesh(c), lam_mesh N^3 contiguous. */
int pm_paint_vjp(pm_ctx* ctx, const uint32_t* u, const uint32_t* id, int64_t n,
                 const float* lam_mesh, float* grad_out, void* stream);
/* VJP of pm_power's auto-spectrum (species_a = species_b = species) with respect to the
 * positions: grad_out[3n] (device, input order) = sum_b dL_dP[b] dP_b / dx, dL_dP a host
 * array of nbins.  dP_b/drho(x) = 2 sum_{k in b} V F_k e^{ikx} / (N^6 rho_bar^2 W_k^2 N_b)
 * (F = FFT of the species mesh, rho_bar its mean, fixed by the species' total mass),
 * then the paint's position VJP.  Synchronous. */
int pm_power_vjp(pm_ctx* ctx, const uint32_t* u, const uint32_t* id, int64_t n, int32_t species,
                 int32_t nbins, const double* dL_dP, float* grad_out, void* stream);
/* VJP of the PM force with respect to positions: grad[3n] = d <lam_f, F(x)> / dx, with
 * F_j = R[G_j rho]: sum_j lam_f,j grad R[G_j rho] + m grad R[B], B = -sum_j G_j paint(lam_f,j)
 * (G_j^T = -G_j: a real convolution with an odd kernel).  Arrays in input order. */
int pm_force_vjp(pm_ctx* ctx, const uint32_t* u, const uint32_t* id, int64_t n, const float* lam_f,
                 float* grad_out, void* stream);
/* VJP of one KDK step a0 -> a1 (ah <= 0: arithmetic mean) at the checkpointed state st
 * (u, p, id, f = F(x0) at a0, any order).  Cotangents lam_x1, lam_p1 of the state at a1
 * and outputs lam_x0, lam_p0 are [3n] arrays indexed by canonical particle id.
 * Positions are treated as continuous (units Mpc/h). */
int pm_step_vjp(pm_ctx* ctx, const pm_state* st, double a0, double ah, double a1,
                const float* lam_x1, const float* lam_p1, float* lam_x0, float* lam_p0,
                void* stream);
/* Transpose of the Zel'dovich initial conditions of pm_ic (same a0 and k_fs; pm_ic must
 * have run on this context with that k_fs): cotangents of the initial positions and
 * momenta (canonical order, [3n]) -> gradient with respect to the white noise
 * (nc^3 contiguous). */
int pm_ic_vjp(pm_ctx* ctx, const float* lam_x0, const float* lam_p0, double a0, double k_fs,
              float* grad_noise, void* stream);

/* ---- learned Green's-function correction (no counterpart in the paper) -------- */

/* A small network m(kappa, a) = 1 + MLP(kappa, a) multiplies the Green's function of
 * the potential: phi_k = -(3/2) Omega_m0 delta_k m(|k| / k_Ny, a) / N^3 / (k^2 W^2),
 * k_Ny = pi N / L, a the scale factor of the force evaluation.  Network:
 * Linear(2, 64) -> SiLU -> Linear(64, 64) -> SiLU -> Linear(64, 1); flat FP32
 * parameters, in order W1[64][2] (row j: weights of kappa and a into unit j), b1[64],
 * W2[64][64] (row = output unit), b2[64], w3[64], b3.  With w3 = b3 = 0 the kernel
 * is the plain one exactly.  m depends on k through s = n_x^2 + n_y^2 + n_z^2 only
 * and is evaluated once per s (table refreshed at every force evaluation). */
enum { PM_MLP_HIDDEN = 64, PM_MLP_NPARAM = 4417 };

/* Copies PM_MLP_NPARAM parameters from host memory and switches the factor on for
 * every later force, potential, step and adjoint call; resets the Adam moments.
 * theta == NULL switches it off.  Synchronous. */
int pm_set_mlp(pm_ctx* ctx, const float* theta, int64_t nparam);
/* Current parameters into host memory (after device work finishes).  Synchronous. */
int pm_get_mlp(pm_ctx* ctx, float* theta, int64_t nparam);
/* Scale factor at which pm_force, pm_potential and pm_force_vjp evaluate the factor
 * (default 1); pm_step and pm_step_vjp use their own a0 and a1. */
int pm_set_force_time(pm_ctx* ctx, double a);
/* The table the Green's-function passes read at scale factor a: out[s] = m(sqrt(s) /
 * (N/2), a) for s = 0 .. 3 (N/2)^2 (device, 3 (N/2)^2 + 1 floats); computed the way the
 * context computes it (FP32, or tensor cores with PM_FLAG_MLP_TENSOR). */
int pm_mlp_table(pm_ctx* ctx, double a, float* out, void* stream);
/* m at n points (device arrays kappa[n], a[n] -> m_out[n]). */
int pm_mlp_eval(pm_ctx* ctx, const float* kappa, const float* a, int64_t n, float* m_out, void* stream);
/* With the factor on, pm_force_vjp and pm_step_vjp also accumulate d L / d theta of
 * the cotangents they are given (FP64 accumulator in the context; needs the
 * three-mesh force path, PM_EINVAL otherwise).  This copies the accumulator to
 * grad_out (device, nparam floats) and clears it when reset != 0. */
int pm_mlp_grad(pm_ctx* ctx, float* grad_out, int64_t nparam, int32_t reset, void* stream);
/* One Adam step (Kingma & Ba 2014) on the context's parameters with gradient grad
 * (device), step count t >= 1 (bias corrections 1 - beta^t). */
int pm_mlp_adam(pm_ctx* ctx, const float* grad, int64_t nparam, double lr, double beta1, double beta2,
                double eps, int64_t t, void* stream);
/* Training loss of the factor: L = sum_i m_i |x_i - y_i|^2 / sum_i m_i over the
 * particles of the selected species (PM_SPECIES_*; the others weigh 0) of a state
 * (u, id) of n particles and a reference run from the same initial conditions
 * (u_ref, id_ref; either id may be NULL for canonical order), x - y the periodic
 * difference int32(u - u_ref) L / 2^32.  lam_x[3n] (device, canonical order)
 * receives dL/dx; *loss (host) receives L.  Ids must lie in [0, n).  Synchronous. */
int pm_displacement_loss(pm_ctx* ctx, const uint32_t* u, const uint32_t* id, const uint32_t* u_ref,
                         const uint32_t* id_ref, int64_t n, int32_t species, float* lam_x, double* loss,
                         void* stream);

/* ---- stage-level entry points (device arrays; for testing each kernel) ------- */

/* Forward r2c FFT (unnormalised, e^{-ikx}) of a real N^3 mesh: out holds
 * N * N * (N/2 + 1) complex values as interleaved floats, kz fastest. */
int pm_fft_r2c(pm_ctx* ctx, const float* mesh, float* out_complex, void* stream);
/* Unnormalised inverse (e^{+ikx}) c2r of a Hermitian half spectrum, same layouts. */
int pm_fft_c2r(pm_ctx* ctx, const float* in_complex, float* mesh_out, void* stream);
/* phi_k of a density mesh: the r2c FFT with the Green's function fused into its
 * last pass.  out_complex as in pm_fft_r2c. */
int pm_potential(pm_ctx* ctx, const float* mesh, float* out_complex, void* stream);
/* F_j mesh (j = 0, 1, 2) from phi_k: -i k_j fused into the first inverse pass. */
int pm_force_mesh(pm_ctx* ctx, const float* phi_complex, int32_t component, float* mesh_out,
                  void* stream);
/* CIC readout of a real N^3 mesh at n particles: out[n]. */
int pm_readout(pm_ctx* ctx, const uint32_t* u, int64_t n, const float* mesh, float* out,
               void* stream);

/* ---- allocation-free variant --------------------------------------------------- */

/* Binned power spectrum of two half-spectrum meshes, without allocating anything.
 * (No counterpart in the paper: a library convenience.)  For callers that cannot
 * call cudaMalloc where they need a spectrum: code running inside a memory pool or
 * arena that owns the device's memory, graph-driven pipelines whose replays must
 * not allocate, hosts that lent their free memory to another framework.  It needs
 * no context (pm_init allocates) and uses, instead of context scratch, one
 * file-scope device array of 3 MiB (256 x 3 x 512 doubles) that every GPU loading
 * the library keeps until exit.
 * delta_a, delta_b: device, N * N * (N/2 + 1) complex values as interleaved floats,
 * kz fastest (the layout pm_fft_r2c writes); they may be the same array.  Each is
 * divided by its own mean (its k = 0 mode over N^3).  Binning as pm_power.
 * k_out, P_out, nmodes_out: device arrays of nbins doubles, written in stream order.
 * Limits: nmesh a power of two in [32, 2048], 1 <= nbins <= 512, box > 0; anything
 * else returns PM_EINVAL without touching the GPU.  The first call on a device
 * resolves the array's device address (cudaGetSymbolAddress with that device
 * current) and keeps it for the life of the process: make that call before any
 * stream capture, and do not call this again on a device after cudaDeviceReset
 * (the reset unloads the module; the kept address would no longer be the array's).
 * All calls share the array, so calls that overlap on the GPU race on it; nothing
 * needs clearing between calls.  The library receives raw pointers and cannot check
 * that delta_a and delta_b hold the N * N * (N/2 + 1) complex values they must. */
int pm_power_bin_noalloc(const float* delta_a, const float* delta_b, int32_t nmesh, double box,
                         int32_t nbins, double* k_out, double* P_out, double* nmodes_out,
                         void* stream);

/* ---- instrumentation --------------------------------------------------------- */

/* Number of kernels this context has launched since pm_init. */
int64_t pm_launch_count(pm_ctx* ctx);
/* Bytes of device memory the context holds now (what pm_config.mem_limit is checked against). */
int64_t pm_memory_used(pm_ctx* ctx);
/* Testing aid for the failure paths (no counterpart in the paper).  what = PM_INJECT_DROP_COPY:
 * in the next TMA-pipelined FFT pass (meshes up to 512^3) the first CTA does not issue its
 * first tile copy, so its bounded wait on that copy runs out (after a short limit), the CTA
 * waits for its other copies in flight and returns, and the next pm_sync reports PM_ETIMEOUT;
 * the pass's output is then invalid, the context stays usable.  One shot: consumed by that
 * launch.  what = 0 cancels a pending injection. */
enum { PM_INJECT_DROP_COPY = 1 };
int pm_test_inject(pm_ctx* ctx, int32_t what);
/* CUDA-event timing of launches on their own stream, per kernel kind: bit k of mask
 * selects kind k (-1 = every kind, 0 = off). */
int pm_profile_enable(pm_ctx* ctx, int32_t mask);
/* Accumulated milliseconds and launches of kernel kind k (0 <= k < pm_kernel_kinds()),
 * synchronous; resets the kind's counters when reset != 0. */
int pm_profile_read(pm_ctx* ctx, int32_t kind, double* ms, int64_t* launches, int32_t reset);
int32_t pm_kernel_kinds(void);
const char* pm_kernel_name(int32_t kind);
/* How pm_step re-sorted the drifted particles (out: 3 int64, host): out[0] steps that
 * used the near-sorted re-sort (the state in the order the context's last step left
 * it: most particles keep their key, only the others are radix-sorted), out[1] steps
 * that sorted from scratch, out[2] the particles the last near-sorted re-sort moved
 * between keys.  Both ways give the same stable permutation of the keys. */
int pm_sort_stats(pm_ctx* ctx, int64_t* out);

#ifdef __cplusplus
}
#endif

#endif /* PMNU_PM_H */
