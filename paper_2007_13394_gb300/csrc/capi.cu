// C-ABI entry points of libpmnu (declared in include/pm.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pm_internal.cuh"

using namespace pmnu;

namespace pmnu {

LaunchScope::LaunchScope(pm_ctx* ctx, cudaStream_t st, int k) : c(ctx), s(st), kind(k) {
  ++c->launches;
  if (c->prof & (1u << k)) {
    if (c->prof_pool.size() < 2) {
      cudaEvent_t a, b;
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      c->prof_pool.push_back(a);
      c->prof_pool.push_back(b);
    }
    e1 = c->prof_pool.back();
    c->prof_pool.pop_back();
    e0 = c->prof_pool.back();
    c->prof_pool.pop_back();
    cudaEventRecord(e0, s);
  }
}

LaunchScope::~LaunchScope() {
  if (e0) {
    cudaEventRecord(e1, s);
    c->prof_live.push_back(Prof{kind, e0, e1});
  }
}

float2* twiddles(pm_ctx* c, int n) {
  auto it = c->tw.find(n);
  if (it != c->tw.end()) return it->second;
  std::vector<float2> h(n);
  for (int t = 0; t < n; ++t) {
    double a = -2.0 * 3.14159265358979323846 * t / n;
    h[t] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  float2* d = nullptr;
  if (ctx_alloc_n(c, &d, (size_t)n) != PM_OK) return nullptr;
  cudaMemcpy(d, h.data(), sizeof(float2) * n, cudaMemcpyHostToDevice);
  c->tw[n] = d;
  return d;
}

int ctx_alloc(pm_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  const int64_t lim = c->cfg.mem_limit;
  if (lim > 0 && c->mem_used + bytes > (size_t)lim) return PM_ENOMEM;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();  // the failed allocation's error is reported as PM_ENOMEM
    return PM_ENOMEM;
  }
  c->allocs[*p] = bytes;
  c->mem_used += bytes;
  return PM_OK;
}

void ctx_free(pm_ctx* c, void* p) {
  if (!p) return;
  auto it = c->allocs.find(p);
  if (it != c->allocs.end()) {
    c->mem_used -= it->second;
    c->allocs.erase(it);
  }
  cudaFree(p);
}

}  // namespace pmnu

namespace {

bool valid(pm_ctx* c) { return c && c->magic == kMagic; }
cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

void drain_profile(pm_ctx* c) {
  for (auto& p : c->prof_live) {
    float ms = 0.f;
    cudaEventSynchronize(p.b);
    cudaEventElapsedTime(&ms, p.a, p.b);
    c->prof_ms[p.kind] += ms;
    c->prof_n[p.kind] += 1;
    c->prof_pool.push_back(p.a);
    c->prof_pool.push_back(p.b);
  }
  c->prof_live.clear();
}

template <class T>
int dalloc(pm_ctx* c, T** p, size_t count) {
  return ctx_alloc_n(c, p, count);
}

void free_all(pm_ctx* c) {
  ctx_free(c, c->meshA);
  ctx_free(c, c->meshB);
  ctx_free(c, c->meshC);
  for (auto& kv : c->tw) ctx_free(c, kv.second);
  ctx_free(c, c->ksq);
  ctx_free(c, c->winv);
  ctx_free(c, c->wforce);
  ctx_free(c, c->kvec0);
  for (int i = 0; i < 2; ++i) {
    ctx_free(c, c->keys[i]);
    ctx_free(c, c->vals[i]);
  }
  ctx_free(c, c->us);
  ctx_free(c, c->ps);
  ctx_free(c, c->ids);
  ctx_free(c, c->counts);
  ctx_free(c, c->bstart);
  ctx_free(c, c->bprev);
  ctx_free(c, c->rs_low);
  ctx_free(c, c->rs_k2);
  ctx_free(c, c->rs_v2);
  ctx_free(c, c->rs_dev);
  if (c->rs_host) cudaFreeHost(c->rs_host);
  ctx_free(c, c->hist);
  ctx_free(c, c->hist_scan);
  ctx_free(c, c->scan_tmp);
  ctx_free(c, c->pk_partial);
  ctx_free(c, c->pk_final);
  ctx_free(c, c->pk_w);
  ctx_free(c, c->ic_amp);
  ctx_free(c, c->ic_amp_nu);
  ctx_free(c, c->err_dev);
  if (c->err_host) cudaFreeHost(c->err_host);
  ctx_free(c, c->hs_u);
  ctx_free(c, c->hs_p);
  ctx_free(c, c->hs_id);
  ctx_free(c, c->hs_f);
  ctx_free(c, c->adj);
  ctx_free(c, c->paint_redo);
  mlp_free(c);
  for (auto& p : c->prof_live) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : c->prof_pool) cudaEventDestroy(e);
}

// sort (u, n) -> vals[0] = perm, keys[0] = sorted keys, bstart = bucket starts
int sort_into_scratch(pm_ctx* c, const uint32_t* u, int64_t n, cudaStream_t s) {
  if (n > c->n_max) return PM_EINVAL;
  return sort_particles(c, u, n, s);
}

// Where the force at the sorted scratch particles goes: with perm, F_out[d n + perm[i]]
// (f_out); else p_out = ps + K F and f_out = F in sorted order, u_out / id_out (when
// set) receive the sorted positions and ids.
struct ForceOut {
  const float* ps;
  float K;
  float* p_out;
  float* f_out;
  uint32_t* u_out;
  uint32_t* id_out;
  const uint32_t* perm;
  const DriftNext* drift = nullptr;  // stencil path only: the next step's kick and drift
};

// The real-space gradient (one potential mesh) unless the k-space form is asked for.
bool stencil_force(const pm_ctx* c) {
  return (c->cfg.flags & (PM_FLAG_SPECTRAL_KERNEL | PM_FLAG_KSPACE_GRADIENT)) == 0;
}

// Paint of the sorted scratch particles into meshA (padded), then the force at every
// sorted particle.  Default: the potential in meshA and the stencil readout.  k-space
// gradient with the third mesh: the fused x pass gives all three component meshes and
// one readout reads them; without it, one component mesh at a time in meshA.
int force_components(pm_ctx* c, int64_t n, double a, const ForceOut& o, cudaStream_t s) {
  float* realA = reinterpret_cast<float*>(c->meshA);
  const int rp = 2 * c->g.pc;
  mlp_table(c, a, s);
  paint_tiles(c, c->us, c->ids, n, PM_SPECIES_ALL, realA, rp, s);
  if (stencil_force(c)) {
    fft_potential(c, c->g, c->meshA, s);
    readout_fd4_kick(c, c->us, o.ps, c->ids, n, realA, rp, o.K, o.p_out, o.f_out, o.u_out, o.id_out, o.perm,
                     s, o.drift);
    return PM_OK;
  }
  if (c->meshC) {
    fft_force_fused(c, c->g, c->meshA, c->meshB, c->meshC, s);
    readout3_kick(c, c->us, o.ps, c->ids, n, realA, reinterpret_cast<float*>(c->meshB),
                  reinterpret_cast<float*>(c->meshC), rp, o.K, o.p_out, o.f_out, o.u_out, o.id_out, o.perm, s);
    return PM_OK;
  }
  fft_forward(c, c->g, c->meshA, c->meshB, 1, s);
  for (int comp = 0; comp < 3; ++comp) {
    fft_inverse_component(c, c->g, c->meshB, c->meshA, comp, s);
    readout_kick(c, c->us, o.ps, c->ids, n, realA, rp, comp, o.K, o.p_out, o.f_out, comp == 0 ? o.u_out : nullptr,
                 comp == 0 ? o.id_out : nullptr, o.perm, s);
  }
  return PM_OK;
}

int check_state(pm_ctx* c, const pm_state* st) {
  if (!st || st->n < 0 || st->n > c->n_max) return PM_EINVAL;
  if (st->n > 0 && (!st->u || !st->p || !st->id || !st->f)) return PM_EINVAL;
  return PM_OK;
}

// Sort of the drifted state (keys and counts from kick_drift_keys or a drifting
// readout) into the scratch copies: the near-sorted re-sort when the state is in the
// order of the last sort, else from scratch.
int sort_drifted(pm_ctx* c, pm_state* st, cudaStream_t s) {
  const int64_t n = st->n;
  int done = 0;
  if (n > 0 && c->rs_n == n) {
    done = resort_near_sorted(c, st->u, st->p, st->id, n, s);
    if (done < 0) return done;
  }
  if (done) {
    ++c->rs_fast;
    return PM_OK;
  }
  ++c->rs_full;
  const int rc = radix_and_buckets(c, n, s);
  if (rc != PM_OK) return rc;
  gather_sorted(c, st->u, st->p, st->id, n, c->vals[0], s);
  return PM_OK;
}

int check_step(double a0, double& ah, double a1) {
  if (!(a0 > 0.0) || !(a1 > a0) || a1 > 2.0) return PM_EINVAL;
  if (ah <= 0.0) ah = 0.5 * (a0 + a1);
  if (!(ah >= a0 && ah <= a1)) return PM_EINVAL;
  return PM_OK;
}

// Force at a0 on a state without a valid force cache (leaves the state in tile order).
int first_force(pm_ctx* c, pm_state* st, double a0, cudaStream_t s) {
  const int64_t n = st->n;
  int rc = sort_into_scratch(c, st->u, n, s);
  if (rc != PM_OK) return rc;
  gather_sorted(c, st->u, st->p, st->id, n, c->vals[0], s);
  force_components(c, n, a0, ForceOut{c->ps, 0.0f, st->p, st->f, st->u, st->id, nullptr}, s);
  st->f_valid = 1;
  std::swap(c->bstart, c->bprev);  // the state is now in this sort's order
  c->rs_n = n;
  return PM_OK;
}

int step_impl(pm_ctx* c, pm_state* st, double a0, double ah, double a1, cudaStream_t s) {
  int rc = check_state(c, st);
  if (rc != PM_OK) return rc;
  rc = check_step(a0, ah, a1);
  if (rc != PM_OK) return rc;
  const int64_t n = st->n;
  double k[3];
  c->cosmo.coeffs(a0, ah, a1, k);
  const float dscale = (float)(k[1] * 4294967296.0 / c->cfg.box);
  if (!st->f_valid) {
    rc = first_force(c, st, a0, s);
    if (rc != PM_OK) return rc;
  }
  // first half kick + drift + keys of the drifted positions; when the state is in the
  // order of the last sort, the near-sorted re-sort, else the radix sort from scratch
  kick_drift_keys(c, st->u, st->p, st->f, n, (float)k[0], dscale, s, n > 0 && c->rs_n == n);
  rc = sort_drifted(c, st, s);
  if (rc != PM_OK) return rc;
  // force at a1 and the second half kick, written back in tile order
  force_components(c, n, a1, ForceOut{c->ps, (float)k[2], st->p, st->f, st->u, st->id, nullptr}, s);
  std::swap(c->bstart, c->bprev);
  c->rs_n = n;
  st->a = a1;
  st->f_valid = 1;
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

// nsteps chained KDK steps (a0, ah, a1 per step, each a0 the previous a1).  On the
// stencil force path the readout that ends step i also applies step i + 1's first half
// kick and drift and writes its keys, so no separate kick/drift pass runs between the
// steps and the force cache is written only by the last one; the state after every
// step is the one pm_step gives, bit for bit.  Other paths loop over step_impl.
int run_impl(pm_ctx* c, pm_state* st, const double* sched, int64_t nsteps, cudaStream_t s) {
  int rc = check_state(c, st);
  if (rc != PM_OK) return rc;
  if (nsteps < 0 || (nsteps > 0 && !sched)) return PM_EINVAL;
  std::vector<double> sc(sched, sched + 3 * nsteps);
  for (int64_t i = 0; i < nsteps; ++i) {
    rc = check_step(sc[3 * i], sc[3 * i + 1], sc[3 * i + 2]);
    if (rc != PM_OK) return rc;
    if (i > 0 && sc[3 * i] != sc[3 * i - 1]) return PM_EINVAL;
  }
  if (nsteps == 0) return PM_OK;
  const int64_t n = st->n;
  if (!stencil_force(c) || n == 0) {
    for (int64_t i = 0; i < nsteps; ++i) {
      rc = step_impl(c, st, sc[3 * i], sc[3 * i + 1], sc[3 * i + 2], s);
      if (rc != PM_OK) return rc;
    }
    return PM_OK;
  }
  std::vector<double> k(3 * nsteps);
  for (int64_t i = 0; i < nsteps; ++i) c->cosmo.coeffs(sc[3 * i], sc[3 * i + 1], sc[3 * i + 2], &k[3 * i]);
  auto dscale = [&](int64_t i) { return (float)(k[3 * i + 1] * 4294967296.0 / c->cfg.box); };
  if (!st->f_valid) {
    rc = first_force(c, st, sc[0], s);
    if (rc != PM_OK) return rc;
  }
  kick_drift_keys(c, st->u, st->p, st->f, n, (float)k[0], dscale(0), s, c->rs_n == n);
  const long long nb1 = c->nbuckets + 1;
  for (int64_t i = 0; i < nsteps; ++i) {
    rc = sort_drifted(c, st, s);
    if (rc != PM_OK) return rc;
    const float K2 = (float)k[3 * i + 2];
    if (i + 1 < nsteps) {
      // counts of the keys the drifting readout writes (the sort above has used its own)
      PM_CUDA_TRY(cudaMemsetAsync(c->counts, 0, sizeof(uint32_t) * 3 * nb1, s));
      PM_CUDA_TRY(cudaMemsetAsync(c->rs_low, 0, sizeof(uint32_t) * nb1, s));
      PM_CUDA_TRY(cudaMemsetAsync(c->rs_dev, 0, sizeof(uint32_t), s));
      DriftNext dn;
      dn.K1 = (float)k[3 * (i + 1)];
      dn.dscale = dscale(i + 1);
      dn.keys = c->keys[0];
      dn.cnt3 = c->counts;
      dn.nb1 = nb1;
      dn.low = c->rs_low;
      ForceOut o{c->ps, K2, st->p, nullptr, st->u, st->id, nullptr};
      o.drift = &dn;
      force_components(c, n, sc[3 * i + 2], o, s);
    } else {
      force_components(c, n, sc[3 * i + 2], ForceOut{c->ps, K2, st->p, st->f, st->u, st->id, nullptr}, s);
    }
    std::swap(c->bstart, c->bprev);
    c->rs_n = n;
  }
  st->a = sc[3 * nsteps - 1];
  st->f_valid = 1;
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

}  // namespace

extern "C" {

const char* pm_strerror(int status) {
  switch (status) {
    case PM_OK: return "ok";
    case PM_EINVAL: return "invalid argument";
    case PM_ENOMEM: return "out of memory";
    case PM_ECUDA: return "CUDA runtime error";
    case PM_EKERNEL: return "a kernel flagged invalid input";
    case PM_ETIMEOUT: return "a bounded device wait timed out";
    case PM_ENOTINIT: return "context not initialised";
    case PM_ENONFINITE: return "a kernel met a non-finite momentum or force";
    default: return "unknown status";
  }
}

int pm_cosmo_growth(const pm_config* cfg, double a, double* out) {
  if (!cfg || !out || !(a > 0.0) || a > 2.0) return PM_EINVAL;
  Cosmo cm;
  int rc = cm.init(*cfg);
  if (rc != PM_OK) return rc;
  out[0] = cm.D(a);
  out[1] = cm.gp(a);
  out[2] = cm.gf(a);
  out[3] = cm.E(a);
  return PM_OK;
}

int pm_cosmo_coeffs(const pm_config* cfg, double a0, double ah, double a1, double* out) {
  if (!cfg || !out || !(a0 > 0.0) || !(a1 > a0) || a1 > 2.0 || ah < a0 || ah > a1) return PM_EINVAL;
  Cosmo cm;
  int rc = cm.init(*cfg);
  if (rc != PM_OK) return rc;
  cm.coeffs(a0, ah, a1, out);
  return PM_OK;
}

int pm_cosmo_params(const pm_config* cfg, double* out) {
  if (!cfg || !out) return PM_EINVAL;
  Cosmo cm;
  int rc = cm.init(*cfg);
  if (rc != PM_OK) return rc;
  out[0] = cm.omega_gamma;
  out[1] = cm.omega_c;
  out[2] = cm.omega_nu;
  out[3] = cm.omega_lambda;
  out[4] = cm.kT_nu0;
  return PM_OK;
}

int pm_nu_shells(const pm_config* cfg, double* edges, double* q_shell, double* m_shell) {
  if (!cfg || !edges || !q_shell || !m_shell) return PM_EINVAL;
  int rc = validate_config(*cfg);
  if (rc != PM_OK) return rc;
  if (cfg->nshell < 1 || cfg->n_nu < 1) return PM_EINVAL;
  return nu_shell_table(cfg->nshell, cfg->m_nu, cfg->n_nu, 40.0, edges, q_shell, m_shell);
}

int pm_init(const pm_config* cfg, pm_ctx** out) {
  if (!cfg || !out) return PM_EINVAL;
  *out = nullptr;
  int rc = validate_config(*cfg);
  if (rc != PM_OK) return rc;
  if (cfg->nsites > 0 && cfg->nshell > kMaxShell) return PM_EINVAL;
  pm_ctx* c = new (std::nothrow) pm_ctx();
  if (!c) return PM_ENOMEM;
  c->cfg = *cfg;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return PM_ECUDA;
  }
  rc = c->cosmo.init(*cfg);
  if (rc != PM_OK) {
    delete c;
    return rc;
  }
  const int N = cfg->nmesh;
  c->g.n = N;
  c->g.logn = 0;
  while ((1 << c->g.logn) < N) ++c->g.logn;
  c->g.pc = N / 2 + 2;
  c->nt = N / kTile;
  c->ntl = c->g.logn - 4;
  c->nbuckets = (long long)c->nt * c->nt * c->nt * 8;
  int bits = 0;
  while ((1LL << bits) < c->nbuckets) ++bits;
  // 18-bit keys or fewer: two 9-bit passes; else 8-bit passes
  c->radix_bits = bits <= 18 ? 9 : 8;
  c->radix_passes = std::max(1, (bits + c->radix_bits - 1) / c->radix_bits);
  c->n_max = cfg->n_max;
  if (c->n_max >= (int64_t)0xffffffffLL) {
    delete c;
    return PM_EINVAL;
  }
  // species masses (units of the mean mass per mesh cell)
  const double cells = (double)N * N * N;
  const double om = c->cosmo.omega_m0;
  c->mt.n_cdm = (int64_t)cfg->nc * cfg->nc * cfg->nc;
  c->m_cdm = cfg->nc > 0 ? c->cosmo.omega_c / om * cells / ((double)cfg->nc * cfg->nc * cfg->nc) : 0.0;
  c->mt.m_cdm = (float)c->m_cdm;
  c->mt.ndir = 2 * cfg->nfib + 1;
  c->mt.nshell = cfg->nsites > 0 ? cfg->nshell : 1;
  c->mt.n_nu = cfg->nsites > 0 ? (int64_t)cfg->nsites * cfg->nsites * cfg->nsites * cfg->nshell *
                                     c->mt.ndir
                               : 0;
  if (cfg->nsites > 0) {
    c->shell_edges.resize(cfg->nshell + 1);
    c->q_shell.resize(cfg->nshell);
    c->m_shell.resize(cfg->nshell);
    rc = nu_shell_table(cfg->nshell, cfg->m_nu, cfg->n_nu, 40.0, c->shell_edges.data(),
                        c->q_shell.data(), c->m_shell.data());
    if (rc != PM_OK) {
      delete c;
      return rc;
    }
    c->m_nu.resize(cfg->nshell);
    const double sites = (double)cfg->nsites * cfg->nsites * cfg->nsites;
    for (int i = 0; i < cfg->nshell; ++i) {
      c->m_nu[i] = c->cosmo.omega_nu / om * c->m_shell[i] / c->mt.ndir * cells / sites;
      c->mt.m_nu[i] = (float)c->m_nu[i];
    }
  }
  // device buffers
  const size_t me = c->g.elems();
  const int64_t nm = std::max<int64_t>(c->n_max, 1);
  const long long hb = (nm + 4095) / 4096;
  c->hist_blocks_max = hb;
  const long long scan_n = std::max<long long>(512 * hb, 3 * (c->nbuckets + 1));
  {  // every level of the recursive scan keeps 2 * blocks words
    size_t need = 64;
    for (long long m = scan_n; m > 1; m = (m + 4095) / 4096) need += 2 * (size_t)((m + 4095) / 4096);
    c->scan_tmp_elems = need;
  }
  // flag bit 0, or a 2048^3 mesh: per-component force path with two meshes (at 2048^3 it is
  // also the faster one: reading three 34 GB meshes at once starves the readout)
  const bool two_mesh = (cfg->flags & PM_FLAG_TWO_MESH) != 0 || N >= 2048;
  if ((!two_mesh && dalloc(c, &c->meshC, me)) || dalloc(c, &c->meshA, me) || dalloc(c, &c->meshB, me) ||
      dalloc(c, &c->ksq, N) ||
      dalloc(c, &c->winv, N) || dalloc(c, &c->wforce, N) || dalloc(c, &c->kvec0, N) || dalloc(c, &c->keys[0], nm) ||
      dalloc(c, &c->keys[1], nm) || dalloc(c, &c->vals[0], nm) || dalloc(c, &c->vals[1], nm) ||
      dalloc(c, &c->us, 3 * nm) || dalloc(c, &c->ps, 3 * nm) || dalloc(c, &c->ids, nm) ||
      dalloc(c, &c->counts, 3 * (c->nbuckets + 1)) || dalloc(c, &c->bstart, 3 * (c->nbuckets + 1)) ||
      dalloc(c, &c->bprev, 3 * (c->nbuckets + 1)) || dalloc(c, &c->rs_low, c->nbuckets + 1) ||
      dalloc(c, &c->rs_k2, nm) || dalloc(c, &c->rs_v2, nm) || dalloc(c, &c->rs_dev, 1) ||
      dalloc(c, &c->hist, 512 * hb) || dalloc(c, &c->hist_scan, 512 * hb) ||
      dalloc(c, &c->scan_tmp, c->scan_tmp_elems) || dalloc(c, &c->pk_partial, (size_t)N * 3 * 2048) ||
      dalloc(c, &c->pk_final, 3 * 2048) || dalloc(c, &c->err_dev, 1) ||
      dalloc(c, &c->paint_redo, (size_t)c->nt * c->nt * c->nt + 1)) {
    free_all(c);
    delete c;
    return PM_ENOMEM;
  }
  if (cudaMallocHost(&c->err_host, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&c->rs_host, 3 * sizeof(uint32_t)) != cudaSuccess) {
    free_all(c);
    delete c;
    return PM_ENOMEM;
  }
  cudaMemset(c->err_dev, 0, sizeof(int));
  // k tables of the force mesh (FP64 on the host, stored as float).  Force kernel:
  // phi_k = -1.5 Omega_m0 delta_k / N^3 / k^2 and the 4-point finite-difference gradient
  // D(k) = (8 sin kH - sin 2kH) / (6H); flags bit 1 selects the deconvolved spectral form
  // (phi_k / W(k)^2, gradient k).  D is 0 on the Nyquist index either way.
  {
    const bool spectral = (cfg->flags & PM_FLAG_SPECTRAL_KERNEL) != 0;
    std::vector<float> ksq(N), winv(N), wf(N), kv(N);
    const double pi = 3.14159265358979323846;
    const double kF = 2.0 * pi / cfg->box, H = cfg->box / N;
    for (int i = 0; i < N; ++i) {
      int ns = i < N / 2 ? i : i - N;
      double k = kF * ns;
      double x = pi * ns / N;
      double sinc = ns == 0 ? 1.0 : std::sin(x) / x;
      ksq[i] = (float)(k * k);
      winv[i] = (float)(1.0 / std::pow(sinc, 4));
      wf[i] = spectral ? winv[i] : 1.0f;
      const double d = spectral ? k : (8.0 * std::sin(k * H) - std::sin(2.0 * k * H)) / (6.0 * H);
      kv[i] = (i == N / 2) ? 0.0f : (float)d;
    }
    cudaMemcpy(c->ksq, ksq.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
    cudaMemcpy(c->winv, winv.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
    cudaMemcpy(c->wforce, wf.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
    cudaMemcpy(c->kvec0, kv.data(), sizeof(float) * N, cudaMemcpyHostToDevice);
  }
  tma_init(c);  // tensor maps for the TMA strided passes (classic kernels if unavailable)
  if (!twiddles(c, N)) {
    free_all(c);
    delete c;
    return PM_ENOMEM;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    free_all(c);
    delete c;
    return PM_ECUDA;
  }
  c->magic = kMagic;
  *out = c;
  return PM_OK;
}

int pm_destroy(pm_ctx* c) {
  if (!valid(c)) return PM_ENOTINIT;
  cudaDeviceSynchronize();
  free_all(c);
  c->magic = 0;
  delete c;
  return PM_OK;
}

int pm_sync(pm_ctx* c, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  cudaStream_t s = S(stream);
  PM_CUDA_TRY(cudaMemcpyAsync(c->err_host, c->err_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
  PM_CUDA_TRY(cudaStreamSynchronize(s));
  int e = *c->err_host;
  if (e) {
    cudaMemsetAsync(c->err_dev, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    return (e & 2) ? PM_ETIMEOUT : ((e & 4) ? PM_ENONFINITE : PM_EKERNEL);
  }
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int pm_coeffs(pm_ctx* c, double a0, double ah, double a1, double* out) {
  if (!valid(c)) return PM_ENOTINIT;
  if (!out || !(a0 > 0.0) || !(a1 > a0) || a1 > 2.0) return PM_EINVAL;
  if (ah <= 0.0) ah = 0.5 * (a0 + a1);
  if (ah < a0 || ah > a1) return PM_EINVAL;
  c->cosmo.coeffs(a0, ah, a1, out);
  out[3] = c->cosmo.D(a0);
  out[4] = c->cosmo.D(a1);
  return PM_OK;
}

int pm_sort(pm_ctx* c, const uint32_t* u, int64_t n, uint32_t* perm_out, uint32_t* key_out,
            void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (n < 0 || (n > 0 && !u)) return PM_EINVAL;
  cudaStream_t s = S(stream);
  int rc = sort_into_scratch(c, u, n, s);
  if (rc != PM_OK) return rc;
  if (n > 0 && perm_out)
    PM_CUDA_TRY(cudaMemcpyAsync(perm_out, c->vals[0], sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
  if (n > 0 && key_out)
    PM_CUDA_TRY(cudaMemcpyAsync(key_out, c->keys[0], sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int pm_paint(pm_ctx* c, const uint32_t* u, const uint32_t* id, int64_t n, int32_t species,
             float* mesh_out, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (n < 0 || !mesh_out || (n > 0 && !u) || species < 1 || species > 3) return PM_EINVAL;
  cudaStream_t s = S(stream);
  int rc = sort_into_scratch(c, u, n, s);
  if (rc != PM_OK) return rc;
  gather_sorted(c, u, nullptr, id, n, c->vals[0], s);
  paint_tiles(c, c->us, c->ids, n, species, mesh_out, c->g.n, s);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int pm_force(pm_ctx* c, const uint32_t* u, const uint32_t* id, int64_t n, float* F_out,
             void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (n < 0 || (n > 0 && (!u || !F_out))) return PM_EINVAL;
  if (n == 0) return PM_OK;
  cudaStream_t s = S(stream);
  int rc = sort_into_scratch(c, u, n, s);
  if (rc != PM_OK) return rc;
  gather_sorted(c, u, nullptr, id, n, c->vals[0], s);
  force_components(c, n, c->force_a, ForceOut{nullptr, 0.0f, nullptr, F_out, nullptr, nullptr, c->vals[0]}, s);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int pm_step(pm_ctx* c, pm_state* st, double a0, double ah, double a1, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  return step_impl(c, st, a0, ah, a1, S(stream));
}

int pm_run(pm_ctx* c, pm_state* st, const double* schedule, int64_t nsteps, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  return run_impl(c, st, schedule, nsteps, S(stream));
}

int pm_step_host(pm_ctx* c, uint32_t* u, float* p, uint32_t* id, float* f, int64_t n,
                 int32_t* f_valid, double a0, double ah, double a1, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (n <= 0 || n > c->n_max || !u || !p || !id || !f || !f_valid) return PM_EINVAL;
  cudaStream_t s = S(stream);
  if (n > c->hs_cap) {
    ctx_free(c, c->hs_u);
    ctx_free(c, c->hs_p);
    ctx_free(c, c->hs_id);
    ctx_free(c, c->hs_f);
    c->hs_u = nullptr;
    c->hs_p = c->hs_f = nullptr;
    c->hs_id = nullptr;
    c->hs_cap = 0;
    if (dalloc(c, &c->hs_u, 3 * n) || dalloc(c, &c->hs_p, 3 * n) || dalloc(c, &c->hs_id, n) ||
        dalloc(c, &c->hs_f, 3 * n))
      return PM_ENOMEM;
    c->hs_cap = n;
  }
  PM_CUDA_TRY(cudaMemcpyAsync(c->hs_u, u, 12 * n, cudaMemcpyHostToDevice, s));
  PM_CUDA_TRY(cudaMemcpyAsync(c->hs_p, p, 12 * n, cudaMemcpyHostToDevice, s));
  PM_CUDA_TRY(cudaMemcpyAsync(c->hs_id, id, 4 * n, cudaMemcpyHostToDevice, s));
  if (*f_valid) PM_CUDA_TRY(cudaMemcpyAsync(c->hs_f, f, 12 * n, cudaMemcpyHostToDevice, s));
  pm_state st{c->hs_u, c->hs_p, c->hs_id, c->hs_f, n, a0, *f_valid, 0};
  int rc = step_impl(c, &st, a0, ah, a1, s);
  if (rc != PM_OK) return rc;
  PM_CUDA_TRY(cudaMemcpyAsync(u, c->hs_u, 12 * n, cudaMemcpyDeviceToHost, s));
  PM_CUDA_TRY(cudaMemcpyAsync(p, c->hs_p, 12 * n, cudaMemcpyDeviceToHost, s));
  PM_CUDA_TRY(cudaMemcpyAsync(id, c->hs_id, 4 * n, cudaMemcpyDeviceToHost, s));
  PM_CUDA_TRY(cudaMemcpyAsync(f, c->hs_f, 12 * n, cudaMemcpyDeviceToHost, s));
  *f_valid = st.f_valid;
  return pm_sync(c, stream);
}

int pm_power(pm_ctx* c, const uint32_t* u, const uint32_t* id, int64_t n, int32_t sa, int32_t sb,
             int32_t nbins, double* k_out, double* P_out, int64_t* nmodes_out, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (n < 0 || (n > 0 && !u) || sa < 1 || sa > 3 || sb < 1 || sb > 3 || !k_out || !P_out ||
      !nmodes_out)
    return PM_EINVAL;
  cudaStream_t s = S(stream);
  int rc = sort_into_scratch(c, u, n, s);
  if (rc != PM_OK) return rc;
  gather_sorted(c, u, nullptr, id, n, c->vals[0], s);
  float* realA = reinterpret_cast<float*>(c->meshA);
  float* realB = reinterpret_cast<float*>(c->meshB);
  paint_tiles(c, c->us, c->ids, n, sa, realA, 2 * c->g.pc, s);
  fft_forward(c, c->g, c->meshA, c->meshA, 0, s);
  const float2* db = c->meshA;
  if (sb != sa) {
    paint_tiles(c, c->us, c->ids, n, sb, realB, 2 * c->g.pc, s);
    fft_forward(c, c->g, c->meshB, c->meshB, 0, s);
    db = c->meshB;
  }
  rc = power_bin(c, c->meshA, db, nbins, k_out, P_out, nmodes_out, s);
  if (rc != PM_OK) return rc;
  return pm_sync(c, stream);
}

int pm_ic(pm_ctx* c, const float* noise, double a0, double k_fs, pm_state* st, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (!noise || !st || !st->u || !st->p || !st->id) return PM_EINVAL;
  return ic_build(c, noise, a0, k_fs, st, S(stream));
}

int pm_ic_pseudo(pm_ctx* c, const float* noise, const float* uniforms, double a0, double k_fs,
                 pm_state* st, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (!noise || !uniforms || !st || !st->u || !st->p || !st->id) return PM_EINVAL;
  return ic_build(c, noise, a0, k_fs, st, S(stream), uniforms);
}

namespace {
// FNV-1a over the fields that define the physics and the mesh
uint64_t config_hash(const pm_config& f) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  };
  mix(&f.box, 8); mix(&f.nmesh, 4); mix(&f.nc, 4); mix(&f.nsites, 4); mix(&f.nshell, 4);
  mix(&f.nfib, 4); mix(&f.h, 8); mix(&f.omega_m, 8); mix(&f.t_cmb, 8); mix(&f.n_eff, 8);
  mix(&f.n_nu, 4); mix(f.m_nu, 24); mix(&f.a_ini_ode, 8);
  return h;
}
constexpr size_t kHeader = 512;
}  // namespace

int pm_state_save(pm_ctx* c, const pm_state* st, const char* path) {
  if (!valid(c)) return PM_ENOTINIT;
  if (!st || !path || st->n < 0 || (st->n > 0 && (!st->u || !st->p || !st->id || !st->f))) return PM_EINVAL;
  const int64_t n = st->n;
  std::vector<char> buf(kHeader + (size_t)n * 40);
  char hdr[kHeader];
  std::memset(hdr, ' ', kHeader);
  int len = std::snprintf(hdr, kHeader,
                          "{\"format\": \"pmnu-state-1\", \"n\": %lld, \"a\": %.17g, \"f_valid\": %d, "
                          "\"nmesh\": %d, \"box\": %.17g, \"config_hash\": \"%016llx\"}",
                          (long long)n, st->a, st->f_valid, c->cfg.nmesh, c->cfg.box,
                          (unsigned long long)config_hash(c->cfg));
  if (len <= 0 || len >= (int)kHeader - 1) return PM_EINVAL;
  hdr[len] = ' ';
  hdr[kHeader - 1] = '\n';
  std::memcpy(buf.data(), hdr, kHeader);
  char* d = buf.data() + kHeader;
  if (n > 0) {
    PM_CUDA_TRY(cudaDeviceSynchronize());
    PM_CUDA_TRY(cudaMemcpy(d, st->u, 12 * n, cudaMemcpyDeviceToHost));
    PM_CUDA_TRY(cudaMemcpy(d + 12 * n, st->p, 12 * n, cudaMemcpyDeviceToHost));
    PM_CUDA_TRY(cudaMemcpy(d + 24 * n, st->id, 4 * n, cudaMemcpyDeviceToHost));
    PM_CUDA_TRY(cudaMemcpy(d + 28 * n, st->f, 12 * n, cudaMemcpyDeviceToHost));
  }
  FILE* fp = std::fopen(path, "wb");
  if (!fp) return PM_EINVAL;
  size_t w = std::fwrite(buf.data(), 1, buf.size(), fp);
  int cl = std::fclose(fp);
  return (w == buf.size() && cl == 0) ? PM_OK : PM_EINVAL;
}

int pm_state_load(pm_ctx* c, pm_state* st, const char* path) {
  if (!valid(c)) return PM_ENOTINIT;
  if (!st || !path) return PM_EINVAL;
  FILE* fp = std::fopen(path, "rb");
  if (!fp) return PM_EINVAL;
  char hdr[kHeader + 1];
  if (std::fread(hdr, 1, kHeader, fp) != kHeader) {
    std::fclose(fp);
    return PM_EINVAL;
  }
  hdr[kHeader] = 0;
  long long n = -1;
  double a = 0.0;
  int fv = 0;
  unsigned long long hash = 0;
  const char* pf = std::strstr(hdr, "\"format\": \"pmnu-state-1\"");
  const char* pn = std::strstr(hdr, "\"n\": ");
  const char* pa = std::strstr(hdr, "\"a\": ");
  const char* pv = std::strstr(hdr, "\"f_valid\": ");
  const char* ph = std::strstr(hdr, "\"config_hash\": \"");
  if (!pf || !pn || !pa || !pv || !ph || std::sscanf(pn + 5, "%lld", &n) != 1 ||
      std::sscanf(pa + 5, "%lf", &a) != 1 || std::sscanf(pv + 11, "%d", &fv) != 1 ||
      std::sscanf(ph + 16, "%16llx", &hash) != 1 || n != st->n || hash != config_hash(c->cfg)) {
    std::fclose(fp);
    return PM_EINVAL;
  }
  std::vector<char> buf((size_t)n * 40);
  size_t r = std::fread(buf.data(), 1, buf.size(), fp);
  std::fclose(fp);
  if (r != buf.size()) return PM_EINVAL;
  if (n > 0) {
    if (!st->u || !st->p || !st->id || !st->f) return PM_EINVAL;
    const char* d = buf.data();
    PM_CUDA_TRY(cudaDeviceSynchronize());
    PM_CUDA_TRY(cudaMemcpy(st->u, d, 12 * n, cudaMemcpyHostToDevice));
    PM_CUDA_TRY(cudaMemcpy(st->p, d + 12 * n, 12 * n, cudaMemcpyHostToDevice));
    PM_CUDA_TRY(cudaMemcpy(st->id, d + 24 * n, 4 * n, cudaMemcpyHostToDevice));
    PM_CUDA_TRY(cudaMemcpy(st->f, d + 28 * n, 12 * n, cudaMemcpyHostToDevice));
  }
  st->a = a;
  st->f_valid = fv;
  return PM_OK;
}

int pm_fft_r2c(pm_ctx* c, const float* mesh, float* out_complex, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (!mesh || !out_complex) return PM_EINVAL;
  cudaStream_t s = S(stream);
  repack_real(c, c->g, mesh, c->g.n, reinterpret_cast<float*>(c->meshA), 2 * c->g.pc, s);
  fft_forward(c, c->g, c->meshA, c->meshA, 0, s);
  repack_complex(c, c->g, c->meshA, c->g.pc, reinterpret_cast<float2*>(out_complex),
                 c->g.n / 2 + 1, s);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int pm_fft_c2r(pm_ctx* c, const float* in_complex, float* mesh_out, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (!in_complex || !mesh_out) return PM_EINVAL;
  cudaStream_t s = S(stream);
  repack_complex(c, c->g, reinterpret_cast<const float2*>(in_complex), c->g.n / 2 + 1, c->meshA,
                 c->g.pc, s);
  fft_inverse_plain(c, c->g, c->meshA, s);
  repack_real(c, c->g, reinterpret_cast<float*>(c->meshA), 2 * c->g.pc, mesh_out, c->g.n, s);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int pm_potential(pm_ctx* c, const float* mesh, float* out_complex, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (!mesh || !out_complex) return PM_EINVAL;
  cudaStream_t s = S(stream);
  repack_real(c, c->g, mesh, c->g.n, reinterpret_cast<float*>(c->meshA), 2 * c->g.pc, s);
  mlp_table(c, c->force_a, s);
  fft_forward(c, c->g, c->meshA, c->meshB, 1, s);
  repack_complex(c, c->g, c->meshB, c->g.pc, reinterpret_cast<float2*>(out_complex),
                 c->g.n / 2 + 1, s);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int pm_force_mesh(pm_ctx* c, const float* phi_complex, int32_t comp, float* mesh_out, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (!phi_complex || !mesh_out || comp < 0 || comp > 2) return PM_EINVAL;
  cudaStream_t s = S(stream);
  repack_complex(c, c->g, reinterpret_cast<const float2*>(phi_complex), c->g.n / 2 + 1, c->meshB,
                 c->g.pc, s);
  fft_inverse_component(c, c->g, c->meshB, c->meshA, comp, s);
  repack_real(c, c->g, reinterpret_cast<float*>(c->meshA), 2 * c->g.pc, mesh_out, c->g.n, s);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int pm_readout(pm_ctx* c, const uint32_t* u, int64_t n, const float* mesh, float* out, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (n < 0 || (n > 0 && (!u || !mesh || !out))) return PM_EINVAL;
  if (n == 0) return PM_OK;
  cudaStream_t s = S(stream);
  // readout of a contiguous (row pitch N) mesh in input order
  readout_kick(c, u, nullptr, nullptr, n, mesh, c->g.n, 0, 0.0f, nullptr, out, nullptr, nullptr,
               nullptr, s);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int pm_paint_T(pm_ctx* c, const uint32_t* u, int64_t n, const float* mesh, float* out, void* stream) {
  return pm_readout(c, u, n, mesh, out, stream);
}

int pm_readout_T(pm_ctx* c, const uint32_t* u, int64_t n, const float* w, float* mesh_out, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (n < 0 || !mesh_out || (n > 0 && (!u || !w))) return PM_EINVAL;
  cudaStream_t s = S(stream);
  int rc = sort_into_scratch(c, u, n, s);
  if (rc != PM_OK) return rc;
  gather_sorted(c, u, nullptr, nullptr, n, c->vals[0], s);
  float* ws = c->ps;  // sorted weights in the momentum scratch
  rc = gather_weights(c, w, n, ws, s);
  if (rc != PM_OK) return rc;
  paint_tiles(c, c->us, c->ids, n, PM_SPECIES_ALL, mesh_out, c->g.n, s, ws);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int pm_paint_vjp(pm_ctx* c, const uint32_t* u, const uint32_t* id, int64_t n, const float* lam_mesh,
                 float* grad_out, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (n < 0 || (n > 0 && (!u || !lam_mesh || !grad_out))) return PM_EINVAL;
  if (n == 0) return PM_OK;
  cudaStream_t s = S(stream);
  int rc = sort_into_scratch(c, u, n, s);
  if (rc != PM_OK) return rc;
  gather_sorted(c, u, nullptr, id, n, c->vals[0], s);
  const float* m[1] = {lam_mesh};
  readout_grad(c, n, m, 1, c->g.n, nullptr, c->vals[0], grad_out, false, s);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int pm_power_vjp(pm_ctx* c, const uint32_t* u, const uint32_t* id, int64_t n, int32_t species,
                 int32_t nbins, const double* dL_dP, float* grad_out, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (n <= 0 || n > c->n_max || !u || !dL_dP || !grad_out || species < 1 || species > 3 || nbins < 1)
    return PM_EINVAL;
  cudaStream_t s = S(stream);
  int rc = sort_into_scratch(c, u, n, s);
  if (rc != PM_OK) return rc;
  gather_sorted(c, u, nullptr, id, n, c->vals[0], s);
  float* realA = reinterpret_cast<float*>(c->meshA);
  paint_tiles(c, c->us, c->ids, n, species, realA, 2 * c->g.pc, s);
  fft_forward(c, c->g, c->meshA, c->meshA, 0, s);
  rc = power_weight(c, nbins, dL_dP, s);
  if (rc != PM_OK) return rc;
  fft_inverse_plain(c, c->g, c->meshA, s);
  const float* m[1] = {realA};
  readout_grad(c, n, m, 1, 2 * c->g.pc, nullptr, c->vals[0], grad_out, false, s, species);
  return pm_sync(c, stream);
}

int pm_force_vjp(pm_ctx* c, const uint32_t* u, const uint32_t* id, int64_t n, const float* lam_f,
                 float* grad_out, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (n < 0 || n > c->n_max || (n > 0 && (!u || !lam_f || !grad_out))) return PM_EINVAL;
  return force_vjp(c, u, id, n, lam_f, c->force_a, grad_out, S(stream));
}

int pm_step_vjp(pm_ctx* c, const pm_state* st, double a0, double ah, double a1, const float* lam_x1,
                const float* lam_p1, float* lam_x0, float* lam_p0, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  int rc = check_state(c, st);
  if (rc != PM_OK) return rc;
  if (!(a0 > 0.0) || !(a1 > a0) || a1 > 2.0) return PM_EINVAL;
  if (ah <= 0.0) ah = 0.5 * (a0 + a1);
  if (!(ah >= a0 && ah <= a1)) return PM_EINVAL;
  if (st->n > 0 && (!lam_x1 || !lam_p1 || !lam_x0 || !lam_p0)) return PM_EINVAL;
  return step_vjp(c, st, a0, ah, a1, lam_x1, lam_p1, lam_x0, lam_p0, S(stream));
}

int pm_ic_vjp(pm_ctx* c, const float* lam_x0, const float* lam_p0, double a0, double k_fs,
              float* grad_noise, void* stream) {
  if (!valid(c)) return PM_ENOTINIT;
  if (!lam_x0 || !lam_p0 || !grad_noise || !(a0 > 0.0)) return PM_EINVAL;
  return ic_vjp(c, lam_x0, lam_p0, a0, k_fs, grad_noise, S(stream));
}

int64_t pm_launch_count(pm_ctx* c) { return valid(c) ? c->launches : -1; }

int64_t pm_memory_used(pm_ctx* c) { return valid(c) ? (int64_t)c->mem_used : -1; }

int pm_test_inject(pm_ctx* c, int32_t what) {
  if (!valid(c)) return PM_ENOTINIT;
  if (what != 0 && what != PM_INJECT_DROP_COPY) return PM_EINVAL;
  c->inject = what;
  return PM_OK;
}

int pm_profile_enable(pm_ctx* c, int32_t mask) {
  if (!valid(c)) return PM_ENOTINIT;
  c->prof = (uint32_t)mask;
  return PM_OK;
}

int pm_profile_read(pm_ctx* c, int32_t kind, double* ms, int64_t* launches, int32_t reset) {
  if (!valid(c)) return PM_ENOTINIT;
  if (kind < 0 || kind >= K_NUM_KINDS || !ms || !launches) return PM_EINVAL;
  drain_profile(c);
  *ms = c->prof_ms[kind];
  *launches = c->prof_n[kind];
  if (reset) {
    c->prof_ms[kind] = 0.0;
    c->prof_n[kind] = 0;
  }
  return PM_OK;
}

int pm_sort_stats(pm_ctx* c, int64_t* out) {
  if (!valid(c)) return PM_ENOTINIT;
  if (!out) return PM_EINVAL;
  out[0] = c->rs_fast;
  out[1] = c->rs_full;
  out[2] = c->rs_last_movers;
  return PM_OK;
}

int32_t pm_kernel_kinds(void) { return K_NUM_KINDS; }

const char* pm_kernel_name(int32_t k) {
  static const char* names[K_NUM_KINDS] = {
      "keys",          "scan",         "radix_hist",   "radix_scatter",   "gather",
      "paint_tiles",   "fft_z_r2c",    "fft_y",        "fft_x_green",     "fft_x_grad",
      "fft_z_c2r",     "fft_x_plain",  "readout_kick", "kick_drift_keys", "power_bin",
      "power_reduce",  "ic_za",        "ic_assemble",  "repack",          "fft_x_fused",
      "readout3_kick", "adjoint",      "mlp_table",    "mlp_backward", "mlp_misc",
      "fft_x_potential", "readout_fd4_kick", "resort_place", "resort_misc", "paint_redo"};
  if (k < 0 || k >= K_NUM_KINDS) return "unknown";
  return names[k];
}

}  // extern "C"
