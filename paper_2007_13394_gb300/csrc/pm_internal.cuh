// Internal context, launch bookkeeping and small device helpers of libpmnu.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <unordered_map>
#include <vector>

#include "../../include/pm.h"
#include "cosmo.h"

namespace pmnu {

// Kernel kinds, for launch counting and per-kind CUDA-event timing.
enum Kind {
  K_KEYS = 0,
  K_SCAN,
  K_RADIX_HIST,
  K_RADIX_SCATTER,
  K_GATHER,
  K_PAINT,
  K_FFT_Z_R2C,
  K_FFT_Y,
  K_FFT_X_GREEN,
  K_FFT_X_GRAD,
  K_FFT_Z_C2R,
  K_FFT_X_PLAIN,
  K_READOUT_KICK,
  K_KICK_DRIFT_KEYS,
  K_POWER_BIN,
  K_POWER_REDUCE,
  K_IC_ZA,
  K_IC_ASSEMBLE,
  K_REPACK,
  K_FFT_X_FUSED,
  K_READOUT3_KICK,
  K_ADJOINT,
  K_MLP_TABLE,
  K_MLP_BACKWARD,
  K_MLP_MISC,
  K_FFT_X_POT,
  K_READOUT_FD4_KICK,
  K_RESORT_PLACE,
  K_RESORT_MISC,
  K_PAINT_REDO,
  K_NUM_KINDS
};

constexpr int kTile = 16;        // tile edge in cells (the sort contract)
constexpr int kMaxShell = 64;    // largest N_shell the mass table carries

// Particle-mass lookup from the canonical id (passed by value to kernels).
struct MassTable {
  int64_t n_cdm;   // ids below are CDM
  int64_t n_nu;    // neutrino ids follow
  int32_t ndir;    // 2 nfib + 1
  int32_t nshell;
  float m_cdm;
  float m_nu[kMaxShell];
};

// The next step's first half kick and drift, fused into a readout (pm_run): K1 and the
// drift's fixed-point scale, where the new keys go and the near-sorted re-sort's counts
// (cnt3: three arrays of nb1 words, low: nb1 words).
struct DriftNext {
  float K1 = 0.0f;
  float dscale = 0.0f;
  uint32_t* keys = nullptr;
  uint32_t* cnt3 = nullptr;
  long long nb1 = 0;
  uint32_t* low = nullptr;
};

// Mesh geometry for one FFT size.
struct Geom {
  int n = 0, logn = 0;   // points per side
  int pc = 0;            // complex row pitch (float2) = n/2 + 2
  long long rows() const { return (long long)n * n; }
  size_t elems() const { return (size_t)n * n * pc; }  // float2 per padded mesh
};

struct Prof {
  int kind;
  cudaEvent_t a, b;
};

}  // namespace pmnu

struct pm_ctx {
  int magic = 0;
  int device = 0;
  pm_config cfg{};
  pmnu::Cosmo cosmo;
  pmnu::Geom g;             // force mesh
  int nt = 0, ntl = 0;      // tiles per side and its log2
  long long nbuckets = 0;   // nt^3 * 8
  int radix_passes = 0;
  int radix_bits = 8;       // digit width of the LSD radix passes
  int64_t n_max = 0;
  // meshes (two padded complex meshes, also viewed as padded real meshes)
  float2* meshA = nullptr;
  float2* meshB = nullptr;
  float2* meshC = nullptr;  // third mesh: the fused force path (null: per-component path)
  // tensor maps of meshA/B/C for the TMA strided passes: [mesh][0: x-pass box, 1: y-pass box]
  CUtensorMap tmap[3][2];
  bool tma_ok = false;
  // per-size tables: twiddles e^{-2 pi i t / n} (n entries); per force-mesh index: |k|^2,
  // 1/sinc^4 (the power spectrum's window compensation), the force Green's function's
  // per-axis factor (1, or 1/sinc^4 for the deconvolved spectral kernel) and the
  // gradient kernel D(k) (4-point finite difference, or k; 0 on the Nyquist index)
  std::map<int, float2*> tw;
  float* ksq = nullptr;
  float* winv = nullptr;
  float* wforce = nullptr;
  float* kvec0 = nullptr;
  // sort / particle scratch
  uint32_t* keys[2] = {nullptr, nullptr};
  uint32_t* vals[2] = {nullptr, nullptr};
  uint32_t* us = nullptr;
  float* ps = nullptr;
  uint32_t* ids = nullptr;
  uint32_t* counts = nullptr;   // 3 (nbuckets + 1), see below
  uint32_t* bstart = nullptr;   // 3 (nbuckets + 1)
  // near-sorted re-sort of pm_step (k_sort.cu).  counts, bstart and bprev hold three
  // arrays of nbuckets + 1 words each: counts = [per new key | stayers per new key |
  // movers per old key], scanned as one array into bstart (bucket starts, then the two
  // other scans offset by n and by n + stayers).  bprev: the same for the order the last
  // step left its state in (valid for rs_n particles, -1: none).
  uint32_t* bprev = nullptr;
  int64_t rs_n = -1;
  uint32_t* rs_low = nullptr;     // movers from a lower old key, per new key (nbuckets + 1)
  uint32_t* rs_k2 = nullptr;      // second (key, index) buffer pair of the movers' radix
  uint32_t* rs_v2 = nullptr;
  uint32_t* rs_dev = nullptr;     // flag bits of k_kick_drift_keys<true>
  uint32_t* rs_host = nullptr;    // pinned: flags, first word of the third scan, last word
  int64_t rs_fast = 0, rs_full = 0;  // re-sorts done the near-sorted way / from scratch
  int64_t rs_last_movers = 0;        // movers of the last near-sorted re-sort
  uint32_t* hist = nullptr;     // 256 * radix blocks, raw
  uint32_t* hist_scan = nullptr;
  uint32_t* scan_tmp = nullptr;
  size_t scan_tmp_elems = 0;
  long long hist_blocks_max = 0;
  // masses
  pmnu::MassTable mt{};
  double m_cdm = 0.0;
  std::vector<double> m_nu, q_shell, m_shell, shell_edges;
  // power binning partials
  double* pk_partial = nullptr;
  double* pk_final = nullptr;
  float* pk_w = nullptr;        // per-bin weights of the spectrum VJP
  // initial-condition tables
  float* ic_amp = nullptr;      // sqrt(P/V) nc^1.5 by integer |n|^2, CDM and filtered neutrino
  float* ic_amp_nu = nullptr;
  long long ic_amp_len = 0;
  double ic_kfs = -1.0;
  // error word
  int* err_dev = nullptr;
  int* err_host = nullptr;
  // host-array state used by pm_step_host
  uint32_t* hs_u = nullptr;
  float* hs_p = nullptr;
  uint32_t* hs_id = nullptr;
  float* hs_f = nullptr;
  int64_t hs_cap = 0;
  // adjoint scratch: 8 x 3n floats (gathered cotangents, drifted positions, partial sums)
  float* adj = nullptr;
  int64_t adj_cap = 0;
  // learned Green's-function factor m(|k| / k_Ny, a) = 1 + MLP (null theta: plain kernel)
  bool mlp_on = false;
  float* mlp_theta = nullptr;     // PM_MLP_NPARAM parameters
  float* mlp_tab = nullptr;       // m at |n|^2 = s for s in [0, mlp_ntab), refreshed per force
  int64_t mlp_ntab = 0;           // 3 (N/2)^2 + 1
  double* mlp_gbin = nullptr;     // d <lambda_F, F> / d m per s (adjoint, then cleared)
  double* mlp_dtheta = nullptr;   // accumulated d L / d theta
  float* mlp_adam = nullptr;      // Adam first and second moments, 2 x PM_MLP_NPARAM
  double* mlp_red = nullptr;      // device scalars of the displacement loss reductions
  double force_a = 1.0;           // scale factor of pm_force / pm_potential / pm_force_vjp
  // device memory held, by allocation, against cfg.mem_limit
  std::unordered_map<void*, size_t> allocs;
  size_t mem_used = 0;
  // the paint's redo list: count, then the tiles whose 32-bit accumulators wrapped
  uint32_t* paint_redo = nullptr;
  // pending test injection (pm_test_inject), consumed by the launch it targets
  int inject = 0;
  // instrumentation
  int64_t launches = 0;
  uint32_t prof = 0;  // bit k: time kernel kind k
  std::vector<pmnu::Prof> prof_live;
  std::vector<cudaEvent_t> prof_pool;
  double prof_ms[pmnu::K_NUM_KINDS] = {};
  int64_t prof_n[pmnu::K_NUM_KINDS] = {};
};

namespace pmnu {

constexpr int kMagic = 0x504d4e55;

// Launch bookkeeping: count, and when profiling, bracket with events on the stream.
struct LaunchScope {
  pm_ctx* c;
  cudaStream_t s;
  int kind;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LaunchScope(pm_ctx* ctx, cudaStream_t st, int k);
  ~LaunchScope();
};

// Device memory of a context, charged against cfg.mem_limit (0: no limit): PM_ENOMEM without
// calling cudaMalloc when the limit would be passed, or when cudaMalloc fails (*p = NULL).
int ctx_alloc(pm_ctx* c, void** p, size_t bytes);
void ctx_free(pm_ctx* c, void* p);  // NULL is a no-op
template <class T>
int ctx_alloc_n(pm_ctx* c, T** p, size_t count) {
  return ctx_alloc(c, reinterpret_cast<void**>(p), sizeof(T) * (count ? count : 1));
}

// host launch helpers implemented in the .cu files
int sort_particles(pm_ctx* c, const uint32_t* u, int64_t n, cudaStream_t s);  // keys + radix -> vals
int build_keys(pm_ctx* c, const uint32_t* u, int64_t n, cudaStream_t s);
int radix_and_buckets(pm_ctx* c, int64_t n, cudaStream_t s);                 // after keys
void scan_exclusive(pm_ctx* c, const uint32_t* in, uint32_t* out, long long n, cudaStream_t s);
void gather_sorted(pm_ctx* c, const uint32_t* u, const float* p, const uint32_t* id, int64_t n,
                   const uint32_t* perm, cudaStream_t s);
// weights (sorted order, signed) replace the species masses when non-null
void paint_tiles(pm_ctx* c, const uint32_t* us, const uint32_t* ids, int64_t n, int species,
                 float* mesh, int row_pitch, cudaStream_t s, const float* weights = nullptr);
void fft_forward(pm_ctx* c, const Geom& g, float2* buf, float2* dst, int green, cudaStream_t s);
void fft_inverse_component(pm_ctx* c, const Geom& g, const float2* phi, float2* buf, int comp,
                           cudaStream_t s);
void fft_inverse_plain(pm_ctx* c, const Geom& g, float2* buf, cudaStream_t s);
// paint mesh in buf (real) -> potential phi (real, unnormalised inverse), in place
void fft_potential(pm_ctx* c, const Geom& g, float2* buf, cudaStream_t s);
// force F = -(4-point gradient of phi) read out at the sorted particles of each tile,
// fused with the kick; arguments as readout3_kick (phi: real mesh, row pitch row_pitch)
// dn non-null: also the next step's first half kick, drift, keys and counts (u_out, p_out
// and id_out required; f_out optional)
void readout_fd4_kick(pm_ctx* c, const uint32_t* us, const float* ps, const uint32_t* ids, int64_t n,
                      const float* phi, int row_pitch, float K, float* p_out, float* f_out,
                      uint32_t* u_out, uint32_t* id_out, const uint32_t* perm_scatter, cudaStream_t s,
                      const DriftNext* dn = nullptr);
// paint mesh in a (real) -> three real force meshes in a, b, cz
void fft_force_fused(pm_ctx* c, const Geom& g, float2* a, float2* b, float2* cz, cudaStream_t s);
void readout3_kick(pm_ctx* c, const uint32_t* us, const float* ps, const uint32_t* ids, int64_t n,
                   const float* mx, const float* my, const float* mz, int row_pitch, float K,
                   float* p_out, float* f_out, uint32_t* u_out, uint32_t* id_out,
                   const uint32_t* perm_scatter, cudaStream_t s);
void readout_kick(pm_ctx* c, const uint32_t* us, const float* ps, const uint32_t* ids, int64_t n,
                  const float* mesh, int row_pitch, int comp, float K, float* p_out, float* f_out,
                  uint32_t* u_out, uint32_t* id_out, const uint32_t* perm_scatter,
                  cudaStream_t s);
// resort: also classify the particles against bprev for resort_near_sorted
void kick_drift_keys(pm_ctx* c, uint32_t* u, float* p, const float* f, int64_t n, float K1,
                     float dscale, cudaStream_t s, bool resort);
// After kick_drift_keys(resort = true): bucket starts, and if the state was in bprev's
// order, the sorted copies us / ps / ids of (u, p, id) with the stable order of keys[0]
// (returns 1); returns 0 (nothing written but bstart) when the caller must sort from
// scratch, a negative status on error.  Synchronises the stream once.
int resort_near_sorted(pm_ctx* c, const uint32_t* u, const float* p, const uint32_t* id, int64_t n,
                       cudaStream_t s);
void repack_real(pm_ctx* c, const Geom& g, const float* src, int src_pitch, float* dst,
                 int dst_pitch, cudaStream_t s);
void repack_complex(pm_ctx* c, const Geom& g, const float2* src, int src_pitch, float2* dst,
                    int dst_pitch, cudaStream_t s);
int power_bin(pm_ctx* c, const float2* da, const float2* db, int nbins, double* k_out,
              double* P_out, int64_t* nmodes_out, cudaStream_t s);
int power_weight(pm_ctx* c, int nbins, const double* dL_dP, cudaStream_t s);
int ic_build(pm_ctx* c, const float* noise, double a0, double k_fs, pm_state* st, cudaStream_t s,
             const float* uniforms = nullptr);
float2* twiddles(pm_ctx* c, int n);
// adjoint (k_adjoint.cu)
void readout_grad(pm_ctx* c, int64_t n, const float* const* meshes, int nmeshes, int row_pitch,
                  const float* wts_sorted, const uint32_t* perm, float* out, bool accumulate,
                  cudaStream_t s, int species = PM_SPECIES_ALL);
int force_vjp(pm_ctx* c, const uint32_t* u, const uint32_t* id, int64_t n, const float* lam_f,
              double a, float* grad, cudaStream_t s);
int step_vjp(pm_ctx* c, const pm_state* st, double a0, double ah, double a1, const float* lx1,
             const float* lp1, float* lx0, float* lp0, cudaStream_t s);
int ic_vjp(pm_ctx* c, const float* lx, const float* lp, double a0, double k_fs, float* grad_noise,
           cudaStream_t s);
int gather_weights(pm_ctx* c, const float* w, int64_t n, float* w_sorted, cudaStream_t s);
bool tma_init(pm_ctx* c);
// learned factor (k_mlp.cu)
int mlp_set(pm_ctx* c, const float* theta_host, int64_t nparam);
void mlp_free(pm_ctx* c);
// refreshes the |n|^2 table for scale factor a when the learned factor is on
void mlp_table(pm_ctx* c, double a, cudaStream_t s);
void mlp_table_tc(pm_ctx* c, double a, cudaStream_t s);  // tensor-core form (k_mlp_tc.cu)
// phi_k = c(k) m(k) rho_k on the force mesh's half spectrum (src and dst padded)
void mlp_green_apply(pm_ctx* c, const float2* rho_k, float2* phi_k, cudaStream_t s);
// d L / d theta += backward of the network over mlp_gbin at scale factor a; clears mlp_gbin
void mlp_backward(pm_ctx* c, double a, cudaStream_t s);

#define PM_CUDA_TRY(expr)                      \
  do {                                         \
    cudaError_t e_ = (expr);                   \
    if (e_ != cudaSuccess) return PM_ECUDA;    \
  } while (0)

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// Sort key of a particle: tile of its cell (16^3 cells, x-major) * 8 + face class.
__device__ __forceinline__ uint32_t tile_key(uint32_t ux, uint32_t uy, uint32_t uz, int shift,
                                             int ntl) {
  uint32_t cx = ux >> shift, cy = uy >> shift, cz = uz >> shift;
  uint32_t tile = ((cx >> 4) << (2 * ntl)) | ((cy >> 4) << ntl) | (cz >> 4);
  uint32_t cls = (((cx & 15u) == 15u) ? 4u : 0u) | (((cy & 15u) == 15u) ? 2u : 0u) |
                 (((cz & 15u) == 15u) ? 1u : 0u);
  return (tile << 3) | cls;
}

// Mass of a canonical id in units of the mean mass per cell; 0 if the species is masked.
// Sets *bad for ids beyond the configured particle count.
__device__ __forceinline__ float id_mass(const MassTable& mt, uint32_t id, int species, bool* bad) {
  if ((int64_t)id < mt.n_cdm) return (species & PM_SPECIES_CDM) ? mt.m_cdm : 0.0f;
  int64_t j = (int64_t)id - mt.n_cdm;
  if (j >= mt.n_nu) {
    *bad = true;
    return 0.0f;
  }
  // 32-bit division: ids are below 2^32 (n_max < 2^32 - 1)
  const int shell = (int)(((uint32_t)j / (uint32_t)mt.ndir) % (uint32_t)mt.nshell);
  return (species & PM_SPECIES_NU) ? mt.m_nu[shell] : 0.0f;
}

}  // namespace pmnu
