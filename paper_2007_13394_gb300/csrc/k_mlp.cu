// Learned multiplicative correction of the Green's function (no counterpart in the
// paper): m(kappa, a) = 1 + MLP(kappa, a), kappa = |k| / k_Ny, a the scale factor of
// the force evaluation; Linear(2, 64) -> SiLU -> Linear(64, 64) -> SiLU -> Linear(64, 1).
//
// The network sees k only through |k|, and |k|^2 = k_F^2 s with the integer
// s = n_x^2 + n_y^2 + n_z^2 <= 3 (N/2)^2.  So instead of running it per mode, one
// launch evaluates it once per s into a table (FP32, weights in shared memory) and
// the Green's-function passes read m from the table: the same numbers, N^3 / 2 modes
// served by 3 N^2 / 4 evaluations.  Training reverses this: the adjoint bins
// d <lambda_F, F> / d m(k) by s (k_adj_combine) and one backward launch takes the
// network's gradient over the bins.
//
// Also here: Adam (Kingma & Ba 2014) on the parameters, and the mass-weighted
// periodic displacement loss the network is trained on with its cotangent.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "pm_internal.cuh"

namespace pmnu {

namespace {

constexpr int H = PM_MLP_HIDDEN;
constexpr int NP = PM_MLP_NPARAM;
// flat parameter layout: W1[H][2], b1[H], W2[H][H] (row = output unit), b2[H], w3[H], b3
constexpr int OW1 = 0, OB1 = 2 * H, OW2 = 3 * H, OB2 = 3 * H + H * H, OW3 = 4 * H + H * H,
              OB3 = 5 * H + H * H;
static_assert(OB3 + 1 == NP, "parameter layout");

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + expf(-z)); }

// 1 + MLP(kappa, a) with the parameters in shared memory
__device__ float mlp_m(const float* __restrict__ th, float kappa, float a) {
  float h1[H];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    const float z = fmaf(th[OW1 + 2 * j], kappa, fmaf(th[OW1 + 2 * j + 1], a, th[OB1 + j]));
    h1[j] = z * sigm(z);
  }
  float out = th[OB3];
  for (int i = 0; i < H; ++i) {
    const float4* w = reinterpret_cast<const float4*>(th + OW2 + i * H);
    float z = th[OB2 + i];
#pragma unroll
    for (int q = 0; q < H / 4; ++q) {
      const float4 v = w[q];
      z = fmaf(v.x, h1[4 * q], z);
      z = fmaf(v.y, h1[4 * q + 1], z);
      z = fmaf(v.z, h1[4 * q + 2], z);
      z = fmaf(v.w, h1[4 * q + 3], z);
    }
    out = fmaf(th[OW3 + i], z * sigm(z), out);
  }
  return 1.0f + out;
}

__device__ __forceinline__ void load_theta(const float* __restrict__ theta, float* th) {
  for (int i = threadIdx.x; i < NP; i += blockDim.x) th[i] = theta[i];
  __syncthreads();
}

// tab[s] = m(sqrt(s) / (N/2), a)
__global__ void __launch_bounds__(256) k_mlp_table(const float* __restrict__ theta, float a, float inv_half,
                                                   int64_t ntab, float* __restrict__ tab) {
  __shared__ __align__(16) float th[NP + 3];
  load_theta(theta, th);
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < ntab;
       s += (int64_t)gridDim.x * blockDim.x)
    tab[s] = mlp_m(th, sqrtf((float)s) * inv_half, a);
}

// out[i] = m(kappa[i], a[i])
__global__ void __launch_bounds__(256) k_mlp_eval(const float* __restrict__ theta, const float* __restrict__ kappa,
                                                  const float* __restrict__ av, int64_t n, float* __restrict__ out) {
  __shared__ __align__(16) float th[NP + 3];
  load_theta(theta, th);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = mlp_m(th, kappa[i], av[i]);
}

// phi = c(k) m(|n|^2) rho on the half spectrum of the force mesh (padded pitch pc)
__global__ void k_green_apply(const float2* __restrict__ rho, float2* __restrict__ phi, int nm, int pc,
                              const float* __restrict__ ksq, const float* __restrict__ winv, float gcoef,
                              const float* __restrict__ mtab) {
  const int x = blockIdx.x / nm, y = blockIdx.x % nm;
  const int nx = x < nm / 2 ? x : x - nm, ny = y < nm / 2 ? y : y - nm;
  for (int kz = threadIdx.x; kz <= nm / 2; kz += blockDim.x) {
    const size_t idx = ((size_t)x * nm + y) * pc + kz;
    const float k2 = ksq[x] + ksq[y] + ksq[kz];
    float g = gcoef * winv[x] * winv[y] * winv[kz] / k2;
    if (k2 == 0.0f) g = 0.0f;
    g *= mtab[nx * nx + ny * ny + kz * kz];
    phi[idx] = cscale(rho[idx], g);
  }
}

// Backward of the network over the bins: dtheta += sum_s gbin[s] dm(kappa_s, a) / dtheta,
// CH entries per block; clears the bins it read.  Shared: parameters and four CH x H
// activation arrays with row pitch HP = H + 1 (H1 = silu(z1), S1 = silu'(z1), D2 = dz2,
// H2 = silu(z2), later dz1).  Loops run the entry index fastest where a parameter row
// is broadcast, the unit index fastest where an activation row is.
constexpr int CH = 64;
constexpr int HP = H + 1;
constexpr int BW_THREADS = 256;
constexpr size_t BW_SMEM = sizeof(float) * ((NP + 3) + 4 * CH * HP + 2 * CH);

__global__ void __launch_bounds__(BW_THREADS) k_mlp_backward(const float* __restrict__ theta, float a,
                                                             float inv_half, int64_t ntab,
                                                             double* __restrict__ gbin,
                                                             double* __restrict__ dtheta) {
  extern __shared__ __align__(16) float sm[];
  float* th = sm;
  float* H1 = th + NP + 3;
  float* S1 = H1 + CH * HP;
  float* D2 = S1 + CH * HP;
  float* H2 = D2 + CH * HP;
  float* kap = H2 + CH * HP;
  float* ge = kap + CH;
  const int64_t e0 = (int64_t)blockIdx.x * CH;
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < CH; e += blockDim.x) {  // upstream gradient per entry
    const int64_t s = e0 + e;
    double g = 0.0;
    if (s < ntab) {
      g = gbin[s];
      gbin[s] = 0.0;
    }
    ge[e] = (float)g;
    kap[e] = sqrtf((float)s) * inv_half;
    if (g != 0.0) any = 1;
  }
  __syncthreads();
  if (!any) return;
  load_theta(theta, th);
  // layer 1
  for (int t = threadIdx.x; t < CH * H; t += blockDim.x) {
    const int e = t % CH, j = t / CH;
    const float z = fmaf(th[OW1 + 2 * j], kap[e], fmaf(th[OW1 + 2 * j + 1], a, th[OB1 + j]));
    const float sg = sigm(z);
    H1[e * HP + j] = z * sg;
    S1[e * HP + j] = sg * (1.0f + z * (1.0f - sg));
  }
  __syncthreads();
  // layer 2: z2 = W2 h1 + b2; h2 and dz2 = g w3 silu'(z2)
  for (int t = threadIdx.x; t < CH * H; t += blockDim.x) {
    const int e = t % CH, i = t / CH;
    float z = th[OB2 + i];
    for (int j = 0; j < H; ++j) z = fmaf(th[OW2 + i * H + j], H1[e * HP + j], z);
    const float sg = sigm(z);
    H2[e * HP + i] = z * sg;
    D2[e * HP + i] = ge[e] * th[OW3 + i] * sg * (1.0f + z * (1.0f - sg));
  }
  __syncthreads();
  // parameter gradients of layers 2 and 3
  for (int t = threadIdx.x; t < H * H; t += blockDim.x) {
    const int i = t / H, j = t % H;
    float acc = 0.0f;
    for (int e = 0; e < CH; ++e) acc = fmaf(D2[e * HP + i], H1[e * HP + j], acc);
    atomicAdd(dtheta + OW2 + t, (double)acc);
  }
  for (int i = threadIdx.x; i < H; i += blockDim.x) {
    float db2 = 0.0f, dw3 = 0.0f;
    for (int e = 0; e < CH; ++e) {
      db2 += D2[e * HP + i];
      dw3 = fmaf(ge[e], H2[e * HP + i], dw3);
    }
    atomicAdd(dtheta + OB2 + i, (double)db2);
    atomicAdd(dtheta + OW3 + i, (double)dw3);
  }
  if (threadIdx.x == 0) {
    float db3 = 0.0f;
    for (int e = 0; e < CH; ++e) db3 += ge[e];
    atomicAdd(dtheta + OB3, (double)db3);
  }
  __syncthreads();  // H2 is read above
  // dz1 = (W2^T dz2) silu'(z1), overwriting H2
  for (int t = threadIdx.x; t < CH * H; t += blockDim.x) {
    const int e = t % CH, j = t / CH;
    float acc = 0.0f;
    for (int i = 0; i < H; ++i) acc = fmaf(th[OW2 + i * H + j], D2[e * HP + i], acc);
    H2[e * HP + j] = acc * S1[e * HP + j];
  }
  __syncthreads();
  for (int j = threadIdx.x; j < H; j += blockDim.x) {
    float dk = 0.0f, db = 0.0f;
    for (int e = 0; e < CH; ++e) {
      const float d = H2[e * HP + j];
      dk = fmaf(d, kap[e], dk);
      db += d;
    }
    atomicAdd(dtheta + OW1 + 2 * j, (double)dk);
    atomicAdd(dtheta + OW1 + 2 * j + 1, (double)(db * a));
    atomicAdd(dtheta + OB1 + j, (double)db);
  }
}

// Adam with bias corrections bc1 = 1 - beta1^t, bc2 = 1 - beta2^t
__global__ void k_adam(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float bc1,
                       float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = grad[i];
  const float mi = b1 * m[i] + (1.0f - b1) * g;
  const float vi = b2 * v[i] + (1.0f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

__global__ void k_grad_out(const double* __restrict__ acc, float* __restrict__ out, int n, int reset,
                           double* __restrict__ acc_w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = (float)acc[i];
  if (reset) acc_w[i] = 0.0;
}

// ref_c[d][id_ref[i]] = u_ref[d][i]
__global__ void k_ref_canonical(const uint32_t* __restrict__ u_ref, const uint32_t* __restrict__ id_ref,
                                int64_t n, uint32_t* __restrict__ ref_c, int* __restrict__ err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t j = id_ref ? (int64_t)id_ref[i] : i;
  if (j >= n) {
    atomicExch(err, PM_EKERNEL);
    return;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) ref_c[d * n + j] = u_ref[d * n + i];
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x / 32); ++k) t += red[k];
  return t;
}

// sum of the particle masses
__global__ void k_mass_sum(const uint32_t* __restrict__ id, int64_t n, MassTable mt, int species,
                           double* __restrict__ out, int* __restrict__ err) {
  __shared__ double red[32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double m = 0.0;
  if (i < n) {
    bool bad = false;
    m = id_mass(mt, id ? id[i] : (uint32_t)i, species, &bad);
    if (bad) atomicExch(err, PM_EKERNEL);
  }
  const double t = block_sum(m, red);
  if (threadIdx.x == 0) atomicAdd(out, t);
}

// L += m_i |d_i|^2 / W, lam[d][id_i] = 2 m_i d_i / W, d_i = int32(u_i - ref_c[id_i]) L / 2^32
__global__ void k_disp_loss(const uint32_t* __restrict__ u, const uint32_t* __restrict__ id, int64_t n,
                            const uint32_t* __restrict__ ref_c, MassTable mt, int species, float scale,
                            const double* __restrict__ wsum, float* __restrict__ lam,
                            double* __restrict__ loss) {
  __shared__ double red[32];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < n) {
    const uint32_t j = id ? id[i] : (uint32_t)i;
    bool bad = false;
    const float m = id_mass(mt, j, species, &bad);
    const double inv_w = 1.0 / *wsum;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int32_t q = (int32_t)(u[d * n + i] - ref_c[d * n + j]);
      const float dd = (float)q * scale;
      l += (double)m * (double)dd * (double)dd * inv_w;
      lam[d * n + j] = (float)(2.0 * (double)m * (double)dd * inv_w);
    }
  }
  const double t = block_sum(l, red);
  if (threadIdx.x == 0) atomicAdd(loss, t);
}

unsigned nblocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int mlp_set(pm_ctx* c, const float* theta_host, int64_t nparam) {
  if (!theta_host) {
    c->mlp_on = false;
    return PM_OK;
  }
  if (nparam != NP) return PM_EINVAL;
  if (!c->mlp_theta) {
    const int64_t half = c->g.n / 2;
    c->mlp_ntab = 3 * half * half + 1;
    if (ctx_alloc_n(c, &c->mlp_theta, NP) != PM_OK || ctx_alloc_n(c, &c->mlp_tab, c->mlp_ntab) != PM_OK ||
        ctx_alloc_n(c, &c->mlp_gbin, c->mlp_ntab) != PM_OK || ctx_alloc_n(c, &c->mlp_dtheta, NP) != PM_OK ||
        ctx_alloc_n(c, &c->mlp_adam, 2 * NP) != PM_OK || (!c->mlp_red && ctx_alloc_n(c, &c->mlp_red, 4) != PM_OK)) {
      mlp_free(c);
      return PM_ENOMEM;
    }
    if (cudaMemset(c->mlp_gbin, 0, sizeof(double) * c->mlp_ntab) != cudaSuccess ||
        cudaMemset(c->mlp_dtheta, 0, sizeof(double) * NP) != cudaSuccess)
      return PM_ECUDA;
  }
  // new parameters restart the optimiser state
  if (cudaMemcpy(c->mlp_theta, theta_host, sizeof(float) * NP, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->mlp_adam, 0, sizeof(float) * 2 * NP) != cudaSuccess)
    return PM_ECUDA;
  c->mlp_on = true;
  return PM_OK;
}

void mlp_free(pm_ctx* c) {
  ctx_free(c, c->mlp_theta);
  ctx_free(c, c->mlp_tab);
  ctx_free(c, c->mlp_gbin);
  ctx_free(c, c->mlp_dtheta);
  ctx_free(c, c->mlp_adam);
  ctx_free(c, c->mlp_red);
  c->mlp_theta = c->mlp_tab = c->mlp_adam = nullptr;
  c->mlp_gbin = c->mlp_dtheta = c->mlp_red = nullptr;
  c->mlp_on = false;
}

void mlp_table(pm_ctx* c, double a, cudaStream_t s) {
  if (!c->mlp_on) return;
  if (c->cfg.flags & PM_FLAG_MLP_TENSOR) {
    mlp_table_tc(c, a, s);
    return;
  }
  LaunchScope L(c, s, K_MLP_TABLE);
  const unsigned grid = (unsigned)std::min<int64_t>(nblocks(c->mlp_ntab), 4 * 152);
  k_mlp_table<<<grid, 256, 0, s>>>(c->mlp_theta, (float)a, 2.0f / (float)c->g.n, c->mlp_ntab, c->mlp_tab);
}

void mlp_green_apply(pm_ctx* c, const float2* rho_k, float2* phi_k, cudaStream_t s) {
  LaunchScope L(c, s, K_MLP_MISC);
  const double nn = (double)c->g.n;
  k_green_apply<<<(unsigned)(c->g.n * c->g.n), 128, 0, s>>>(rho_k, phi_k, c->g.n, c->g.pc, c->ksq, c->wforce,
                                                           (float)(-1.5 * c->cosmo.omega_m0 / (nn * nn * nn)),
                                                           c->mlp_tab);
}

void mlp_backward(pm_ctx* c, double a, cudaStream_t s) {
  if (!c->mlp_on) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BW_SMEM);
    attr = true;
  }
  LaunchScope L(c, s, K_MLP_BACKWARD);
  k_mlp_backward<<<nblocks(c->mlp_ntab, CH), BW_THREADS, BW_SMEM, s>>>(
      c->mlp_theta, (float)a, 2.0f / (float)c->g.n, c->mlp_ntab, c->mlp_gbin, c->mlp_dtheta);
}

}  // namespace pmnu

using namespace pmnu;

extern "C" {

int pm_set_mlp(pm_ctx* c, const float* theta, int64_t nparam) {
  if (!c || c->magic != kMagic) return PM_ENOTINIT;
  return mlp_set(c, theta, nparam);
}

int pm_get_mlp(pm_ctx* c, float* theta, int64_t nparam) {
  if (!c || c->magic != kMagic) return PM_ENOTINIT;
  if (!theta || nparam != NP || !c->mlp_theta) return PM_EINVAL;
  if (cudaDeviceSynchronize() != cudaSuccess) return PM_ECUDA;
  return cudaMemcpy(theta, c->mlp_theta, sizeof(float) * NP, cudaMemcpyDeviceToHost) == cudaSuccess
             ? PM_OK
             : PM_ECUDA;
}

int pm_set_force_time(pm_ctx* c, double a) {
  if (!c || c->magic != kMagic) return PM_ENOTINIT;
  if (!(a > 0.0) || a > 2.0) return PM_EINVAL;
  c->force_a = a;
  return PM_OK;
}

int pm_mlp_eval(pm_ctx* c, const float* kappa, const float* a, int64_t n, float* m_out, void* stream) {
  if (!c || c->magic != kMagic) return PM_ENOTINIT;
  if (!c->mlp_theta || n < 0 || (n > 0 && (!kappa || !a || !m_out))) return PM_EINVAL;
  if (n == 0) return PM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LaunchScope L(c, s, K_MLP_MISC);
  const unsigned grid = (unsigned)std::min<int64_t>(nblocks(n), 4 * 152);
  k_mlp_eval<<<grid, 256, 0, s>>>(c->mlp_theta, kappa, a, n, m_out);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int pm_mlp_table(pm_ctx* c, double a, float* out, void* stream) {
  if (!c || c->magic != kMagic) return PM_ENOTINIT;
  if (!c->mlp_theta || !out || !(a > 0.0) || a > 2.0) return PM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool on = c->mlp_on;
  c->mlp_on = true;  // evaluate even while the factor is switched off
  mlp_table(c, a, s);
  c->mlp_on = on;
  PM_CUDA_TRY(cudaMemcpyAsync(out, c->mlp_tab, sizeof(float) * c->mlp_ntab, cudaMemcpyDeviceToDevice, s));
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int pm_mlp_grad(pm_ctx* c, float* grad_out, int64_t nparam, int32_t reset, void* stream) {
  if (!c || c->magic != kMagic) return PM_ENOTINIT;
  if (!c->mlp_theta || nparam != NP || !grad_out) return PM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LaunchScope L(c, s, K_MLP_MISC);
  k_grad_out<<<nblocks(NP), 256, 0, s>>>(c->mlp_dtheta, grad_out, NP, reset ? 1 : 0, c->mlp_dtheta);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int pm_mlp_adam(pm_ctx* c, const float* grad, int64_t nparam, double lr, double beta1, double beta2,
                double eps, int64_t t, void* stream) {
  if (!c || c->magic != kMagic) return PM_ENOTINIT;
  if (!c->mlp_theta || nparam != NP || !grad || t < 1 || !(lr > 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) ||
      !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0))
    return PM_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double bc1 = 1.0 - std::pow(beta1, (double)t), bc2 = 1.0 - std::pow(beta2, (double)t);
  LaunchScope L(c, s, K_MLP_MISC);
  k_adam<<<nblocks(NP), 256, 0, s>>>(c->mlp_theta, grad, c->mlp_adam, c->mlp_adam + NP, NP, (float)lr,
                                     (float)beta1, (float)beta2, (float)eps, (float)bc1, (float)bc2);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int pm_displacement_loss(pm_ctx* c, const uint32_t* u, const uint32_t* id, const uint32_t* u_ref,
                         const uint32_t* id_ref, int64_t n, int32_t species, float* lam_x, double* loss,
                         void* stream) {
  if (!c || c->magic != kMagic) return PM_ENOTINIT;
  if (n <= 0 || n > c->n_max || !u || !u_ref || !lam_x || !loss || species < 1 || species > 3)
    return PM_EINVAL;
  if (!c->mlp_red && ctx_alloc_n(c, &c->mlp_red, 4) != PM_OK) return PM_ENOMEM;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // canonical copy of the reference positions in the adjoint scratch
  if (n > c->adj_cap) {
    ctx_free(c, c->adj);
    c->adj = nullptr;
    c->adj_cap = 0;
    if (ctx_alloc_n(c, &c->adj, 8 * 3 * (size_t)n) != PM_OK) return PM_ENOMEM;
    c->adj_cap = n;
  }
  uint32_t* ref_c = reinterpret_cast<uint32_t*>(c->adj);
  PM_CUDA_TRY(cudaMemsetAsync(c->mlp_red, 0, sizeof(double) * 2, s));
  {
    LaunchScope L(c, s, K_MLP_MISC);
    k_ref_canonical<<<nblocks(n), 256, 0, s>>>(u_ref, id_ref, n, ref_c, c->err_dev);
  }
  {
    LaunchScope L(c, s, K_MLP_MISC);
    k_mass_sum<<<nblocks(n), 256, 0, s>>>(id, n, c->mt, species, c->mlp_red, c->err_dev);
  }
  {
    LaunchScope L(c, s, K_MLP_MISC);
    k_disp_loss<<<nblocks(n), 256, 0, s>>>(u, id, n, ref_c, c->mt, species, (float)(c->cfg.box / 4294967296.0),
                                           c->mlp_red, lam_x, c->mlp_red + 1);
  }
  double h[2];
  PM_CUDA_TRY(cudaMemcpyAsync(h, c->mlp_red, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
  const int rc = pm_sync(c, s);
  if (rc != PM_OK) return rc;
  *loss = h[1];
  return PM_OK;
}

}  // extern "C"
