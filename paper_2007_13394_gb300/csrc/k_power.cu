// Binned (cross) power spectrum of two half-spectrum meshes.
//
// P_ab(k) = (V / N^6) Re(delta_a delta_b^*) / W(k)^2 per mode, W the CIC window, each
// species mesh divided by its own mean (read from its k = 0 mode);
// bins of width k_F from k_F / 2: mode n (integer wavevector) falls in bin b when
// (b + 1/2)^2 <= |n|^2 < (b + 3/2)^2, decided exactly in integers.  Modes with
// 0 < n_z < N/2 count twice (Hermitian partners not stored).  Per CTA (one x plane)
// the sums go to shared memory in FP64, then a second kernel adds the per-plane
// partials in plane order.
#include <cuda_runtime.h>

#include <vector>

#include "pm_internal.cuh"

namespace pmnu {

namespace {

constexpr int kPowThreads = 256;
constexpr int kMaxBins = 2048;

__device__ __forceinline__ int bin_of(long long n2) {
  int b = (int)floorf(sqrtf((float)n2) - 0.5f);
  if (b < 0) b = 0;
  while ((long long)(b + 1) * (b + 1) + (b + 1) < n2) ++b;   // n2 > (b+1)^2 + (b+1): next bin
  while (b > 0 && (long long)b * b + b >= n2) --b;            // n2 <= b^2 + b: previous bin
  return b;
}

__global__ void __launch_bounds__(kPowThreads) k_power_bin(const float2* __restrict__ da,
                                                           const float2* __restrict__ db, int nm,
                                                           int pc, int nbins,
                                                           const float* __restrict__ winv,
                                                           float norm, double kf,
                                                           double* __restrict__ partial) {
  extern __shared__ double sh[];  // 3 * nbins: count, k sum, P sum
  for (int i = threadIdx.x; i < 3 * nbins; i += kPowThreads) sh[i] = 0.0;
  __syncthreads();
  const int x = blockIdx.x;
  const int nx = x < nm / 2 ? x : x - nm;
  const int nzc = nm / 2 + 1;
  const float wx = __ldg(winv + x);
  // delta_s = rho_s / mean_s: the k = 0 mode holds N^3 mean_s
  const float nn3 = (float)nm * (float)nm * (float)nm;
  const float ma = da[0].x / nn3, mb = db[0].x / nn3;
  const float scale = (ma != 0.0f && mb != 0.0f) ? norm / (ma * mb) : 0.0f;
  for (int q = threadIdx.x; q < nm * nzc; q += kPowThreads) {
    const int y = q / nzc, kz = q % nzc;
    const int ny = y < nm / 2 ? y : y - nm;
    const long long n2 = (long long)nx * nx + (long long)ny * ny + (long long)kz * kz;
    if (n2 == 0) continue;
    const int b = bin_of(n2);
    if (b >= nbins) continue;
    const size_t idx = ((size_t)x * nm + y) * pc + kz;
    const float2 a = da[idx], bb = db[idx];
    const float re = a.x * bb.x + a.y * bb.y;
    const float pk = scale * re * wx * __ldg(winv + y) * __ldg(winv + kz);
    const double w = (kz == 0 || kz == nm / 2) ? 1.0 : 2.0;
    atomicAdd(&sh[b], w);
    atomicAdd(&sh[nbins + b], w * kf * sqrt((double)n2));
    atomicAdd(&sh[2 * nbins + b], w * (double)pk);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * nbins; i += kPowThreads)
    partial[(size_t)blockIdx.x * 3 * nbins + i] = sh[i];
}

__global__ void k_power_reduce(const double* __restrict__ partial, int nplanes, int nbins,
                               double* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * nbins) return;
  double s = 0.0;
  for (int p = 0; p < nplanes; ++p) s += partial[(size_t)p * 3 * nbins + i];
  out[i] = s;
}

// d *= cw[b(n)] / W(k)^2 on the half spectrum (0 at k = 0 and beyond the last bin): the
// k-space cotangent of a binned auto-spectrum (the factor 2 and V / (N^6 rho_bar^2 N_b)
// folded into cw on the host).
__global__ void k_power_weight(float2* __restrict__ d, int nm, int pc, int nbins,
                               const float* __restrict__ winv, const float* __restrict__ cw) {
  const int x = blockIdx.x;
  const int nx = x < nm / 2 ? x : x - nm;
  const int nzc = nm / 2 + 1;
  const float wx = __ldg(winv + x);
  for (int q = threadIdx.x; q < nm * nzc; q += blockDim.x) {
    const int y = q / nzc, kz = q % nzc;
    const int ny = y < nm / 2 ? y : y - nm;
    const long long n2 = (long long)nx * nx + (long long)ny * ny + (long long)kz * kz;
    const size_t idx = ((size_t)x * nm + y) * pc + kz;
    float w = 0.0f;
    if (n2 > 0) {
      const int b = bin_of(n2);
      if (b < nbins) w = __ldg(cw + b) * wx * __ldg(winv + y) * __ldg(winv + kz);
    }
    d[idx] = cscale(d[idx], w);
  }
}

}  // namespace

// Cotangent mesh of sum_b dL_dP[b] P_b (auto-spectrum of the half spectrum in meshA, in
// place): meshA <- c_k F_k, c_k = 2 dL_dP[b] V / (N^6 rho_bar^2 W_k^2 N_b).  Synchronous
// (the mode counts N_b and rho_bar come from the binning pass).
int power_weight(pm_ctx* c, int nbins, const double* dL_dP, cudaStream_t s) {
  if (nbins < 1 || nbins > kMaxBins) return PM_EINVAL;
  std::vector<double> kb(nbins), Pb(nbins);
  std::vector<int64_t> nb(nbins);
  float2 f0;
  PM_CUDA_TRY(cudaMemcpyAsync(&f0, c->meshA, sizeof(float2), cudaMemcpyDeviceToHost, s));
  int rc = power_bin(c, c->meshA, c->meshA, nbins, kb.data(), Pb.data(), nb.data(), s);
  if (rc != PM_OK) return rc;
  const Geom& g = c->g;
  const double nn = (double)g.n, n3 = nn * nn * nn;
  const double rho_bar = (double)f0.x / n3;
  std::vector<float> cw(nbins, 0.0f);
  if (rho_bar != 0.0) {
    const double V = c->cfg.box * c->cfg.box * c->cfg.box;
    for (int b = 0; b < nbins; ++b)
      if (nb[b] > 0) cw[b] = (float)(2.0 * dL_dP[b] * V / (n3 * n3 * rho_bar * rho_bar * (double)nb[b]));
  }
  if (!c->pk_w && ctx_alloc_n(c, &c->pk_w, kMaxBins) != PM_OK) return PM_ENOMEM;
  PM_CUDA_TRY(cudaMemcpyAsync(c->pk_w, cw.data(), sizeof(float) * nbins, cudaMemcpyHostToDevice, s));
  LaunchScope L(c, s, K_POWER_BIN);
  k_power_weight<<<g.n, kPowThreads, 0, s>>>(c->meshA, g.n, g.pc, nbins, c->winv, c->pk_w);
  PM_CUDA_TRY(cudaStreamSynchronize(s));  // cw lives on this stack frame until the copy ends
  return PM_OK;
}

int power_bin(pm_ctx* c, const float2* da, const float2* db, int nbins, double* k_out,
              double* P_out, int64_t* nmodes_out, cudaStream_t s) {
  if (nbins < 1 || nbins > kMaxBins) return PM_EINVAL;
  const Geom& g = c->g;
  const double nn = (double)g.n;
  const float norm = (float)(c->cfg.box * c->cfg.box * c->cfg.box / (nn * nn * nn * nn * nn * nn));
  const double kf = 2.0 * 3.14159265358979323846 / c->cfg.box;
  const size_t smem = sizeof(double) * 3 * nbins;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_power_bin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(3 * kMaxBins * 8));
    attr = true;
  }
  {
    LaunchScope L(c, s, K_POWER_BIN);
    k_power_bin<<<g.n, kPowThreads, smem, s>>>(da, db, g.n, g.pc, nbins, c->winv, norm, kf,
                                               c->pk_partial);
  }
  {
    LaunchScope L(c, s, K_POWER_REDUCE);
    k_power_reduce<<<(3 * nbins + 255) / 256, 256, 0, s>>>(c->pk_partial, g.n, nbins, c->pk_final);
  }
  std::vector<double> h(3 * nbins);
  PM_CUDA_TRY(cudaMemcpyAsync(h.data(), c->pk_final, sizeof(double) * 3 * nbins,
                              cudaMemcpyDeviceToHost, s));
  PM_CUDA_TRY(cudaStreamSynchronize(s));
  for (int b = 0; b < nbins; ++b) {
    double cnt = h[b];
    nmodes_out[b] = (int64_t)cnt;
    k_out[b] = cnt > 0 ? h[nbins + b] / cnt : 0.0;
    P_out[b] = cnt > 0 ? h[2 * nbins + b] / cnt : 0.0;
  }
  return PM_OK;
}

}  // namespace pmnu
