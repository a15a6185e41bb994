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

}  // namespace

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
