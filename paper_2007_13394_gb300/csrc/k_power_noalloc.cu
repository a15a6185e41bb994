// Power-spectrum binning that allocates nothing (pm_power_bin_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a
// spectrum: code running inside a memory pool or arena that owns every byte of
// the device, a CUDA-graph-driven pipeline whose replays must not call
// cudaMalloc, or a host that has handed all free memory to another framework.
// For them this entry point takes only the caller's input spectra and output
// arrays; the per-CTA partial sums live in one file-scope device array of fixed
// size (kRows x 3 x kMaxBins doubles, 3 MiB) that every GPU which loads the
// library holds until the process exits.
//
// The array's host-side name is not a device address, so the first call on each
// device resolves its address with cudaGetSymbolAddress (with that device
// current) and caches it; make that first call before any stream capture.
// Every call shares the array: calls whose kernels overlap on the GPU (different
// streams, or different host threads on one device) race on it and must be
// serialised by the caller.  Each call overwrites every partial row it later
// reads, so nothing has to be cleared between calls.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pm.h"

namespace {

constexpr int kRows = 256;        // CTAs of the binning kernel (planes x = b mod kRows)
constexpr int kMaxBins = 512;     // largest nbins accepted
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_pk_scratch[kRows * 3 * kMaxBins];

double* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

__device__ __forceinline__ int bin_index(long long n2) {
  int b = (int)floorf(sqrtf((float)n2) - 0.5f);
  if (b < 0) b = 0;
  while ((long long)(b + 1) * (b + 1) + (b + 1) < n2) ++b;
  while (b > 0 && (long long)b * b + b >= n2) --b;
  return b;
}

// 1 / sinc^4(pi n_s / N) for the signed index of position i
__device__ __forceinline__ float inv_window4(int i, int nm) {
  const int ns = i < nm / 2 ? i : i - nm;
  if (ns == 0) return 1.0f;
  const float x = (float)ns / (float)nm;
  const float s = sinpif(x) / (3.14159265358979f * x);
  const float s2 = s * s;
  return 1.0f / (s2 * s2);
}

__global__ void __launch_bounds__(kThreads) k_bin_noalloc(const float2* __restrict__ da,
                                                          const float2* __restrict__ db, int nm,
                                                          int nbins, float norm, double kf,
                                                          double* __restrict__ rows) {
  __shared__ double sh[3 * kMaxBins];
  for (int i = threadIdx.x; i < 3 * nbins; i += kThreads) sh[i] = 0.0;
  __syncthreads();
  const int nzc = nm / 2 + 1;
  const float nn3 = (float)nm * (float)nm * (float)nm;
  const float ma = da[0].x / nn3, mb = db[0].x / nn3;
  const float scale = (ma != 0.0f && mb != 0.0f) ? norm / (ma * mb) : 0.0f;
  for (int x = blockIdx.x; x < nm; x += gridDim.x) {
    const int nx = x < nm / 2 ? x : x - nm;
    const float wx = inv_window4(x, nm);
    for (int q = threadIdx.x; q < nm * nzc; q += kThreads) {
      const int y = q / nzc, kz = q % nzc;
      const int ny = y < nm / 2 ? y : y - nm;
      const long long n2 = (long long)nx * nx + (long long)ny * ny + (long long)kz * kz;
      if (n2 == 0) continue;
      const int b = bin_index(n2);
      if (b >= nbins) continue;
      const size_t idx = ((size_t)x * nm + y) * nzc + kz;
      const float2 a = da[idx], c = db[idx];
      const float pk = scale * (a.x * c.x + a.y * c.y) * wx * inv_window4(y, nm) * inv_window4(kz, nm);
      const double w = (kz == 0 || kz == nm / 2) ? 1.0 : 2.0;
      atomicAdd(&sh[b], w);
      atomicAdd(&sh[nbins + b], w * kf * sqrt((double)n2));
      atomicAdd(&sh[2 * nbins + b], w * (double)pk);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * nbins; i += kThreads)
    rows[(size_t)blockIdx.x * 3 * nbins + i] = sh[i];
}

__global__ void k_reduce_noalloc(const double* __restrict__ rows, int nrows, int nbins,
                                 double* __restrict__ k_out, double* __restrict__ P_out,
                                 double* __restrict__ nmodes_out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbins) return;
  double c = 0.0, ks = 0.0, ps = 0.0;
  for (int r = 0; r < nrows; ++r) {
    const double* row = rows + (size_t)r * 3 * nbins;
    c += row[b];
    ks += row[nbins + b];
    ps += row[2 * nbins + b];
  }
  nmodes_out[b] = c;
  k_out[b] = c > 0.0 ? ks / c : 0.0;
  P_out[b] = c > 0.0 ? ps / c : 0.0;
}

// Address of the scratch array on the current device, resolved once per device.
int scratch_on_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PM_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return PM_EINVAL;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_pk_scratch) != cudaSuccess || !p) return PM_ECUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return PM_OK;
}

}  // namespace

extern "C" int pm_power_bin_noalloc(const float* delta_a, const float* delta_b, int32_t nmesh,
                                    double box, int32_t nbins, double* k_out, double* P_out,
                                    double* nmodes_out, void* stream) {
  if (!delta_a || !delta_b || !k_out || !P_out || !nmodes_out) return PM_EINVAL;
  if (nmesh < 32 || nmesh > 2048 || (nmesh & (nmesh - 1))) return PM_EINVAL;
  if (nbins < 1 || nbins > kMaxBins) return PM_EINVAL;
  if (!(box > 0.0)) return PM_EINVAL;
  double* rows = nullptr;
  int rc = scratch_on_current_device(&rows);
  if (rc != PM_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const double nn = (double)nmesh;
  const float norm = (float)(box * box * box / (nn * nn * nn * nn * nn * nn));
  const double kf = 2.0 * 3.14159265358979323846 / box;
  const int grid = nmesh < kRows ? nmesh : kRows;
  // launch errors are peeked, not cleared: an error left by earlier, unrelated work on this
  // thread stays for its owner to read (it is also reported here, as PM_ECUDA)
  k_bin_noalloc<<<grid, kThreads, 0, s>>>(reinterpret_cast<const float2*>(delta_a),
                                          reinterpret_cast<const float2*>(delta_b), nmesh, nbins,
                                          norm, kf, rows);
  if (cudaPeekAtLastError() != cudaSuccess) return PM_ECUDA;
  k_reduce_noalloc<<<(nbins + 127) / 128, 128, 0, s>>>(rows, grid, nbins, k_out, P_out, nmodes_out);
  return cudaPeekAtLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}
