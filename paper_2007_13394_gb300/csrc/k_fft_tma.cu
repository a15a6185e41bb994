// Strided FFT passes (y and x) with TMA-prefetched column tiles.
//
// A persistent CTA walks its share of the column tiles (TK adjacent kz columns of
// one y plane or one x line set).  One thread issues the tensor-memory-accelerator
// copies (cp.async.bulk.tensor.3d) of the tiles one and two ahead (one ahead in the
// two-transform passes) into further shared-memory buffers while the whole CTA
// transforms the current one, so DRAM stays busy during the radix stages.  The tile arrives dense, element (column c, line index i) at
// i * TK + c, which is exactly what the first Stockham stage reads.  Results go
// back to global memory with ordinary coalesced stores.
//
// Variants: plain (y or x), x with the Green's function epilogue, x with the
// -i k_j prologue, the x pass of the potential (forward, Green's function, inverse;
// in place), and the fused x pass of the k-space force (forward, Green's function,
// then IFFT(-i k_x phi) and IFFT(phi) scaled by -i k_y and -i k_z; phi parks in the
// tile's own input buffer, which nothing else touches until the next prefetch).
// In-place passes are safe: a tile's columns are read (by its CTA's prefetch) and
// written (by the same CTA, later) by one CTA only.
//
// Every wait on a copy is bounded: after kSpinLimit polls the CTA records
// PM_ETIMEOUT's bit in the error word, waits (bounded) for its other copies in
// flight, and returns.  pm_test_inject exercises that path: the first CTA then skips
// its first tile's copy (and gives up after a shorter limit).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "fft_engine.cuh"
#include "pm_internal.cuh"

namespace pmnu {

namespace {

using namespace fft;

constexpr int kSpinLimit = 1 << 22;
constexpr int kSpinLimitInjected = 1 << 12;  // a dropped copy (pm_test_inject) gives up sooner

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int limit) {
  for (int i = 0; i < limit; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

// Shared memory.  Single-transform passes (plain, Green's function, gradient): three
// tile buffers (copies run two tiles ahead of the transform), each sized for the
// padded work layout (rounded up to 128 bytes, the alignment of a tensor copy's
// destination) because the Stockham stages run in the buffer of the tile just read.
// Two-transform passes (potential, fused) keep two tile buffers and a separate work
// area: measured with 16 values a thread, where the in-buffer layout meant three CTAs
// at 80 registers, the spills and the extra barrier cost more than the deeper prefetch
// gained; the potential pass is close to issue-bound, so prefetch depth is not its limit.
// values a thread holds: 8 (radix-8 stages, 64 registers, twice the resident warps of
// the 16-value form) from 256-point lines up
template <int LOGM>
constexpr int vpt_tma() {
  return LOGM >= 8 ? 8 : 16;
}

template <int LOGM, int TK, int MODE>
struct TmaShape {
  static constexpr int M = 1 << LOGM;
  static constexpr int V = vpt_tma<LOGM>();
  static constexpr int BOXR = M < 256 ? M : 256;
  static constexpr int NBOX = M / BOXR;
  static constexpr int THREADS = TK * M / V;
  static constexpr uint32_t TILE_BYTES = (uint32_t)M * TK * 8;
  static constexpr size_t WORK_BYTES = (size_t)(M + M / 16 + 1) * TK * 8;
  static constexpr bool WORK_IN_TILE = MODE != MODE_FUSED && MODE != MODE_POT;
  static constexpr int NBUF = WORK_IN_TILE ? 3 : 2;
  static constexpr size_t BUF_BYTES = WORK_IN_TILE ? (WORK_BYTES + 127) / 128 * 128 : (size_t)TILE_BYTES;
  static constexpr size_t SMEM = NBUF * BUF_BYTES + (WORK_IN_TILE ? 0 : WORK_BYTES);
};

// WIN: the Green's function's per-axis window factors are loaded (false: all 1, skipped).
template <int LOGM, int TK, bool INV, int MODE, bool WIN>
__global__ void __launch_bounds__(TmaShape<LOGM, TK, MODE>::THREADS, 2) k_fft_strided_tma(
    const __grid_constant__ CUtensorMap map, float2* __restrict__ d0, float2* __restrict__ d1,
    float2* __restrict__ d2, int axis, int pc, int ntiles_z, int ntiles,
    const float2* __restrict__ tw, KTables kt, int comp, int* __restrict__ err, int drop) {
  using S = TmaShape<LOGM, TK, MODE>;
  constexpr int M = S::M, V = S::V, Q = M / V, NBUF = S::NBUF;
  extern __shared__ __align__(128) unsigned char smraw[];
  auto buf = [&](int b) { return reinterpret_cast<float2*>(smraw + (size_t)b * S::BUF_BYTES); };
  float2* const work_sep = reinterpret_cast<float2*>(smraw + NBUF * S::BUF_BYTES);
  __shared__ __align__(8) uint64_t bars[NBUF];
  __shared__ int fail;
  const int c = threadIdx.x % TK, j = threadIdx.x / TK;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int b = 0; b < NBUF; ++b) mbar_init(&bars[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fail = 0;
  }
  __syncthreads();
  // drop != 0 (a test injection): CTA 0 never issues its first tile's copy, so the wait on
  // it runs out after the short limit and the CTA takes the timeout path below
  const int limit = drop ? kSpinLimitInjected : kSpinLimit;
  auto issue = [&](int tile, int b) {
    if (drop && blockIdx.x == 0 && tile == 0) return;
    const int outer = tile / ntiles_z, kz0 = (tile % ntiles_z) * TK;
    mbar_expect_tx(&bars[b], S::TILE_BYTES);
#pragma unroll
    for (int q = 0; q < S::NBOX; ++q) {
      float2* dst = buf(b) + q * S::BOXR * TK;
      if (axis == 1)
        tma_load_3d(dst, &map, kz0, q * S::BOXR, outer, &bars[b]);
      else
        tma_load_3d(dst, &map, kz0, outer, q * S::BOXR, &bars[b]);
    }
  };
  const long long stride = axis == 1 ? (long long)pc : (long long)M * pc;
  constexpr int NTW = tw_count<M, 1, V>();
  float2 twr[NTW];  // this thread's twiddles, for every tile of the walk
  load_twiddles<M, M, 1, 0, NTW, V>(twr, j, tw);
  uint32_t parity[NBUF];
#pragma unroll
  for (int b = 0; b < NBUF; ++b) parity[b] = 0u;
  int tile = blockIdx.x;
  if (threadIdx.x == 0) {
    for (int q = 0; q < NBUF - 1; ++q)
      if (tile + q * (int)gridDim.x < ntiles) issue(tile + q * (int)gridDim.x, q);
  }
  for (int it = 0; tile < ntiles; tile += gridDim.x, ++it) {
    const int b = it % NBUF;
    const int ahead = tile + (NBUF - 1) * (int)gridDim.x;
    if (threadIdx.x == 0 && ahead < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(ahead, (it + NBUF - 1) % NBUF);  // the buffer released at the end of the last iteration
    }
    if (!mbar_wait_bounded(&bars[b], parity[b], limit)) fail = 1;
    parity[b] ^= 1u;
    __syncthreads();
    if (fail) {
      if (threadIdx.x == 0) {
        atomicOr(err, 2);
        for (int q = 1; q < NBUF; ++q)  // copies still in flight: wait for them (bounded)
          if (tile + q * (int)gridDim.x < ntiles)
            mbar_wait_bounded(&bars[(it + q) % NBUF], parity[(it + q) % NBUF], kSpinLimit);
      }
      return;
    }
    const int outer = tile / ntiles_z;
    const int kz = (tile % ntiles_z) * TK + c;
    const bool ok = kz <= M / 2;
    const long long base = (axis == 1 ? (long long)outer * M * pc : (long long)outer * pc) + kz;
    float2* in = buf(b);
    float2* const work = S::WORK_IN_TILE ? in : work_sep;
    float2 v[V];
#pragma unroll
    for (int s = 0; s < V; ++s) v[s] = in[(j + s * Q) * TK + c];
    if constexpr (S::WORK_IN_TILE) __syncthreads();  // every input read before the stages overwrite it
    if constexpr (MODE == MODE_GRAD) {  // v *= -i k_comp; x pass: element index kx, outer ky
#pragma unroll
      for (int s = 0; s < V; ++s) {
        const int kx = j + s * Q;
        const float kk = comp == 0 ? __ldg(kt.kvec0 + kx)
                                   : (comp == 1 ? __ldg(kt.kvec0 + outer) : (ok ? __ldg(kt.kvec0 + kz) : 0.f));
        v[s] = make_float2(kk * v[s].y, -kk * v[s].x);
      }
    }
    run_stages_reg<M, 1, INV, 0, NTW, V>(v, j, work + c, TK, twr);
    if constexpr (MODE == MODE_GREEN || MODE == MODE_FUSED || MODE == MODE_POT) {
      const float wy = WIN ? __ldg(kt.winv + outer) : 1.0f, ky2 = __ldg(kt.ksq + outer);
      const float wz = !ok ? 0.f : (WIN ? __ldg(kt.winv + kz) : 1.0f), kz2 = ok ? __ldg(kt.ksq + kz) : 0.f;
#pragma unroll
      for (int s = 0; s < V; ++s) {
        const int kx = j + s * Q;
        const float k2 = __ldg(kt.ksq + kx) + ky2 + kz2;
        // fast division (2 ulp), as in the classic passes
        float g = kt.gcoef * (WIN ? __ldg(kt.winv + kx) : 1.0f) * wy * wz / k2;
        if (k2 == 0.0f) g = 0.0f;
        if (kt.mtab && ok) g *= __ldg(kt.mtab + nsq_index<M>(kx, outer, kz));
        v[s] = cscale(v[s], g);
        if constexpr (MODE == MODE_FUSED) {
          in[(j + s * Q) * TK + c] = v[s];               // phi, read back by this thread only
          const float kk = __ldg(kt.kvec0 + kx);
          v[s] = make_float2(kk * v[s].y, -kk * v[s].x);  // -i k_x phi
        }
      }
    }
    if constexpr (MODE == MODE_POT) run_stages_reg<M, 1, true, 0, NTW, V>(v, j, work + c, TK, twr);
    if constexpr (MODE == MODE_FUSED) {
      run_stages_reg<M, 1, true, 0, NTW, V>(v, j, work + c, TK, twr);
      if (ok) {
#pragma unroll
        for (int s = 0; s < V; ++s) d0[base + (long long)(j + s * Q) * stride] = v[s];
      }
#pragma unroll
      for (int s = 0; s < V; ++s) v[s] = in[(j + s * Q) * TK + c];
      run_stages_reg<M, 1, true, 0, NTW, V>(v, j, work + c, TK, twr);
      if (ok) {
        const float ky0 = __ldg(kt.kvec0 + outer), kz0 = __ldg(kt.kvec0 + kz);
#pragma unroll
        for (int s = 0; s < V; ++s) {
          const long long idx = base + (long long)(j + s * Q) * stride;
          d1[idx] = make_float2(ky0 * v[s].y, -ky0 * v[s].x);
          d2[idx] = make_float2(kz0 * v[s].y, -kz0 * v[s].x);
        }
      }
    } else {
      if (ok) {
#pragma unroll
        for (int s = 0; s < V; ++s) d0[base + (long long)(j + s * Q) * stride] = v[s];
      }
    }
    __syncthreads();  // this tile's buffer is free for the copy issued next iteration
  }
}

// columns per tile: TK * M = 4096 points, 8..16 columns
template <int LOGM>
constexpr int tk_tma() {
  return LOGM >= 11 ? 2 : (LOGM == 10 ? 4 : (LOGM == 9 ? 8 : 16));
}

template <int LOGM, bool INV, int MODE>
int launch(pm_ctx* c, const CUtensorMap* map, float2* d0, float2* d1, float2* d2, int axis, int pc,
           const float2* tw, const KTables& kt, int comp, cudaStream_t s) {
  constexpr int TK = tk_tma<LOGM>();
  using SH = TmaShape<LOGM, TK, MODE>;
  constexpr int M = SH::M;
  constexpr bool GREEN = MODE == MODE_GREEN || MODE == MODE_FUSED || MODE == MODE_POT;  // read the window
  const int w = (GREEN && kt.winv) ? 1 : 0;
  auto kern = w ? k_fft_strided_tma<LOGM, TK, INV, MODE, GREEN> : k_fft_strided_tma<LOGM, TK, INV, MODE, false>;
  static int blocks_per_sm[2] = {0, 0};
  if (blocks_per_sm[w] == 0) {
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SH::SMEM) != cudaSuccess)
      return PM_ECUDA;
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, SH::THREADS, SH::SMEM);
    blocks_per_sm[w] = b > 0 ? b : 1;
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const int ntz = (M / 2 + 1 + TK - 1) / TK;
  const int ntiles = M * ntz;
  int grid = sms * blocks_per_sm[w];
  if (grid > ntiles) grid = ntiles;
  const int drop = c->inject == PM_INJECT_DROP_COPY ? 1 : 0;
  c->inject = 0;  // one shot
  kern<<<grid, SH::THREADS, SH::SMEM, s>>>(*map, d0, d1, d2, axis, pc, ntz, ntiles, tw, kt, comp,
                                            c->err_dev, drop);
  return PM_OK;
}

template <bool INV, int MODE>
int dispatch(pm_ctx* c, const Geom& g, const CUtensorMap* map, float2* d0, float2* d1, float2* d2,
             int axis, const float2* tw, const KTables& kt, int comp, cudaStream_t s) {
  switch (g.logn) {
    case 5: return launch<5, INV, MODE>(c, map, d0, d1, d2, axis, g.pc, tw, kt, comp, s);
    case 6: return launch<6, INV, MODE>(c, map, d0, d1, d2, axis, g.pc, tw, kt, comp, s);
    case 7: return launch<7, INV, MODE>(c, map, d0, d1, d2, axis, g.pc, tw, kt, comp, s);
    case 8: return launch<8, INV, MODE>(c, map, d0, d1, d2, axis, g.pc, tw, kt, comp, s);
    case 9: return launch<9, INV, MODE>(c, map, d0, d1, d2, axis, g.pc, tw, kt, comp, s);
    case 10: return launch<10, INV, MODE>(c, map, d0, d1, d2, axis, g.pc, tw, kt, comp, s);
    case 11: return launch<11, INV, MODE>(c, map, d0, d1, d2, axis, g.pc, tw, kt, comp, s);
    default: return PM_EINVAL;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

// Tensor maps of the three force meshes, one per pass direction (box TK x 256 along y
// or along x).  Returns false (and the callers keep the non-TMA kernels) when the
// driver entry point is missing.
bool tma_init(pm_ctx* c) {
  c->tma_ok = false;
  auto enc = encoder();
  if (!enc) return false;
  const Geom& g = c->g;
  const int M = g.n, BOXR = M < 256 ? M : 256;
  int tk = 16;
  if (g.logn >= 11) tk = 2;
  else if (g.logn == 10) tk = 4;
  else if (g.logn == 9) tk = 8;
  float2* bufs[3] = {c->meshA, c->meshB, c->meshC};
  for (int b = 0; b < 3; ++b) {
    for (int axis = 0; axis < 2; ++axis) {  // 0: x pass box, 1: y pass box
      if (!bufs[b]) continue;
      cuuint64_t dims[3] = {(cuuint64_t)(g.n / 2 + 1), (cuuint64_t)g.n, (cuuint64_t)g.n};
      cuuint64_t strides[2] = {(cuuint64_t)g.pc * 8, (cuuint64_t)g.n * g.pc * 8};
      cuuint32_t box[3] = {(cuuint32_t)tk, axis == 1 ? (cuuint32_t)BOXR : 1u,
                           axis == 1 ? 1u : (cuuint32_t)BOXR};
      cuuint32_t es[3] = {1, 1, 1};
      CUresult r = enc(&c->tmap[b][axis], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, bufs[b], dims, strides,
                       box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return false;
    }
  }
  c->tma_ok = true;
  return true;
}

// Index of a force-mesh buffer, or -1.
static int mesh_index(pm_ctx* c, const float2* p) {
  if (p == c->meshA) return 0;
  if (p == c->meshB) return 1;
  if (p == c->meshC && p) return 2;
  return -1;
}

int strided_tma(pm_ctx* c, const Geom& g, const float2* src, float2* d0, float2* d1, float2* d2,
                int axis, bool inv, int mode, int comp, const float2* tw, const fft::KTables& kt,
                cudaStream_t s) {
  using namespace fft;
  if (!c->tma_ok || g.n != c->g.n) return PM_EINVAL;
  // Columns of 1024 or more points only fit 2- or 4-column tiles (16-32 B rows), which the
  // TMA engine serves far below the classic kernels' rate: TMA for up to 512 points.
  if (g.logn >= 10) return PM_EINVAL;
  const int bi = mesh_index(c, src);
  if (bi < 0) return PM_EINVAL;
  const CUtensorMap* map = &c->tmap[bi][axis == 1 ? 1 : 0];
  if (!inv && mode == MODE_PLAIN) return dispatch<false, MODE_PLAIN>(c, g, map, d0, d1, d2, axis, tw, kt, comp, s);
  if (inv && mode == MODE_PLAIN) return dispatch<true, MODE_PLAIN>(c, g, map, d0, d1, d2, axis, tw, kt, comp, s);
  if (!inv && mode == MODE_GREEN) return dispatch<false, MODE_GREEN>(c, g, map, d0, d1, d2, axis, tw, kt, comp, s);
  if (inv && mode == MODE_GRAD) return dispatch<true, MODE_GRAD>(c, g, map, d0, d1, d2, axis, tw, kt, comp, s);
  if (!inv && mode == MODE_FUSED) return dispatch<false, MODE_FUSED>(c, g, map, d0, d1, d2, axis, tw, kt, comp, s);
  if (!inv && mode == MODE_POT) return dispatch<false, MODE_POT>(c, g, map, d0, d1, d2, axis, tw, kt, comp, s);
  return PM_EINVAL;
}

}  // namespace pmnu
