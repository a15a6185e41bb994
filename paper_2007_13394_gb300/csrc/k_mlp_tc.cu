// Tensor-core (tcgen05, BF16 operands, FP32 accumulation) form of the learned factor's
// table m(sqrt(s) / (N/2), a) = 1 + MLP: the hidden 64 x 64 layer of 128 table entries
// is one M = 128, N = 64, K = 64 matrix product, D = H1 W2^T.
//
// One CTA of 128 threads (4 warps) per 128 entries:
//   1. thread r computes h1 = SiLU(W1 (kappa_r, a) + b1) in FP32 and stores it as BF16
//      row r of A in shared memory; W2 (row = output unit) is B, also BF16.  Both use
//      the canonical K-major layout without swizzle: 8-row x 16-byte core matrices,
//      the 8 K-groups of a row block adjacent (leading-dimension byte offset 128), row
//      blocks 1024 bytes apart (stride-dimension byte offset).
//   2. warp 0 allocates 64 TMEM columns; thread 0 issues four tcgen05.mma (K = 16
//      each) into them and commits to an mbarrier that every thread waits on (bounded:
//      on time-out the CTA flags PM_ETIMEOUT in the error word and writes nothing).
//   3. warp w reads TMEM lanes 32 w .. 32 w + 31 (its row per thread, 64 FP32 columns)
//      with tcgen05.ld, adds b2, applies SiLU, dots with w3, adds b3 and 1.
// Used when the context's flags ask for it (PM_FLAG_MLP_TENSOR); the FP32 table stays
// the default (tighter: BF16 rounding of h1 and W2 costs ~3 significant digits).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "pm_internal.cuh"

namespace pmnu {

namespace {

constexpr int H = PM_MLP_HIDDEN;  // 64 = N = K
constexpr int NP = PM_MLP_NPARAM;
constexpr int OW1 = 0, OB1 = 2 * H, OW2 = 3 * H, OB2 = 3 * H + H * H, OW3 = 4 * H + H * H,
              OB3 = 5 * H + H * H;
constexpr int TM = 128;              // entries (rows of A) per CTA
constexpr int kThreads = 128;
constexpr int kTmemCols = 64;        // FP32 accumulator columns (N)
constexpr int kSpin = 1 << 22;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) of a K-major, no-swizzle operand with K = 64 bf16
__device__ __forceinline__ int kmajor_offset(int row, int k) {
  return (row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// sm_100 shared-memory matrix descriptor: start >> 4 (bits 0-13), leading-dimension
// byte offset >> 4 (16-29), stride-dimension byte offset >> 4 (32-45), version 1
// (46-47), base offset 0, no swizzle (61-63 = 0)
__device__ __forceinline__ uint64_t smem_desc(uint32_t start, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((start >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (7-9 = 1,
// 10-12 = 1), both K-major (15, 16 = 0), N >> 3 (17-22), M >> 4 (24-28)
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(H >> 3) << 17) |
                            ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + expf(-z)); }

__global__ void __launch_bounds__(kThreads) k_mlp_table_tc(const float* __restrict__ theta, float a,
                                                           float inv_half, int64_t ntab,
                                                           float* __restrict__ tab, int* __restrict__ err) {
  __shared__ __align__(1024) unsigned char sa[TM * H * 2];  // A: 16 KB
  __shared__ __align__(1024) unsigned char sb[H * H * 2];   // B: 8 KB
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ float th[NP + 3];
  __shared__ int timed_out;
  const int t = threadIdx.x, w = t >> 5;
  for (int i = t; i < NP; i += kThreads) th[i] = theta[i];
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    timed_out = 0;
  }
  if (w == 0) {  // 64 TMEM columns for the accumulator
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  // B = W2 in BF16 (row n = output unit, k = input unit)
  for (int i = t; i < H * H; i += kThreads) {
    const int n = i / H, k = i % H;
    *reinterpret_cast<__nv_bfloat16*>(sb + kmajor_offset(n, k)) = __float2bfloat16_rn(th[OW2 + n * H + k]);
  }
  // A row t = h1 of entry e0 + t
  const int64_t e = (int64_t)blockIdx.x * TM + t;
  const float kappa = sqrtf((float)e) * inv_half;
#pragma unroll 8
  for (int k = 0; k < H; ++k) {
    const float z = fmaf(th[OW1 + 2 * k], kappa, fmaf(th[OW1 + 2 * k + 1], a, th[OB1 + k]));
    *reinterpret_cast<__nv_bfloat16*>(sa + kmajor_offset(t, k)) = __float2bfloat16_rn(z * sigm(z));
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor core
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (t == 0) {
#pragma unroll
    for (int kk = 0; kk < H / 16; ++kk) {  // K = 16 per instruction: two core matrices along K
      const uint64_t da = smem_desc(saddr(sa) + kk * 256, 128, 1024);
      const uint64_t db = smem_desc(saddr(sb) + kk * 256, 128, 1024);
      const uint32_t acc = kk > 0 ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
          "l"(da), "l"(db), "r"(kIdesc), "r"(acc)
          : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(&bar))
                 : "memory");
  }
  // bounded wait for the products (phase 0)
  bool done = false;
  for (int i = 0; i < kSpin && !done; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(&bar))
        : "memory");
    done = ok != 0;
  }
  if (!done) timed_out = 1;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncthreads();
  if (!timed_out) {
    // warp w: TMEM lanes 32 w + lane (its rows), columns 0..63 in four loads of 16
    float out = th[OB3];
#pragma unroll
    for (int c0 = 0; c0 < H; c0 += 16) {
      uint32_t r[16];
      const uint32_t addr = tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
          "%12, %13, %14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
            "=r"(r[15])
          : "r"(addr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float z = __uint_as_float(r[j]) + th[OB2 + c0 + j];
        out = fmaf(th[OW3 + c0 + j], z * sigm(z), out);
      }
    }
    if (e < ntab) tab[e] = 1.0f + out;
  } else if (t == 0) {
    atomicOr(err, 2);  // the ETIMEOUT bit of the error word
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (w == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

void mlp_table_tc(pm_ctx* c, double a, cudaStream_t s) {
  LaunchScope L(c, s, K_MLP_TABLE);
  const unsigned grid = (unsigned)((c->mlp_ntab + TM - 1) / TM);
  k_mlp_table_tc<<<grid, kThreads, 0, s>>>(c->mlp_theta, (float)a, 2.0f / (float)c->g.n, c->mlp_ntab, c->mlp_tab,
                                            c->err_dev);
}

}  // namespace pmnu
