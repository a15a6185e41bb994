// 3D real FFT of the padded mesh, built from three axis passes.
//
// Layout: complex mesh C[x][y][kz], kz in [0, N/2], row pitch P = N/2 + 2 float2
// (the same bytes as a real mesh with row pitch 2P floats, so every pass can run
// in place).  Forward: z pass r2c (rows of N reals -> N/2 + 1 complex), y pass
// c2c, x pass c2c with the Green's function multiply fused into its epilogue
// (written to a second buffer).  Inverse for force component j: x pass with the
// -i k_j multiply fused into its prologue (second buffer -> first), y pass, z
// pass c2r.  The potential (the default force path) runs five passes in place on
// one mesh: z r2c, y, x forward + Green's function + x inverse in one kernel, y
// inverse, z c2r.
//
// Each line of M points is held by M/V threads, V = 16 values each (value s of thread
// j is element j + s M/V); z rows of 1024 and 2048 points use V = 32, so that their
// M = 512 and 1024 complex points take two stages instead of three.  Stockham stages of
// radix V (the last stage radix 2..V) run in registers; between stages the line goes
// through shared memory, padded by one float2 per 16 (per 32 when V = 32) to keep the
// stride-V writes free of bank conflicts.  The first stage reads global memory directly and the last stage
// writes it directly, both coalesced.  Twiddles come from a table e^{-2 pi i t / N}
// computed in double precision on the host.
//
// The strided passes (y, x) put TK adjacent kz columns in one CTA, lane-fastest,
// so each global access covers TK consecutive float2.
#include <cuda_runtime.h>

#include "fft_engine.cuh"
#include "pm_internal.cuh"

namespace pmnu {

namespace {

using namespace fft;

// z-pass CTA size: 128 threads from 1024-point rows up (rows held 32 values a thread,
// four or eight rows a CTA, 128 registers a thread), so that more CTAs in different
// load / transform / store phases share an SM; 256 below (16 values, 64 registers).
template <int LOGN>
constexpr int z_threads() {
  return LOGN >= 10 ? 128 : 256;
}
template <int LOGN>
constexpr int z_min_blocks() {
  return (z_values<LOGN>() >= 32 ? 512 : 1024) / z_threads<LOGN>();
}

// z pass, real -> complex, in place on rows of pitch P float2.
template <int LOGN, int NT = z_threads<LOGN>()>
__global__ void __launch_bounds__(NT, z_min_blocks<LOGN>()) k_fft_z_r2c(float2* __restrict__ data, long long nrows,
                                                                        int pc, const float2* __restrict__ tw) {
  constexpr int N = 1 << LOGN, M = N / 2, V = z_values<LOGN>(), TPL = M / V, LPC = NT / TPL;
  constexpr int LS = z_line<LOGN>();  // line stride in shared memory
  constexpr bool WARP = TPL <= 32;    // a row's threads within one warp: warp barriers suffice
  extern __shared__ float2 sm[];
  const int line = threadIdx.x / TPL, j = threadIdx.x % TPL;
  const long long row = (long long)blockIdx.x * LPC + line;
  z_r2c_row<LOGN, WARP, V>(data + row * pc, row < nrows, j, sm + line * LS, tw);
}

// z pass, complex -> real, in place.
template <int LOGN, int NT = z_threads<LOGN>()>
__global__ void __launch_bounds__(NT, z_min_blocks<LOGN>()) k_fft_z_c2r(float2* __restrict__ data, long long nrows,
                                                                        int pc, const float2* __restrict__ tw) {
  constexpr int N = 1 << LOGN, M = N / 2, V = z_values<LOGN>(), TPL = M / V, LPC = NT / TPL;
  constexpr int LS = z_line<LOGN>();
  constexpr bool WARP = TPL <= 32;  // a row's threads within one warp: warp barriers suffice
  extern __shared__ float2 sm[];
  const int line = threadIdx.x / TPL, j = threadIdx.x % TPL;
  const long long row = (long long)blockIdx.x * LPC + line;
  z_c2r_row<LOGN, WARP, V>(data + row * pc, row < nrows, j, sm + line * LS, tw);
}



// Strided c2c pass along y (axis = 1) or x (axis = 0) for kz columns [kz0, kz0 + TK),
// V values a thread.  MINB CTAs per SM: 1024 threads in all (64 registers a thread) by
// default.
// WIN: the Green's function's per-axis window factors are loaded (false: all 1, skipped).
template <int LOGM, int TK, bool INV, int EPI, int PRO, int V = 16,
          int MINB = 1024 / (TK * (1 << LOGM) / V), bool WIN = true>
__global__ void __launch_bounds__(TK*(1 << LOGM) / V, MINB) k_fft_strided(
    const float2* __restrict__ src, float2* __restrict__ dst, int axis, int pc, int ntiles_z,
    const float2* __restrict__ tw, KTables kt, int comp) {
  constexpr int M = 1 << LOGM, Q = M / V;
  extern __shared__ float2 sm[];
  const int c = threadIdx.x % TK, j = threadIdx.x / TK;
  const int outer = blockIdx.x / ntiles_z;
  const int kz = (blockIdx.x % ntiles_z) * TK + c;
  const bool ok = kz <= M / 2;
  const long long stride = axis == 1 ? (long long)pc : (long long)M * pc;
  const long long base = (axis == 1 ? (long long)outer * M * pc : (long long)outer * pc) + kz;
  float2 v[V];
#pragma unroll
  for (int s = 0; s < V; ++s)
    v[s] = ok ? src[base + (long long)(j + s * Q) * stride] : make_float2(0.f, 0.f);
  if constexpr (PRO == PRO_GRAD) {  // v *= -i k_comp; x pass: element index is kx, outer is ky
#pragma unroll
    for (int s = 0; s < V; ++s) {
      const int kx = j + s * Q;
      const float kk = comp == 0 ? __ldg(kt.kvec0 + kx)
                                 : (comp == 1 ? __ldg(kt.kvec0 + outer) : __ldg(kt.kvec0 + kz));
      v[s] = make_float2(kk * v[s].y, -kk * v[s].x);
    }
  }
  run_stages<M, M, 1, INV, V>(v, j, sm + c, TK, tw);
  if constexpr (EPI == EPI_GREEN || EPI == EPI_POT) {
    const float wy = WIN ? __ldg(kt.winv + outer) : 1.0f, ky2 = __ldg(kt.ksq + outer);
    const float wz = !ok ? 0.f : (WIN ? __ldg(kt.winv + kz) : 1.0f), kz2 = ok ? __ldg(kt.ksq + kz) : 0.f;
    const float kf2 = __ldg(kt.ksq + 1);  // k_F^2
#pragma unroll
    for (int s = 0; s < V; ++s) {
      const int kx = j + s * Q;
      const int nx = kx < M / 2 ? kx : kx - M;  // signed index: k_x^2 = k_F^2 n_x^2, no table load
      const float k2 = kf2 * (float)(nx * nx) + ky2 + kz2;
      // fast division (2 ulp): the IEEE divide's extra instructions and registers cost 15 % of
      // this issue-bound pass at 2048^3, for a 2e-7 relative change of phi_k
      float g = __fdividef(kt.gcoef * (WIN ? __ldg(kt.winv + kx) : 1.0f) * wy * wz, k2);
      if (k2 == 0.0f) g = 0.0f;
      if (kt.mtab && ok) g *= __ldg(kt.mtab + nsq_index<M>(kx, outer, kz));
      v[s] = cscale(v[s], g);
    }
  }
  if constexpr (EPI == EPI_POT) run_stages<M, M, 1, true, V>(v, j, sm + c, TK, tw);
  if (!ok) return;
#pragma unroll
  for (int s = 0; s < V; ++s) dst[base + (long long)(j + s * Q) * stride] = v[s];
}

// Fused x pass of the force: forward x FFT of one column tile, Green's function,
// then the three force components.  k_y and k_z are constant along an x line, so
// IFFT_x(-i k_y phi) = -i k_y IFFT_x(phi) (same for z): two inverse transforms give
// all three components.  Writes component x in place over the input, y and z to
// two further meshes.  phi is parked in shared memory between the inverses.
template <int LOGM, int TK>
__global__ void __launch_bounds__(TK*(1 << LOGM) / 16, 1024 / (TK * (1 << LOGM) / 16)) k_fft_x_fused(
    float2* __restrict__ a, float2* __restrict__ b, float2* __restrict__ cz, int pc, int ntiles_z,
    const float2* __restrict__ tw, KTables kt) {
  constexpr int M = 1 << LOGM, Q = M / 16;
  extern __shared__ float2 sm[];
  float2* work = sm;
  float2* phis = sm + (M + M / 16 + 1) * TK;
  const int c = threadIdx.x % TK, j = threadIdx.x / TK;
  const int outer = blockIdx.x / ntiles_z;                  // ky index
  const int kz = (blockIdx.x % ntiles_z) * TK + c;
  const bool ok = kz <= M / 2;
  const long long stride = (long long)M * pc;
  const long long base = (long long)outer * pc + kz;
  float2 v[16];
#pragma unroll
  for (int s = 0; s < 16; ++s)
    v[s] = ok ? a[base + (long long)(j + s * Q) * stride] : make_float2(0.f, 0.f);
  run_stages<M, M, 1, false>(v, j, work + c, TK, tw);
  {
    const bool win = kt.winv != nullptr;  // null: unit window (no loads)
    const float wy = win ? __ldg(kt.winv + outer) : 1.0f, ky2 = __ldg(kt.ksq + outer);
    const float wz = !ok ? 0.f : (win ? __ldg(kt.winv + kz) : 1.0f), kz2 = ok ? __ldg(kt.ksq + kz) : 0.f;
#pragma unroll
    for (int s = 0; s < 16; ++s) {
      const int kx = j + s * Q;
      const float k2 = __ldg(kt.ksq + kx) + ky2 + kz2;
      float g = kt.gcoef * (win ? __ldg(kt.winv + kx) : 1.0f) * wy * wz / k2;
      if (k2 == 0.0f) g = 0.0f;
      if (kt.mtab && ok) g *= __ldg(kt.mtab + nsq_index<M>(kx, outer, kz));
      v[s] = cscale(v[s], g);
      phis[(j + s * Q) * TK + c] = v[s];                   // read back by this thread only
      const float kk = __ldg(kt.kvec0 + kx);
      v[s] = make_float2(kk * v[s].y, -kk * v[s].x);       // -i k_x phi
    }
  }
  run_stages<M, M, 1, true>(v, j, work + c, TK, tw);
  if (ok) {
#pragma unroll
    for (int s = 0; s < 16; ++s) a[base + (long long)(j + s * Q) * stride] = v[s];
  }
#pragma unroll
  for (int s = 0; s < 16; ++s) v[s] = phis[(j + s * Q) * TK + c];
  run_stages<M, M, 1, true>(v, j, work + c, TK, tw);
  if (!ok) return;
  const float ky0 = __ldg(kt.kvec0 + outer), kz0 = __ldg(kt.kvec0 + kz);
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const long long idx = base + (long long)(j + s * Q) * stride;
    b[idx] = make_float2(ky0 * v[s].y, -ky0 * v[s].x);
    cz[idx] = make_float2(kz0 * v[s].y, -kz0 * v[s].x);
  }
}

template <int LOGM>
constexpr int tk_fused() {
  return LOGM >= 10 ? 4 : (LOGM == 9 ? 8 : 16);
}

template <int LOGM>
void launch_x_fused(float2* a, float2* b, float2* cz, int pc, const float2* tw, const KTables& kt,
                    cudaStream_t s) {
  constexpr int M = 1 << LOGM, TK = tk_fused<LOGM>();
  constexpr int threads = TK * M / 16;
  const int ntz = (M / 2 + 1 + TK - 1) / TK;
  const size_t smem = sizeof(float2) * ((size_t)(M + M / 16 + 1) * TK + (size_t)M * TK);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_fft_x_fused<LOGM, TK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  k_fft_x_fused<LOGM, TK><<<(unsigned)(M * ntz), threads, smem, s>>>(a, b, cz, pc, ntz, tw, kt);
}

// Shape of the classic strided kernel: TK columns a CTA, V values a thread, MINB CTAs per SM.
template <int LOGM, int EPI>
struct StridedShape {
  static constexpr int TK = LOGM >= 10 ? 8 : 16;
  static constexpr int V = 16;
  static constexpr int MINB = 1024 / (TK * (1 << LOGM) / V);
};

template <int LOGM, bool INV, int EPI, int PRO>
void launch_strided(const float2* src, float2* dst, int axis, int pc, const float2* tw,
                    const KTables& kt, int comp, cudaStream_t s) {
  using SS = StridedShape<LOGM, EPI>;
  constexpr int M = 1 << LOGM, TK = SS::TK;
  constexpr int threads = TK * M / SS::V;
  const int ntz = (M / 2 + 1 + TK - 1) / TK;
  const size_t smem = sizeof(float2) * (size_t)(M + M / 16 + 1) * TK;
  constexpr bool GREEN = EPI == EPI_GREEN || EPI == EPI_POT;  // only these read the window
  const int w = (GREEN && kt.winv) ? 1 : 0;
  auto kern = w ? k_fft_strided<LOGM, TK, INV, EPI, PRO, SS::V, SS::MINB, GREEN>
                : k_fft_strided<LOGM, TK, INV, EPI, PRO, SS::V, SS::MINB, false>;
  static bool attr[2] = {false, false};
  if (!attr[w]) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr[w] = true;
  }
  kern<<<(unsigned)(M * ntz), threads, smem, s>>>(src, dst, axis, pc, ntz, tw, kt, comp);
}

template <int LOGN>
void launch_z(float2* data, long long nrows, int pc, const float2* tw, bool inverse, cudaStream_t s) {
  constexpr int kZThreads = z_threads<LOGN>();
  constexpr int N = 1 << LOGN, M = N / 2, TPL = M / z_values<LOGN>(), LPC = kZThreads / TPL;
  constexpr int LS = z_line<LOGN>();
  const size_t smem = sizeof(float2) * (size_t)LS * LPC;
  unsigned grid = (unsigned)((nrows + LPC - 1) / LPC);
  if (inverse) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_fft_z_c2r<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      attr = true;
    }
    k_fft_z_c2r<LOGN><<<grid, kZThreads, smem, s>>>(data, nrows, pc, tw);
  } else {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_fft_z_r2c<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      attr = true;
    }
    k_fft_z_r2c<LOGN><<<grid, kZThreads, smem, s>>>(data, nrows, pc, tw);
  }
}

void dispatch_z(const Geom& g, float2* data, const float2* tw, bool inverse, cudaStream_t s) {
  switch (g.logn) {
    case 5: launch_z<5>(data, g.rows(), g.pc, tw, inverse, s); break;
    case 6: launch_z<6>(data, g.rows(), g.pc, tw, inverse, s); break;
    case 7: launch_z<7>(data, g.rows(), g.pc, tw, inverse, s); break;
    case 8: launch_z<8>(data, g.rows(), g.pc, tw, inverse, s); break;
    case 9: launch_z<9>(data, g.rows(), g.pc, tw, inverse, s); break;
    case 10: launch_z<10>(data, g.rows(), g.pc, tw, inverse, s); break;
    case 11: launch_z<11>(data, g.rows(), g.pc, tw, inverse, s); break;
    default: break;
  }
}

template <bool INV, int EPI, int PRO>
void dispatch_strided(const Geom& g, const float2* src, float2* dst, int axis, const float2* tw,
                      const KTables& kt, int comp, cudaStream_t s) {
  switch (g.logn) {
    case 5: launch_strided<5, INV, EPI, PRO>(src, dst, axis, g.pc, tw, kt, comp, s); break;
    case 6: launch_strided<6, INV, EPI, PRO>(src, dst, axis, g.pc, tw, kt, comp, s); break;
    case 7: launch_strided<7, INV, EPI, PRO>(src, dst, axis, g.pc, tw, kt, comp, s); break;
    case 8: launch_strided<8, INV, EPI, PRO>(src, dst, axis, g.pc, tw, kt, comp, s); break;
    case 9: launch_strided<9, INV, EPI, PRO>(src, dst, axis, g.pc, tw, kt, comp, s); break;
    case 10: launch_strided<10, INV, EPI, PRO>(src, dst, axis, g.pc, tw, kt, comp, s); break;
    case 11: launch_strided<11, INV, EPI, PRO>(src, dst, axis, g.pc, tw, kt, comp, s); break;
    default: break;
  }
}

// Strided pass: the TMA-pipelined kernel when it applies, else the classic one.
template <bool INV, int EPI, int PRO>
void strided(pm_ctx* c, const Geom& g, const float2* src, float2* dst, int axis, const float2* tw,
             const KTables& kt, int comp, cudaStream_t s) {
  const int mode = EPI == EPI_GREEN ? MODE_GREEN
                   : EPI == EPI_POT  ? MODE_POT
                                     : (PRO == PRO_GRAD ? MODE_GRAD : MODE_PLAIN);
  if (strided_tma(c, g, src, dst, nullptr, nullptr, axis, INV, mode, comp, tw, kt, s) == PM_OK) return;
  dispatch_strided<INV, EPI, PRO>(g, src, dst, axis, tw, kt, comp, s);
}

KTables ktables(pm_ctx* c, const Geom& g) {
  KTables kt;
  kt.ksq = c->ksq;
  // the per-axis window factors of the Green's function: all 1 for the default kernel,
  // where the passes skip them (null), 1 / sinc^4 for the deconvolved spectral one
  kt.winv = (c->cfg.flags & PM_FLAG_SPECTRAL_KERNEL) ? c->wforce : nullptr;
  kt.kvec0 = c->kvec0;
  double nn = (double)g.n;
  kt.gcoef = (float)(-1.5 * c->cosmo.omega_m0 / (nn * nn * nn));
  kt.mtab = (c->mlp_on && g.n == c->g.n) ? c->mlp_tab : nullptr;
  return kt;
}

}  // namespace

void fft_forward(pm_ctx* c, const Geom& g, float2* buf, float2* dst, int green, cudaStream_t s) {
  const float2* tw = twiddles(c, g.n);
  KTables kt = ktables(c, g);
  {
    LaunchScope L(c, s, K_FFT_Z_R2C);
    dispatch_z(g, buf, tw, false, s);
  }
  {
    LaunchScope L(c, s, K_FFT_Y);
    strided<false, EPI_NONE, PRO_NONE>(c, g, buf, buf, 1, tw, kt, 0, s);
  }
  if (green) {
    LaunchScope L(c, s, K_FFT_X_GREEN);
    strided<false, EPI_GREEN, PRO_NONE>(c, g, buf, dst, 0, tw, kt, 0, s);
  } else {
    LaunchScope L(c, s, K_FFT_X_PLAIN);
    strided<false, EPI_NONE, PRO_NONE>(c, g, buf, dst, 0, tw, kt, 0, s);
  }
}

void fft_inverse_component(pm_ctx* c, const Geom& g, const float2* phi, float2* buf, int comp,
                           cudaStream_t s) {
  const float2* tw = twiddles(c, g.n);
  KTables kt = ktables(c, g);
  {
    LaunchScope L(c, s, K_FFT_X_GRAD);
    strided<true, EPI_NONE, PRO_GRAD>(c, g, phi, buf, 0, tw, kt, comp, s);
  }
  {
    LaunchScope L(c, s, K_FFT_Y);
    strided<true, EPI_NONE, PRO_NONE>(c, g, buf, buf, 1, tw, kt, 0, s);
  }
  {
    LaunchScope L(c, s, K_FFT_Z_C2R);
    dispatch_z(g, buf, tw, true, s);
  }
}

void fft_force_fused(pm_ctx* c, const Geom& g, float2* a, float2* b, float2* cz, cudaStream_t s) {
  const float2* tw = twiddles(c, g.n);
  KTables kt = ktables(c, g);
  {
    LaunchScope L(c, s, K_FFT_Z_R2C);
    dispatch_z(g, a, tw, false, s);
  }
  {
    LaunchScope L(c, s, K_FFT_Y);
    strided<false, EPI_NONE, PRO_NONE>(c, g, a, a, 1, tw, kt, 0, s);
  }
  {
    LaunchScope L(c, s, K_FFT_X_FUSED);
    if (strided_tma(c, g, a, a, b, cz, 0, false, MODE_FUSED, 0, tw, kt, s) == PM_OK) goto fused_done;
    switch (g.logn) {
      case 5: launch_x_fused<5>(a, b, cz, g.pc, tw, kt, s); break;
      case 6: launch_x_fused<6>(a, b, cz, g.pc, tw, kt, s); break;
      case 7: launch_x_fused<7>(a, b, cz, g.pc, tw, kt, s); break;
      case 8: launch_x_fused<8>(a, b, cz, g.pc, tw, kt, s); break;
      case 9: launch_x_fused<9>(a, b, cz, g.pc, tw, kt, s); break;
      case 10: launch_x_fused<10>(a, b, cz, g.pc, tw, kt, s); break;
      case 11: launch_x_fused<11>(a, b, cz, g.pc, tw, kt, s); break;
      default: break;
    }
  fused_done:;
  }
  float2* bufs[3] = {a, b, cz};
  for (int comp = 0; comp < 3; ++comp) {
    {
      LaunchScope L(c, s, K_FFT_Y);
      strided<true, EPI_NONE, PRO_NONE>(c, g, bufs[comp], bufs[comp], 1, tw, kt, 0, s);
    }
    {
      LaunchScope L(c, s, K_FFT_Z_C2R);
      dispatch_z(g, bufs[comp], tw, true, s);
    }
  }
}

void fft_potential(pm_ctx* c, const Geom& g, float2* buf, cudaStream_t s) {
  const float2* tw = twiddles(c, g.n);
  KTables kt = ktables(c, g);
  {
    LaunchScope L(c, s, K_FFT_Z_R2C);
    dispatch_z(g, buf, tw, false, s);
  }
  {
    LaunchScope L(c, s, K_FFT_Y);
    strided<false, EPI_NONE, PRO_NONE>(c, g, buf, buf, 1, tw, kt, 0, s);
  }
  {
    LaunchScope L(c, s, K_FFT_X_POT);
    strided<false, EPI_POT, PRO_NONE>(c, g, buf, buf, 0, tw, kt, 0, s);
  }
  {
    LaunchScope L(c, s, K_FFT_Y);
    strided<true, EPI_NONE, PRO_NONE>(c, g, buf, buf, 1, tw, kt, 0, s);
  }
  {
    LaunchScope L(c, s, K_FFT_Z_C2R);
    dispatch_z(g, buf, tw, true, s);
  }
}

void fft_inverse_plain(pm_ctx* c, const Geom& g, float2* buf, cudaStream_t s) {
  const float2* tw = twiddles(c, g.n);
  KTables kt = ktables(c, g);
  {
    LaunchScope L(c, s, K_FFT_X_PLAIN);
    strided<true, EPI_NONE, PRO_NONE>(c, g, buf, buf, 0, tw, kt, 0, s);
  }
  {
    LaunchScope L(c, s, K_FFT_Y);
    strided<true, EPI_NONE, PRO_NONE>(c, g, buf, buf, 1, tw, kt, 0, s);
  }
  {
    LaunchScope L(c, s, K_FFT_Z_C2R);
    dispatch_z(g, buf, tw, true, s);
  }
}

}  // namespace pmnu
