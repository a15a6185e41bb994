// Adjoint (vector-Jacobian products) of the particle-mesh step, for gradients of a
// final-field loss with respect to the initial modes (reconstruction).
//
// * CIC readout gradient: d/dx sum_c W(x - c) M(c), with dw/dx = -+1/H per axis.
// * Paint transpose = readout; readout transpose = paint of per-particle weights
//   (the deterministic tile paint with signed weights).
// * Force VJP for a cotangent lambda_F (F_j = R[G_j rho], G_j real with an odd
//   kernel so G_j^T = -G_j):
//     dL/dx_i = sum_j lambda_F,ij grad R[G_j rho](x_i) + m_i grad R[B](x_i),
//     B_k = sum_j i D(k_j) g(k) FFT(paint(lambda_F,j))_k, D the gradient kernel.
//   With the 4-point kernel (and no learned factor) both terms run on one potential
//   mesh at a time: G_j rho = -S_j phi, and B = G * (sum_j S_j paint(lambda_F,j)).
// * KDK step VJP (p_h = p0 + K1 F(x0), x1 = x0 + Delta p_h, p1 = p_h + K2 F(x1)).
// * Zel'dovich IC transpose: s_j = T_j omega with T_j = IFFT diag(S_j) FFT, so
//   dL/domega = IFFT(sum_j conj(S_j) FFT(lambda_s,j)), neutrino sites with the
//   conjugate phase.
// Cotangent arrays at the C-ABI are indexed by canonical particle id.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "pm_internal.cuh"

namespace pmnu {

namespace {

// out[d][perm[i]] (+)= sum_j a_j(i) d/dx_d R[M_j](x_i) for the sorted particle i.
// a_j(i) = wts[j * n + i] when wts is set, else the particle's mass.
__global__ void k_readout_grad(const uint32_t* __restrict__ us, const uint32_t* __restrict__ ids,
                               int64_t n, const float* __restrict__ m0, const float* __restrict__ m1,
                               const float* __restrict__ m2, int nmesh_used, int nm, int shift,
                               int row_pitch, float inv_h, const float* __restrict__ wts, MassTable mt,
                               const uint32_t* __restrict__ perm, float* __restrict__ out,
                               int accumulate, int species) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t ux = us[i], uy = us[n + i], uz = us[2 * n + i];
  const float fscale = 1.0f / (float)(1u << shift);
  const uint32_t fmask = (1u << shift) - 1u;
  const int cx = ux >> shift, cy = uy >> shift, cz = uz >> shift;
  const int cx1 = (cx + 1) & (nm - 1), cy1 = (cy + 1) & (nm - 1), cz1 = (cz + 1) & (nm - 1);
  const float fx = (float)(ux & fmask) * fscale, fy = (float)(uy & fmask) * fscale,
              fz = (float)(uz & fmask) * fscale;
  const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
  const size_t r00 = ((size_t)cx * nm + cy) * row_pitch, r01 = ((size_t)cx * nm + cy1) * row_pitch;
  const size_t r10 = ((size_t)cx1 * nm + cy) * row_pitch, r11 = ((size_t)cx1 * nm + cy1) * row_pitch;
  const float* ms[3] = {m0, m1, m2};
  bool bad = false;
  const float mass = wts ? 0.0f : id_mass(mt, ids[i], species, &bad);
  float o[3] = {0.f, 0.f, 0.f};
  for (int j = 0; j < nmesh_used; ++j) {
    const float* M = ms[j];
    const float a = wts ? wts[(int64_t)j * n + i] : mass;
    if (a == 0.0f) continue;
    const float v000 = __ldg(M + r00 + cz), v001 = __ldg(M + r00 + cz1);
    const float v010 = __ldg(M + r01 + cz), v011 = __ldg(M + r01 + cz1);
    const float v100 = __ldg(M + r10 + cz), v101 = __ldg(M + r10 + cz1);
    const float v110 = __ldg(M + r11 + cz), v111 = __ldg(M + r11 + cz1);
    // d/dx: (x1 plane - x0 plane) weighted in y, z; likewise for y and z
    const float dX = gy * (gz * (v100 - v000) + fz * (v101 - v001)) +
                     fy * (gz * (v110 - v010) + fz * (v111 - v011));
    const float dY = gx * (gz * (v010 - v000) + fz * (v011 - v001)) +
                     fx * (gz * (v110 - v100) + fz * (v111 - v101));
    const float dZ = gx * (gy * (v001 - v000) + fy * (v011 - v010)) +
                     fx * (gy * (v101 - v100) + fy * (v111 - v110));
    o[0] += a * dX;
    o[1] += a * dY;
    o[2] += a * dZ;
  }
  const int64_t dst = perm ? (int64_t)perm[i] : i;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float v = o[d] * inv_h;
    if (accumulate)
      out[(int64_t)d * n + dst] += v;
    else
      out[(int64_t)d * n + dst] = v;
  }
}

// B_k (+)= i D(k_j) g(k) m(k) A_k on the half spectrum (padded pitch pc), the transpose
// of -G_j (D the gradient kernel); m = 1 without the learned factor.  With rho (the
// density's half spectrum) it also bins d <lambda_F, F> / d m(k) =
// Re[(-i D(k_j)) g rho_k conj(A_k)] (twice for 0 < k_z < N/2) by s = |n|^2 into gbin.
__global__ void k_adj_combine(const float2* __restrict__ a, float2* __restrict__ b, int nm, int pc,
                              const float* __restrict__ ksq, const float* __restrict__ winv,
                              const float* __restrict__ kvec0, float gcoef, int comp, int accumulate,
                              const float* __restrict__ mtab, const float2* __restrict__ rho,
                              double* __restrict__ gbin) {
  const int x = blockIdx.x / nm, y = blockIdx.x % nm;
  const int nx = x < nm / 2 ? x : x - nm, ny = y < nm / 2 ? y : y - nm;
  for (int kz = threadIdx.x; kz <= nm / 2; kz += blockDim.x) {
    const size_t idx = ((size_t)x * nm + y) * pc + kz;
    const int sidx = nx * nx + ny * ny + kz * kz;
    const float k2 = ksq[x] + ksq[y] + ksq[kz];
    float g = gcoef * winv[x] * winv[y] * winv[kz] / k2;
    if (k2 == 0.0f) g = 0.0f;
    const float kj = comp == 0 ? kvec0[x] : (comp == 1 ? kvec0[y] : kvec0[kz]);
    const float2 v = a[idx];
    if (rho) {
      const float2 r = rho[idx];
      const float mult = (kz > 0 && kz < nm / 2) ? 2.0f : 1.0f;
      const float q = mult * kj * g * (r.y * v.x - r.x * v.y);
      if (q != 0.0f) atomicAdd(gbin + sidx, (double)q);
    }
    const float s = kj * (mtab ? g * mtab[sidx] : g);
    const float2 r = make_float2(-s * v.y, s * v.x);  // i s v
    if (accumulate) {
      float2 o = b[idx];
      b[idx] = make_float2(o.x + r.x, o.y + r.y);
    } else {
      b[idx] = r;
    }
  }
}

// ---- one-mesh force VJP (4-point kernel): the forward force is F_j = -S_j phi with S_j
// the 4-point stencil along axis j (transfer function i D(k_j)), so
//   term 1: sum_j lambda_j grad R[F_j] from the potential staged per tile, and
//   term 2: B = G * (sum_j S_j paint(lambda_j)) (IFFT[g sum_j i D(k_j) FFT(paint_j)]).
constexpr int kVjpThreads = 256;
constexpr int kVjpSpanXY = kTile + 5;  // cells -2 .. 18 along x and y
constexpr int kVjpSpanZ = kTile + 8;   // cells -4 .. 19 along z (16-byte aligned rows)
constexpr int kVjpChunksZ = kVjpSpanZ / 4;
constexpr int kVjpStage = kVjpSpanXY * kVjpSpanXY * kVjpChunksZ;
constexpr int kVjpSY = kVjpSpanZ, kVjpSX = kVjpSpanXY * kVjpSpanZ;

__device__ __forceinline__ void vjp_cp_async16(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gmem_src)
               : "memory");
}

// out[d][perm[i]] = sum_j lambda_j(i) d/dx_d R[F_j](x_i), F_j = -S_j phi, one CTA per
// tile: the tile's potential with the stencil halo staged like the forward readout's,
// F_j at the particle's 8 CIC corners from the 56 values, then the CIC weight
// derivatives (the pattern of k_readout_grad).
__global__ void __launch_bounds__(kVjpThreads) k_readout_grad_fd4(
    const uint32_t* __restrict__ us, int64_t n, const uint32_t* __restrict__ bstart,
    const float* __restrict__ phi, int nm, int shift, int ntl, int row_pitch, float inv12h, float inv_h,
    const float* __restrict__ lam, const uint32_t* __restrict__ perm, float* __restrict__ out,
    int* __restrict__ err) {
  __shared__ __align__(16) float sp[kVjpSpanXY * kVjpSpanXY * kVjpSpanZ];
  const int t = threadIdx.x;
  const uint32_t tile = blockIdx.x;
  const uint32_t lo = bstart[8 * tile], hi = bstart[8 * tile + 8];
  if (lo == hi) return;
  const int nt = 1 << ntl;
  const int ox = (int)(tile >> (2 * ntl)) * kTile, oy = (int)((tile >> ntl) & (nt - 1)) * kTile,
            oz = (int)(tile & (nt - 1)) * kTile;
  const int wrap = nm - 1;
  for (int c = t; c < kVjpStage; c += kVjpThreads) {
    const int x = c / (kVjpSpanXY * kVjpChunksZ), r = c - x * (kVjpSpanXY * kVjpChunksZ);
    const int y = r / kVjpChunksZ, k = r - y * kVjpChunksZ;
    const int gx = (ox + x - 2) & wrap, gy = (oy + y - 2) & wrap, gz = (oz - 4 + 4 * k) & wrap;
    vjp_cp_async16(sp + x * kVjpSX + y * kVjpSY + 4 * k, phi + ((size_t)gx * nm + gy) * (size_t)row_pitch + gz);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const float fscale = 1.0f / (float)(1u << shift);
  const uint32_t fmask = (1u << shift) - 1u;
  bool bad = false;
  for (uint32_t i = lo + t; i < hi; i += kVjpThreads) {
    const uint32_t ux = us[i], uy = us[n + i], uz = us[2 * n + i];
    const int lx = (int)(ux >> shift) - ox, ly = (int)(uy >> shift) - oy, lz = (int)(uz >> shift) - oz;
    if ((unsigned)lx >= (unsigned)kTile || (unsigned)ly >= (unsigned)kTile || (unsigned)lz >= (unsigned)kTile) {
      bad = true;
      continue;
    }
    const float fx = (float)(ux & fmask) * fscale, fy = (float)(uy & fmask) * fscale,
                fz = (float)(uz & fmask) * fscale;
    const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
    const float* q = sp + (lx + 2) * kVjpSX + (ly + 2) * kVjpSY + (lz + 4);
    // F_j at corner (a, b, c) of the cell, Fj[a][b][c] = -S_j phi / ... (scaled below)
    float Fx[2][2][2], Fy[2][2][2], Fz[2][2][2];
    auto line = [](const float* q0, int S, float& c0, float& c1) {  // stencil sums at corners 0, 1
      const float m2 = q0[-2 * S], m1 = q0[-S], p0 = q0[0], p1 = q0[S], p2 = q0[2 * S], p3 = q0[3 * S];
      c0 = 8.0f * (p1 - m1) - (p2 - m2);
      c1 = 8.0f * (p2 - p0) - (p3 - m1);
    };
#pragma unroll
    for (int a = 0; a < 2; ++a) {
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        line(q + a * kVjpSY + b, kVjpSX, Fx[0][a][b], Fx[1][a][b]);  // x line at (y, z) = (a, b)
        line(q + a * kVjpSX + b, kVjpSY, Fy[a][0][b], Fy[a][1][b]);  // y line at (x, z) = (a, b)
        line(q + a * kVjpSX + b * kVjpSY, 1, Fz[a][b][0], Fz[a][b][1]);  // z line at (x, y) = (a, b)
      }
    }
    const float l0 = lam[i], l1 = lam[n + i], l2 = lam[2 * n + i];
    float o[3] = {0.f, 0.f, 0.f};
    const float (*Fs[3])[2][2] = {Fx, Fy, Fz};
    const float ls[3] = {l0, l1, l2};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const float (*v)[2][2] = Fs[j];
      const float dX = gy * (gz * (v[1][0][0] - v[0][0][0]) + fz * (v[1][0][1] - v[0][0][1])) +
                       fy * (gz * (v[1][1][0] - v[0][1][0]) + fz * (v[1][1][1] - v[0][1][1]));
      const float dY = gx * (gz * (v[0][1][0] - v[0][0][0]) + fz * (v[0][1][1] - v[0][0][1])) +
                       fx * (gz * (v[1][1][0] - v[1][0][0]) + fz * (v[1][1][1] - v[1][0][1]));
      const float dZ = gx * (gy * (v[0][0][1] - v[0][0][0]) + fy * (v[0][1][1] - v[0][1][0])) +
                       fx * (gy * (v[1][0][1] - v[1][0][0]) + fy * (v[1][1][1] - v[1][1][0]));
      o[0] += ls[j] * dX;
      o[1] += ls[j] * dY;
      o[2] += ls[j] * dZ;
    }
    const int64_t dst = perm ? (int64_t)perm[i] : (int64_t)i;
    const float scale = -inv12h * inv_h;  // F_j = -(stencil sum) / (12 H); d/dx: 1 / H
#pragma unroll
    for (int d = 0; d < 3; ++d) out[(int64_t)d * n + dst] = scale * o[d];
  }
  if (bad) atomicOr(err, 1);
}

// B (+)= S_j A on real meshes (row pitch rp): the 4-point stencil along axis j, periodic.
__global__ void k_stencil_axis(const float* __restrict__ A, float* __restrict__ B, int nm, int rp, int axis,
                               float inv12h, int accumulate) {
  const int x = blockIdx.x / nm, y = blockIdx.x % nm;
  const int w = nm - 1;
  const size_t row = ((size_t)x * nm + y) * rp;
  for (int z = threadIdx.x; z < nm; z += blockDim.x) {
    auto at = [&](int o) -> float {  // A at offset o along the axis
      if (axis == 0) return __ldg(A + ((size_t)((x + o) & w) * nm + y) * rp + z);
      if (axis == 1) return __ldg(A + ((size_t)x * nm + ((y + o) & w)) * rp + z);
      return __ldg(A + row + ((z + o) & w));
    };
    const float v = inv12h * (8.0f * (at(1) - at(-1)) - (at(2) - at(-2)));
    B[row + z] = accumulate ? B[row + z] + v : v;
  }
}

// u1 = u0 + rne(Delta (p0 + K1 f0) 2^32 / L), p_h = p0 + K1 f0 (no sort keys)
__global__ void k_drift_only(const uint32_t* __restrict__ u0, const float* __restrict__ p0,
                             const float* __restrict__ f0, int64_t n, float K1, float dscale,
                             uint32_t* __restrict__ u1) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float ph = p0[d * n + i] + K1 * f0[d * n + i];
    const long long step = __float2ll_rn(dscale * ph);
    u1[d * n + i] = u0[d * n + i] + (uint32_t)(unsigned long long)step;
  }
}

// dst[d][i] = src[d][id[i]] (canonical -> state order) or dst[d][id[i]] = src[d][i]
__global__ void k_by_id(const float* __restrict__ src, float* __restrict__ dst,
                        const uint32_t* __restrict__ id, int64_t n, int to_canonical, float scale) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t j = id ? (int64_t)id[i] : i;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (to_canonical)
      dst[d * n + j] = scale * src[d * n + i];
    else
      dst[d * n + i] = scale * src[d * n + j];
  }
}

// y = a x + b y over 3n
__global__ void k_axpby(const float* __restrict__ x, float* __restrict__ y, int64_t m, float a, float b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) y[i] = a * x[i] + b * y[i];
}

// gather per-component weights into the sorted order: ws[j][k] = w[j][perm[k]]
__global__ void k_gather3(const float* __restrict__ w, const uint32_t* __restrict__ perm, int64_t n,
                          int ncomp, float* __restrict__ ws) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const uint32_t i = perm[k];
  for (int j = 0; j < ncomp; ++j) ws[(int64_t)j * n + k] = w[(int64_t)j * n + i];
}

// IC transpose: lattice mesh (padded real, nc) of lambda_s for CDM nodes (canonical order)
__global__ void k_icadj_cdm(const float* __restrict__ lx, const float* __restrict__ lp, int nc,
                            int rp, int comp, float D0, float gp0, int64_t n_total,
                            float* __restrict__ mesh) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ncell = (int64_t)nc * nc * nc;
  if (i >= ncell) return;
  const int ix = (int)(i / ((int64_t)nc * nc)), iy = (int)((i / nc) % nc), iz = (int)(i % nc);
  mesh[((size_t)ix * nc + iy) * rp + iz] =
      D0 * lx[comp * n_total + i] + gp0 * lp[comp * n_total + i];
}

// neutrino sites: sum of lambda_s over the site's shell x direction particles
__global__ void k_icadj_nu(const float* __restrict__ lx, const float* __restrict__ lp, int nc,
                           int rp, int comp, float D0, float gp0, int nsites, int stride, int j0,
                           int per_site, int64_t n_offset, int64_t n_total, float* __restrict__ mesh) {
  const int64_t site = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nsite3 = (int64_t)nsites * nsites * nsites;
  if (site >= nsite3) return;
  float s = 0.f;
  for (int q = 0; q < per_site; ++q) {
    const int64_t i = n_offset + site * per_site + q;
    s += D0 * lx[comp * n_total + i] + gp0 * lp[comp * n_total + i];
  }
  const int sx = (int)(site / ((int64_t)nsites * nsites)), sy = (int)((site / nsites) % nsites),
            sz = (int)(site % nsites);
  const int ix = (j0 + stride * sx) % nc, iy = (j0 + stride * sy) % nc, iz = (j0 + stride * sz) % nc;
  mesh[((size_t)ix * nc + iy) * rp + iz] = s;
}

// K (+)= conj(S_j) A_k with S_j = i f e^{i theta}, f = amp(|n|^2) n_j / |n|^2 (the forward
// ZA multiplier of k_ic_za), theta = pi (n_x + n_y + n_z) / nc for shifted sites.
__global__ void k_icadj_kspace(const float2* __restrict__ a, float2* __restrict__ kacc, int nc, int pc,
                               const float* __restrict__ amp, int comp, int phase_shift,
                               int accumulate) {
  const int x = blockIdx.x / nc, y = blockIdx.x % nc;
  const int nx = x < nc / 2 ? x : x - nc, ny = y < nc / 2 ? y : y - nc;
  for (int kz = threadIdx.x; kz <= nc / 2; kz += blockDim.x) {
    const size_t idx = ((size_t)x * nc + y) * pc + kz;
    const long long n2 = (long long)nx * nx + (long long)ny * ny + (long long)kz * kz;
    float2 r = make_float2(0.f, 0.f);
    const bool nyq = (x == nc / 2) || (y == nc / 2) || (kz == nc / 2);
    if (n2 > 0 && !nyq) {
      const int nj = comp == 0 ? nx : (comp == 1 ? ny : kz);
      const float f = __ldg(amp + n2) * (float)nj / (float)n2;
      float2 cs = make_float2(0.f, -f);  // conj(i f) = -i f
      if (phase_shift) {
        float sn, co;
        sincospif((float)(nx + ny + kz) / (float)nc, &sn, &co);
        cs = cmul(cs, make_float2(co, -sn));  // conj(e^{i theta})
      }
      r = cmul(cs, a[idx]);
    }
    if (accumulate) {
      const float2 o = kacc[idx];
      kacc[idx] = make_float2(o.x + r.x, o.y + r.y);
    } else {
      kacc[idx] = r;
    }
  }
}

int ensure_adj(pm_ctx* c, int64_t n) {
  if (n <= c->adj_cap) return PM_OK;
  ctx_free(c, c->adj);
  c->adj = nullptr;
  c->adj_cap = 0;
  if (ctx_alloc_n(c, &c->adj, 8 * 3 * (size_t)std::max<int64_t>(n, 1)) != PM_OK) return PM_ENOMEM;
  c->adj_cap = n;
  return PM_OK;
}

unsigned blocks(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

int gather_weights(pm_ctx* c, const float* w, int64_t n, float* w_sorted, cudaStream_t s) {
  if (n == 0) return PM_OK;
  LaunchScope L(c, s, K_ADJOINT);
  k_gather3<<<blocks(n), 256, 0, s>>>(w, c->vals[0], n, 1, w_sorted);
  return PM_OK;
}

// Readout gradient of up to three padded meshes at the sorted scratch particles
void readout_grad(pm_ctx* c, int64_t n, const float* const* meshes, int nmeshes, int row_pitch,
                  const float* wts_sorted, const uint32_t* perm, float* out, bool accumulate,
                  cudaStream_t s, int species) {
  if (n == 0) return;
  LaunchScope L(c, s, K_ADJOINT);
  const float inv_h = (float)(c->g.n / c->cfg.box);
  k_readout_grad<<<blocks(n), 256, 0, s>>>(c->us, c->ids, n, meshes[0], nmeshes > 1 ? meshes[1] : nullptr,
                                           nmeshes > 2 ? meshes[2] : nullptr, nmeshes, c->g.n,
                                           32 - c->g.logn, row_pitch, inv_h, wts_sorted, c->mt, perm,
                                           out, accumulate ? 1 : 0, species);
}

// Force VJP: u (any order, with id), cotangent lam_f[3n] in the same order -> grad[3n].
// With the learned factor (evaluated at scale factor a) it also accumulates
// d <lam_f, F> / d theta; that needs the third mesh, which holds rho_k meanwhile.
int force_vjp(pm_ctx* c, const uint32_t* u, const uint32_t* id, int64_t n, const float* lam_f,
              double a, float* grad, cudaStream_t s) {
  if (n == 0) return PM_OK;
  const bool learned = c->mlp_on;
  if (learned && !c->meshC) return PM_EINVAL;
  int rc = ensure_adj(c, n);
  if (rc != PM_OK) return rc;
  rc = sort_particles(c, u, n, s);
  if (rc != PM_OK) return rc;
  gather_sorted(c, u, nullptr, id, n, c->vals[0], s);
  float* lam_s = c->adj + 6 * 3 * n;  // sorted cotangent, 3n
  {
    LaunchScope L(c, s, K_ADJOINT);
    k_gather3<<<blocks(n), 256, 0, s>>>(lam_f, c->vals[0], n, 3, lam_s);
  }
  float* realA = reinterpret_cast<float*>(c->meshA);
  float* realB = reinterpret_cast<float*>(c->meshB);
  const int rp = 2 * c->g.pc;
  if (!learned && (c->cfg.flags & (PM_FLAG_SPECTRAL_KERNEL | PM_FLAG_KSPACE_GRADIENT)) == 0) {
    // one mesh at a time, five FFT passes a term (see k_readout_grad_fd4)
    const float inv12h = (float)((double)c->g.n / (12.0 * c->cfg.box));
    const float inv_h = (float)(c->g.n / c->cfg.box);
    paint_tiles(c, c->us, c->ids, n, PM_SPECIES_ALL, realA, rp, s);
    fft_potential(c, c->g, c->meshA, s);
    {
      LaunchScope L(c, s, K_ADJOINT);
      k_readout_grad_fd4<<<(unsigned)(c->nt * c->nt * c->nt), kVjpThreads, 0, s>>>(
          c->us, n, c->bstart, realA, c->g.n, 32 - c->g.logn, c->ntl, rp, inv12h, inv_h, lam_s, c->vals[0], grad,
          c->err_dev);
    }
    for (int j = 0; j < 3; ++j) {
      paint_tiles(c, c->us, c->ids, n, PM_SPECIES_ALL, realA, rp, s, lam_s + (int64_t)j * n);
      LaunchScope L(c, s, K_ADJOINT);
      k_stencil_axis<<<(unsigned)(c->g.n * c->g.n), 256, 0, s>>>(realA, realB, c->g.n, rp, j, inv12h, j > 0);
    }
    fft_potential(c, c->g, c->meshB, s);
    const float* m[1] = {realB};
    readout_grad(c, n, m, 1, rp, nullptr, c->vals[0], grad, true, s);
    return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
  }
  // term 1: sum_j lambda_j grad R[G_j rho]
  paint_tiles(c, c->us, c->ids, n, PM_SPECIES_ALL, realA, rp, s);
  if (learned) {
    mlp_table(c, a, s);
    fft_forward(c, c->g, c->meshA, c->meshC, 0, s);  // rho_k, kept for the factor's gradient
    mlp_green_apply(c, c->meshC, c->meshB, s);
  } else {
    fft_forward(c, c->g, c->meshA, c->meshB, 1, s);
  }
  for (int j = 0; j < 3; ++j) {
    fft_inverse_component(c, c->g, c->meshB, c->meshA, j, s);
    const float* m[1] = {realA};
    readout_grad(c, n, m, 1, rp, lam_s + (int64_t)j * n, c->vals[0], grad, j > 0, s);
  }
  // term 2: m_i grad R[B], B_k = sum_j i D(k_j) g FFT(paint(lambda_j))
  const double nn = (double)c->g.n;
  const float gcoef = (float)(-1.5 * c->cosmo.omega_m0 / (nn * nn * nn));
  for (int j = 0; j < 3; ++j) {
    paint_tiles(c, c->us, c->ids, n, PM_SPECIES_ALL, realA, rp, s, lam_s + (int64_t)j * n);
    fft_forward(c, c->g, c->meshA, c->meshA, 0, s);
    LaunchScope L(c, s, K_ADJOINT);
    k_adj_combine<<<(unsigned)(c->g.n * c->g.n), 128, 0, s>>>(
        c->meshA, c->meshB, c->g.n, c->g.pc, c->ksq, c->wforce, c->kvec0, gcoef, j, j > 0,
        learned ? c->mlp_tab : nullptr, learned ? c->meshC : nullptr, c->mlp_gbin);
  }
  fft_inverse_plain(c, c->g, c->meshB, s);
  const float* m[1] = {realB};
  readout_grad(c, n, m, 1, rp, nullptr, c->vals[0], grad, true, s);
  if (learned) mlp_backward(c, a, s);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int step_vjp(pm_ctx* c, const pm_state* st, double a0, double ah, double a1, const float* lx1,
             const float* lp1, float* lx0, float* lp0, cudaStream_t s) {
  const int64_t n = st->n;
  if (n == 0) return PM_OK;
  int rc = ensure_adj(c, n);
  if (rc != PM_OK) return rc;
  double k[3];
  c->cosmo.coeffs(a0, ah, a1, k);
  const int64_t m3 = 3 * n;
  float* Lx = c->adj;             // lambda_x in state order
  float* Lp = c->adj + m3;        // lambda_p in state order
  float* lamF = c->adj + 2 * m3;
  float* g = c->adj + 3 * m3;
  uint32_t* u1 = reinterpret_cast<uint32_t*>(c->adj + 4 * m3);
#define ADJ(launch)                      \
  do {                                   \
    LaunchScope L_(c, s, K_ADJOINT);     \
    launch;                              \
  } while (0)
  ADJ((k_by_id<<<blocks(n), 256, 0, s>>>(lx1, Lx, st->id, n, 0, 1.0f)));
  ADJ((k_by_id<<<blocks(n), 256, 0, s>>>(lp1, Lp, st->id, n, 0, 1.0f)));
  ADJ((k_drift_only<<<blocks(n), 256, 0, s>>>(st->u, st->p, st->f, n, (float)k[0],
                                              (float)(k[1] * 4294967296.0 / c->cfg.box), u1)));
  // lambda_x1' = lambda_x1 + F_vjp(x1; K2 lambda_p1)
  ADJ((k_by_id<<<blocks(n), 256, 0, s>>>(Lp, lamF, nullptr, n, 0, (float)k[2])));
  rc = force_vjp(c, u1, st->id, n, lamF, a1, g, s);
  if (rc != PM_OK) return rc;
  ADJ((k_axpby<<<blocks(m3), 256, 0, s>>>(g, Lx, m3, 1.0f, 1.0f)));
  // lambda_ph = lambda_p1 + Delta lambda_x1'
  ADJ((k_axpby<<<blocks(m3), 256, 0, s>>>(Lx, Lp, m3, (float)k[1], 1.0f)));
  // lambda_x0 = lambda_x1' + F_vjp(x0; K1 lambda_ph)
  ADJ((k_by_id<<<blocks(n), 256, 0, s>>>(Lp, lamF, nullptr, n, 0, (float)k[0])));
  rc = force_vjp(c, st->u, st->id, n, lamF, a0, g, s);
  if (rc != PM_OK) return rc;
  ADJ((k_axpby<<<blocks(m3), 256, 0, s>>>(g, Lx, m3, 1.0f, 1.0f)));
  ADJ((k_by_id<<<blocks(n), 256, 0, s>>>(Lx, lx0, st->id, n, 1, 1.0f)));
  ADJ((k_by_id<<<blocks(n), 256, 0, s>>>(Lp, lp0, st->id, n, 1, 1.0f)));
#undef ADJ
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

int ic_vjp(pm_ctx* c, const float* lx, const float* lp, double a0, double k_fs, float* grad_noise,
           cudaStream_t s) {
  const pm_config& cf = c->cfg;
  const int nc = cf.nc;
  if (nc < 32 || (nc & (nc - 1)) || nc > c->g.n) return PM_EINVAL;
  if (!c->ic_amp || k_fs != c->ic_kfs) return PM_EINVAL;  // pm_ic with the same k_fs first
  Geom gi;
  gi.n = nc;
  gi.logn = 0;
  while ((1 << gi.logn) < nc) ++gi.logn;
  gi.pc = nc / 2 + 2;
  const int64_t n_cdm = (int64_t)nc * nc * nc;
  const int ndir = 2 * cf.nfib + 1;
  const int64_t n_nu = cf.nsites > 0 ? (int64_t)cf.nsites * cf.nsites * cf.nsites * cf.nshell * ndir : 0;
  const int64_t n = n_cdm + n_nu;
  const float D0 = (float)c->cosmo.D(a0), gp0 = (float)c->cosmo.gp(a0);
  const int stride = cf.nsites > 0 ? nc / cf.nsites : 1;
  const bool even = (stride % 2) == 0;
  const int j0 = even ? stride / 2 : (stride + 1) / 2;
  float* realA = reinterpret_cast<float*>(c->meshA);
  const int rp = 2 * gi.pc;
  bool first = true;
  for (int species = 0; species < 2; ++species) {
    if (species == 1 && n_nu == 0) break;
    for (int comp = 0; comp < 3; ++comp) {
      PM_CUDA_TRY(cudaMemsetAsync(c->meshA, 0, sizeof(float2) * gi.elems(), s));
      {
        LaunchScope L(c, s, K_ADJOINT);
        if (species == 0)
          k_icadj_cdm<<<blocks(n_cdm), 256, 0, s>>>(lx, lp, nc, rp, comp, D0, gp0, n, realA);
        else
          k_icadj_nu<<<blocks((int64_t)cf.nsites * cf.nsites * cf.nsites), 256, 0, s>>>(
              lx, lp, nc, rp, comp, D0, gp0, cf.nsites, stride, j0, cf.nshell * ndir, n_cdm, n, realA);
      }
      fft_forward(c, gi, c->meshA, c->meshA, 0, s);
      LaunchScope L(c, s, K_ADJOINT);
      k_icadj_kspace<<<(unsigned)(nc * nc), 128, 0, s>>>(c->meshA, c->meshB, nc, gi.pc,
                                                         species == 0 ? c->ic_amp : c->ic_amp_nu, comp,
                                                         species == 1 && even ? 1 : 0, first ? 0 : 1);
      first = false;
    }
  }
  fft_inverse_plain(c, gi, c->meshB, s);
  repack_real(c, gi, reinterpret_cast<float*>(c->meshB), rp, grad_noise, nc, s);
  return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ECUDA;
}

}  // namespace pmnu
