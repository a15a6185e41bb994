// Particle <-> mesh kernels: deterministic tile paint, CIC readout fused with the
// kick (of force meshes, or of the potential with the 4-point gradient applied in
// shared memory), the first kick fused with the drift and the next sort keys.
//
// Paint (CIC of rho / rho_bar): one CTA per 16^3 tile.  The tile's own particles
// are the bucket range [bstart[8 t], bstart[8 t + 8]); a particle on the tile's
// high face layer (class bits) also reaches the neighbouring tile, which reads
// exactly those classes of its seven low-side neighbours.  Each (particle,
// corner) pair is therefore counted by the one CTA that owns the corner cell.
// Contributions are accumulated in shared memory as fixed-point integers: integer
// addition is associative, so the result does not depend on thread scheduling, and
// no float atomics are used.  Mass paints use 2^-24 resolution: each contribution
// q < 2^31 goes to a 32-bit accumulator with one atomic add, whose returned old value
// shows when the sum wrapped past 2^32, and then a second word counts the carry
// (value = carry 2^32 + low word: exact, whatever the order).  A wrap needs a cell of
// 256 mean cell masses, so nearly every corner costs one 32-bit shared atomic (those
// run ~4x faster than 64-bit ones, and the 32-bit conversions of the write-out avoid
// the narrow FP64 pipe that 64-bit float <-> integer conversions use).  Masses of 128
// or more and the signed weights of the adjoint use one 64-bit accumulator instead
// (resolution 2^-24 for masses, so both forms give the same bits; 2^-32 for weights).
#include <cuda_runtime.h>

#include <algorithm>

#include "pm_internal.cuh"

namespace pmnu {

namespace {

constexpr int kPaintThreads = 256;
constexpr float kFixW = 4294967296.0f;              // 2^32: signed weights
constexpr float kUnfixW = 2.3283064365386963e-10f;  // 2^-32
constexpr float kFixM = 16777216.0f;                // 2^24: masses
constexpr float kUnfixM = 5.9604644775390625e-08f;  // 2^-24

// The 14 bucket runs a tile reads, as (neighbour offset o, first class, end class):
// its own tile (all classes), then for each low-side neighbour o the classes that
// contain every bit of o, merged where they are contiguous.
__constant__ int8_t c_runs[14][3] = {{0, 0, 8}, {4, 4, 8}, {2, 2, 4}, {2, 6, 8}, {1, 1, 2},
                                     {1, 3, 4}, {1, 5, 6}, {1, 7, 8}, {6, 6, 8}, {5, 5, 6},
                                     {5, 7, 8}, {3, 3, 4}, {3, 7, 8}, {7, 7, 8}};

// Shared accumulator layout: cell (x, y, z) of the tile at x * kSx + y * kSy + z.  With
// kSy = 18 and kSx = 292 (4 and 2 modulo 16) the 8 CIC corners of one particle land in
// 8 distinct 8-byte bank pairs.
constexpr int kSy = 18, kSx = 292;
constexpr int kAccWords = kTile * kSx;
// fast paint: wrap bitmap words, event list capacity, and the whole shared area in words
// (low words, bitmap, event count, 16-bit events, rounded up to whole 16-byte groups)
constexpr int kWrapBits = (kAccWords + 31) / 32;
constexpr unsigned int kWraps = 1024;
constexpr int kFastWords = ((kAccWords + kWrapBits + 1 + kWraps / 2) + 3) / 4 * 4;

// Records that the fast paint's low word ad wrapped: its bit in the bitmap and an event in
// the list (layout of paint_tile); false when the list is full.  Out of line: rarely taken,
// and it keeps the paint's inner loop at fewer registers.
__device__ __noinline__ bool record_wrap(unsigned int* accw, unsigned int ad) {
  atomicOr(accw + kAccWords + (ad >> 5), 1u << (ad & 31));
  const unsigned int e = atomicAdd(accw + kAccWords + kWrapBits, 1u);
  if (e >= kWraps) return false;
  reinterpret_cast<unsigned short*>(accw + kAccWords + kWrapBits + 1)[e] = (unsigned short)ad;
  return true;
}

// Paint of one tile.  FAST: 32-bit low words only (half the shared memory of the carry form:
// zeroed, and read at the write-out, once per cell).  A low word that wraps past 2^32 (the
// cell passes another 256 mean cell masses) is recorded as an event -- the cell's bit in a
// bitmap, its index in a list of up to kWraps events -- and at the write-out a cell whose
// bit is set counts its events in the list: value = events 2^32 + low word.  A tile with
// more events than the list holds is written to the redo list and left unwritten; the redo
// pass paints it in full with the 32-bit carry (or 64-bit) form.  Every form sums the same
// exact integers, so all give the same floats.
template <bool FAST>
__device__ __forceinline__ void paint_tile(
    uint32_t tile, unsigned int* __restrict__ accw, uint32_t* __restrict__ run_lo, uint32_t* __restrict__ run_pre,
    const uint32_t* __restrict__ us, const uint32_t* __restrict__ ids, int64_t n,
    const uint32_t* __restrict__ bstart, float* __restrict__ mesh, const MassTable& mt, int species, int nm,
    int shift, int ntl, int row_pitch, int* __restrict__ err, const float* __restrict__ wts, float mmax,
    uint32_t* __restrict__ redo) {
  // FAST: low words, then the wrap bitmap, the event count and the event list.  Else one
  // 64-bit accumulator, or the same bytes as two 32-bit halves (hi words, then lo words) in the
  // carry form.
  long long* const acc = reinterpret_cast<long long*>(accw);
  unsigned int* const acc_hi = accw;
  unsigned int* const acc_lo = FAST ? accw : accw + kAccWords;
  volatile unsigned int* const wbits = accw + kAccWords;          // FAST: kWrapBits words
  unsigned int* const wcount = accw + kAccWords + kWrapBits;       // FAST: one word
  volatile unsigned short* const wlist = reinterpret_cast<unsigned short*>(accw + kAccWords + kWrapBits + 1);
  const int t = threadIdx.x;
  if constexpr (FAST) {
    for (int i = t; i < (kAccWords + kWrapBits + 1) / 4 + 1; i += kPaintThreads)
      reinterpret_cast<uint4*>(accw)[i] = make_uint4(0, 0, 0, 0);
  } else {
    for (int i = t; i < kAccWords; i += kPaintThreads) acc[i] = 0;
  }
  const int nt = 1 << ntl;
  const int tx = tile >> (2 * ntl), ty = (tile >> ntl) & (nt - 1), tz = tile & (nt - 1);
  if (t < 32) {  // one warp resolves the 14 runs and their prefix
    uint32_t lo = 0, len = 0;
    if (t < 14) {
      const int o = c_runs[t][0];
      const int ox = (o >> 2) & 1, oy = (o >> 1) & 1, oz = o & 1;
      const uint32_t nb = ((uint32_t)((tx - ox) & (nt - 1)) << (2 * ntl)) |
                          ((uint32_t)((ty - oy) & (nt - 1)) << ntl) | (uint32_t)((tz - oz) & (nt - 1));
      lo = bstart[nb * 8 + c_runs[t][1]];
      len = bstart[nb * 8 + c_runs[t][2]] - lo;
    }
    uint32_t x = len;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (t >= d) x += y;
    }
    if (t < 14) {
      run_lo[t] = lo;
      run_pre[t + 1] = x;
    }
    if (t == 0) run_pre[0] = 0;
  }
  __syncthreads();
  const float fscale = 1.0f / (float)(1u << shift);
  const uint32_t fmask = (1u << shift) - 1u;
  const uint32_t total = run_pre[14];
  // One particle per thread (coalesced loads in bucket order), its 8 corners added by
  // the same thread.
  // carry form: 32-bit accumulators and conversions (GB300's FP64 pipe, which runs the
  // 64-bit float <-> integer conversions, is narrow); w 2^24 < 2^31 needs mmax < 128
  const bool carry = FAST || (wts == nullptr && mmax < 128.0f);
  const float fix = wts ? kFixW : kFixM;
  const int ox = tx * kTile, oy = ty * kTile, oz = tz * kTile;
  bool bad = false, wrap = false;
  int r = 0;
  // the particle of iteration v + kPaintThreads is loaded while v's corners are added
  auto locate = [&](uint32_t v) {
    while (v >= run_pre[r + 1]) ++r;  // v only grows, so the run index only grows
    return run_lo[r] + (v - run_pre[r]);
  };
  uint32_t k = 0, qid = 0, qu0 = 0, qu1 = 0, qu2 = 0;
  float qw = 0.0f;
  if ((uint32_t)t < total) {
    k = locate(t);
    if (wts) qw = wts[k]; else qid = ids[k];
    qu0 = us[k];
    qu1 = us[n + k];
    qu2 = us[2 * n + k];
  }
  for (uint32_t v = t; v < total; v += kPaintThreads) {
    const uint32_t u0 = qu0, u1 = qu1, u2 = qu2, idv = qid;
    const float wv = qw;
    const uint32_t vn = v + kPaintThreads;
    if (vn < total) {
      const uint32_t kn = locate(vn);
      if (wts) qw = wts[kn]; else qid = ids[kn];
      qu0 = us[kn];
      qu1 = us[n + kn];
      qu2 = us[2 * n + kn];
    }
    const float m = wts ? wv : id_mass(mt, idv, species, &bad);  // weights: signed, sorted order
    if (m == 0.0f) continue;
    int l[3] = {(int)(u0 >> shift) - ox, (int)(u1 >> shift) - oy, (int)(u2 >> shift) - oz};
    int lo_ok = 0;  // bit d: lower corner inside along d; bit 3 + d: upper inside
#pragma unroll
    for (int d = 0; d < 3; ++d) {  // periodic wrap relative to the tile origin
      if (l[d] > nm / 2) l[d] -= nm;
      if (l[d] < -nm / 2) l[d] += nm;
      if (l[d] >= 0 && l[d] < kTile) lo_ok |= 1 << d;
      if (l[d] + 1 >= 0 && l[d] + 1 < kTile) lo_ok |= 8 << d;
    }
    const int cell = l[0] * kSx + l[1] * kSy + l[2];
    const float fx = (float)(u0 & fmask) * fscale, fy = (float)(u1 & fmask) * fscale,
                fz = (float)(u2 & fmask) * fscale;
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
      const int bx = corner >> 2, by = (corner >> 1) & 1, bz = corner & 1;
      const bool inside = ((lo_ok >> (bx ? 3 : 0)) & 1) && ((lo_ok >> (by ? 4 : 1)) & 1) &&
                          ((lo_ok >> (bz ? 5 : 2)) & 1);
      if (inside) {
        const float w = (bx ? fx : 1.0f - fx) * (by ? fy : 1.0f - fy) * (bz ? fz : 1.0f - fz) * m;
        const int ad = cell + bx * kSx + by * kSy + bz;
        if (carry) {
          const unsigned int q = __float2uint_rn(w * fix);  // < 2^31: masses below 128
          const unsigned int old = atomicAdd(&acc_lo[ad], q);
          if (old + q < old) {  // the low word wrapped
            if constexpr (FAST) {
              if (!record_wrap(accw, ad)) wrap = true;  // the list is full: the tile is repainted
            } else {
              atomicAdd(&acc_hi[ad], 1u);
            }
          }
        } else {
          const long long q = __float2ll_rn(w * fix);
          atomicAdd((unsigned long long*)&acc[ad], (unsigned long long)q);
        }
      }
    }
  }
  if (bad) atomicOr(err, 1);
  if constexpr (FAST) {
    // the barrier's vote tells every thread whether the event list overflowed (the redo pass
    // then paints this tile)
    if (__syncthreads_or(wrap ? 1 : 0)) {
      if (t == 0) redo[1 + atomicAdd(redo, 1u)] = tile;
      return;
    }
  } else {
    __syncthreads();
  }
  // FAST: whether any low word of the tile wrapped (else the write-out reads low words only)
  bool any_wrap = false;
  if constexpr (FAST) any_wrap = *(volatile unsigned int*)wcount != 0u;
  // write the tile: 256 rows of 16 floats, as float4
  for (int q = t; q < kTile * kTile * kTile / 4; q += kPaintThreads) {
    int row = q >> 2, z4 = (q & 3) * 4;
    int lx = row >> 4, ly = row & 15;
    const int a0 = lx * kSx + ly * kSy + z4;
    float fv[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if constexpr (FAST) {
        const unsigned int ad = a0 + e, lo = acc_lo[ad];
        if (any_wrap && ((wbits[ad >> 5] >> (ad & 31)) & 1u)) {  // the cell wrapped: count its events
          const unsigned int ne = *(volatile unsigned int*)wcount;
          unsigned int hi = 0;
          for (unsigned int k = 0; k < ne; ++k) hi += wlist[k] == ad ? 1u : 0u;
          fv[e] = __ull2float_rn(((unsigned long long)hi << 32) + (unsigned long long)lo);
        } else {
          fv[e] = __uint2float_rn(lo);
        }
      } else if (carry) {
        // value = carry 2^32 + low word: without a carry the correctly rounded 32-bit
        // conversion is that of the 64-bit sum
        const unsigned int hi = acc_hi[a0 + e], lo = acc_lo[a0 + e];
        fv[e] = hi == 0u ? __uint2float_rn(lo)
                         : __ull2float_rn(((unsigned long long)hi << 32) + (unsigned long long)lo);
      } else {
        fv[e] = __ll2float_rn(acc[a0 + e]);
      }
    }
    const float un = wts ? kUnfixW : kUnfixM;
    float4 v = make_float4(fv[0] * un, fv[1] * un, fv[2] * un, fv[3] * un);
    size_t off = ((size_t)(ox + lx) * nm + (oy + ly)) * (size_t)row_pitch + oz + z4;
    *reinterpret_cast<float4*>(mesh + off) = v;
  }
}

// One CTA per tile.  FAST: the 32-bit form with wrap events, tiles whose event list
// overflows sent to the redo list (redo[0] = count, redo[1 ..] = tiles); else the carry or
// 64-bit form.
template <bool FAST>
__global__ void __launch_bounds__(kPaintThreads, FAST ? 8 : 1) k_paint_tiles(
    const uint32_t* __restrict__ us, const uint32_t* __restrict__ ids, int64_t n,
    const uint32_t* __restrict__ bstart, float* __restrict__ mesh, MassTable mt, int species,
    int nm, int shift, int ntl, int row_pitch, int* __restrict__ err, const float* __restrict__ wts,
    float mmax, uint32_t* __restrict__ redo) {
  __shared__ __align__(16) unsigned int accw[FAST ? kFastWords : 2 * kAccWords];
  __shared__ uint32_t run_lo[14], run_pre[15];
  paint_tile<FAST>(blockIdx.x, accw, run_lo, run_pre, us, ids, n, bstart, mesh, mt, species, nm, shift, ntl,
                   row_pitch, err, wts, mmax, redo);
}

// The redo pass: the tiles the fast pass listed, painted with the 32-bit carry form
// (persistent CTAs walk the list; an empty list, the normal case, costs one launch).
__global__ void __launch_bounds__(kPaintThreads) k_paint_redo(
    const uint32_t* __restrict__ us, const uint32_t* __restrict__ ids, int64_t n,
    const uint32_t* __restrict__ bstart, float* __restrict__ mesh, MassTable mt, int species,
    int nm, int shift, int ntl, int row_pitch, int* __restrict__ err, float mmax,
    const uint32_t* __restrict__ redo) {
  __shared__ __align__(16) unsigned int accw[2 * kAccWords];
  __shared__ uint32_t run_lo[14], run_pre[15];
  const uint32_t count = redo[0];
  for (uint32_t q = blockIdx.x; q < count; q += gridDim.x) {
    paint_tile<false>(redo[1 + q], accw, run_lo, run_pre, us, ids, n, bstart, mesh, mt, species, nm, shift, ntl,
                      row_pitch, err, nullptr, mmax, nullptr);
    __syncthreads();  // the shared accumulators are reused by the next tile
  }
}

// CIC readout of one real mesh component fused with the kick p_j += K F_j.
__global__ void k_readout_kick(const uint32_t* __restrict__ us, const float* __restrict__ ps,
                               const uint32_t* __restrict__ ids, int64_t n,
                               const float* __restrict__ mesh, int nm, int shift, int row_pitch,
                               int comp, float K, float* __restrict__ p_out,
                               float* __restrict__ f_out, uint32_t* __restrict__ u_out,
                               uint32_t* __restrict__ id_out, const uint32_t* __restrict__ perm) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t ux = us[i], uy = us[n + i], uz = us[2 * n + i];
  const float fscale = 1.0f / (float)(1u << shift);
  const uint32_t fmask = (1u << shift) - 1u;
  const int cx = ux >> shift, cy = uy >> shift, cz = uz >> shift;
  const int cx1 = (cx + 1) & (nm - 1), cy1 = (cy + 1) & (nm - 1), cz1 = (cz + 1) & (nm - 1);
  const float fx = (float)(ux & fmask) * fscale, fy = (float)(uy & fmask) * fscale,
              fz = (float)(uz & fmask) * fscale;
  const size_t r00 = ((size_t)cx * nm + cy) * row_pitch, r01 = ((size_t)cx * nm + cy1) * row_pitch;
  const size_t r10 = ((size_t)cx1 * nm + cy) * row_pitch, r11 = ((size_t)cx1 * nm + cy1) * row_pitch;
  const float v000 = __ldg(mesh + r00 + cz), v001 = __ldg(mesh + r00 + cz1);
  const float v010 = __ldg(mesh + r01 + cz), v011 = __ldg(mesh + r01 + cz1);
  const float v100 = __ldg(mesh + r10 + cz), v101 = __ldg(mesh + r10 + cz1);
  const float v110 = __ldg(mesh + r11 + cz), v111 = __ldg(mesh + r11 + cz1);
  const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
  const float F = gx * (gy * (gz * v000 + fz * v001) + fy * (gz * v010 + fz * v011)) +
                  fx * (gy * (gz * v100 + fz * v101) + fy * (gz * v110 + fz * v111));
  if (perm) {  // stage-level readout / force in the caller's order
    uint32_t j = perm[i];
    f_out[(int64_t)comp * n + j] = F;
    return;
  }
  if (p_out) p_out[(int64_t)comp * n + i] = __fmaf_rn(K, F, ps[(int64_t)comp * n + i]);
  if (f_out) f_out[(int64_t)comp * n + i] = F;
  if (u_out) {
    u_out[i] = ux;
    u_out[n + i] = uy;
    u_out[2 * n + i] = uz;
    id_out[i] = ids[i];
  }
}

// CIC readout of all three force meshes at once, fused with the kick p += K F.
__global__ void k_readout3_kick(const uint32_t* __restrict__ us, const float* __restrict__ ps,
                                const uint32_t* __restrict__ ids, int64_t n,
                                const float* __restrict__ mx, const float* __restrict__ my,
                                const float* __restrict__ mz, int nm, int shift, int row_pitch,
                                float K, float* __restrict__ p_out, float* __restrict__ f_out,
                                uint32_t* __restrict__ u_out, uint32_t* __restrict__ id_out,
                                const uint32_t* __restrict__ perm) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
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
  const float w000 = gx * gy * gz, w001 = gx * gy * fz, w010 = gx * fy * gz, w011 = gx * fy * fz;
  const float w100 = fx * gy * gz, w101 = fx * gy * fz, w110 = fx * fy * gz, w111 = fx * fy * fz;
  const float* m[3] = {mx, my, mz};
  float F[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float* g = m[d];
    F[d] = w000 * __ldg(g + r00 + cz) + w001 * __ldg(g + r00 + cz1) + w010 * __ldg(g + r01 + cz) +
           w011 * __ldg(g + r01 + cz1) + w100 * __ldg(g + r10 + cz) + w101 * __ldg(g + r10 + cz1) +
           w110 * __ldg(g + r11 + cz) + w111 * __ldg(g + r11 + cz1);
  }
  if (perm) {  // force in the caller's order
    const uint32_t j = perm[i];
#pragma unroll
    for (int d = 0; d < 3; ++d) f_out[(int64_t)d * n + j] = F[d];
    return;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (p_out) p_out[(int64_t)d * n + i] = __fmaf_rn(K, F[d], ps[(int64_t)d * n + i]);
    if (f_out) f_out[(int64_t)d * n + i] = F[d];
  }
  if (u_out) {
    u_out[i] = ux;
    u_out[n + i] = uy;
    u_out[2 * n + i] = uz;
    id_out[i] = ids[i];
  }
}

// Force from the potential mesh with the 4-point gradient in real space, fused with
// the kick.  The finite-difference gradient [8 (phi(x+H) - phi(x-H)) - (phi(x+2H) -
// phi(x-2H))] / (12 H) has exactly the transfer function i D(k) of the k-space kernel
// (0 on the Nyquist index), so this equals the CIC readout of IFFT(-i D(k_j) phi_k)
// while the mesh side needs one inverse transform instead of three.
//
// One CTA per 16^3 tile.  The tile's potential with a halo of 2 cells below and 3
// above along x and y, and of 4 below and 3 above along z (so that every z row splits
// into 16-byte aligned chunks, also where it wraps), is staged in shared memory with
// asynchronous 16-byte copies (21 x 21 x 24 floats).  Each thread then takes particles
// of the tile's bucket range [bstart[8 t], bstart[8 t + 8]), all of whose cells lie
// in the tile, and gathers the 56 potential values its 8 CIC corners' stencils touch;
// the first particle's position is loaded while the copies are in flight, the next
// one's while the current one is computed.  Differences of neighbouring values are
// formed first, so FP32 rounding scales with the gradient, not with the potential.
// A particle outside its tile (a bucket range that does not match the positions)
// sets the error word's invalid-input bit.
// The next step's first half kick and drift, fused into the readout that ends a step
// (pm_run): p = (ps + K2 F) + K1' F, u' = u + rne(Delta' p 2^32 / L), in the operations
// and order of the unfused path (readout, then k_kick_drift_keys), so the state is
// bit-identical.  Writes the new key and the near-sorted re-sort's counts (the
// particle's old key is its current bucket, so it is in range by construction).
__device__ __forceinline__ uint32_t drift_fixed(uint32_t u, float dscale, float p) {
  const float x = dscale * p;
  const uint32_t step = fabsf(x) < 2147483648.0f ? (uint32_t)__float2int_rn(x)
                                                 : (uint32_t)(unsigned long long)__float2ll_rn(x);
  return u + step;
}

__device__ __forceinline__ void drift_next(const DriftNext& dn, const float (&F)[3], const float (&pv)[3],
                                           float K2, int64_t n, uint32_t i, uint32_t ux, uint32_t uy, uint32_t uz,
                                           int shift, int ntl, float* __restrict__ p_out, float* __restrict__ f_out,
                                           uint32_t* __restrict__ u_out) {
  uint32_t uu[3] = {ux, uy, uz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float p1 = __fmaf_rn(K2, F[d], pv[d]);
    const float p2 = __fmaf_rn(dn.K1, F[d], p1);
    p_out[(int64_t)d * n + i] = p2;
    if (f_out) f_out[(int64_t)d * n + i] = F[d];
    uu[d] = drift_fixed(uu[d], dn.dscale, p2);
    u_out[(int64_t)d * n + i] = uu[d];
  }
  const uint32_t kn = tile_key(uu[0], uu[1], uu[2], shift, ntl);
  const uint32_t ko = tile_key(ux, uy, uz, shift, ntl);
  dn.keys[i] = kn;
  // counts: all particles by new key, stayers by new key, movers by old key, movers from a
  // lower key by new key.  The lanes here hold consecutive particles of the tile's sorted
  // range, so their old keys never decrease from lane to lane: stayers (new key = old key)
  // and movers are counted per run of equal old keys with ballots, and only the movers'
  // new keys need a match over the lanes.
  const unsigned act = __activemask();
  const int lane = threadIdx.x & 31;
  const bool stay = kn == ko;
  const unsigned below = act & ((1u << lane) - 1u);
  const int prev = below ? 31 - __clz(below) : lane;  // the nearest active lane below
  const uint32_t ko_prev = __shfl_sync(act, ko, prev);
  const bool head = prev == lane || ko_prev != ko;
  const unsigned heads = __ballot_sync(act, head);
  const unsigned stays = __ballot_sync(act, stay);
  const unsigned lows = __ballot_sync(act, !stay && ko < kn);
  if (head) {
    const unsigned after = heads & ~((2u << lane) - 1u);  // heads above this lane (lane 31: none)
    const unsigned upto = after ? (1u << (__ffs(after) - 1)) - 1u : 0xffffffffu;
    const unsigned run = act & upto & ~((1u << lane) - 1u);
    const uint32_t ns = (uint32_t)__popc(run & stays), nmv = (uint32_t)__popc(run & ~stays);
    if (ns) {
      atomicAdd(dn.cnt3 + ko, ns);
      atomicAdd(dn.cnt3 + dn.nb1 + ko, ns);
    }
    if (nmv) atomicAdd(dn.cnt3 + 2 * dn.nb1 + ko, nmv);
  }
  if (!stay) {
    const unsigned peers = __match_any_sync(act & ~stays, kn);
    if (lane == __ffs(peers) - 1) {
      atomicAdd(dn.cnt3 + kn, (uint32_t)__popc(peers));
      const uint32_t nl = (uint32_t)__popc(peers & lows);
      if (nl) atomicAdd(dn.low + kn, nl);
    }
  }
}

constexpr int kFd4Threads = 256;
constexpr int kSpanXY = kTile + 5;                 // cells -2 .. 18 along x and y
constexpr int kSpanZ = kTile + 8;                  // cells -4 .. 19 along z
constexpr int kChunksZ = kSpanZ / 4;               // 16-byte chunks per staged z row
constexpr int kStageChunks = kSpanXY * kSpanXY * kChunksZ;
constexpr int kFd4SY = kSpanZ, kFd4SX = kSpanXY * kSpanZ;

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gmem_src)
               : "memory");
}

template <bool DRIFT>
__global__ void __launch_bounds__(kFd4Threads) k_readout_fd4_kick(
    const uint32_t* __restrict__ us, const float* __restrict__ ps, const uint32_t* __restrict__ ids,
    int64_t n, const uint32_t* __restrict__ bstart, const float* __restrict__ phi, int nm, int shift,
    int ntl, int row_pitch, float inv12h, float K, float* __restrict__ p_out, float* __restrict__ f_out,
    uint32_t* __restrict__ u_out, uint32_t* __restrict__ id_out, const uint32_t* __restrict__ perm,
    int* __restrict__ err, DriftNext dn) {
  __shared__ __align__(16) float sp[kSpanXY * kSpanXY * kSpanZ];
  const int t = threadIdx.x;
  const uint32_t tile = blockIdx.x;
  const uint32_t lo = bstart[8 * tile], hi = bstart[8 * tile + 8];
  if (lo == hi) return;
  const int nt = 1 << ntl;
  const int ox = (int)(tile >> (2 * ntl)) * kTile, oy = (int)((tile >> ntl) & (nt - 1)) * kTile,
            oz = (int)(tile & (nt - 1)) * kTile;
  const int wrap = nm - 1;
  // chunk k of staged row (x, y) holds cells oz - 4 + 4k .. oz - 1 + 4k (mod N): contiguous
  // and 16-byte aligned because N, oz and the row pitch are multiples of 4 floats
  for (int c = t; c < kStageChunks; c += kFd4Threads) {
    const int x = c / (kSpanXY * kChunksZ), r = c - x * (kSpanXY * kChunksZ);
    const int y = r / kChunksZ, k = r - y * kChunksZ;
    const int gx = (ox + x - 2) & wrap, gy = (oy + y - 2) & wrap, gz = (oz - 4 + 4 * k) & wrap;
    cp_async16(sp + x * kFd4SX + y * kFd4SY + 4 * k, phi + ((size_t)gx * nm + gy) * (size_t)row_pitch + gz);
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  // a particle's position, momentum and id are loaded one iteration ahead
  const bool kick = ps != nullptr && perm == nullptr;
  auto load = [&](uint32_t j, uint32_t (&uq)[3], float (&pq)[3], uint32_t& idq) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      uq[d] = us[(int64_t)d * n + j];
      pq[d] = kick ? ps[(int64_t)d * n + j] : 0.0f;
    }
    idq = id_out ? ids[j] : 0u;
  };
  uint32_t i = lo + t;
  uint32_t cu[3] = {0u, 0u, 0u}, cid = 0u;
  float cp[3] = {0.f, 0.f, 0.f};
  if (i < hi) load(i, cu, cp, cid);
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  const float fscale = 1.0f / (float)(1u << shift);
  const uint32_t fmask = (1u << shift) - 1u;
  bool bad = false, nonfinite = false;
  for (; i < hi; i += kFd4Threads) {
    const uint32_t inext = i + kFd4Threads;
    uint32_t nu[3] = {0u, 0u, 0u}, nid = 0u;
    float np[3] = {0.f, 0.f, 0.f};
    if (inext < hi) load(inext, nu, np, nid);
    const uint32_t ux = cu[0], uy = cu[1], uz = cu[2];
    const int lx = (int)(ux >> shift) - ox, ly = (int)(uy >> shift) - oy, lz = (int)(uz >> shift) - oz;
    if ((unsigned)lx < (unsigned)kTile && (unsigned)ly < (unsigned)kTile && (unsigned)lz < (unsigned)kTile) {
      const float fx = (float)(ux & fmask) * fscale, fy = (float)(uy & fmask) * fscale,
                  fz = (float)(uz & fmask) * fscale;
      const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
      const float* q = sp + (lx + 2) * kFd4SX + (ly + 2) * kFd4SY + (lz + 4);  // phi at the particle's cell
      // stencil sum of one axis at the two corners 0 (weight g) and 1 (weight f) of a
      // line through q0 with stride S: g (8 (p1 - m1) - (p2 - m2)) + f (8 (p2 - p0) - (p3 - m1))
      auto axis_sum = [](const float* q0, int S, float g, float f) {
        const float m2 = q0[-2 * S], m1 = q0[-S], p0 = q0[0], p1 = q0[S], p2 = q0[2 * S], p3 = q0[3 * S];
        return g * (8.0f * (p1 - m1) - (p2 - m2)) + f * (8.0f * (p2 - p0) - (p3 - m1));
      };
      float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
#pragma unroll
      for (int a = 0; a < 2; ++a) {
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          // x lines at (y, z) = (b, a); y lines at (x, z) = (b, a); z lines at (x, y) = (b, a)
          Fx = fmaf((b ? fy : gy) * (a ? fz : gz), axis_sum(q + b * kFd4SY + a, kFd4SX, gx, fx), Fx);
          Fy = fmaf((b ? fx : gx) * (a ? fz : gz), axis_sum(q + b * kFd4SX + a, kFd4SY, gy, fy), Fy);
          Fz = fmaf((b ? fx : gx) * (a ? fy : gy), axis_sum(q + b * kFd4SX + a * kFd4SY, 1, gz, fz), Fz);
        }
      }
      const float F[3] = {-inv12h * Fx, -inv12h * Fy, -inv12h * Fz};
      // a NaN or infinity in the force or the incoming momentum poisons the sum
      if (!isfinite(F[0] + F[1] + F[2] + cp[0] + cp[1] + cp[2])) nonfinite = true;
      if (perm) {  // force in the caller's order
        const uint32_t j = perm[i];
#pragma unroll
        for (int d = 0; d < 3; ++d) f_out[(int64_t)d * n + j] = F[d];
      } else if constexpr (DRIFT) {
        drift_next(dn, F, cp, K, n, i, ux, uy, uz, shift, ntl, p_out, f_out, u_out);
        id_out[i] = cid;
      } else {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          if (p_out) p_out[(int64_t)d * n + i] = __fmaf_rn(K, F[d], cp[d]);
          if (f_out) f_out[(int64_t)d * n + i] = F[d];
        }
        if (u_out) {
          u_out[i] = ux;
          u_out[n + i] = uy;
          u_out[2 * n + i] = uz;
          id_out[i] = cid;
        }
      }
    } else {
      bad = true;
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      cu[d] = nu[d];
      cp[d] = np[d];
    }
    cid = nid;
  }
  if (bad) atomicOr(err, 1);
  if (nonfinite) atomicOr(err, 4);
}

// First half kick with the cached force, drift in fixed point, next sort key.
// RESORT (the state is in the tile order of the last step, whose bucket starts are
// bprev): also classify each particle for the near-sorted re-sort of k_sort.cu.  A
// stayer keeps its key ko; every other particle is a mover.  Counts (cnt3 holds three
// arrays of nbuckets + 1): cnt3[0][kn] all particles of new key kn, cnt3[1][kn]
// stayers, cnt3[2][ko] movers out of old key ko; low[kn] movers from a lower old key.
// Flag bit 1: a particle outside its old key's range [bprev[ko], bprev[ko + 1]) (the
// state is not in bprev's order: the caller sorts from scratch).
template <bool RESORT>
__global__ void k_kick_drift_keys(uint32_t* __restrict__ u, float* __restrict__ p,
                                  const float* __restrict__ f, int64_t n, float K1, float dscale,
                                  int shift, int ntl, uint32_t* __restrict__ keys,
                                  uint32_t* __restrict__ cnt3, long long nb1, const uint32_t* __restrict__ bprev,
                                  uint32_t* __restrict__ low, uint32_t* __restrict__ flags, int* __restrict__ err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool ok = i < n;
  uint32_t key = 0xffffffffu, cat = 0xffffffffu, ko = 0xffffffffu;
  uint32_t flag = 0u;
  if (ok) {
    uint32_t uu[3], u0[3];
    float chk = 0.0f;  // a NaN or infinity in p or f poisons the sum
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const float pv = __fmaf_rn(K1, f[d * n + i], p[d * n + i]);
      chk += pv;
      p[d * n + i] = pv;
      // u += rne(Delta p 2^32 / L), modulo 2^32; the 32-bit conversion (same rounding)
      // whenever the step fits, the 64-bit one (FP64 pipe) only for steps of 2^31 or more
      u0[d] = u[d * n + i];
      uu[d] = drift_fixed(u0[d], dscale, pv);
      u[d * n + i] = uu[d];
    }
    key = tile_key(uu[0], uu[1], uu[2], shift, ntl);
    keys[i] = key;
    if (!isfinite(chk)) atomicOr(err, 4);
    if constexpr (RESORT) {
      const uint32_t k0 = tile_key(u0[0], u0[1], u0[2], shift, ntl);
      const bool in_range = (uint32_t)i >= bprev[k0] && (uint32_t)i < bprev[k0 + 1];
      if (!in_range) {
        flag = 1u;
      } else if (k0 == key) {
        cat = key << 1;  // stayer
      } else {
        ko = k0;
        if (k0 < key) cat = (key << 1) | 1u;  // mover from a lower key
      }
    }
  }
  unsigned act = __ballot_sync(0xffffffffu, ok);
  if (ok) {
    unsigned peers = __match_any_sync(act, key);
    int leader = __ffs(peers) - 1;
    if ((int)(threadIdx.x & 31) == leader) atomicAdd(cnt3 + key, (uint32_t)__popc(peers));
  }
  if constexpr (RESORT) {
    const int lane = threadIdx.x & 31;
    const unsigned has = __ballot_sync(0xffffffffu, cat != 0xffffffffu);
    if (cat != 0xffffffffu) {
      const unsigned peers = __match_any_sync(has, cat);
      if (lane == __ffs(peers) - 1) {
        if (cat & 1u)
          atomicAdd(low + (cat >> 1), (uint32_t)__popc(peers));
        else
          atomicAdd(cnt3 + nb1 + (cat >> 1), (uint32_t)__popc(peers));
      }
    }
    const unsigned hasm = __ballot_sync(0xffffffffu, ko != 0xffffffffu);
    if (ko != 0xffffffffu) {
      const unsigned peers = __match_any_sync(hasm, ko);
      if (lane == __ffs(peers) - 1) atomicAdd(cnt3 + 2 * nb1 + ko, (uint32_t)__popc(peers));
    }
    unsigned fl = flag;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fl |= __shfl_xor_sync(0xffffffffu, fl, o);
    if (fl && lane == 0) atomicOr(flags, fl);
  }
}

__global__ void k_repack_real(const float* __restrict__ src, int sp, float* __restrict__ dst,
                              int dp, int nm) {
  long long row = blockIdx.x;
  for (int z = threadIdx.x; z < nm; z += blockDim.x) dst[row * dp + z] = src[row * sp + z];
}

__global__ void k_repack_complex(const float2* __restrict__ src, int sp, float2* __restrict__ dst,
                                 int dp, int ncols) {
  long long row = blockIdx.x;
  for (int z = threadIdx.x; z < ncols; z += blockDim.x) dst[row * dp + z] = src[row * sp + z];
}

}  // namespace

void paint_tiles(pm_ctx* c, const uint32_t* us, const uint32_t* ids, int64_t n, int species,
                 float* mesh, int row_pitch, cudaStream_t s, const float* weights) {
  unsigned grid = (unsigned)(c->nt * c->nt * c->nt);
  float mmax = 0.0f;  // largest particle mass of the painted species
  if (species & PM_SPECIES_CDM) mmax = std::max(mmax, c->mt.m_cdm);
  if (species & PM_SPECIES_NU)
    for (int i = 0; i < c->mt.nshell && i < kMaxShell; ++i) mmax = std::max(mmax, c->mt.m_nu[i]);
  if (weights == nullptr && mmax < 128.0f && c->paint_redo) {
    // 32-bit pass, then the tiles whose words wrapped, in the carry form
    cudaMemsetAsync(c->paint_redo, 0, sizeof(uint32_t), s);
    {
      LaunchScope L(c, s, K_PAINT);
      k_paint_tiles<true><<<grid, kPaintThreads, 0, s>>>(us, ids, n, c->bstart, mesh, c->mt, species, c->g.n,
                                                         32 - c->g.logn, c->ntl, row_pitch, c->err_dev, nullptr,
                                                         mmax, c->paint_redo);
    }
    // persistent CTAs, as many as fit: the list is short, or empty, in most steps
    static int per_sm = 0, sms = 0;
    if (per_sm == 0) {
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_paint_redo, kPaintThreads, 0);
      if (per_sm < 1) per_sm = 1;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    }
    LaunchScope L(c, s, K_PAINT_REDO);
    k_paint_redo<<<(unsigned)std::min<long long>((long long)per_sm * sms, grid), kPaintThreads, 0, s>>>(
        us, ids, n, c->bstart, mesh, c->mt, species, c->g.n, 32 - c->g.logn, c->ntl, row_pitch, c->err_dev, mmax,
        c->paint_redo);
    return;
  }
  LaunchScope L(c, s, K_PAINT);
  k_paint_tiles<false><<<grid, kPaintThreads, 0, s>>>(us, ids, n, c->bstart, mesh, c->mt, species, c->g.n,
                                                      32 - c->g.logn, c->ntl, row_pitch, c->err_dev, weights, mmax,
                                                      nullptr);
}

void readout_kick(pm_ctx* c, const uint32_t* us, const float* ps, const uint32_t* ids, int64_t n,
                  const float* mesh, int row_pitch, int comp, float K, float* p_out, float* f_out,
                  uint32_t* u_out, uint32_t* id_out, const uint32_t* perm_scatter,
                  cudaStream_t s) {
  if (n == 0) return;
  LaunchScope L(c, s, K_READOUT_KICK);
  k_readout_kick<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
      us, ps, ids, n, mesh, c->g.n, 32 - c->g.logn, row_pitch, comp, K, p_out, f_out, u_out,
      id_out, perm_scatter);
}

void readout3_kick(pm_ctx* c, const uint32_t* us, const float* ps, const uint32_t* ids, int64_t n,
                   const float* mx, const float* my, const float* mz, int row_pitch, float K,
                   float* p_out, float* f_out, uint32_t* u_out, uint32_t* id_out,
                   const uint32_t* perm_scatter, cudaStream_t s) {
  if (n == 0) return;
  LaunchScope L(c, s, K_READOUT3_KICK);
  k_readout3_kick<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
      us, ps, ids, n, mx, my, mz, c->g.n, 32 - c->g.logn, row_pitch, K, p_out, f_out, u_out, id_out,
      perm_scatter);
}

void readout_fd4_kick(pm_ctx* c, const uint32_t* us, const float* ps, const uint32_t* ids, int64_t n,
                      const float* phi, int row_pitch, float K, float* p_out, float* f_out,
                      uint32_t* u_out, uint32_t* id_out, const uint32_t* perm_scatter, cudaStream_t s,
                      const DriftNext* dn) {
  if (n == 0) return;
  LaunchScope L(c, s, K_READOUT_FD4_KICK);
  const float inv12h = (float)((double)c->g.n / (12.0 * c->cfg.box));
  const unsigned grid = (unsigned)(c->nt * c->nt * c->nt);
  if (dn)
    k_readout_fd4_kick<true><<<grid, kFd4Threads, 0, s>>>(us, ps, ids, n, c->bstart, phi, c->g.n, 32 - c->g.logn,
                                                          c->ntl, row_pitch, inv12h, K, p_out, f_out, u_out,
                                                          id_out, nullptr, c->err_dev, *dn);
  else
    k_readout_fd4_kick<false><<<grid, kFd4Threads, 0, s>>>(us, ps, ids, n, c->bstart, phi, c->g.n,
                                                           32 - c->g.logn, c->ntl, row_pitch, inv12h, K, p_out,
                                                           f_out, u_out, id_out, perm_scatter, c->err_dev,
                                                           DriftNext{});
}

void kick_drift_keys(pm_ctx* c, uint32_t* u, float* p, const float* f, int64_t n, float K1,
                     float dscale, cudaStream_t s, bool resort) {
  const long long nb1 = c->nbuckets + 1;
  cudaMemsetAsync(c->counts, 0, sizeof(uint32_t) * (resort ? 3 * nb1 : nb1), s);
  if (resort) {
    cudaMemsetAsync(c->rs_low, 0, sizeof(uint32_t) * nb1, s);
    cudaMemsetAsync(c->rs_dev, 0, sizeof(uint32_t), s);
  }
  if (n == 0) return;
  LaunchScope L(c, s, K_KICK_DRIFT_KEYS);
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (resort)
    k_kick_drift_keys<true><<<grid, 256, 0, s>>>(u, p, f, n, K1, dscale, 32 - c->g.logn, c->ntl, c->keys[0],
                                                  c->counts, nb1, c->bprev, c->rs_low, c->rs_dev, c->err_dev);
  else
    k_kick_drift_keys<false><<<grid, 256, 0, s>>>(u, p, f, n, K1, dscale, 32 - c->g.logn, c->ntl, c->keys[0],
                                                   c->counts, nb1, nullptr, nullptr, nullptr, c->err_dev);
}

void repack_real(pm_ctx* c, const Geom& g, const float* src, int sp, float* dst, int dp,
                 cudaStream_t s) {
  LaunchScope L(c, s, K_REPACK);
  k_repack_real<<<(unsigned)g.rows(), 256, 0, s>>>(src, sp, dst, dp, g.n);
}

void repack_complex(pm_ctx* c, const Geom& g, const float2* src, int sp, float2* dst, int dp,
                    cudaStream_t s) {
  LaunchScope L(c, s, K_REPACK);
  k_repack_complex<<<(unsigned)g.rows(), 256, 0, s>>>(src, sp, dst, dp, g.n / 2 + 1);
}

}  // namespace pmnu
