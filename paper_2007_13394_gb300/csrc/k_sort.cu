// Stable counting sort of particles into 16^3-cell tiles of the mesh.
//
// key = tile * 8 + face class (see pm.h, pm_sort).  The per-key counts (an
// integer histogram, order independent) give every bucket's start by an
// exclusive scan; the particle order inside the key space comes from a stable
// least-significant-digit radix sort of (key, incoming index) with 8- or 9-bit
// digits (two 9-bit passes cover the 18-bit keys of meshes up to 512^3):
// per pass, an upsweep histogram per 4096-key block, a scan of the
// digit-major histogram, and a downsweep that ranks each key stably inside
// its block (warp match inside a round, warp-private digit counters across the
// warp's contiguous 512 keys, one block scan over (digit, warp)) and writes it
// through shared memory so that global writes stay coalesced.
//
// Near-sorted re-sort (pm_step): the state is in the order of the last step's sort,
// bucket starts bprev, and most particles keep their key.  A stayer (same key, inside
// its old key's range) keeps its relative order; movers are compacted in index order
// and radix-sorted alone.  Old ranges are ordered by key, so among the particles of new
// key B those with index below bprev[B] are exactly the movers from lower keys, those
// inside B's old range are B's stayers, the rest came from higher keys: bucket B is
// [lower movers | stayers | higher movers], which is the stable order.  The result is
// the same permutation as the radix sort from scratch; a particle outside its old
// key's range (a state not in bprev's order) sends the caller to that sort.
#include <cuda_runtime.h>

#include "pm_internal.cuh"

namespace pmnu {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096

constexpr int kRadixThreads = 256;
constexpr int kRadixRounds = 16;
constexpr int kRadixTile = kRadixThreads * kRadixRounds;  // 4096 keys per block
constexpr int kRadixWarps = kRadixThreads / 32;

// ------------------------------------------------------------------ keys
__global__ void k_keys(const uint32_t* __restrict__ u, int64_t n, int shift, int ntl,
                       uint32_t* __restrict__ keys, uint32_t* __restrict__ counts) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool ok = i < n;
  uint32_t key = 0xffffffffu;
  if (ok) {
    key = tile_key(u[i], u[n + i], u[2 * n + i], shift, ntl);
    keys[i] = key;
  }
  // warp-aggregated histogram increment
  unsigned act = __ballot_sync(0xffffffffu, ok);
  if (ok) {
    unsigned peers = __match_any_sync(act, key);
    int leader = __ffs(peers) - 1;
    if ((int)(threadIdx.x & 31) == leader) atomicAdd(counts + key, (uint32_t)__popc(peers));
  }
}

// ------------------------------------------------------------------ scan
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums,
                                                         uint32_t* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t s = lane < nw ? warp_sums[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) warp_sums[lane] = s;  // inclusive warp prefix
  }
  __syncthreads();
  uint32_t before = (w > 0 ? warp_sums[w - 1] : 0u) + (x - v);
  if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
  return before;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const uint32_t* __restrict__ in,
                                                            long long n,
                                                            uint32_t* __restrict__ sums) {
  __shared__ uint32_t ws[32];
  long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (base + k < n) s += in[base + k];
  uint32_t tot;
  block_exclusive_scan(s, ws, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t* __restrict__ in,
                                                             long long n,
                                                             const uint32_t* __restrict__ offs,
                                                             uint32_t* __restrict__ out) {
  __shared__ uint32_t ws[32];
  long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  uint32_t v[kScanItems], s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? in[base + k] : 0u;
    s += v[k];
  }
  uint32_t run = block_exclusive_scan(s, ws, nullptr) + (offs ? offs[blockIdx.x] : 0u);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
}

// ------------------------------------------------------------------ radix
// Digit width BITS (8 or 9): DIG digits, each of the 256 threads owns DIG / 256 of them.
template <int BITS>
__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const uint32_t* __restrict__ keys,
                                                              int64_t n, int shift,
                                                              long long nblk,
                                                              uint32_t* __restrict__ hist) {
  constexpr int DIG = 1 << BITS, PER = DIG / kRadixThreads;
  constexpr uint32_t MASK = DIG - 1;
  __shared__ uint32_t cnt[DIG];
#pragma unroll
  for (int q = 0; q < PER; ++q) cnt[threadIdx.x + q * kRadixThreads] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kRadixTile;
#pragma unroll 4
  for (int r = 0; r < kRadixRounds; ++r) {
    int64_t i = base + r * kRadixThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & MASK], 1u);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int d = threadIdx.x + q * kRadixThreads;
    hist[(long long)d * nblk + blockIdx.x] = cnt[d];
  }
}

// Stable scatter of one 4096-key block: warp w ranks the contiguous keys [512 w, 512 w + 512)
// of the block in 16 rounds of 32 (warp match for the rank inside a round, a warp-private
// per-digit counter across rounds), so the order inside each digit is the index order;
// one block-wide scan over (digit, warp) turns the counters into staging offsets; the
// keys are staged in digit order in shared memory and written out in coalesced runs.
template <int BITS>
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(
    const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, int64_t n, int shift,
    long long nblk, const uint32_t* __restrict__ hist, const uint32_t* __restrict__ hist_scan,
    uint32_t* __restrict__ kout, uint32_t* __restrict__ vout) {
  constexpr int DIG = 1 << BITS, PER = DIG / kRadixThreads;
  constexpr uint32_t MASK = DIG - 1;
  constexpr int KPW = kRadixTile / kRadixWarps;  // keys per warp
  constexpr int RPW = KPW / 32;                  // rounds per warp
  extern __shared__ uint32_t stage_kv[];  // keys then values of the block, in digit order
  uint32_t* sk = stage_kv;
  uint32_t* sv = stage_kv + kRadixTile;
  __shared__ uint32_t wcnt[kRadixWarps][DIG];  // per-warp digit counts, then staging offsets
  __shared__ uint32_t dstart[DIG];             // block-local start of each digit
  __shared__ uint32_t gbase[DIG];              // global start of this block's run of each digit
  __shared__ uint32_t ws[32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
  for (int i = t; i < kRadixWarps * DIG; i += kRadixThreads) (&wcnt[0][0])[i] = 0;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int d = t + q * kRadixThreads;
    gbase[d] = hist_scan[(long long)d * nblk + blockIdx.x];
  }
  __syncthreads();
  // 1. ranks inside the warp's digit runs
  const unsigned lt = (1u << lane) - 1u;
  uint32_t key[RPW], val[RPW], rk[RPW];
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int64_t i = base + w * KPW + r * 32 + lane;
    const bool ok = i < n;
    key[r] = ok ? kin[i] : 0u;
    val[r] = ok ? (vin ? vin[i] : (uint32_t)i) : 0u;
    const uint32_t d = ok ? ((key[r] >> shift) & MASK) : (uint32_t)(DIG + lane);
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t below = (uint32_t)__popc(peers & lt);
    const uint32_t c0 = ok ? wcnt[w][d] : 0u;  // every peer reads the count before this round
    rk[r] = c0 + below;
    __syncwarp();
    if (ok && below == 0) wcnt[w][d] = c0 + (uint32_t)__popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // 2. digit totals -> block-exclusive digit starts -> per-warp staging offsets
  {
    uint32_t c[PER], sum = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int d = t * PER + q;
      uint32_t tot = 0;
#pragma unroll
      for (int ww = 0; ww < kRadixWarps; ++ww) tot += wcnt[ww][d];
      c[q] = tot;
      sum += tot;
    }
    uint32_t ex = block_exclusive_scan(sum, ws, nullptr);
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int d = t * PER + q;
      dstart[d] = ex;
      uint32_t run = ex;
#pragma unroll
      for (int ww = 0; ww < kRadixWarps; ++ww) {
        const uint32_t cw = wcnt[ww][d];
        wcnt[ww][d] = run;
        run += cw;
      }
      ex += c[q];
    }
  }
  __syncthreads();
  // 3. stage in digit order
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int64_t i = base + w * KPW + r * 32 + lane;
    if (i < n) {
      const uint32_t d = (key[r] >> shift) & MASK;
      const uint32_t pos = wcnt[w][d] + rk[r];
      sk[pos] = key[r];
      sv[pos] = val[r];
    }
  }
  __syncthreads();
  // 4. coalesced runs to the digit's global position
  const int64_t cnt = (n - base) < kRadixTile ? (n - base) : kRadixTile;
  for (int j = t; j < cnt; j += kRadixThreads) {
    uint32_t k = sk[j];
    uint32_t d = (k >> shift) & MASK;
    uint32_t dst = gbase[d] + (j - dstart[d]);
    kout[dst] = k;
    vout[dst] = sv[j];
  }
}

// ------------------------------------------------------------------ gather
__global__ void k_gather(const uint32_t* __restrict__ u, const float* __restrict__ p,
                         const uint32_t* __restrict__ id, int64_t n,
                         const uint32_t* __restrict__ perm, uint32_t* __restrict__ us,
                         float* __restrict__ ps, uint32_t* __restrict__ ids) {
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  uint32_t i = perm[k];
  us[k] = u[i];
  us[n + k] = u[n + i];
  us[2 * n + k] = u[2 * n + i];
  if (p) {
    ps[k] = p[i];
    ps[n + k] = p[n + i];
    ps[2 * n + k] = p[2 * n + i];
  }
  ids[k] = id ? id[i] : i;
}

// ------------------------------------------------------------------ near-sorted re-sort
__device__ __forceinline__ void copy_particle(const uint32_t* __restrict__ u, const float* __restrict__ p,
                                              const uint32_t* __restrict__ id, int64_t n, uint32_t i,
                                              uint32_t dst, uint32_t* __restrict__ us, float* __restrict__ ps,
                                              uint32_t* __restrict__ ids) {
  us[dst] = u[i];
  us[n + dst] = u[n + i];
  us[2 * n + dst] = u[2 * n + i];
  if (p) {
    ps[dst] = p[i];
    ps[n + dst] = p[n + i];
    ps[2 * n + dst] = p[2 * n + i];
  }
  ids[dst] = id ? id[i] : i;
}

// One CTA per old tile O: walks O's range [bprev[8 O], bprev[8 O + 8]) in chunks of the
// block size, in index order.  With stage, a mover's position, momentum and id also go to a
// 32-byte record at its list position (the placement then reads one sector a mover
// instead of seven scattered words), and mv holds that position.  A block scan of the mover flags gives every particle the
// number of movers of its own old key before it (mrank); a stayer goes to
// bstart[B] + low[B] + (i - bprev[B]) - mrank, a mover's (new key, index) to its old
// key's slot of the mover list, mstart3[ko] - base3 + mrank (movers in index order).
constexpr int kResortThreads = 256;

__global__ void __launch_bounds__(kResortThreads) k_resort_old_tiles(
    const uint32_t* __restrict__ u, const float* __restrict__ p, const uint32_t* __restrict__ id, int64_t n,
    const uint32_t* __restrict__ keys, const uint32_t* __restrict__ bprev, const uint32_t* __restrict__ bstart3,
    long long nb1, const uint32_t* __restrict__ low, uint32_t* __restrict__ us, float* __restrict__ ps,
    uint32_t* __restrict__ ids, uint32_t* __restrict__ mk, uint32_t* __restrict__ mv, int64_t nm,
    int* __restrict__ err, uint4* __restrict__ stage) {
  constexpr int W = kResortThreads / 32;
  __shared__ uint32_t cls_lo[9];   // bprev[8 O + c]
  __shared__ uint32_t cls_m0[8];   // movers of the tile before class c's first particle
  __shared__ uint32_t wsum[W];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const uint32_t O = blockIdx.x;
  if (t < 9) cls_lo[t] = bprev[8 * O + t];
  __syncthreads();
  const uint32_t lo = cls_lo[0], hi = cls_lo[8];
  if (lo == hi) return;
  const uint32_t base3 = bstart3[2 * nb1];  // n + all stayers: offset of the third scan
  const unsigned lt = (1u << lane) - 1u;
  uint32_t run = 0;  // movers of the tile before this chunk
  for (uint32_t chunk = lo; chunk < hi; chunk += kResortThreads) {
    const uint32_t i = chunk + t;
    const bool ok = i < hi;
    uint32_t kn = 0, c = 0;
    uint32_t pu[3] = {0u, 0u, 0u}, pid = 0u;
    float pp[3] = {0.f, 0.f, 0.f};
    if (ok) {  // the particle's data is loaded before the block scan, not after it
      kn = keys[i];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        pu[d] = u[d * n + i];
        if (p) pp[d] = p[d * n + i];
      }
      pid = id ? id[i] : i;
#pragma unroll
      for (int k = 1; k < 8; ++k) c += i >= cls_lo[k] ? 1u : 0u;
    }
    const uint32_t ko = 8 * O + c;
    const bool mover = ok && kn != ko;
    // where the particle's run starts: B's stayers, or old key ko's slot of the mover list
    const uint32_t run0 = !ok ? 0u : (mover ? bstart3[2 * nb1 + ko] - base3 : bstart3[ko] + low[ko]);
    const unsigned bal = __ballot_sync(0xffffffffu, mover);
    if (lane == 0) wsum[w] = (uint32_t)__popc(bal);
    __syncthreads();
    uint32_t before = run, total = 0;
#pragma unroll
    for (int ww = 0; ww < W; ++ww) {
      before += ww < w ? wsum[ww] : 0u;
      total += wsum[ww];
    }
    const uint32_t mex = before + (uint32_t)__popc(bal & lt);  // movers of the tile before i
    if (ok && i == cls_lo[c]) cls_m0[c] = mex;                   // class c starts here
    __syncthreads();
    if (ok) {
      const uint32_t mrank = mex - cls_m0[c];
      if (!mover) {
        const uint32_t dst = run0 + (i - cls_lo[c]) - mrank;
        if (dst < (uint64_t)n) {
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            us[d * n + dst] = pu[d];
            if (p) ps[d * n + dst] = pp[d];
          }
          ids[dst] = pid;
        } else {
          atomicOr(err, 1);  // inconsistent counts: never written out of range
        }
      } else {
        const uint32_t pos = run0 + mrank;
        if (pos < (uint64_t)nm) {
          mk[pos] = kn;
          if (stage) {  // the mover's 28 bytes as one 32-byte record at its list position
            mv[pos] = pos;
            stage[2 * (size_t)pos] = make_uint4(pu[0], pu[1], pu[2], pid);
            stage[2 * (size_t)pos + 1] = make_uint4(__float_as_uint(pp[0]), __float_as_uint(pp[1]),
                                                    __float_as_uint(pp[2]), 0u);
          } else {
            mv[pos] = i;
          }
        } else {
          atomicOr(err, 1);
        }
      }
    }
    run += total;
    __syncthreads();  // wsum is rewritten by the next chunk
  }
}

// Mover r of new key B in the movers' stable order: destination bstart[B] + r, behind B's
// stayers when it came from a higher key (r >= low[B]).  The movers of keys below B
// number bstart[B] - sstart[B], sstart = the stayers' scan (bstart3's second third
// minus n).
__global__ void k_place_movers(const uint32_t* __restrict__ mk, const uint32_t* __restrict__ mv, int64_t nm,
                               const uint32_t* __restrict__ u, const float* __restrict__ p,
                               const uint32_t* __restrict__ id, int64_t n, const uint32_t* __restrict__ bstart3,
                               long long nb1, long long nbuckets, const uint32_t* __restrict__ low,
                               uint32_t* __restrict__ us, float* __restrict__ ps, uint32_t* __restrict__ ids,
                               int* __restrict__ err, const uint4* __restrict__ stage) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nm) return;
  const uint32_t B = mk[j];
  if (B >= (uint64_t)nbuckets || mv[j] >= (uint64_t)(stage ? nm : n)) {
    atomicOr(err, 1);
    return;
  }
  const uint32_t s0 = bstart3[nb1 + B], s1 = bstart3[nb1 + B + 1];
  const uint32_t r = (uint32_t)j - (bstart3[B] - (s0 - (uint32_t)n));
  const uint32_t dst = bstart3[B] + r + (r >= low[B] ? s1 - s0 : 0u);
  if (dst >= (uint64_t)n) {
    atomicOr(err, 1);
    return;
  }
  if (stage) {  // one 32-byte record (mv: its position in the mover list)
    const uint4 a = stage[2 * (size_t)mv[j]], b = stage[2 * (size_t)mv[j] + 1];
    us[dst] = a.x;
    us[n + dst] = a.y;
    us[2 * n + dst] = a.z;
    ids[dst] = a.w;
    if (p) {
      ps[dst] = __uint_as_float(b.x);
      ps[n + dst] = __uint_as_float(b.y);
      ps[2 * n + dst] = __uint_as_float(b.z);
    }
  } else {
    copy_particle(u, p, id, n, mv[j], dst, us, ps, ids);
  }
}

}  // namespace

namespace {
// Reduce-then-scan; level k keeps its block sums and their scanned offsets in tmp,
// the next level works further along tmp (total < 2.001 * ceil(n / 4096) words).
void scan_rec(pm_ctx* c, const uint32_t* in, uint32_t* out, long long n, uint32_t* tmp,
              cudaStream_t s) {
  long long nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 1) {
    LaunchScope L(c, s, K_SCAN);
    k_scan_apply<<<1, kScanThreads, 0, s>>>(in, n, nullptr, out);
    return;
  }
  uint32_t* sums = tmp;
  uint32_t* offs = tmp + nb;
  {
    LaunchScope L(c, s, K_SCAN);
    k_scan_sums<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
  }
  scan_rec(c, sums, offs, nb, tmp + 2 * nb, s);
  {
    LaunchScope L(c, s, K_SCAN);
    k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, offs, out);
  }
}
}  // namespace

void scan_exclusive(pm_ctx* c, const uint32_t* in, uint32_t* out, long long n, cudaStream_t s) {
  if (n <= 0) return;
  scan_rec(c, in, out, n, c->scan_tmp, s);
}

int build_keys(pm_ctx* c, const uint32_t* u, int64_t n, cudaStream_t s) {
  if (cudaMemsetAsync(c->counts, 0, sizeof(uint32_t) * (c->nbuckets + 1), s) != cudaSuccess)
    return PM_ECUDA;
  if (n > 0) {
    LaunchScope L(c, s, K_KEYS);
    unsigned grid = (unsigned)((n + 255) / 256);
    k_keys<<<grid, 256, 0, s>>>(u, n, 32 - c->g.logn, c->ntl, c->keys[0], c->counts);
  }
  return PM_OK;
}

namespace {
// LSD radix passes of the context's digit width over n (key, value) pairs in buffer pair
// 0 (values absent: the incoming index), pair 1 the other buffers.  Returns which pair
// holds the result.
int radix_passes(pm_ctx* c, uint32_t* const kb[2], uint32_t* const vb[2], bool index_vals, int64_t n,
                 cudaStream_t s) {
  const long long nblk = (n + kRadixTile - 1) / kRadixTile;
  int cur = 0;
  const int bits = c->radix_bits;
  for (int pass = 0; pass < c->radix_passes; ++pass) {
    int shift = bits * pass;
    {
      LaunchScope L(c, s, K_RADIX_HIST);
      if (bits == 9)
        k_radix_hist<9><<<(unsigned)nblk, kRadixThreads, 0, s>>>(kb[cur], n, shift, nblk, c->hist);
      else
        k_radix_hist<8><<<(unsigned)nblk, kRadixThreads, 0, s>>>(kb[cur], n, shift, nblk, c->hist);
    }
    scan_exclusive(c, c->hist, c->hist_scan, (1LL << bits) * nblk, s);
    {
      LaunchScope L(c, s, K_RADIX_SCATTER);
      const uint32_t* vin = (pass == 0 && index_vals) ? nullptr : vb[cur];
      const int dyn = 2 * kRadixTile * (int)sizeof(uint32_t);
      static bool attr = false;
      if (!attr) {
        cudaFuncSetAttribute(k_radix_scatter<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        cudaFuncSetAttribute(k_radix_scatter<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        attr = true;
      }
      if (bits == 9)
        k_radix_scatter<9><<<(unsigned)nblk, kRadixThreads, dyn, s>>>(kb[cur], vin, n, shift, nblk, c->hist,
                                                                      c->hist_scan, kb[cur ^ 1], vb[cur ^ 1]);
      else
        k_radix_scatter<8><<<(unsigned)nblk, kRadixThreads, dyn, s>>>(kb[cur], vin, n, shift, nblk, c->hist,
                                                                      c->hist_scan, kb[cur ^ 1], vb[cur ^ 1]);
    }
    cur ^= 1;
  }
  return cur;
}
}  // namespace

int radix_and_buckets(pm_ctx* c, int64_t n, cudaStream_t s) {
  // bucket starts: exclusive scan of the nbuckets + 1 counts (last count is 0 -> total)
  scan_exclusive(c, c->counts, c->bstart, c->nbuckets + 1, s);
  if (n == 0) return PM_OK;
  if ((n + kRadixTile - 1) / kRadixTile > c->hist_blocks_max) return PM_EINVAL;
  uint32_t* const kb[2] = {c->keys[0], c->keys[1]};
  uint32_t* const vb[2] = {c->vals[0], c->vals[1]};
  if (radix_passes(c, kb, vb, true, n, s) != 0) {  // keep the result in keys[0] / vals[0]
    std::swap(c->keys[0], c->keys[1]);
    std::swap(c->vals[0], c->vals[1]);
  }
  return PM_OK;
}

int sort_particles(pm_ctx* c, const uint32_t* u, int64_t n, cudaStream_t s) {
  int st = build_keys(c, u, n, s);
  if (st != PM_OK) return st;
  return radix_and_buckets(c, n, s);
}

void gather_sorted(pm_ctx* c, const uint32_t* u, const float* p, const uint32_t* id, int64_t n,
                   const uint32_t* perm, cudaStream_t s) {
  if (n == 0) return;
  LaunchScope L(c, s, K_GATHER);
  k_gather<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(u, p, id, n, perm, c->us, c->ps, c->ids);
}

int resort_near_sorted(pm_ctx* c, const uint32_t* u, const float* p, const uint32_t* id, int64_t n,
                       cudaStream_t s) {
  const long long nb1 = c->nbuckets + 1;
  // bucket starts, stayers' and old keys' movers' starts in one scan
  scan_exclusive(c, c->counts, c->bstart, 3 * nb1, s);
  if (n == 0) return 1;
  PM_CUDA_TRY(cudaMemcpyAsync(c->rs_host, c->rs_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  PM_CUDA_TRY(cudaMemcpyAsync(c->rs_host + 1, c->bstart + 2 * nb1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  PM_CUDA_TRY(cudaMemcpyAsync(c->rs_host + 2, c->bstart + 3 * nb1 - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  PM_CUDA_TRY(cudaStreamSynchronize(s));
  if (c->rs_host[0] & 1u) return 0;  // not the order of bprev: sort from scratch
  const int64_t nm = (int64_t)c->rs_host[2] - (int64_t)c->rs_host[1];
  if (nm < 0 || nm > n || (nm + kRadixTile - 1) / kRadixTile > c->hist_blocks_max) return PM_EINVAL;
  c->rs_last_movers = nm;
  // the movers' records go to the second mesh, free during a step, when they fit (32 bytes a
  // mover: up to 2^30 movers at 2048^3); else the placement gathers from the state itself
  uint4* stage = nullptr;
  if (c->meshB && (size_t)nm * 32 <= c->g.elems() * sizeof(float2)) stage = reinterpret_cast<uint4*>(c->meshB);
  {
    LaunchScope L(c, s, K_RESORT_PLACE);
    k_resort_old_tiles<<<(unsigned)((long long)c->nt * c->nt * c->nt), kResortThreads, 0, s>>>(
        u, p, id, n, c->keys[0], c->bprev, c->bstart, nb1, c->rs_low, c->us, c->ps, c->ids, c->keys[1], c->vals[1],
        nm, c->err_dev, stage);
  }
  if (nm > 0) {
    uint32_t* const kb[2] = {c->keys[1], c->rs_k2};
    uint32_t* const vb[2] = {c->vals[1], c->rs_v2};
    const int r = radix_passes(c, kb, vb, false, nm, s);
    LaunchScope L(c, s, K_RESORT_MISC);
    k_place_movers<<<(unsigned)((nm + 255) / 256), 256, 0, s>>>(kb[r], vb[r], nm, u, p, id, n, c->bstart, nb1,
                                                                 c->nbuckets, c->rs_low, c->us, c->ps, c->ids,
                                                                 c->err_dev, stage);
  }
  return 1;
}

}  // namespace pmnu
