// Stockham FFT engine shared by the FFT kernels (device code only).
//
// A line of M points (M a power of two, 16 <= M <= 2048) is held by M/V threads,
// V = 16 (8 or 32) values each (value s of thread j is element j + s M/V).  Stockham
// stages of radix V (the last stage radix 2..V) run in registers; between stages the line
// goes through shared memory, padded by one float2 per 16 (per 32 when V = 32) so that
// the stride-V writes of the first stage are free of bank conflicts.  A line's elements may be
// interleaved with other lines' (column stride cs in shared memory).  Twiddles
// come from a table e^{-2 pi i t / TWN} computed in double precision on the host.
#pragma once

#include "pm_internal.cuh"

namespace pmnu {
namespace fft {

__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }

// shared-memory index of element i of a line held V values a thread
template <int V>
__device__ __forceinline__ int padv(int i) {
  return V >= 32 ? i + (i >> 5) : padi(i);
}

// e^{s 2 pi i m / 16} for compile-time m, s = -1 forward, +1 inverse
template <int m, bool INV>
__device__ __forceinline__ float2 w16() {
  constexpr float C[16] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                           0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                           -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
                           0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
  constexpr float cv = C[m & 15];
  constexpr float sv = C[(m + 12) & 15];  // sin(2 pi m / 16) = cos(2 pi (m - 4) / 16)
  return INV ? make_float2(cv, sv) : make_float2(cv, -sv);
}

template <int m, bool INV>
__device__ __forceinline__ float2 rot16(float2 a) {
  if constexpr ((m & 15) == 0) {
    return a;
  } else if constexpr ((m & 15) == 4) {  // multiply by -i (forward) or +i (inverse)
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
  } else if constexpr ((m & 15) == 8) {
    return make_float2(-a.x, -a.y);
  } else if constexpr ((m & 15) == 12) {
    return INV ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
  } else {
    return cmul(a, w16<m, INV>());
  }
}

// e^{s 2 pi i m / 32} for odd compile-time m (the last layer of a 32-point DFT)
template <int m, bool INV>
__device__ __forceinline__ float2 w32() {
  // cos(2 pi t / 32), t = 0 .. 8
  constexpr float C[9] = {1.0f, 0.98078528040323044913f, 0.92387953251128675613f, 0.83146961230254523708f,
                          0.70710678118654752440f, 0.55557023301960222474f, 0.38268343236508977173f,
                          0.19509032201612826785f, 0.0f};
  constexpr int t = m & 31;  // cos and sin of 2 pi t / 32 from the first quadrant
  constexpr int q = t & 7, qq = t >> 3;
  constexpr float c0 = C[q], s0 = C[8 - q];
  constexpr float cv = qq == 0 ? c0 : qq == 1 ? -s0 : qq == 2 ? -c0 : s0;
  constexpr float sv = qq == 0 ? s0 : qq == 1 ? c0 : qq == 2 ? -s0 : -c0;
  return INV ? make_float2(cv, sv) : make_float2(cv, -sv);
}

// rotation by e^{s 2 pi i K / LEN} in a radix-2 layer of length LEN <= 32
template <int K, int LEN, bool INV>
__device__ __forceinline__ float2 rotl(float2 a) {
  if constexpr (LEN <= 16) {
    return rot16<K * (16 / LEN), INV>(a);
  } else if constexpr ((K & 1) == 0) {
    return rot16<K / 2, INV>(a);
  } else {
    return cmul(a, w32<K, INV>());
  }
}

template <int R>
__host__ __device__ constexpr int brev(int i) {
  int r = 0;
  for (int b = 1, k = R >> 1; b < R; b <<= 1, k >>= 1)
    if (i & b) r |= k;
  return r;
}

// In-register DFT of size R (2, 4, 8, 16, 32): radix-2 decimation in time.
template <int R, bool INV, int LEN = 2>
__device__ __forceinline__ void dft_layers(float2 (&x)[R]);

template <int R, bool INV, int LEN, int I, int K>
__device__ __forceinline__ void dft_bfly(float2 (&x)[R]) {
  if constexpr (I < R) {
    if constexpr (K < LEN / 2) {
      float2 a = x[I + K];
      float2 b = rotl<K, LEN, INV>(x[I + K + LEN / 2]);
      x[I + K] = cadd(a, b);
      x[I + K + LEN / 2] = csub(a, b);
      dft_bfly<R, INV, LEN, I, K + 1>(x);
    } else {
      dft_bfly<R, INV, LEN, I + LEN, 0>(x);
    }
  }
}

template <int R, bool INV, int LEN>
__device__ __forceinline__ void dft_layers(float2 (&x)[R]) {
  if constexpr (LEN <= R) {
    dft_bfly<R, INV, LEN, 0, 0>(x);
    dft_layers<R, INV, LEN * 2>(x);
  }
}

template <int R, int I>
__device__ __forceinline__ void bitrev_perm(float2 (&x)[R]) {
  if constexpr (I < R) {
    constexpr int J = brev<R>(I);
    if constexpr (J > I) {
      float2 t = x[I];
      x[I] = x[J];
      x[J] = t;
    }
    bitrev_perm<R, I + 1>(x);
  }
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2 (&x)[R]) {
  bitrev_perm<R, 0>(x);
  dft_layers<R, INV, 2>(x);
}

// Barrier between the shared-memory phases of a stage: the block, or only the warp when
// every line the warp touches is held by that warp alone (WARP).
template <bool WARP>
__device__ __forceinline__ void line_sync() {
  if constexpr (WARP) {
    __syncwarp();
  } else {
    __syncthreads();
  }
}

// One Stockham stage on a line of M points (sub-transform length NS, radix R), V values
// a thread (value s of thread j is element j + s M / V).
template <int M, int TWN, int NS, int R, bool INV, bool LAST, int V = 16, bool WARP = false>
__device__ __forceinline__ void stage(float2 (&v)[V], int j, float2* sm, int cs,
                                      const float2* __restrict__ tw) {
  constexpr int B = V / R;  // butterflies per thread
  constexpr int Q = M / V;
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int jj = j + b * Q;
    const int k = jj & (NS - 1);
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = v[b + r * B];
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = __ldg(tw + ((k * r * (TWN / (NS * R))) & (TWN - 1)));
        x[r] = cmul(x[r], INV ? cconj(w) : w);
      }
    }
    dft<R, INV>(x);
    if constexpr (LAST) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[b + r * B] = x[r];
    } else {
      const int base = (jj / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) sm[padv<V>(base + r * NS) * cs] = x[r];
    }
  }
  if constexpr (!LAST) {
    line_sync<WARP>();
#pragma unroll
    for (int s = 0; s < V; ++s) v[s] = sm[padv<V>(j + s * Q) * cs];
    line_sync<WARP>();
  }
}

template <int M, int TWN, int NS, bool INV, int V = 16, bool WARP = false>
__device__ __forceinline__ void run_stages(float2 (&v)[V], int j, float2* sm, int cs,
                                           const float2* __restrict__ tw) {
  constexpr int REM = M / NS;
  constexpr int R = REM >= V ? V : REM;
  constexpr bool LAST = (NS * R == M);
  stage<M, TWN, NS, R, INV, LAST, V, WARP>(v, j, sm, cs, tw);
  if constexpr (!LAST) run_stages<M, TWN, NS * R, INV, V, WARP>(v, j, sm, cs, tw);
}

// Twiddles a thread's stages use, held in registers.  They depend only on the thread's
// place j in its line, so a persistent kernel loads them once and reuses them for
// every tile.  Stage NS (radix R, B = V / R butterflies a thread) takes B (R - 1)
// entries, butterfly b's factor r at offset b (R - 1) + r - 1; the first stage (NS = 1)
// takes none.
template <int M, int NS, int V = 16>
__host__ __device__ constexpr int tw_count() {
  constexpr int REM = M / NS;
  constexpr int R = REM >= V ? V : REM;
  constexpr int own = NS > 1 ? (V / R) * (R - 1) : 0;
  if constexpr (NS * R == M) {
    return own;
  } else {
    return own + tw_count<M, NS * R, V>();
  }
}

template <int M, int TWN, int NS, int OFF, int NTW, int V = 16>
__device__ __forceinline__ void load_twiddles(float2 (&w)[NTW], int j, const float2* __restrict__ tw) {
  constexpr int REM = M / NS;
  constexpr int R = REM >= V ? V : REM;
  constexpr int B = V / R;
  constexpr int Q = M / V;
  if constexpr (NS > 1) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int k = (j + b * Q) & (NS - 1);
#pragma unroll
      for (int r = 1; r < R; ++r) w[OFF + b * (R - 1) + r - 1] = __ldg(tw + ((k * r * (TWN / (NS * R))) & (TWN - 1)));
    }
  }
  if constexpr (NS * R < M) load_twiddles<M, TWN, NS * R, OFF + (NS > 1 ? B * (R - 1) : 0), NTW, V>(w, j, tw);
}

// One Stockham stage with the twiddles from registers (see stage()).
template <int M, int NS, int R, bool INV, bool LAST, int OFF, int NTW, int V = 16>
__device__ __forceinline__ void stage_reg(float2 (&v)[V], int j, float2* sm, int cs, const float2 (&w)[NTW]) {
  constexpr int B = V / R;
  constexpr int Q = M / V;
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int jj = j + b * Q;
    const int k = jj & (NS - 1);
    float2 x[R];
#pragma unroll
    for (int r = 0; r < R; ++r) x[r] = v[b + r * B];
    if constexpr (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const float2 t = w[OFF + b * (R - 1) + r - 1];
        x[r] = cmul(x[r], INV ? cconj(t) : t);
      }
    }
    dft<R, INV>(x);
    if constexpr (LAST) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[b + r * B] = x[r];
    } else {
      const int base = (jj / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) sm[padv<V>(base + r * NS) * cs] = x[r];
    }
  }
  if constexpr (!LAST) {
    __syncthreads();
#pragma unroll
    for (int s = 0; s < V; ++s) v[s] = sm[padv<V>(j + s * Q) * cs];
    __syncthreads();
  }
}

template <int M, int NS, bool INV, int OFF, int NTW, int V = 16>
__device__ __forceinline__ void run_stages_reg(float2 (&v)[V], int j, float2* sm, int cs, const float2 (&w)[NTW]) {
  constexpr int REM = M / NS;
  constexpr int R = REM >= V ? V : REM;
  constexpr bool LAST = (NS * R == M);
  stage_reg<M, NS, R, INV, LAST, OFF, NTW, V>(v, j, sm, cs, w);
  if constexpr (!LAST) run_stages_reg<M, NS * R, INV, OFF + (NS > 1 ? (V / R) * (R - 1) : 0), NTW, V>(v, j, sm, cs, w);
}

// z pass, real -> complex, of one row: N reals read as M = N/2 complex values, held by
// M/V threads (j = 0 .. M/V - 1) with V values each (V = 16, or 32 for rows of 1024 and
// 2048 points: one exchange through shared memory fewer); ls is the row's shared-memory
// line (z_line<LOGN, V>() float2).  Writes the N/2 + 1 modes k = 0 .. M over the row in
// place.  ok = false: the thread takes part in the barriers only.
// The split of the half-length transform Z into the real transform needs Z_k and
// conj(Z_{M-k}): Z_k is the thread's own value, so only the mirrored one goes through
// shared memory, unpadded (a lane-contiguous descending read, free of bank conflicts).
template <int LOGN, bool WARP, int V = 16>
__device__ __forceinline__ void z_r2c_row(float2* __restrict__ rp, bool ok, int j, float2* ls,
                                          const float2* __restrict__ tw) {
  constexpr int N = 1 << LOGN, M = N / 2, TPL = M / V;
  float2 v[V];
#pragma unroll
  for (int s = 0; s < V; ++s) v[s] = ok ? rp[j + s * TPL] : make_float2(0.f, 0.f);
  run_stages<M, N, 1, false, V, WARP>(v, j, ls, 1, tw);
#pragma unroll
  for (int s = 0; s < V; ++s) ls[j + s * TPL] = v[s];
  line_sync<WARP>();
  if (ok) {
    auto mode = [&](int k, float2 zk, float2 zm) {
      const float2 e = cscale(cadd(zk, zm), 0.5f);
      const float2 o = cscale(csub(zk, zm), 0.5f);
      const float2 w = __ldg(tw + k);           // e^{-2 pi i k / N}
      const float2 wo = cmul(w, o);
      rp[k] = make_float2(e.x + wo.y, e.y - wo.x);  // e - i w o
    };
#pragma unroll
    for (int s = 0; s < V; ++s) {
      const int k = j + s * TPL;
      mode(k, v[s], cconj(ls[(M - k) & (M - 1)]));
    }
    if (j == 0) mode(M, v[0], cconj(v[0]));  // k = M: Z_0 and its own mirror
  }
}

// z pass, complex -> real, of one row in place (the inverse of z_r2c_row, unnormalised).
// X_k is the thread's own loaded value; only conj(X_{M-k}) is read back from shared memory.
template <int LOGN, bool WARP, int V = 16>
__device__ __forceinline__ void z_c2r_row(float2* __restrict__ rp, bool ok, int j, float2* ls,
                                          const float2* __restrict__ tw) {
  constexpr int N = 1 << LOGN, M = N / 2, TPL = M / V;
  float2 v[V];
#pragma unroll
  for (int s = 0; s < V; ++s) {
    v[s] = ok ? rp[j + s * TPL] : make_float2(0.f, 0.f);
    ls[j + s * TPL] = v[s];
  }
  if (j == 0) ls[M] = ok ? rp[M] : make_float2(0.f, 0.f);
  line_sync<WARP>();
#pragma unroll
  for (int s = 0; s < V; ++s) {
    const int k = j + s * TPL;
    const float2 xm = cconj(ls[M - k]);
    const float2 e = cadd(v[s], xm);
    const float2 d = csub(v[s], xm);
    const float2 w = cconj(__ldg(tw + k));   // e^{+2 pi i k / N}
    const float2 wd = cmul(w, d);
    v[s] = make_float2(e.x - wd.y, e.y + wd.x);  // e + i w d
  }
  line_sync<WARP>();
  run_stages<M, N, 1, true, V, WARP>(v, j, ls, 1, tw);
  if (ok) {
#pragma unroll
    for (int s = 0; s < V; ++s) rp[j + s * TPL] = v[s];  // (x[2n], x[2n+1])
  }
}

// values a thread and shared-memory line length (float2) of the z passes
template <int LOGN>
__host__ __device__ constexpr int z_values() {
  return LOGN >= 10 ? 32 : 16;
}
// A row's M + M/V-pad + 2 float2, rounded up so that rows sharing a 16-lane phase of a
// warp's 8-byte accesses (rows held by TPL < 16 threads) start TPL float2 apart modulo 16
// and so fall into disjoint banks.
template <int LOGN, int V = z_values<LOGN>()>
__host__ __device__ constexpr int z_line() {
  constexpr int M = 1 << (LOGN - 1), TPL = M / V;
  constexpr int base = M + M / (V >= 32 ? 32 : 16) + 2;
  if constexpr (TPL >= 16) {
    return base;
  } else {
    return base + ((TPL - base % 16) % 16 + 16) % 16;
  }
}

// Fused epilogue / prologue of the x pass.
struct KTables {
  const float* ksq;    // k_n^2, n in [0, N) (signed wavenumber of index n)
  const float* winv;   // per-axis factor of the Green's function, 1 / sinc^4(pi n_s / N) for the
                       // deconvolved spectral kernel; null: all factors 1 (the default kernel)
  const float* kvec0;  // gradient kernel D(k_n), 0 on the Nyquist index
  float gcoef;         // -1.5 Omega_m0 / N^3
  const float* mtab;   // learned factor by |n|^2 (n signed indices), null: plain kernel
};

// |n|^2 of a half-spectrum mode from its unsigned indices (kz <= M/2 is its own |n_z|)
template <int M>
__device__ __forceinline__ int nsq_index(int kx, int ky, int kz) {
  const int nx = kx < M / 2 ? kx : kx - M, ny = ky < M / 2 ? ky : ky - M;
  return nx * nx + ny * ny + kz * kz;
}

enum { EPI_NONE = 0, EPI_GREEN = 1, EPI_POT = 2 };  // EPI_POT: Green's function, then inverse
enum { PRO_NONE = 0, PRO_GRAD = 1 };

// MODE_POT: forward x FFT, Green's function, inverse x FFT (the potential, one output)
enum { MODE_PLAIN = 0, MODE_GREEN = 1, MODE_GRAD = 2, MODE_FUSED = 3, MODE_POT = 4 };

}  // namespace fft

// TMA-pipelined strided pass over one of the context's force meshes (k_fft_tma.cu);
// returns PM_EINVAL when it does not apply (no tensor maps, foreign buffer or size),
// so the caller runs the classic kernel instead.
int strided_tma(pm_ctx* c, const Geom& g, const float2* src, float2* d0, float2* d1, float2* d2,
                int axis, bool inv, int mode, int comp, const float2* tw, const fft::KTables& kt,
                cudaStream_t s);

}  // namespace pmnu
