// Shared-memory / register radix FFT building blocks for M x M complex64 tiles.
//
// The far-field propagator of Eq. 1 is a 2-D DFT; the near-field Fresnel
// transfer-function propagator is a DFT, a pointwise product and an inverse
// DFT. One CTA transforms one M x M tile (M a power of two, 8..256) with
// T = M * G threads, G = M / E, E = min(16, M): every thread keeps E complex
// values in registers.
//
// A length-M 1-D DFT is split as M = E x G (Cooley-Tukey four-step):
//   pass 1  DFT-E over j of x[t + G j]            (thread t = 0..G-1, in registers)
//           times the twiddle W_M^(t k2)
//   swap    through shared memory (exchange "A")
//   pass 2  DFT-G over t for the E/G values k2 this thread owns
//           -> X[k2 + E k1]
// The 2-D transform runs rows then columns with a transpose (exchange "B")
// between them. The inverse runs the same steps mirrored, so it consumes the
// register layout that the forward leaves and returns to the starting one.
//
// Thread mappings (virtual thread vt in [0, T)):
//   ROW phase   (line, t) = (vt / G, vt % G); register j holds element (line, t + G j)
//   COLUMN phase (c, t)   = (vt / G, vt % G); after the forward transform register
//               r = i2 * G + k1 holds frequency (u, c), u = t * (E / G) + i2 + E k1
// The G threads of one line sit in one warp, so the line-internal swaps need
// only a warp barrier; the transpose needs the whole CTA.
//
// Shared-memory layouts are affine in the thread's fixed coordinates plus a
// compile-time offset (so no per-element address survives across phases), and
// every exchange is bank-conflict-free for 8-byte elements:
//   line-internal swap     line * LDA + k2 * SA + t * ST   (SA, ST, LDA per M below)
//   transpose              x * M + (y ^ hB(x)), hB(x) = (x' & ~m) ^ ((x' & m) << (log2 E - s)),
//                          x' = x mod E, m = 2^s - 1, s = log2(E / G)  (XOR swizzle)
//   twiddles W_M^(t k2)    t * (E + 1) + k2
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ptycho {

// ------------------------------------------------------------------ complex helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// conj(a) * b
__device__ __forceinline__ float2 cconjmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// multiply by the primitive 4th root used by the transform direction:
// forward (e^{-2 pi i / 4} = -i), inverse (+i)
template <bool INV>
__device__ __forceinline__ float2 mul_w4(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos(2 pi m / 16) and sin(2 pi m / 16), m = 0..15, from the exact values
// cos(pi/8) = sqrt(2 + sqrt 2) / 2, sin(pi/8) = sqrt(2 - sqrt 2) / 2, sqrt(2)/2.
__host__ __device__ constexpr float cos16(int m) {
  return (m & 15) == 0 ? 1.0f : (m & 15) == 1 ? 0.92387953251128674f : (m & 15) == 2 ? 0.70710678118654752f
       : (m & 15) == 3 ? 0.38268343236508978f : (m & 15) == 4 ? 0.0f : (m & 15) == 5 ? -0.38268343236508978f
       : (m & 15) == 6 ? -0.70710678118654752f : (m & 15) == 7 ? -0.92387953251128674f : (m & 15) == 8 ? -1.0f
       : (m & 15) == 9 ? -0.92387953251128674f : (m & 15) == 10 ? -0.70710678118654752f
       : (m & 15) == 11 ? -0.38268343236508978f : (m & 15) == 12 ? 0.0f : (m & 15) == 13 ? 0.38268343236508978f
       : (m & 15) == 14 ? 0.70710678118654752f : 0.92387953251128674f;
}
__host__ __device__ constexpr float sin16(int m) { return cos16(m + 12); }  // sin(a) = cos(a - pi/2)

// x * W_16^m, W = e^{-2 pi i / 16} (forward) or its conjugate (inverse)
template <bool INV, int m>
__device__ __forceinline__ float2 mul_w16(float2 a) {
  constexpr int mm = m & 15;
  if constexpr (mm == 0) return a;
  else if constexpr (mm == 4) return mul_w4<INV>(a);
  else if constexpr (mm == 8) return make_float2(-a.x, -a.y);
  else if constexpr (mm == 12) return mul_w4<!INV>(a);
  else {
    constexpr float c = cos16(mm);
    constexpr float s = INV ? sin16(mm) : -sin16(mm);
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
  }
}

// ------------------------------------------------------------------ register DFTs (natural order in and out)
template <bool INV>
__device__ __forceinline__ void dft2(float2& a0, float2& a1) {
  float2 t = a0;
  a0 = cadd(t, a1);
  a1 = csub(t, a1);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
  float2 s13 = cadd(a1, a3), d13 = mul_w4<INV>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

template <bool INV>
__device__ __forceinline__ void dft8(float2* a) {
  // decimation in time: even / odd halves
  float2 e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  float2 o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  o1 = mul_w16<INV, 2>(o1);
  o2 = mul_w16<INV, 4>(o2);
  o3 = mul_w16<INV, 6>(o3);
  a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
  a[1] = cadd(e1, o1); a[5] = csub(e1, o1);
  a[2] = cadd(e2, o2); a[6] = csub(e2, o2);
  a[3] = cadd(e3, o3); a[7] = csub(e3, o3);
}

template <bool INV>
__device__ __forceinline__ void dft16(float2* a) {
  // j = j1 + 4 j2: DFT-4 over j2 for each j1, twiddle W16^(j1 k2), DFT-4 over j1: X[k2 + 4 k1]
  float2 b[16];
#pragma unroll
  for (int j1 = 0; j1 < 4; ++j1) {
    float2 x0 = a[j1], x1 = a[j1 + 4], x2 = a[j1 + 8], x3 = a[j1 + 12];
    dft4<INV>(x0, x1, x2, x3);
    b[j1 * 4 + 0] = x0; b[j1 * 4 + 1] = x1; b[j1 * 4 + 2] = x2; b[j1 * 4 + 3] = x3;
  }
  b[1 * 4 + 1] = mul_w16<INV, 1>(b[1 * 4 + 1]);
  b[1 * 4 + 2] = mul_w16<INV, 2>(b[1 * 4 + 2]);
  b[1 * 4 + 3] = mul_w16<INV, 3>(b[1 * 4 + 3]);
  b[2 * 4 + 1] = mul_w16<INV, 2>(b[2 * 4 + 1]);
  b[2 * 4 + 2] = mul_w16<INV, 4>(b[2 * 4 + 2]);
  b[2 * 4 + 3] = mul_w16<INV, 6>(b[2 * 4 + 3]);
  b[3 * 4 + 1] = mul_w16<INV, 3>(b[3 * 4 + 1]);
  b[3 * 4 + 2] = mul_w16<INV, 6>(b[3 * 4 + 2]);
  b[3 * 4 + 3] = mul_w16<INV, 9>(b[3 * 4 + 3]);
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    float2 x0 = b[0 * 4 + k2], x1 = b[1 * 4 + k2], x2 = b[2 * 4 + k2], x3 = b[3 * 4 + k2];
    dft4<INV>(x0, x1, x2, x3);
    a[k2 + 0] = x0; a[k2 + 4] = x1; a[k2 + 8] = x2; a[k2 + 12] = x3;
  }
}

// cos(2 pi m / 32): cos(pi k / 16) for k = 0..8 from the half-angle identities (exact decimal expansions of
// cos(pi/16) = sqrt(2 + sqrt(2 + sqrt 2)) / 2 and its neighbours), extended by symmetry
__host__ __device__ constexpr float cos32(int m) {
  constexpr float C[9] = {1.0f, 0.98078528040323044913f, 0.92387953251128675613f, 0.83146961230254523708f,
                          0.70710678118654752440f, 0.55557023301960222474f, 0.38268343236508977173f,
                          0.19509032201612826785f, 0.0f};
  const int r = m & 31, a = r > 16 ? 32 - r : r;
  return a <= 8 ? C[a] : -C[16 - a];
}
__host__ __device__ constexpr float sin32(int m) { return cos32(m - 8); }  // sin(a) = cos(a - pi/2)

// x * W_32^m, W = e^{-2 pi i / 32} (forward) or its conjugate (inverse)
template <bool INV, int m>
__device__ __forceinline__ float2 mul_w32(float2 a) {
  if constexpr ((m & 1) == 0) {
    return mul_w16<INV, m / 2>(a);
  } else {
    constexpr float c = cos32(m);
    constexpr float s = INV ? sin32(m) : -sin32(m);
    return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.x, s, a.y * c));
  }
}

// butterflies k, k + 1, .., 15 of the DFT-32: a[k] = e[k] + W_32^k o[k], a[k + 16] = e[k] - W_32^k o[k]
template <bool INV, int K>
__device__ __forceinline__ void bfly32(float2* a, const float2* e, const float2* o) {
  const float2 t = mul_w32<INV, K>(o[K]);
  a[K] = cadd(e[K], t);
  a[K + 16] = csub(e[K], t);
  if constexpr (K < 15) bfly32<INV, K + 1>(a, e, o);
}

// DFT-32 in registers, natural order in and out: even and odd halves by DFT-16, then the butterflies
template <bool INV>
__device__ __forceinline__ void dft32(float2* a) {
  float2 e[16], o[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    e[j] = a[2 * j];
    o[j] = a[2 * j + 1];
  }
  dft16<INV>(e);
  dft16<INV>(o);
  bfly32<INV, 0>(a, e, o);
}

template <int N, bool INV>
__device__ __forceinline__ void dft(float2* a) {
  if constexpr (N == 1) {
  } else if constexpr (N == 2) {
    dft2<INV>(a[0], a[1]);
  } else if constexpr (N == 4) {
    dft4<INV>(a[0], a[1], a[2], a[3]);
  } else if constexpr (N == 8) {
    dft8<INV>(a);
  } else if constexpr (N == 16) {
    dft16<INV>(a);
  } else if constexpr (N == 32) {
    dft32<INV>(a);
  } else {
    static_assert(N == 1, "unsupported register DFT size");
  }
}

// ------------------------------------------------------------------ tile geometry
template <int M_>
struct Tile {
  static constexpr int M = M_;
  static constexpr int E = M < 16 ? M : 16;  // registers per line
  static constexpr int G = M / E;             // threads per line
  static constexpr int T = M * G;             // virtual threads per tile
  static constexpr int EG = E / G;            // pass-2 DFTs per thread
  static_assert(M == 8 || M == 16 || M == 32 || M == 64 || M == 128 || M == 256, "M must be 8..256");
  // row-internal swap strides (searched for conflict-free half-warps)
  static constexpr int SA = M == 32 ? 3 : M == 64 ? 5 : M == 128 ? 1 : M == 256 ? 17 : 1;
  static constexpr int ST = M == 32 ? 8 : M == 64 ? 4 : M == 128 ? 18 : M == 256 ? 1 : 1;
  static constexpr int LDA = M == 32 ? 55 : M == 64 ? 89 : M == 128 ? 143 : M == 256 ? 271 : E;
  static constexpr int LDN = G > 1 ? M + G : M + 1;   // natural [y][x] layout row stride
  static constexpr int LDW = E + 1;                   // twiddle table row stride
  static constexpr int LOG2E = E == 16 ? 4 : E == 8 ? 3 : 0;
  static constexpr int S = EG == 16 ? 4 : EG == 8 ? 3 : EG == 4 ? 2 : EG == 2 ? 1 : 0;
  static constexpr int cmax(int a, int b) { return a > b ? a : b; }
  static constexpr int SMEM = cmax(cmax(G > 1 ? M * LDA : 0, M * M), M * LDN);  // float2 slots

  __device__ __forceinline__ static int idxA(int line, int t, int k2) { return line * LDA + k2 * SA + t * ST; }
  __device__ __forceinline__ static int idxB(int y, int x) {
    constexpr int m = (1 << S) - 1;
    const int xl = x & (E - 1);
    return x * M + (y ^ ((xl & ~m) ^ ((xl & m) << (LOG2E - S))));
  }
  __device__ __forceinline__ static int idxN(int y, int x) { return y * LDN + x; }
};

// ------------------------------------------------------------------ 2-D transform steps
// tw[m] = W_M^m for m in [0, M) (forward convention); the inverse uses conj.
// A CTA of T / V threads runs the tile: thread `tid` plays the V virtual
// threads vtid = tid + v * (T / V), v in [0, V), and keeps V x E registers.

// a[v][k2] *= W_M^(t k2) (INV: times the conjugate) for k2 = 1 .. E-1, t the part of virtual thread
// v. When the CTA's thread count is a multiple of G every virtual thread of a thread has the same
// part, and each twiddle is read from shared memory once for all V lines.
template <int M, int V, bool INV>
__device__ __forceinline__ void twiddle(float2 (&a)[V][Tile<M>::E], const float2* tw, int tid) {
  using TL = Tile<M>;
  constexpr int E = TL::E, G = TL::G, TR = TL::T / V, W = TL::LDW;
  if constexpr (TR % G == 0) {
    const int t = tid % G;
#pragma unroll
    for (int k2 = 1; k2 < E; ++k2) {
      const float2 w = tw[t * W + k2];
#pragma unroll
      for (int v = 0; v < V; ++v) a[v][k2] = INV ? cmulc(a[v][k2], w) : cmul(a[v][k2], w);
    }
  } else {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int t = (tid + v * TR) % G;
#pragma unroll
      for (int k2 = 1; k2 < E; ++k2) a[v][k2] = INV ? cmulc(a[v][k2], tw[t * W + k2]) : cmul(a[v][k2], tw[t * W + k2]);
    }
  }
}

// ROW layout registers -> COL layout registers (forward 2-D DFT, unscaled).
// tw: twiddle table, tw[t * (E + 1) + k2] = W_M^(t k2) for t < G.
// The shared buffer must be free on entry; it is free again on return.
template <int M, int V>
__device__ __forceinline__ void fft2_forward(float2 (&a)[V][Tile<M>::E], float2* sm, const float2* tw, int tid) {
  using TL = Tile<M>;
  constexpr int E = TL::E, G = TL::G, EG = TL::EG, TR = TL::T / V;
  // ---- rows: pass 1 (ROW mapping)
#pragma unroll
  for (int v = 0; v < V; ++v) dft<E, false>(a[v]);
  twiddle<M, V, false>(a, tw, tid);
  if constexpr (G > 1) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int line = (tid + v * TR) / G, t = (tid + v * TR) % G;
#pragma unroll
      for (int k2 = 0; k2 < E; ++k2) sm[TL::idxA(line, t, k2)] = a[v][k2];
    }
    __syncwarp();  // the swap stays inside the warp
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int line = (tid + v * TR) / G, t = (tid + v * TR) % G;
#pragma unroll
      for (int i2 = 0; i2 < EG; ++i2)
#pragma unroll
        for (int tt = 0; tt < G; ++tt) a[v][i2 * G + tt] = sm[TL::idxA(line, tt, t * EG + i2)];
      // ---- rows: pass 2
#pragma unroll
      for (int i2 = 0; i2 < EG; ++i2) dft<G, false>(&a[v][i2 * G]);
    }
    __syncthreads();
  }
  // ---- transpose: ROW thread (line, t) holds x = t * EG + i2 + E k1 at register i2 * G + k1
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int line = (tid + v * TR) / G, t = (tid + v * TR) % G;
#pragma unroll
    for (int i2 = 0; i2 < EG; ++i2)
#pragma unroll
      for (int k1 = 0; k1 < G; ++k1) sm[TL::idxB(line, t * EG + i2 + E * k1)] = a[v][i2 * G + k1];
  }
  __syncthreads();
  // ---- columns (COLUMN mapping): column c reads y = t + G j
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int c = (tid + v * TR) / G, t = (tid + v * TR) % G;
#pragma unroll
    for (int j = 0; j < E; ++j) a[v][j] = sm[TL::idxB(t + G * j, c)];
    dft<E, false>(a[v]);
  }
  twiddle<M, V, false>(a, tw, tid);
  if constexpr (G > 1) {
    __syncthreads();
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int c = (tid + v * TR) / G, t = (tid + v * TR) % G;
#pragma unroll
      for (int k2 = 0; k2 < E; ++k2) sm[TL::idxA(c, t, k2)] = a[v][k2];
    }
    __syncwarp();  // the swap stays inside the warp
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int c = (tid + v * TR) / G, t = (tid + v * TR) % G;
#pragma unroll
      for (int i2 = 0; i2 < EG; ++i2)
#pragma unroll
        for (int tt = 0; tt < G; ++tt) a[v][i2 * G + tt] = sm[TL::idxA(c, tt, t * EG + i2)];
#pragma unroll
      for (int i2 = 0; i2 < EG; ++i2) dft<G, false>(&a[v][i2 * G]);
    }
  }
  __syncthreads();
}

// COL layout registers -> ROW layout registers (inverse 2-D DFT, unscaled: times M^2).
// The shared buffer must be free on entry; it is free again on return.
template <int M, int V>
__device__ __forceinline__ void fft2_inverse(float2 (&a)[V][Tile<M>::E], float2* sm, const float2* tw, int tid) {
  using TL = Tile<M>;
  constexpr int E = TL::E, G = TL::G, EG = TL::EG, TR = TL::T / V;
  // ---- columns: undo pass 2
  if constexpr (G > 1) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int c = (tid + v * TR) / G, t = (tid + v * TR) % G;
#pragma unroll
      for (int i2 = 0; i2 < EG; ++i2) dft<G, true>(&a[v][i2 * G]);
#pragma unroll
      for (int i2 = 0; i2 < EG; ++i2)
#pragma unroll
        for (int tt = 0; tt < G; ++tt) sm[TL::idxA(c, tt, t * EG + i2)] = a[v][i2 * G + tt];
    }
    __syncwarp();  // the swap stays inside the warp
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int c = (tid + v * TR) / G, t = (tid + v * TR) % G;
#pragma unroll
      for (int k2 = 0; k2 < E; ++k2) a[v][k2] = sm[TL::idxA(c, t, k2)];
    }
    __syncthreads();
  }
  // ---- columns: undo pass 1, then transpose back
  twiddle<M, V, true>(a, tw, tid);
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int c = (tid + v * TR) / G, t = (tid + v * TR) % G;
    dft<E, true>(a[v]);
#pragma unroll
    for (int j = 0; j < E; ++j) sm[TL::idxB(t + G * j, c)] = a[v][j];
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int line = (tid + v * TR) / G, t = (tid + v * TR) % G;
#pragma unroll
    for (int i2 = 0; i2 < EG; ++i2)
#pragma unroll
      for (int k1 = 0; k1 < G; ++k1) a[v][i2 * G + k1] = sm[TL::idxB(line, t * EG + i2 + E * k1)];
  }
  __syncthreads();
  // ---- rows: undo pass 2
  if constexpr (G > 1) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int line = (tid + v * TR) / G, t = (tid + v * TR) % G;
#pragma unroll
      for (int i2 = 0; i2 < EG; ++i2) dft<G, true>(&a[v][i2 * G]);
#pragma unroll
      for (int i2 = 0; i2 < EG; ++i2)
#pragma unroll
        for (int tt = 0; tt < G; ++tt) sm[TL::idxA(line, tt, t * EG + i2)] = a[v][i2 * G + tt];
    }
    __syncwarp();  // the swap stays inside the warp
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int line = (tid + v * TR) / G, t = (tid + v * TR) % G;
#pragma unroll
      for (int k2 = 0; k2 < E; ++k2) a[v][k2] = sm[TL::idxA(line, t, k2)];
    }
    __syncthreads();
  }
  // ---- rows: undo pass 1
  twiddle<M, V, true>(a, tw, tid);
#pragma unroll
  for (int v = 0; v < V; ++v) dft<E, true>(a[v]);
}

// frequency index of COL-layout register r = i2 * G + k1 for thread part t
template <int M>
__device__ __forceinline__ int col_freq(int t, int r) {
  using TL = Tile<M>;
  return t * TL::EG + (r / TL::G) + TL::E * (r % TL::G);
}

}  // namespace ptycho
