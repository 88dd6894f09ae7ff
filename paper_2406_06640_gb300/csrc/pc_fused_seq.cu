// Fused per-position pc-engine kernel, one CTA per scan position with the K probe modes in
// sequence. Everything between the object gather and the per-position contributions stays on
// the SM; no CTA exchanges data with another, so no cluster barrier and no distributed shared
// memory is involved, and every SM of the GPU takes positions.
//
//   o_n     = O[y_n : y_n + M, x_n : x_n + M]                (Fig. 1: object box) -> TMEM
//   pass 1, k = 0 .. K-1:
//     psi_k = P_k o_n                                         (Eq. 1, mixed-state modes)
//     Psi_k = centred FFT2 (far field, checkerboard trick)    (Eq. 1)
//           | IFFT2(FFT2(psi_k) H) (near field, Fresnel transfer function)
//     S    += |Psi_k|^2   (shared memory, each thread its own detector pixels)
//     Psi_{K-1} is kept in TMEM for pass 2
//   A^G     = sqrt(S) (x) g   (Eq. 6)  or  I_m = S (x) g  (Eq. 2), g of Eq. 7 normalised,
//             separable, zero padded
//   R       = sqrt(I_n) / (A^G + eps)  or  sqrt(I_n) / sqrt(I_m + eps^2)     (Fig. 1 box 1)
//   error  += sum (Ihat - I_n)^2 with I_n = (sqrt I_n)^2, Ihat = (A^G)^2 or I_m
//   pass 2, k = K-1, 0, 1, .. K-2 (mode K-1 from TMEM, the others propagated again):
//     Psi'_k = R Psi_k;  psi'_k = inverse propagation;  dpsi_k = psi'_k - P_k o_n
//     c_n   += conj(P_k) dpsi_k                 (TMEM; written once per position)
//     pacc_k += conj(o_n) dpsi_k, dacc += |o_n|^2   (per-slot partials: reductions at L2 into
//                                                  the slot's own array, each element always
//                                                  added to by the same thread, so in a fixed order)
//
// Cost against the cluster form: one more forward propagation for each of K - 1 modes (cheaper on
// this GPU than a store and a load of their detector fields through L2 and HBM), in exchange for no
// exchanges and all SMs busy. Persistent: CTA `slot` takes positions slot,
// slot + slots, ... and owns partial `slot`, so every sum is taken in a fixed order and the
// iteration is bitwise reproducible.
//
// Storage per CTA (M = 128): the FFT exchange buffer (146 KB of shared memory; the blur's
// intermediate aliases it), S and then R (66 KB), twiddles and taps; in tensor memory, per
// thread, its 32 object-box values and its 32 contribution accumulators (512 columns). Probe
// modes and partials are read from L2.
#include <cuda_runtime.h>

#include "cluster.cuh"
#include "engine.h"
#include "fft.cuh"
#include "fused_common.cuh"

namespace ptycho {

// L2 eviction policies: the per-slot probe partials are added to once per position and mode and
// must survive in L2 between those visits; the streamed data (sqrt I, c_n) must not push them out
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// stores of the partials, which this kernel never reads back: no memory clobber, so the compiler may
// move later loads above them
__device__ __forceinline__ void st_part(float2* a, float2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(a), "f"(v.x), "f"(v.y), "l"(pol));
}
__device__ __forceinline__ void st_part(float* a, float v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol));
}
// fire-and-forget add at L2. A partial element is only ever added to by one thread of one CTA, and
// reductions of one thread to one address take effect in program order, so the sums keep their order
// (position by position) and stay bitwise reproducible; no register waits for the old value
__device__ __forceinline__ void red_hint(float2* a, float2 v, uint64_t pol) {
  asm volatile("red.global.add.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(a), "f"(v.x), "f"(v.y), "l"(pol));
}
__device__ __forceinline__ void red_hint(float* a, float v, uint64_t pol) {
  asm volatile("red.global.add.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol));
}
// bring `bytes` (a multiple of 16, 16-byte aligned) into L2 ahead of use
__device__ __forceinline__ void prefetch_l2(const void* a, uint32_t bytes, uint64_t pol) {
  asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(a), "r"(bytes), "l"(pol)
               : "memory");
}

template <int M>
struct SeqShape {
  using TL = Tile<M>;
  static constexpr int V = M == 128 ? 2 : 1;  // lines per thread (M = 128: 512 threads x 2 lines)
  static constexpr int TR = TL::T / V;        // threads per CTA
  // TMEM holds the object box and the contributions (V E complex values each per thread) when the
  // CTA has whole groups of 4 warps; smaller tiles keep them in registers
  static constexpr bool TMEM = TR % 128 == 0;
  static constexpr int COLS_PER_THREAD = 4 * V * TL::E;
  static constexpr int TMEM_COLS = TMEM ? (TR / 128) * COLS_PER_THREAD : 0;
  static_assert(!TMEM || (TMEM_COLS >= 32 && TMEM_COLS <= 512 && (TMEM_COLS & (TMEM_COLS - 1)) == 0),
                "TMEM allocation must be a power of two in [32, 512] columns");
  static constexpr int MIN_BLOCKS = M == 64 ? 2 : 1;
};

template <int M>
struct SeqSmem {
  static constexpr int LD = M + 1;  // padded row stride of the f32 detector buffers
  static constexpr size_t kX = (size_t)Tile<M>::SMEM * 8;  // FFT exchange buffer
  static constexpr size_t kB = (size_t)M * LD * 4;         // one f32 detector buffer
  static constexpr size_t CBUF = ((kX > kB ? kX : kB) + 15) / 16 * 16;
  static constexpr size_t ZBUF = (kB + 15) / 16 * 16;      // S, then R
  static constexpr size_t TWT = ((size_t)Tile<M>::G * Tile<M>::LDW * 8 + 15) / 16 * 16;
  static constexpr size_t HQ = (size_t)M * 8;
  static constexpr size_t TAPS = 2 * kMaxTaps * 4 + 8;  // taps, TMEM address
  static constexpr size_t BYTES = CBUF + ZBUF + TWT + HQ + TAPS;
  static_assert(BYTES <= 232448, "shared memory budget of one CTA");
  static_assert((size_t)SeqShape<M>::TR * 8 <= CBUF, "error reduction buffer");
};

template <int M, bool NEAR, int KH>
__global__ void __launch_bounds__(SeqShape<M>::TR, SeqShape<M>::MIN_BLOCKS) pc_seq_kernel(const FusedArgs a) {
  using TL = Tile<M>;
  using SM = SeqSmem<M>;
  constexpr int E = TL::E, G = TL::G, LD = SM::LD;
  constexpr int V = SeqShape<M>::V, TR = SeqShape<M>::TR;
  constexpr int NB = E > 8 ? 8 : E;  // outputs per blur strip
  constexpr bool TM = SeqShape<M>::TMEM;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* cbuf = reinterpret_cast<float2*>(smem);
  float* X = reinterpret_cast<float*>(smem);               // x-blurred S (aliases the exchange buffer)
  float* Z = reinterpret_cast<float*>(smem + SM::CBUF);    // S during pass 1, then R
  float2* s_tw = reinterpret_cast<float2*>(smem + SM::CBUF + SM::ZBUF);
  float2* s_h = reinterpret_cast<float2*>(smem + SM::CBUF + SM::ZBUF + SM::TWT);
  float* s_gx = reinterpret_cast<float*>(smem + SM::CBUF + SM::ZBUF + SM::TWT + SM::HQ);
  float* s_gy = s_gx + kMaxTaps;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_gy + kMaxTaps);

  const int tid = threadIdx.x;
  const int K = a.K;
  const int slot = blockIdx.x, nslots = gridDim.x;
  const float inv_m2 = 1.0f / (float)(M * M);

  for (int i = tid; i < G * TL::LDW; i += TR) {
    const int t = i / TL::LDW, k2 = i % TL::LDW;
    s_tw[i] = k2 < E ? a.tw[(t * k2) % M] : make_float2(0.f, 0.f);
  }
  if constexpr (NEAR)
    for (int i = tid; i < M; i += TR) s_h[i] = a.hq[i];
  for (int i = tid; i < 2 * KH + 1; i += TR) {
    const int d = i - KH;
    const bool in = d >= -a.kh && d <= a.kh;
    s_gx[i] = in ? a.gx[d + a.kh] : 0.f;
    s_gy[i] = in ? a.gy[d + a.kh] : 0.f;
  }
  int line[V], tp[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    line[v] = (tid + v * TR) / G;
    tp[v] = (tid + v * TR) % G;
  }
  // ---- TMEM: columns [colO, colO + 2 V E) hold the object box, [colC, colC + 2 V E) the
  // contributions (and, between the passes, Psi_{K-1})
  uint32_t t_lane = 0, colO = 0, colC = 0;
  if constexpr (TM) {
    const int warp = tid / 32;
    if (warp == 0) tmem_alloc(smem_addr(s_tmem), SeqShape<M>::TMEM_COLS);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    t_lane = *s_tmem + ((uint32_t)(32 * (warp % 4)) << 16);
    colO = (uint32_t)((warp / 4) * SeqShape<M>::COLS_PER_THREAD);
    colC = colO + 2 * V * E;
  } else {
    __syncthreads();
  }
  // register storage of the small tiles (unused with TMEM)
  float2 o_r[V][E], c_r[V][E], st_r[V][E];
  float err_s = 0.f, err_c = 0.f;  // compensated per-thread sum of (Ihat - I)^2
  const uint64_t keep = policy_evict_last(), stream = policy_evict_first();

  for (int n = slot; n < a.N; n += nslots) {
    const bool first = n == slot;
    const int2 pn = a.pos[n];
    const float2* On = a.O + (size_t)pn.x * a.obj_w + pn.y;
    const float* Qn = a.sqrtI + (size_t)n * M * M;
    // sqrt(I_n) is read once, by the modulus step: start moving it into L2 now
    if (tid == 0) prefetch_l2(Qn, (uint32_t)(M * M * 4), stream);
    float2 v[V][E];

    // ---- the object box in ROW layout into TMEM (every load in flight at once)
#pragma unroll
    for (int q = 0; q < V; ++q)
#pragma unroll
      for (int j = 0; j < E; ++j) v[q][j] = On[(size_t)line[q] * a.obj_w + tp[q] + G * j];
    if constexpr (TM) {
#pragma unroll
      for (int q = 0; q < V; ++q)
#pragma unroll
        for (int h = 0; h < E / 8; ++h) {
          float pr[16];
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            pr[2 * jj] = v[q][8 * h + jj].x;
            pr[2 * jj + 1] = v[q][8 * h + jj].y;
          }
          tmem_st16(t_lane + colO + 2 * (q * E + 8 * h), pr);
        }
      tmem_wait_st();
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q)
#pragma unroll
        for (int j = 0; j < E; ++j) o_r[q][j] = v[q][j];
    }

    // ---- exit wave P_k o_n in ROW layout; far field: times (-1)^(y + x), which centres the transform
    auto exit_wave = [&](int k) {
      const float2* Pk = a.P + (size_t)k * M * M;
#pragma unroll
      for (int q = 0; q < V; ++q)
#pragma unroll
        for (int j = 0; j < E; ++j) v[q][j] = __ldg(&Pk[line[q] * M + tp[q] + G * j]);
#pragma unroll
      for (int q = 0; q < V; ++q) {
        float2 o[E];
        if constexpr (TM) {
#pragma unroll
          for (int h = 0; h < E / 8; ++h) {
            float pr[16];
            tmem_ld16(t_lane + colO + 2 * (q * E + 8 * h), pr);
            tmem_wait_ld();
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) o[8 * h + jj] = make_float2(pr[2 * jj], pr[2 * jj + 1]);
          }
        } else {
#pragma unroll
          for (int j = 0; j < E; ++j) o[j] = o_r[q][j];
        }
#pragma unroll
        for (int j = 0; j < E; ++j) {
          float2 psi = cmul(v[q][j], o[j]);
          if (!NEAR && ((line[q] + tp[q] + G * j) & 1)) psi = make_float2(-psi.x, -psi.y);
          v[q][j] = psi;
        }
      }
    };
    // ---- forward propagation to the detector (far: COL layout; near: ROW layout, scaled)
    auto forward = [&]() {
      fft2_forward<M, V>(v, cbuf, s_tw, tid);
      if constexpr (NEAR) {
#pragma unroll
        for (int q = 0; q < V; ++q)
#pragma unroll
          for (int r = 0; r < E; ++r) {
            const int vt = tid + q * TR;
            v[q][r] = cmul(v[q][r], cmul(s_h[col_freq<M>(vt % G, r)], s_h[vt / G]));
          }
        fft2_inverse<M, V>(v, cbuf, s_tw, tid);
#pragma unroll
        for (int q = 0; q < V; ++q)
#pragma unroll
          for (int j = 0; j < E; ++j) v[q][j] = cscale(v[q][j], inv_m2);
      }
    };

    // ---- pass 1: S = sum_k |Psi_k|^2 in Z, each thread on its own detector pixels; the last
    // mode's sum is turned into the blur's input (sqrt for the amplitude model) in place
    for (int k = 0; k < K; ++k) {
      exit_wave(k);
      forward();
      const bool last = k == K - 1;
#pragma unroll
      for (int q = 0; q < V; ++q)
#pragma unroll
        for (int r = 0; r < E; ++r) {
          int row, col;
          det_coords<M, NEAR>(tid + q * TR, r, row, col);
          float s = cabs2(v[q][r]);
          if (k > 0) s += Z[row * LD + col];
          if (last && !a.blur_intensity) s = sqrtf(s);
          Z[row * LD + col] = s;
        }
    }
    // Psi_{K-1} waits in the contribution columns (registers for the small tiles)
    if constexpr (TM) {
#pragma unroll
      for (int q = 0; q < V; ++q)
#pragma unroll
        for (int h = 0; h < E / 8; ++h) {
          float pr[16];
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            pr[2 * jj] = v[q][8 * h + jj].x;
            pr[2 * jj + 1] = v[q][8 * h + jj].y;
          }
          tmem_st16(t_lane + colC + 2 * (q * E + 8 * h), pr);
        }
      tmem_wait_st();
    } else {
#pragma unroll
      for (int q = 0; q < V; ++q)
#pragma unroll
        for (int j = 0; j < E; ++j) st_r[q][j] = v[q][j];
    }
    __syncthreads();  // Z complete; the exchange buffer is free (forward ended with a barrier)

    // ---- the pc intensity model: blur along x (columns, sigma_1), Z -> X
    for (int w = tid; w < M * (M / NB); w += TR) {
      const int row = w % M, c0 = (w / M) * NB;
      float out[NB];
      blur_strip<NB, KH>(Z, row * LD, 1, c0, 0, M, s_gx, out);
#pragma unroll
      for (int o = 0; o < NB; ++o) X[row * LD + c0 + o] = out[o];
    }
    __syncthreads();
    // ---- blur along y (rows, sigma_2), X -> model; the error and the modulus ratio R -> Z
    for (int w = tid; w < M * (M / NB); w += TR) {
      const int col = w % M, rs = (w / M) * NB;
      float sq[NB];
#pragma unroll
      for (int o = 0; o < NB; ++o) sq[o] = __ldcs(&Qn[(rs + o) * M + col]);
      float out[NB];
      blur_strip<NB, KH>(X, col, LD, rs, 0, M, s_gy, out);
#pragma unroll
      for (int o = 0; o < NB; ++o) {
        const float acc = out[o];
        const float im = sq[o] * sq[o];
        const float ihat = a.blur_intensity ? acc : acc * acc;
        const float d = ihat - im;
        const float y = fmaf(d, d, -err_c);
        const float tt = err_s + y;
        err_c = (tt - err_s) - y;
        err_s = tt;
        Z[(rs + o) * LD + col] =
            a.blur_intensity ? sq[o] * rsqrtf(acc + a.eps * a.eps) : __fdividef(sq[o], acc + a.eps);
      }
    }
    __syncthreads();

    // ---- pass 2: mode K-1 from storage, then modes 0 .. K-2 propagated again
    for (int i = 0; i < K; ++i) {
      const int k = i == 0 ? K - 1 : i - 1;
      if (i == 0) {
        if constexpr (TM) {
#pragma unroll
          for (int q = 0; q < V; ++q)
#pragma unroll
            for (int h = 0; h < E / 8; ++h) {
              float pr[16];
              tmem_ld16(t_lane + colC + 2 * (q * E + 8 * h), pr);
              tmem_wait_ld();
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) v[q][8 * h + jj] = make_float2(pr[2 * jj], pr[2 * jj + 1]);
            }
        } else {
#pragma unroll
          for (int q = 0; q < V; ++q)
#pragma unroll
            for (int j = 0; j < E; ++j) v[q][j] = st_r[q][j];
        }
      } else {
        exit_wave(k);
        forward();
      }
      // Psi' = R Psi
#pragma unroll
      for (int q = 0; q < V; ++q)
#pragma unroll
        for (int r = 0; r < E; ++r) {
          int row, col;
          det_coords<M, NEAR>(tid + q * TR, r, row, col);
          v[q][r] = cscale(v[q][r], Z[row * LD + col]);
        }
      // back-propagation to ROW layout (times M^2)
      if constexpr (NEAR) {
        fft2_forward<M, V>(v, cbuf, s_tw, tid);
#pragma unroll
        for (int q = 0; q < V; ++q)
#pragma unroll
          for (int r = 0; r < E; ++r) {
            const int vt = tid + q * TR;
            v[q][r] = cmulc(v[q][r], cmul(s_h[col_freq<M>(vt % G, r)], s_h[vt / G]));
          }
      }
      fft2_inverse<M, V>(v, cbuf, s_tw, tid);
      // dpsi = psi' - P_k o_n; contributions, probe partials
      const float2* Pk = a.P + (size_t)k * M * M;
      float2* pk = a.pacc + ((size_t)slot * K + k) * M * M;
      float* dk = a.dacc + (size_t)slot * M * M;
#pragma unroll
      for (int q = 0; q < V; ++q) {
        const int ln = line[q];
#pragma unroll
        for (int h = 0; h < E / 4; ++h) {
          float2 p[4];
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) p[jj] = __ldg(&Pk[ln * M + tp[q] + G * (4 * h + jj)]);
          float2 o[4], c[4];
          if constexpr (TM) {
            float pr[8], ac[8];
            tmem_ld8(t_lane + colO + 2 * (q * E + 4 * h), pr);
            if (i > 0) tmem_ld8(t_lane + colC + 2 * (q * E + 4 * h), ac);
            tmem_wait_ld();
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              o[jj] = make_float2(pr[2 * jj], pr[2 * jj + 1]);
              c[jj] = i > 0 ? make_float2(ac[2 * jj], ac[2 * jj + 1]) : make_float2(0.f, 0.f);
            }
          } else {
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              o[jj] = o_r[q][4 * h + jj];
              c[jj] = i > 0 ? c_r[q][4 * h + jj] : make_float2(0.f, 0.f);
            }
          }
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int j = 4 * h + jj;
            const int x = tp[q] + G * j;
            float2 psi_new = cscale(v[q][j], inv_m2);
            if (!NEAR && ((ln + x) & 1)) psi_new = make_float2(-psi_new.x, -psi_new.y);
            const float2 dpsi = csub(psi_new, cmul(p[jj], o[jj]));
            c[jj] = cadd(c[jj], cconjmul(p[jj], dpsi));
            // the slot's first position sets its partials, the later ones add to them
            const float2 dp = cconjmul(o[jj], dpsi);
            if (first) {
              st_part(&pk[ln * M + x], dp, keep);
              if (i == 0) st_part(&dk[ln * M + x], cabs2(o[jj]), keep);
            } else {
              red_hint(&pk[ln * M + x], dp, keep);
              if (i == 0) red_hint(&dk[ln * M + x], cabs2(o[jj]), keep);
            }
          }
          if constexpr (TM) {
            float ac[8];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              ac[2 * jj] = c[jj].x;
              ac[2 * jj + 1] = c[jj].y;
            }
            tmem_st8(t_lane + colC + 2 * (q * E + 4 * h), ac);
          } else {
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) c_r[q][4 * h + jj] = c[jj];
          }
        }
      }
      if constexpr (TM) tmem_wait_st();
    }
    // ---- c_n, written once (streaming: the object gather reads it after this launch)
    float2* cn = a.cn + (size_t)n * M * M;
#pragma unroll
    for (int q = 0; q < V; ++q) {
      float2 c[E];
      if constexpr (TM) {
#pragma unroll
        for (int h = 0; h < E / 8; ++h) {
          float ac[16];
          tmem_ld16(t_lane + colC + 2 * (q * E + 8 * h), ac);
          tmem_wait_ld();
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) c[8 * h + jj] = make_float2(ac[2 * jj], ac[2 * jj + 1]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < E; ++j) c[j] = c_r[q][j];
      }
#pragma unroll
      for (int j = 0; j < E; ++j) __stcs(&cn[line[q] * M + tp[q] + G * j], c[j]);
    }
    // the next position's pass 1 rewrites Z, which other threads read above
    __syncthreads();
  }

  // ---- per-CTA FP64 error numerator (the compensated FP32 thread sums, added in a fixed tree);
  // the slot's other K - 1 entries are zero (the error is per position, not per mode)
  double* red = reinterpret_cast<double*>(smem);
  red[tid] = (double)err_s - (double)err_c;
  __syncthreads();
  for (int w = TR / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid < K) a.errpart[(size_t)slot * K + tid] = tid == 0 ? red[0] : 0.0;
  if constexpr (TM) {
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (tid / 32 == 0) tmem_dealloc(*s_tmem, SeqShape<M>::TMEM_COLS);
  }
}

// ------------------------------------------------------------------ launches
template <int M, bool NEAR, int KH>
static cudaError_t launch_seq_kh(const FusedArgs& a, int slots, cudaStream_t s) {
  auto kern = pc_seq_kernel<M, NEAR, KH>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SeqSmem<M>::BYTES);
  if (e != cudaSuccess) return e;
  kern<<<slots, SeqShape<M>::TR, SeqSmem<M>::BYTES, s>>>(a);
  return cudaGetLastError();
}

// the paper's 11 x 11 kernel (Sec. 3.1) has its own instantiation; any other odd size up to 31
// runs with the taps zero-padded to 31
template <int M, bool NEAR>
static cudaError_t launch_seq_t(const FusedArgs& a, int slots, cudaStream_t s) {
  return a.kh == 5 ? launch_seq_kh<M, NEAR, 5>(a, slots, s) : launch_seq_kh<M, NEAR, 15>(a, slots, s);
}

// co-resident CTAs over the whole GPU, the smallest count over the instantiations; CTAs on one SM
// must not ask for more than its 512 TMEM columns together (tcgen05.alloc would wait for columns
// that a persistent CTA never frees), which the shared-memory and register budgets guarantee
template <int M>
static cudaError_t seq_slots_t(int* slots) {
  int dev = 0, sms = 0, best = 1 << 30;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const void* kerns[4] = {(const void*)pc_seq_kernel<M, false, 5>, (const void*)pc_seq_kernel<M, false, 15>,
                          (const void*)pc_seq_kernel<M, true, 5>, (const void*)pc_seq_kernel<M, true, 15>};
  for (const void* k : kerns) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SeqSmem<M>::BYTES);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, SeqShape<M>::TR, SeqSmem<M>::BYTES);
    if (e != cudaSuccess) return e;
    if (SeqShape<M>::TMEM && per_sm * SeqShape<M>::TMEM_COLS > 512) return cudaErrorInvalidConfiguration;
    best = per_sm < best ? per_sm : best;
  }
  *slots = best * sms;
  return cudaSuccess;
}

cudaError_t launch_fused(int M, const FusedArgs& a, int slots, cudaStream_t s) {
  const bool nf = a.near_field != 0;
  switch (M) {
    case 8: return nf ? launch_seq_t<8, true>(a, slots, s) : launch_seq_t<8, false>(a, slots, s);
    case 16: return nf ? launch_seq_t<16, true>(a, slots, s) : launch_seq_t<16, false>(a, slots, s);
    case 32: return nf ? launch_seq_t<32, true>(a, slots, s) : launch_seq_t<32, false>(a, slots, s);
    case 64: return nf ? launch_seq_t<64, true>(a, slots, s) : launch_seq_t<64, false>(a, slots, s);
    case 128: return nf ? launch_seq_t<128, true>(a, slots, s) : launch_seq_t<128, false>(a, slots, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t fused_max_slots(int M, int /*K*/, int* slots) {
  switch (M) {
    case 8: return seq_slots_t<8>(slots);
    case 16: return seq_slots_t<16>(slots);
    case 32: return seq_slots_t<32>(slots);
    case 64: return seq_slots_t<64>(slots);
    case 128: return seq_slots_t<128>(slots);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ptycho
