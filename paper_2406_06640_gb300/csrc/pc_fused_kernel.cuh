// Device code of the fused per-position kernel (see pc_fused.cu for what it computes); included by
// the translation units that instantiate it (pc_fused.cu: single-problem and work-queue launches;
// pc_fused_dm.cu: the pc-DM engine).
#pragma once
#include <cuda_runtime.h>

#include "engine.h"
#include "cluster.cuh"
#include "fft.cuh"
#include "fused_common.cuh"

namespace ptycho {

// fire-and-forget adds at L2 for the per-slot partials: every element is added to by one thread of one
// CTA only, and one thread's adds to one address take effect in program order, so each sum keeps its
// position order (bitwise reproducible) while no thread waits for the old value
__device__ __forceinline__ void red_add_l2(float2* a, float2 v) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(a), "f"(v.x), "f"(v.y));
}
__device__ __forceinline__ void red_add_l2(float* a, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(a), "f"(v));
}

// set when a bounded device wait of the fused kernel gave up (one flag per translation unit that
// instantiates the kernel; read and cleared by fused_timed_out)
static __device__ int g_fused_timeout;

// ---- bounded mbarrier wait (global timer); false once `budget_ns` has passed without the phase
constexpr unsigned long long kFusedWaitNs = 2000000000ull;  // 2 s
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t phase,
                                                  unsigned long long budget_ns = kFusedWaitNs) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P1;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P1;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    if (ok) return true;
    if (global_ns() - t0 > budget_ns) return false;
  }
}
// largest K * ceil(M / K) over the cluster sizes 1..8 (rows of the per-source slots)
constexpr int max_slot_rows(int M) {
  int best = 0;
  for (int K = 1; K <= 8; ++K) {
    const int r = K * ((M + K - 1) / K);
    best = r > best ? r : best;
  }
  return best;
}

template <int M, int KH>
struct FusedSmem {
  static constexpr int LD = M + 1;  // padded row stride of the f32 detector buffers
  static constexpr size_t kX = (size_t)Tile<M>::SMEM * 8;  // FFT exchange buffer
  // modulus phase (aliases the exchange buffer): R (M rows) + own x-blurred rows with halos
  static constexpr size_t kF = (size_t)(M + M + 2 * KH) * LD * 4;
  // contributions received from every rank for the own rows
  static constexpr size_t kR = (size_t)max_slot_rows(M) * Tile<M>::LDN * 8;
  static constexpr size_t kXF = kX > kF ? kX : kF;
  static constexpr size_t CBUF = ((kXF > kR ? kXF : kR) + 15) / 16 * 16;
  static constexpr size_t IBUF = ((size_t)max_slot_rows(M) * LD * 4 + 15) / 16 * 16;
  static constexpr size_t TWT = ((size_t)Tile<M>::G * Tile<M>::LDW * 8 + 15) / 16 * 16;  // twiddle table
  static constexpr size_t HQ = (size_t)M * 8;                                             // Fresnel factors
  static constexpr size_t TAPS = 2 * kMaxTaps * 4 + 8 + 16;  // taps, TMEM address, mbarrier (16-byte aligned)
  static constexpr size_t BYTES = CBUF + IBUF + TWT + HQ + TAPS;
  // queued launches: the current problem's arguments and the chunk index handed out by rank 0
  static constexpr size_t DESC = (sizeof(FusedArgs) + 15) / 16 * 16 + 16;
  static_assert(BYTES + DESC <= 232448, "shared memory budget of one CTA");
};

// lines per thread: the 128 x 128 tile runs on 512 threads with two lines each
// (128 registers per thread instead of 64 at 1024 threads)
template <int M>
struct FusedShape {
  static constexpr int V = M == 128 ? 2 : 1;
  static constexpr int TR = Tile<M>::T / V;
  // TMEM keeps this CTA's probe mode and its probe-numerator partial (V E complex
  // values each per thread) when the CTA has whole groups of 4 warps
  static constexpr bool TMEM = TR % 128 == 0;
  static constexpr int COLS_PER_THREAD = 4 * V * Tile<M>::E;
  static constexpr int TMEM_COLS = TMEM ? (TR / 128) * COLS_PER_THREAD : 0;
  static_assert(!TMEM || (TMEM_COLS >= 32 && TMEM_COLS <= 512 && (TMEM_COLS & (TMEM_COLS - 1)) == 0),
                "TMEM allocation must be a power of two in [32, 512] columns");
};

template <int M, bool NEAR, int KH, bool QUEUED, bool DM = false>
__global__ void __launch_bounds__(FusedShape<M>::TR, 1) pc_fused_kernel(const FusedArgs a_in) {
  using TL = Tile<M>;
  using SM = FusedSmem<M, KH>;
  constexpr int E = TL::E, G = TL::G, LD = SM::LD, LDN = TL::LDN;
  constexpr int V = FusedShape<M>::V, TR = FusedShape<M>::TR;
  constexpr int NB = E > 8 ? 8 : E;  // outputs per blur strip
  extern __shared__ __align__(16) unsigned char smem[];
  float2* cbuf = reinterpret_cast<float2*>(smem);
  float* Z = reinterpret_cast<float*>(smem);  // R for the whole tile, M x LD
  float* X = Z;                               // own rows of A (aliases Z, dead before R arrives)
  float* Yb = Z + M * LD;                     // own x-blurred rows with KH halo rows on each side
  float2* recv = cbuf;                        // contributions for the own rows, one slot per source rank
  float* ibuf = reinterpret_cast<float*>(smem + SM::CBUF);  // |Psi|^2 for the own rows, one slot per rank
  float2* s_tw = reinterpret_cast<float2*>(smem + SM::CBUF + SM::IBUF);
  float2* s_h = reinterpret_cast<float2*>(smem + SM::CBUF + SM::IBUF + SM::TWT);
  float* s_gx = reinterpret_cast<float*>(smem + SM::CBUF + SM::IBUF + SM::TWT + SM::HQ);
  float* s_gy = s_gx + kMaxTaps;

  const int tid = threadIdx.x;
  const int K = a_in.K;
  const int rank = (int)cluster_ctarank();
  const int slot = blockIdx.x / K;
  const int nslots = gridDim.x / K;

  // twiddle table s_tw[t * (E + 1) + k2] = W_M^(t k2), t < G, from the host table W_M^m (same for every
  // problem of a launch: one M)
  for (int i = tid; i < G * TL::LDW; i += TR) {
    const int t = i / TL::LDW, k2 = i % TL::LDW;
    s_tw[i] = k2 < E ? a_in.tw[(t * k2) % M] : make_float2(0.f, 0.f);
  }
  int line[V], tp[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    line[v] = (tid + v * TR) / G;
    tp[v] = (tid + v * TR) % G;
  }
  // ---- TMEM: columns [colP, colP + 2 V E) hold P_k, [colA, colA + 2 V E) the probe numerator
  constexpr bool TM = FusedShape<M>::TMEM;
  uint32_t t_lane = 0, colP = 0, colA = 0;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_gy + kMaxTaps);
  if constexpr (TM) {
    const int warp = tid / 32;
    if (warp == 0) tmem_alloc(smem_addr(s_tmem), FusedShape<M>::TMEM_COLS);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    t_lane = *s_tmem + ((uint32_t)(32 * (warp % 4)) << 16);
    colP = (uint32_t)((warp / 4) * FusedShape<M>::COLS_PER_THREAD);
    colA = colP + 2 * V * E;
  }
  const int RPO = (M + K - 1) / K;  // rows per owner
  const int r0 = min(M, rank * RPO), r1 = min(M, r0 + RPO), nrow = r1 - r0;
  const float inv_m2 = 1.0f / (float)(M * M);
  const uint32_t ibuf_s = smem_addr(ibuf), z_s = smem_addr(Z), yb_s = smem_addr(Yb), recv_s = smem_addr(recv);
  float err_s = 0.f, err_c = 0.f;  // compensated per-thread sum of (Ihat - I)^2 over own rows
  // staging of the own rows' measured data behind Z and Yb in the exchange buffer, when it fits
  const size_t meas_off = ((size_t)(M + nrow + 2 * KH) * LD * 4 + 15) / 16 * 16;
  const bool pre = meas_off + (size_t)2 * nrow * M * 4 <= SM::CBUF;
  const float* s_meas = reinterpret_cast<const float*>(smem + meas_off);
  const uint32_t meas_s = smem_addr(smem + meas_off);
  const uint32_t bar_s = smem_addr(s_gy + kMaxTaps) + 8u;  // after the TMEM address word; 16-byte aligned
  uint32_t mphase = 0;
  bool waits_ok = true;
  if (tid == 0) mbar_init(bar_s, 1);
  __syncthreads();

  // ---- per problem (one unit of work): Fresnel factors, taps, this rank's probe mode into TMEM.
  // Called between CTA barriers.
  auto setup_unit = [&](const FusedArgs& a) {
    if constexpr (NEAR)
      for (int i = tid; i < M; i += TR) s_h[i] = a.hq[i];
    // taps centred at index KH; zero outside the requested kernel
    for (int i = tid; i < 2 * KH + 1; i += TR) {
      const int d = i - KH;
      const bool in = d >= -a.kh && d <= a.kh;
      s_gx[i] = in ? a.gx[d + a.kh] : 0.f;
      s_gy[i] = in ? a.gy[d + a.kh] : 0.f;
    }
    if constexpr (TM) {
      const float2* Pk = a.P + (size_t)rank * M * M;
#pragma unroll
      for (int q = 0; q < V; ++q)
#pragma unroll
        for (int h = 0; h < E / 8; ++h) {
          float pr[16];
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const float2 p = Pk[line[q] * M + tp[q] + G * (8 * h + jj)];
            pr[2 * jj] = p.x;
            pr[2 * jj + 1] = p.y;
          }
          tmem_st16(t_lane + colP + 2 * (q * E + 8 * h), pr);
        }
      tmem_wait_st();
    }
  };

  // ---- one scan position n of problem a; `first` starts this unit's probe partials
  auto run_position = [&](const FusedArgs& a, int n, bool first, float2* pacc, float* dacc) {
    const float2* Pk = a.P + (size_t)rank * M * M;
    const float eps = a.eps;
    // pc-DM: this position's exit-wave state of mode `rank` (P o_n itself when the state starts)
    float2* Sn = DM ? a.psi + ((size_t)n * K + rank) * M * M : nullptr;
    const bool dm_init = DM && a.dm_init;
    const int2 pn = a.pos[n];
    const float2* On = a.O + (size_t)pn.x * a.obj_w + pn.y;
    float2 v[V][E];

    // ---- exit wave in ROW layout: P o_n, or (pc-DM, CHI) the reflected wave 2 P o_n - psi_n;
    // far field: times (-1)^(y + x), which centres the transform
    auto exit_wave = [&](auto chi_c) {
      constexpr bool CHI = decltype(chi_c)::value != 0;
      if constexpr (TM) {
        // every object load of this thread in flight at once (the TMEM waits below are compiler
        // barriers: loads issued after them would expose one L2 round trip per group)
#pragma unroll
        for (int q = 0; q < V; ++q)
#pragma unroll
          for (int j = 0; j < E; ++j) v[q][j] = On[(size_t)line[q] * a.obj_w + tp[q] + G * j];
#pragma unroll
        for (int q = 0; q < V; ++q)
#pragma unroll
          for (int h = 0; h < E / 4; ++h) {
            float pr[8];
            tmem_ld8(t_lane + colP + 2 * (q * E + 4 * h), pr);
            tmem_wait_ld();
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              const int x = tp[q] + G * (4 * h + jj);
              float2 psi = cmul(make_float2(pr[2 * jj], pr[2 * jj + 1]), v[q][4 * h + jj]);
              if constexpr (CHI) {
                const float2 st = dm_init ? psi : Sn[line[q] * M + x];
                psi = make_float2(2.f * psi.x - st.x, 2.f * psi.y - st.y);
              }
              if (!NEAR && ((line[q] + x) & 1)) psi = make_float2(-psi.x, -psi.y);
              v[q][4 * h + jj] = psi;
            }
          }
      } else {
#pragma unroll
        for (int q = 0; q < V; ++q)
#pragma unroll
          for (int j = 0; j < E; ++j) {
            const int x = tp[q] + G * j;
            float2 psi = cmul(Pk[line[q] * M + x], On[(size_t)line[q] * a.obj_w + x]);
            if constexpr (CHI) {
              const float2 st = dm_init ? psi : Sn[line[q] * M + x];
              psi = make_float2(2.f * psi.x - st.x, 2.f * psi.y - st.y);
            }
            if (!NEAR && ((line[q] + x) & 1)) psi = make_float2(-psi.x, -psi.y);
            v[q][j] = psi;
          }
      }
    };

    // ---- propagation to the detector and the pc intensity model of Fig. 1 box 1 on the own rows.
    // PS bit 0: accumulate the error of the model intensity; bit 1: push the modulus ratio R to
    // every rank (then Z holds R for the whole tile)
    auto detector = [&](auto ps_c) {
      constexpr int PS = decltype(ps_c)::value;
      // ---- forward propagation
      fft2_forward<M, V>(v, cbuf, s_tw, tid);  // COL layout
      if constexpr (NEAR) {
#pragma unroll
        for (int q = 0; q < V; ++q)
#pragma unroll
          for (int r = 0; r < E; ++r) {
            const int vt = tid + q * TR;
            v[q][r] = cmul(v[q][r], cmul(s_h[col_freq<M>(vt % G, r)], s_h[vt / G]));
          }
        fft2_inverse<M, V>(v, cbuf, s_tw, tid);  // ROW layout, times M^2
#pragma unroll
        for (int q = 0; q < V; ++q)
#pragma unroll
          for (int j = 0; j < E; ++j) v[q][j] = cscale(v[q][j], inv_m2);
      }
      // ---- own rows of sqrt(I) and I into free shared memory (bulk copies, used in step 4); the
      // exchange buffer is free here (the propagation ended with a CTA barrier)
      if (pre && tid == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const uint32_t bytes = (uint32_t)(nrow * M * 4);
        mbar_arrive_expect_tx(bar_s, 2u * bytes);
        if (bytes) {
          bulk_g2s(meas_s, a.sqrtI + ((size_t)n * M + r0) * M, bytes, bar_s);
          bulk_g2s(meas_s + bytes, a.I + ((size_t)n * M + r0) * M, bytes, bar_s);
        }
      }
      // ---- (1) push |Psi_k|^2 into slot `rank` of the row owner's buffer
#pragma unroll
      for (int q = 0; q < V; ++q)
#pragma unroll
        for (int r = 0; r < E; ++r) {
          int row, col;
          det_coords<M, NEAR>(tid + q * TR, r, row, col);
          const int ow = row / RPO;
          const int lr = row - ow * RPO;
          st_cluster_f32(map_rank(ibuf_s + (uint32_t)(((rank * RPO + lr) * LD + col) * 4), (unsigned)ow),
                         cabs2(v[q][r]));
        }
      cluster_sync_all();
      // ---- (2) own rows: mode sum in rank order -> X; zero the halo rows that lie outside the tile
      for (int p = tid; p < nrow * M; p += TR) {
        const int lr = p / M, col = p % M;
        float s = 0.f;
        for (int q = 0; q < K; ++q) s += ibuf[(q * RPO + lr) * LD + col];
        X[lr * LD + col] = a.blur_intensity ? s : sqrtf(s);
      }
      for (int p = tid; p < 2 * KH * M; p += TR) {
        const int h = p / M, col = p % M;
        const int gr = h < KH ? r0 - KH + h : r1 + (h - KH);
        if (gr < 0 || gr >= M) Yb[(gr - r0 + KH) * LD + col] = 0.f;
      }
      __syncthreads();
      // ---- (3) blur along x (columns, sigma_1) of the own rows; push the rows other ranks need as
      // halo (strips of NB outputs: enough work items for every thread at K = 4)
      for (int w = tid; w < nrow * (M / NB); w += TR) {
        const int lr = w % nrow, c0 = (w / nrow) * NB;
        const int gr = r0 + lr;
        float out[NB];
        blur_strip<NB, KH>(X, lr * LD, 1, c0, 0, M, s_gx, out);
#pragma unroll
        for (int o = 0; o < NB; ++o) Yb[(lr + KH) * LD + c0 + o] = out[o];
        for (int q = 0; q < K; ++q) {
          if (q == rank) continue;
          const int q0 = min(M, q * RPO), q1 = min(M, q0 + RPO);
          if ((gr >= q0 - KH && gr < q0) || (gr >= q1 && gr < q1 + KH)) {
            const uint32_t base = map_rank(yb_s + (uint32_t)(((gr - q0 + KH) * LD + c0) * 4), (unsigned)q);
#pragma unroll
            for (int o = 0; o < NB; ++o) st_cluster_f32(base + 4u * o, out[o]);
          }
        }
      }
      cluster_sync_all();
      // ---- (4) blur along y (rows, sigma_2), then the error and / or the modulus ratio R
      {
        const float* In = a.I + (size_t)n * M * M;
        const float* Qn = a.sqrtI + (size_t)n * M * M;
        if (pre && waits_ok) {
          if (!mbar_wait_bounded(bar_s, mphase)) {
            waits_ok = false;  // report once and stop waiting; the results are flagged invalid
            atomicExch(&g_fused_timeout, 1);
          }
          mphase ^= 1u;
        }
        const int nstrip = (nrow + NB - 1) / NB;
        for (int w = tid; w < M * nstrip; w += TR) {
          const int col = w % M, rs = (w / M) * NB;
          float out[NB];
          blur_strip<NB, KH>(Yb, col, LD, rs + KH, 0, nrow + 2 * KH, s_gy, out);
#pragma unroll
          for (int o = 0; o < NB; ++o) {
            const int lr = rs + o;
            if (lr >= nrow) break;
            const int gr = r0 + lr;
            const float acc = out[o];
            if constexpr ((PS & 1) != 0) {
              const float im = pre ? s_meas[(nrow + lr) * M + col] : In[gr * M + col];
              const float ihat = a.blur_intensity ? acc : acc * acc;
              const float d = ihat - im;
              const float y = fmaf(d, d, -err_c);
              const float tt = err_s + y;
              err_c = (tt - err_s) - y;
              err_s = tt;
            }
            if constexpr ((PS & 2) != 0) {
              const float sq = pre ? s_meas[lr * M + col] : Qn[gr * M + col];
              const float R = a.blur_intensity ? sq * rsqrtf(acc + eps * eps) : __fdividef(sq, acc + eps);
              const uint32_t zoff = z_s + (uint32_t)((gr * LD + col) * 4);
              for (int q = 0; q < K; ++q) st_cluster_f32(map_rank(zoff, (unsigned)q), R);
            }
          }
        }
      }
      // R arrives from every rank; without R only this CTA's shared memory was read
      if constexpr ((PS & 2) != 0) cluster_sync_all();
      else __syncthreads();
    };

    if constexpr (DM) {
      exit_wave(IntC<0>{});  // the estimate P o_n: its model error is E
      detector(IntC<1>{});
      exit_wave(IntC<1>{});  // the reflected wave: its modulus ratio
      detector(IntC<2>{});
    } else {
      exit_wave(IntC<0>{});
      detector(IntC<3>{});
    }
    // ---- (5) Psi' = R Psi
#pragma unroll
    for (int q = 0; q < V; ++q)
#pragma unroll
      for (int r = 0; r < E; ++r) {
        int row, col;
        det_coords<M, NEAR>(tid + q * TR, r, row, col);
        v[q][r] = cscale(v[q][r], Z[row * LD + col]);
      }
    __syncthreads();  // Z aliases the exchange buffer
    // ---- (6) back-propagation to ROW layout
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
    cluster_sync_all();  // every rank is done with its exchange buffer, which now receives contributions
    // ---- (7) dpsi; probe partials; conj(P) dpsi pushed to the row owner
#pragma unroll
    for (int q = 0; q < V; ++q) {
      const int ln = line[q];
      const int ow = ln / RPO;
      const uint32_t dst = map_rank(recv_s + (uint32_t)((rank * RPO + ln - ow * RPO) * LDN * 8), (unsigned)ow);
      if constexpr (TM) {
        // this line's object values and (own rows) denominator partials, all loads in flight at once
        float2 o[E];
#pragma unroll
        for (int j = 0; j < E; ++j) o[j] = On[(size_t)ln * a.obj_w + tp[q] + G * j];
        const bool own = ln >= r0 && ln < r1;
#pragma unroll
        for (int h = 0; h < E / 4; ++h) {
          float pr[8], ac[8];
          tmem_ld8(t_lane + colP + 2 * (q * E + 4 * h), pr);
          if (!DM && !first) tmem_ld8(t_lane + colA + 2 * (q * E + 4 * h), ac);
          tmem_wait_ld();
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int j = 4 * h + jj;
            const int x = tp[q] + G * j;
            float2 psi_new = cscale(v[q][j], inv_m2);
            if (!NEAR && ((ln + x) & 1)) psi_new = make_float2(-psi_new.x, -psi_new.y);
            const float2 p = make_float2(pr[2 * jj], pr[2 * jj + 1]);
            float2 dpsi = csub(psi_new, cmul(p, o[j]));
            if constexpr (DM) {  // psi_n <- psi_n + Pi_F(chi) - P o_n; the overlap step takes psi_n - P o_n
              const float2 ov = cmul(p, o[j]);
              const float2 st = cadd(dm_init ? ov : Sn[ln * M + x], dpsi);
              Sn[ln * M + x] = st;
              dpsi = csub(st, ov);
            }
            st_cluster_f2(dst + 8u * x, cconjmul(p, dpsi));
            if constexpr (!DM) {  // pc-DM takes its probe step after the object step, from its state
              const float2 pc = cconjmul(o[j], dpsi);
              ac[2 * jj] = first ? pc.x : ac[2 * jj] + pc.x;
              ac[2 * jj + 1] = first ? pc.y : ac[2 * jj + 1] + pc.y;
              if (own) {
                if (first) dacc[ln * M + x] = cabs2(o[j]);
                else red_add_l2(&dacc[ln * M + x], cabs2(o[j]));
              }
            }
          }
          if constexpr (!DM) tmem_st8(t_lane + colA + 2 * (q * E + 4 * h), ac);
        }
        if constexpr (!DM) tmem_wait_st();
      } else {
#pragma unroll
        for (int j = 0; j < E; ++j) {
          const int x = tp[q] + G * j;
          float2 psi_new = cscale(v[q][j], inv_m2);
          if (!NEAR && ((ln + x) & 1)) psi_new = make_float2(-psi_new.x, -psi_new.y);
          const float2 p = Pk[ln * M + x];
          const float2 o = On[(size_t)ln * a.obj_w + x];
          float2 dpsi = csub(psi_new, cmul(p, o));
          if constexpr (DM) {  // psi_n <- psi_n + Pi_F(chi) - P o_n; the overlap step takes psi_n - P o_n
            const float2 ov = cmul(p, o);
            const float2 st = cadd(dm_init ? ov : Sn[ln * M + x], dpsi);
            Sn[ln * M + x] = st;
            dpsi = csub(st, ov);
          }
          st_cluster_f2(dst + 8u * x, cconjmul(p, dpsi));
          if constexpr (!DM) {
            const int qi = ln * M + x;
            const float2 pc = cconjmul(o, dpsi);
            if (first) pacc[qi] = pc;
            else red_add_l2(&pacc[qi], pc);
            if (ln >= r0 && ln < r1) {
              if (first) dacc[qi] = cabs2(o);
              else red_add_l2(&dacc[qi], cabs2(o));
            }
          }
        }
      }
    }
    cluster_sync_all();
    // ---- (8) own rows of c_n: sum over the source ranks in order
    {
      float2* cn = a.cn + (size_t)n * M * M;
      for (int p = tid; p < nrow * M; p += TR) {
        const int lr = p / M, col = p % M;
        float2 s = make_float2(0.f, 0.f);
        for (int q = 0; q < K; ++q) s = cadd(s, recv[(q * RPO + lr) * LDN + col]);
        cn[(size_t)(r0 + lr) * M + col] = s;
      }
    }
    __syncthreads();  // the next position reuses the exchange buffer
  };

  // ---- end of a unit: probe-numerator partial from TMEM to global; per-CTA FP64 error
  // numerator (the compensated FP32 thread sums, added in thread order) into partial `part`
  auto finish_unit = [&](const FusedArgs& a, float2* pacc, int part) {
    if constexpr (TM && !DM) {
#pragma unroll
      for (int q = 0; q < V; ++q)
#pragma unroll
        for (int h = 0; h < E / 4; ++h) {
          float ac[8];
          tmem_ld8(t_lane + colA + 2 * (q * E + 4 * h), ac);
          tmem_wait_ld();
#pragma unroll
          for (int jj = 0; jj < 4; ++jj)
            pacc[line[q] * M + tp[q] + G * (4 * h + jj)] = make_float2(ac[2 * jj], ac[2 * jj + 1]);
        }
    }
    double* red = reinterpret_cast<double*>(smem);
    red[tid] = (double)err_s - (double)err_c;
    __syncthreads();
    for (int w = TR / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    if (tid == 0) a.errpart[(size_t)part * K + rank] = red[0];
    err_s = 0.f;
    err_c = 0.f;
    __syncthreads();  // red aliases the exchange buffer
  };

  if constexpr (!QUEUED) {
    // one problem: cluster `slot` takes positions slot, slot + slots, ... and owns partial `slot`
    setup_unit(a_in);
    __syncthreads();
    float2* pacc = a_in.pacc + ((size_t)slot * K + rank) * M * M;
    float* dacc = a_in.dacc + (size_t)slot * M * M;
    for (int n = slot; n < a_in.N; n += nslots) run_position(a_in, n, n == slot, pacc, dacc);
    finish_unit(a_in, pacc, slot);
  } else {
    // work queue over every problem of this launch: chunk (problem, first position, end, partial);
    // rank 0 takes the next chunk index and hands it to every rank of the cluster
    FusedArgs* s_desc = reinterpret_cast<FusedArgs*>(smem + SM::BYTES);
    int* s_item = reinterpret_cast<int*>(smem + SM::BYTES + SM::DESC - 16);
    for (;;) {
      if (rank == 0 && tid == 0) {
        const int c = atomicAdd(a_in.queue, 1);
        for (int q = 0; q < K; ++q) st_cluster_s32(map_rank(smem_addr(s_item), (unsigned)q), c);
      }
      cluster_sync_all();
      const int c = *s_item;
      if (c >= a_in.nchunks) break;
      const int4 ch = a_in.chunks[c];
      const int* src = reinterpret_cast<const int*>(a_in.probs + ch.x);
      for (int i = tid; i < (int)(sizeof(FusedArgs) / 4); i += TR) reinterpret_cast<int*>(s_desc)[i] = src[i];
      __syncthreads();
      setup_unit(*s_desc);
      __syncthreads();
      float2* pacc = s_desc->pacc + ((size_t)ch.w * K + rank) * M * M;
      float* dacc = s_desc->dacc + (size_t)ch.w * M * M;
      for (int n = ch.y; n < ch.z; ++n) run_position(*s_desc, n, n == ch.y, pacc, dacc);
      finish_unit(*s_desc, pacc, ch.w);
    }
  }
  if constexpr (TM) {
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (tid / 32 == 0) tmem_dealloc(*s_tmem, FusedShape<M>::TMEM_COLS);
  }
}

}  // namespace ptycho
