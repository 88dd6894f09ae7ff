// Numerical monochromatisation by CGLS (Sec. 4.2, Eqs. 12-13).
//
// Broadband pattern b = C m, C = sum_j w_j T_j (w_j: spectral weight / a_j^2), where T_j samples m at
// c + (i - c) / a_j along both axes (c = M / 2, a_j = lambda_j / lambda_c) with linear interpolation
// and zero outside the grid. k CGLS steps from x_0 = 0 give the least-squares solution over the
// Krylov subspace of Eq. 13.
//
// One CTA per pattern runs all k steps on chip: the search direction p (with a one-pixel zero
// border, so samples outside the grid read zeros) and the residual r live in shared memory; x and
// the step's product vector live in registers (thread t owns the pixels t + m TPB, one column per
// thread). C p gathers four neighbours per wavelength. C^T r runs separably per wavelength, r S_j
// then S_j^T (.), from a table of the transposed interpolation built in shared memory with the same
// coordinate formula as C, so the GPU's C^T is exactly the transpose of its C. Step sizes and norms
// are FP64 block reductions in a fixed order (bitwise reproducible).
#include <cuda_runtime.h>
#include <math.h>

#include "cluster.cuh"
#include "engine.h"

namespace ptycho {

namespace {

constexpr int kTapsT = 8;  // entries of one column of S_j (a_j <= 2.5: at most 2 a_j + 3)

template <int M>
struct MonoShape {
  static constexpr int TPB = M == 128 ? 1024 : (M == 8 ? 64 : 256);
  static constexpr int PPT = M * M / TPB;  // pixels per thread
  static constexpr int LDP = M + 2;        // padded row of p
  static constexpr size_t P_BYTES = (size_t)LDP * LDP * 4;
  static constexpr int LDR = M + 1;         // padded row of r and T (conflict-free column walks)
  static constexpr size_t R_BYTES = (size_t)M * LDR * 4;
  static constexpr size_t TAB_BYTES = (size_t)M * kTapsT * 8 + (size_t)M * 4;  // taps, then counts
  static constexpr size_t RED_BYTES = (size_t)(TPB / 32 + 1) * 2 * 8;
  static constexpr size_t SPEC_BYTES = (size_t)3 * kMonoMaxJ * 4;
  static constexpr size_t ROW_BYTES = (size_t)2 * M * 8;  // C p: row samples (i0, f), two buffers
  static constexpr size_t BYTES = P_BYTES + 2 * R_BYTES + TAB_BYTES + RED_BYTES + SPEC_BYTES + ROW_BYTES;
  static_assert(M * M % TPB == 0 && TPB % M == 0, "pixel ownership");
};

// sample position of output index i under scale 1 / a: i0 in [-1, M - 1] and fraction f (zero
// weight outside the grid: i0 = -1, f = 0 reads the zero border)
__device__ __forceinline__ void interp_at(int i, float c, float inv_a, int M, int& i0, float& f) {
  const float t = fmaf((float)i - c, inv_a, c);
  if (!(t >= -1.f && t < (float)M)) {
    i0 = -1;
    f = 0.f;
    return;
  }
  const float fl = floorf(t);
  i0 = (int)fl;
  f = t - fl;
}

// FP64 sums of two per-thread values over the CTA, in a fixed order; every thread gets both. The
// warps' sums are finished by warp 0 alone (shuffle tree) and broadcast through shared memory.
template <int TPB>
__device__ __forceinline__ void block_sum2(double a, double b, double* red, double& oa, double& ob) {
  constexpr int NW = TPB / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  __syncthreads();  // red is free (previous readers are done)
  if (lane == 0) {
    red[2 * warp] = a;
    red[2 * warp + 1] = b;
  }
  __syncthreads();
  if (warp == 0) {
    double x = lane < NW ? red[2 * lane] : 0.0, y = lane < NW ? red[2 * lane + 1] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane == 0) {
      red[2 * NW] = x;
      red[2 * NW + 1] = y;
    }
  }
  __syncthreads();
  oa = red[2 * NW];
  ob = red[2 * NW + 1];
}

template <int M>
__global__ void __launch_bounds__(MonoShape<M>::TPB, 1) k_mono_cgls(const MonoArgs a) {
  using SH = MonoShape<M>;
  constexpr int TPB = SH::TPB, PPT = SH::PPT, LDP = SH::LDP, LDR = SH::LDR, RSTEP = TPB / M;
  extern __shared__ __align__(16) unsigned char smem[];
  float* Pp = reinterpret_cast<float*>(smem);                        // (M + 2)^2, zero border
  float* R = reinterpret_cast<float*>(smem + SH::P_BYTES);               // M x LDR
  float* T = reinterpret_cast<float*>(smem + SH::P_BYTES + SH::R_BYTES);  // M x LDR, r S_j
  // column u of S_j: its non-zero taps (weight, source index as float bits) in increasing source
  // order, zero-filled to kTapsT, and their count
  float2* tab = reinterpret_cast<float2*>(smem + SH::P_BYTES + 2 * SH::R_BYTES);
  const float4* tab4 = reinterpret_cast<const float4*>(tab);
  int* tab_n = reinterpret_cast<int*>(tab + M * kTapsT);
  double* red = reinterpret_cast<double*>(smem + SH::P_BYTES + 2 * SH::R_BYTES + SH::TAB_BYTES);
  // spectrum: 1 / a_j, a_j, w_j
  float* s_inv = reinterpret_cast<float*>(smem + SH::P_BYTES + 2 * SH::R_BYTES + SH::TAB_BYTES + SH::RED_BYTES);
  float* s_a = s_inv + kMonoMaxJ;
  float* s_w = s_a + kMonoMaxJ;
  float2* s_rt = reinterpret_cast<float2*>(smem + SH::P_BYTES + 2 * SH::R_BYTES + SH::TAB_BYTES + SH::RED_BYTES +
                                           SH::SPEC_BYTES);  // 2 x M

  const int tid = threadIdx.x;
  const int col = tid % M, row0 = tid / M;
  const float c = 0.5f * (float)M;
  const int n = blockIdx.x;
  const float* bn = a.b + (size_t)n * M * M;
  float* xn = a.x + (size_t)n * M * M;
  double* rs = a.resid ? a.resid + (size_t)n * (a.k + 1) : nullptr;

  // C^T v for the own pixels into acc, v in R (separable per wavelength, through T)
  auto adjoint = [&](float (&acc)[PPT]) {
#pragma unroll
    for (int m = 0; m < PPT; ++m) acc[m] = 0.f;
    for (int j = 0; j < a.J; ++j) {
      const float inv_a = s_inv[j], sa = s_a[j];
      // column u of S_j: the sources x with i0(x) in {u - 1, u}; weight 1 - f (i0 = u) or f (i0 = u - 1)
      // (M * kTapsT is a multiple of 32 and so is TPB: every warp runs whole iterations, and the 8
      // lanes of one column sit in one warp)
      for (int e = tid; e < M * kTapsT; e += TPB) {
        const int u = e / kTapsT, l = e % kTapsT;
        const int lo = max(0, (int)ceilf(fmaf((float)(u - 1) - c, sa, c)) - 1);
        const int hi = min(M - 1, (int)floorf(fmaf((float)(u + 1) - c, sa, c)) + 1);
        const int src = lo + l;
        float w = 0.f;
        if (src <= hi) {
          int i0;
          float f;
          interp_at(src, c, inv_a, M, i0, f);
          w = i0 == u ? 1.f - f : (i0 == u - 1 ? f : 0.f);
        }
        const unsigned nz = __ballot_sync(0xffffffffu, w != 0.f);
        const unsigned grp = (nz >> ((tid & 31) & ~(kTapsT - 1))) & ((1u << kTapsT) - 1u);
        const int cnt = __popc(grp);
        if (w != 0.f) tab[u * kTapsT + __popc(grp & ((1u << l) - 1u))] = make_float2(w, __int_as_float(src));
        if (l >= cnt) tab[u * kTapsT + l] = make_float2(0.f, __int_as_float(0));
        if (l == 0) tab_n[u] = cnt;
      }
      __syncthreads();
      // T(y, v) = sum_x S_j[x, v] R(y, x); zero-filled taps add exact zeros
      if constexpr (M >= 32) {
        // a warp walks 32 consecutive rows of one column: the column's taps are a broadcast and the
        // padded rows put the 32 loads (and the store) in 32 different banks
        const int lane = tid & 31, warp = tid >> 5;
#pragma unroll 4
        for (int m = 0; m < PPT; ++m) {
          const int unit = warp * PPT + m;
          const int v = unit % M, y = (unit / M) * 32 + lane;
          const int nt = tab_n[v];
          float s = 0.f;
#pragma unroll
          for (int h = 0; h < kTapsT / 2; ++h)
            if (2 * h < nt) {
              const float4 e = tab4[v * (kTapsT / 2) + h];
              s = fmaf(e.x, R[y * LDR + __float_as_int(e.y)], s);
              s = fmaf(e.z, R[y * LDR + __float_as_int(e.w)], s);
            }
          T[y * LDR + v] = s;
        }
      } else {
        int ci[kTapsT];
        float cw[kTapsT];
#pragma unroll
        for (int h = 0; h < kTapsT / 2; ++h) {
          const float4 e = tab4[col * (kTapsT / 2) + h];
          cw[2 * h] = e.x;
          ci[2 * h] = __float_as_int(e.y);
          cw[2 * h + 1] = e.z;
          ci[2 * h + 1] = __float_as_int(e.w);
        }
        const int nt = __reduce_max_sync(0xffffffffu, tab_n[col]);
#pragma unroll
        for (int m = 0; m < PPT; ++m) {
          const int y = row0 + m * RSTEP;
          float s = 0.f;
#pragma unroll
          for (int l = 0; l < kTapsT; ++l)
            if (l < nt) s = fmaf(cw[l], R[y * LDR + ci[l]], s);
          T[y * LDR + col] = s;
        }
      }
      __syncthreads();
      // acc(u, v) += w_j sum_y S_j[y, u] T(y, v)
      const float wj = s_w[j];
#pragma unroll
      for (int m = 0; m < PPT; ++m) {
        const int u = row0 + m * RSTEP;
        const int nh = (__reduce_max_sync(0xffffffffu, tab_n[u]) + 1) / 2;
        float s = 0.f;
#pragma unroll
        for (int h = 0; h < kTapsT / 2; ++h)
          if (h < nh) {
            const float4 e = tab4[u * (kTapsT / 2) + h];
            s = fmaf(e.x, T[__float_as_int(e.y) * LDR + col], s);
            s = fmaf(e.z, T[__float_as_int(e.w) * LDR + col], s);
          }
        acc[m] = fmaf(wj, s, acc[m]);
      }
      __syncthreads();  // the table and T are rebuilt for the next wavelength
    }
  };

  // C p for the own pixels into acc, p in Pp. The row samples of a wavelength are the same for a
  // whole row of pixels: a table per wavelength (two buffers: the barrier that publishes table j
  // also ends every read of table j - 2)
  auto forward = [&](float (&acc)[PPT]) {
#pragma unroll
    for (int m = 0; m < PPT; ++m) acc[m] = 0.f;
    for (int j = 0; j < a.J; ++j) {
      const float inv_a = s_inv[j], wj = s_w[j];
      float2* rt = s_rt + (j & 1) * M;
      for (int i = tid; i < M; i += TPB) {
        int i0;
        float f;
        interp_at(i, c, inv_a, M, i0, f);
        rt[i] = make_float2(__int_as_float(i0), f);
      }
      __syncthreads();
      int x0;
      float fx;
      interp_at(col, c, inv_a, M, x0, fx);
      const float gx = 1.f - fx;
#pragma unroll
      for (int m = 0; m < PPT; ++m) {
        const float2 ry = rt[row0 + m * RSTEP];
        const int y0 = __float_as_int(ry.x);
        const float fy = ry.y;
        const float* p0 = Pp + (y0 + 1) * LDP + (x0 + 1);
        const float top = fmaf(fx, p0[1], gx * p0[0]);
        const float bot = fmaf(fx, p0[LDP + 1], gx * p0[LDP]);
        acc[m] = fmaf(wj, fmaf(fy, bot, (1.f - fy) * top), acc[m]);
      }
    }
  };

  // ---- start: spectrum to shared memory, zero border of p, r = b, x = 0
  for (int i = tid; i < a.J; i += TPB) {
    s_inv[i] = a.inv_a[i];
    s_a[i] = a.a[i];
    s_w[i] = a.w[i];
  }
  for (int i = tid; i < LDP * LDP; i += TPB) Pp[i] = 0.f;
  float xk[PPT], acc[PPT];
  float rr = 0.f;  // per-thread partial sums in FP32 (PPT terms), CTA sums in FP64
#pragma unroll
  for (int m = 0; m < PPT; ++m) {
    const int y = row0 + m * RSTEP;
    const float v = bn[y * M + col];
    R[y * LDR + col] = v;
    rr = fmaf(v, v, rr);
    xk[m] = 0.f;
  }
  __syncthreads();
  adjoint(acc);  // s_0 = C^T b
  double gamma = 0.0, rr_all = 0.0;
  {
    float g = 0.f;
#pragma unroll
    for (int m = 0; m < PPT; ++m) g = fmaf(acc[m], acc[m], g);
    block_sum2<TPB>(g, rr, red, gamma, rr_all);
  }
  if (rs && tid == 0) rs[0] = sqrt(rr_all);
#pragma unroll
  for (int m = 0; m < PPT; ++m) Pp[(row0 + m * RSTEP + 1) * LDP + col + 1] = acc[m];
  __syncthreads();

  for (int it = 0; it < a.k; ++it) {
    if (!(gamma > 0.0)) {  // C^T r = 0: x is the least-squares solution already
      if (rs && tid == 0) rs[it + 1] = sqrt(rr_all);
      continue;
    }
    forward(acc);  // q = C p
    double qq = 0.0;
    {
      float l = 0.f;
#pragma unroll
      for (int m = 0; m < PPT; ++m) l = fmaf(acc[m], acc[m], l);
      double unused;
      block_sum2<TPB>(l, 0.0, red, qq, unused);
    }
    if (!(qq > 0.0)) {
      if (rs && tid == 0) rs[it + 1] = sqrt(rr_all);
      continue;
    }
    const float alpha = (float)(gamma / qq);
    rr = 0.f;
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      const int y = row0 + m * RSTEP;
      xk[m] = fmaf(alpha, Pp[(y + 1) * LDP + col + 1], xk[m]);
      const float r = fmaf(-alpha, acc[m], R[y * LDR + col]);
      R[y * LDR + col] = r;
      rr = fmaf(r, r, rr);
    }
    __syncthreads();
    adjoint(acc);  // s = C^T r
    double gnew = 0.0;
    {
      float g = 0.f;
#pragma unroll
      for (int m = 0; m < PPT; ++m) g = fmaf(acc[m], acc[m], g);
      block_sum2<TPB>(g, rr, red, gnew, rr_all);
    }
    if (rs && tid == 0) rs[it + 1] = sqrt(rr_all);
    const float beta = (float)(gnew / gamma);
    gamma = gnew;
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      float* pp = Pp + (row0 + m * RSTEP + 1) * LDP + col + 1;
      *pp = fmaf(beta, *pp, acc[m]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < PPT; ++m) {
    const float v = xk[m];
    xn[(row0 + m * RSTEP) * M + col] = a.clamp ? fmaxf(v, 0.f) : v;
  }
}

// ---- M = 256: one cluster of kBands CTAs per pattern, CTA rank b owns rows [b BR, (b + 1) BR) of p,
// r and T. C p reads its four neighbours from whichever band holds them (distributed shared memory),
// the first adjoint pass works on the own rows, the second reads T across the bands; CTA sums meet
// in rank 0's shared memory and every rank adds them in rank order (identical step sizes on all
// ranks).
constexpr int kBands = 4;

__device__ __forceinline__ double ld_cluster_f64(uint32_t addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void st_cluster_f64(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}

struct MonoBandShape {
  static constexpr int M = 256, BR = M / kBands, TPB = 1024, PPT = BR * M / TPB, RSTEP = TPB / M;
  static constexpr int LDR = M + 1;
  static constexpr size_t P_BYTES = (size_t)BR * M * 4;
  static constexpr size_t R_BYTES = (size_t)BR * LDR * 4;
  static constexpr size_t TAB_BYTES = (size_t)M * kTapsT * 8 + (size_t)M * 4;
  static constexpr size_t RED_BYTES = (size_t)(TPB / 32 + 1) * 2 * 8 + (size_t)kBands * 2 * 8;
  static constexpr size_t SPEC_BYTES = (size_t)3 * kMonoMaxJ * 4;
  static constexpr size_t BYTES = P_BYTES + 2 * R_BYTES + TAB_BYTES + RED_BYTES + SPEC_BYTES;
  static_assert(BR % 32 == 0 && TPB % M == 0 && (BR * M) % TPB == 0, "band ownership");
};

__global__ void __launch_bounds__(MonoBandShape::TPB, 1) k_mono_cgls_band(const MonoArgs a) {
  using SH = MonoBandShape;
  constexpr int M = SH::M, BR = SH::BR, TPB = SH::TPB, PPT = SH::PPT, RSTEP = SH::RSTEP, LDR = SH::LDR;
  constexpr int NW = TPB / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  float* Pb = reinterpret_cast<float*>(smem);                              // BR x M
  float* R = reinterpret_cast<float*>(smem + SH::P_BYTES);                 // BR x LDR
  float* T = reinterpret_cast<float*>(smem + SH::P_BYTES + SH::R_BYTES);  // BR x LDR, r S_j
  float2* tab = reinterpret_cast<float2*>(smem + SH::P_BYTES + 2 * SH::R_BYTES);
  const float4* tab4 = reinterpret_cast<const float4*>(tab);
  int* tab_n = reinterpret_cast<int*>(tab + M * kTapsT);
  double* red = reinterpret_cast<double*>(smem + SH::P_BYTES + 2 * SH::R_BYTES + SH::TAB_BYTES);
  double* slots = red + 2 * (NW + 1);  // kBands x 2 CTA sums (used in rank 0)
  float* s_inv = reinterpret_cast<float*>(smem + SH::P_BYTES + 2 * SH::R_BYTES + SH::TAB_BYTES + SH::RED_BYTES);
  float* s_a = s_inv + kMonoMaxJ;
  float* s_w = s_a + kMonoMaxJ;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned band = cluster_ctarank();
  const int n = blockIdx.x / kBands;
  const int y_base = (int)band * BR;
  const int col = tid % M, lrow0 = tid / M;  // own pixels: local rows lrow0 + RSTEP m, column col
  const float c = 0.5f * (float)M;
  const float* bn = a.b + (size_t)n * M * M;
  float* xn = a.x + (size_t)n * M * M;
  double* rs = a.resid ? a.resid + (size_t)n * (a.k + 1) : nullptr;
  const uint32_t pb_s = smem_addr(Pb), t_s = smem_addr(T), slots_s = smem_addr(slots);

  // two FP64 sums over the cluster (per-CTA fixed-order sums, then the ranks in order)
  auto cluster_sum2 = [&](double x, double y, double& ox, double& oy) {
    double cx, cy;
    block_sum2<TPB>(x, y, red, cx, cy);
    cluster_sync_all();  // the slots are free (every rank read the previous sums)
    if (tid == 0) {
      st_cluster_f64(map_rank(slots_s + 16u * band, 0), cx);
      st_cluster_f64(map_rank(slots_s + 16u * band + 8u, 0), cy);
    }
    cluster_sync_all();
    double sx = 0.0, sy = 0.0;
    for (int q = 0; q < kBands; ++q) {
      sx += ld_cluster_f64(map_rank(slots_s + 16u * q, 0));
      sy += ld_cluster_f64(map_rank(slots_s + 16u * q + 8u, 0));
    }
    ox = sx;
    oy = sy;
  };
  // p at global (yy, xx), zero outside the grid
  auto p_at = [&](int yy, int xx) -> float {
    if (yy < 0 || yy >= M || xx < 0 || xx >= M) return 0.f;
    return ld_cluster_f32(map_rank(pb_s + (uint32_t)(((yy % BR) * M + xx) * 4), (unsigned)(yy / BR)));
  };

  auto adjoint = [&](float (&acc)[PPT]) {
#pragma unroll
    for (int m = 0; m < PPT; ++m) acc[m] = 0.f;
    for (int j = 0; j < a.J; ++j) {
      const float inv_a = s_inv[j], sa = s_a[j];
      for (int e = tid; e < M * kTapsT; e += TPB) {
        const int u = e / kTapsT, l = e % kTapsT;
        const int lo = max(0, (int)ceilf(fmaf((float)(u - 1) - c, sa, c)) - 1);
        const int hi = min(M - 1, (int)floorf(fmaf((float)(u + 1) - c, sa, c)) + 1);
        const int src = lo + l;
        float w = 0.f;
        if (src <= hi) {
          int i0;
          float f;
          interp_at(src, c, inv_a, M, i0, f);
          w = i0 == u ? 1.f - f : (i0 == u - 1 ? f : 0.f);
        }
        const unsigned nz = __ballot_sync(0xffffffffu, w != 0.f);
        const unsigned grp = (nz >> ((tid & 31) & ~(kTapsT - 1))) & ((1u << kTapsT) - 1u);
        const int cnt = __popc(grp);
        if (w != 0.f) tab[u * kTapsT + __popc(grp & ((1u << l) - 1u))] = make_float2(w, __int_as_float(src));
        if (l >= cnt) tab[u * kTapsT + l] = make_float2(0.f, __int_as_float(0));
        if (l == 0) tab_n[u] = cnt;
      }
      __syncthreads();
      // T(y, v) = sum_x S_j[x, v] R(y, x) on the own rows: a warp walks 32 rows of one column
#pragma unroll 4
      for (int m = 0; m < PPT; ++m) {
        const int unit = warp * PPT + m;
        const int v = unit % M, ly = (unit / M) * 32 + lane;
        const int nt = tab_n[v];
        float sum = 0.f;
#pragma unroll
        for (int h = 0; h < kTapsT / 2; ++h)
          if (2 * h < nt) {
            const float4 e = tab4[v * (kTapsT / 2) + h];
            sum = fmaf(e.x, R[ly * LDR + __float_as_int(e.y)], sum);
            sum = fmaf(e.z, R[ly * LDR + __float_as_int(e.w)], sum);
          }
        T[ly * LDR + v] = sum;
      }
      cluster_sync_all();  // every band's T is complete
      // acc(u, v) += w_j sum_y S_j[y, u] T(y, v), T rows from their bands
      const float wj = s_w[j];
#pragma unroll
      for (int m = 0; m < PPT; ++m) {
        const int u = y_base + lrow0 + m * RSTEP;
        const int nh = (__reduce_max_sync(0xffffffffu, tab_n[u]) + 1) / 2;
        float sum = 0.f;
#pragma unroll
        for (int h = 0; h < kTapsT / 2; ++h)
          if (h < nh) {
            const float4 e = tab4[u * (kTapsT / 2) + h];
            const int y1 = __float_as_int(e.y), y2 = __float_as_int(e.w);
            const float t1 = ld_cluster_f32(map_rank(t_s + (uint32_t)(((y1 % BR) * LDR + col) * 4), (unsigned)(y1 / BR)));
            const float t2 = ld_cluster_f32(map_rank(t_s + (uint32_t)(((y2 % BR) * LDR + col) * 4), (unsigned)(y2 / BR)));
            sum = fmaf(e.x, t1, sum);
            sum = fmaf(e.z, t2, sum);
          }
        acc[m] = fmaf(wj, sum, acc[m]);
      }
      cluster_sync_all();  // no rank reads this T any more; the table is rebuilt
    }
  };

  auto forward = [&](float (&acc)[PPT]) {
#pragma unroll
    for (int m = 0; m < PPT; ++m) acc[m] = 0.f;
    for (int j = 0; j < a.J; ++j) {
      const float inv_a = s_inv[j], wj = s_w[j];
      int x0;
      float fx;
      interp_at(col, c, inv_a, M, x0, fx);
      const float gx = 1.f - fx;
#pragma unroll 4
      for (int m = 0; m < PPT; ++m) {
        int y0;
        float fy;
        interp_at(y_base + lrow0 + m * RSTEP, c, inv_a, M, y0, fy);
        const float top = fmaf(fx, p_at(y0, x0 + 1), gx * p_at(y0, x0));
        const float bot = fmaf(fx, p_at(y0 + 1, x0 + 1), gx * p_at(y0 + 1, x0));
        acc[m] = fmaf(wj, fmaf(fy, bot, (1.f - fy) * top), acc[m]);
      }
    }
  };

  // ---- start: spectrum to shared memory, r = b (own rows), x = 0
  for (int i = tid; i < a.J; i += TPB) {
    s_inv[i] = a.inv_a[i];
    s_a[i] = a.a[i];
    s_w[i] = a.w[i];
  }
  float xk[PPT], acc[PPT];
  float rr = 0.f;
#pragma unroll
  for (int m = 0; m < PPT; ++m) {
    const int ly = lrow0 + m * RSTEP;
    const float v = bn[(size_t)(y_base + ly) * M + col];
    R[ly * LDR + col] = v;
    rr = fmaf(v, v, rr);
    xk[m] = 0.f;
  }
  __syncthreads();
  adjoint(acc);  // s_0 = C^T b
  double gamma = 0.0, rr_all = 0.0;
  {
    float g = 0.f;
#pragma unroll
    for (int m = 0; m < PPT; ++m) g = fmaf(acc[m], acc[m], g);
    cluster_sum2(g, rr, gamma, rr_all);
  }
  if (rs && band == 0 && tid == 0) rs[0] = sqrt(rr_all);
#pragma unroll
  for (int m = 0; m < PPT; ++m) Pb[(lrow0 + m * RSTEP) * M + col] = acc[m];
  cluster_sync_all();  // p complete in every band

  for (int it = 0; it < a.k; ++it) {
    if (!(gamma > 0.0)) {
      if (rs && band == 0 && tid == 0) rs[it + 1] = sqrt(rr_all);
      continue;
    }
    forward(acc);  // q = C p
    double qq = 0.0;
    {
      float l = 0.f;
#pragma unroll
      for (int m = 0; m < PPT; ++m) l = fmaf(acc[m], acc[m], l);
      double unused;
      cluster_sum2(l, 0.0, qq, unused);
    }
    if (!(qq > 0.0)) {
      if (rs && band == 0 && tid == 0) rs[it + 1] = sqrt(rr_all);
      continue;
    }
    const float alpha = (float)(gamma / qq);
    rr = 0.f;
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      const int ly = lrow0 + m * RSTEP;
      xk[m] = fmaf(alpha, Pb[ly * M + col], xk[m]);
      const float r = fmaf(-alpha, acc[m], R[ly * LDR + col]);
      R[ly * LDR + col] = r;
      rr = fmaf(r, r, rr);
    }
    __syncthreads();
    adjoint(acc);  // s = C^T r
    double gnew = 0.0;
    {
      float g = 0.f;
#pragma unroll
      for (int m = 0; m < PPT; ++m) g = fmaf(acc[m], acc[m], g);
      cluster_sum2(g, rr, gnew, rr_all);
    }
    if (rs && band == 0 && tid == 0) rs[it + 1] = sqrt(rr_all);
    const float beta = (float)(gnew / gamma);
    gamma = gnew;
    // every rank finished reading p in the forward pass (cluster barriers since); update the own band
#pragma unroll
    for (int m = 0; m < PPT; ++m) {
      float* pp = Pb + (lrow0 + m * RSTEP) * M + col;
      *pp = fmaf(beta, *pp, acc[m]);
    }
    cluster_sync_all();
  }
#pragma unroll
  for (int m = 0; m < PPT; ++m) {
    const float v = xk[m];
    xn[(size_t)(y_base + lrow0 + m * RSTEP) * M + col] = a.clamp ? fmaxf(v, 0.f) : v;
  }
  cluster_sync_all();  // no rank exits while another may still read its shared memory
}

cudaError_t launch_mono_band(const MonoArgs& a, cudaStream_t s) {
  using SH = MonoBandShape;
  cudaError_t e = cudaFuncSetAttribute(k_mono_cgls_band, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SH::BYTES);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(a.N * kBands));
  cfg.blockDim = dim3(SH::TPB);
  cfg.dynamicSmemBytes = SH::BYTES;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kBands;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_mono_cgls_band, a);
}

template <int M>
cudaError_t launch_mono_t(const MonoArgs& a, cudaStream_t s) {
  using SH = MonoShape<M>;
  auto kern = k_mono_cgls<M>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SH::BYTES);
  if (e != cudaSuccess) return e;
  kern<<<a.N, SH::TPB, SH::BYTES, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mono(const MonoArgs& a, cudaStream_t s) {
  if (a.N == 0) return cudaSuccess;
  switch (a.M) {
    case 8: return launch_mono_t<8>(a, s);
    case 16: return launch_mono_t<16>(a, s);
    case 32: return launch_mono_t<32>(a, s);
    case 64: return launch_mono_t<64>(a, s);
    case 128: return launch_mono_t<128>(a, s);
    case 256: return launch_mono_band(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ptycho
