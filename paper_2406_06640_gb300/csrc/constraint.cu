// Complex constraint of Fig. 1 box 2 (Eqs. 9-11) for the data-parallel engine.
//
//   a = max(|O|, 1e-6), phi = arg O in (-pi, pi]
//   C_n    = clamp( sum_box |ln a| / max(sum_box |phi|, 1e-30), cbar_min, cbar_max )   (Eq. 11, Sec. 4.8)
//   C(r)   = mean of C_n over the boxes that cover r
//   A^c    = exp((1 - alpha1) ln a + alpha1 C phi)                                       (Eq. 9)
//   phi^c  = (1 - alpha2) phi + alpha2 ln a / C                                          (Eq. 10)
//   O      = A^c exp(i phi^c) on covered pixels; uncovered pixels are unchanged.
//
// The paper applies the constraint per box inside its sequential loop; with
// every box updated at once, overlapping boxes are reconciled by the per-pixel
// mean of their C_n.
//
// All box sums are exact: values are held in 32.32 fixed point (int64) and
// summed with integer arithmetic, so the results do not depend on order.
//   (1) |ln a| and |phi| of every object pixel in 32.32 fixed point, as prefix sums along the
//       object rows;
//   (2) one warp per box: each box sum is M differences of two row prefix sums -> C_n, and C_n
//       in fixed point;
//   (3) one block per 32 x 32 object tile: the boxes of the tile's position list, clipped to the
//       tile, add their fixed-point C_n at the corners of a difference array in shared memory;
//       its prefix sums give every pixel the sum over the boxes that contain it and their
//       count; then Eqs. 9-10.
// Every sum is an exact integer sum, so the results do not depend on the order of the terms.
#include <cuda_runtime.h>
#include <math.h>

#include "engine.h"
#include "fft.cuh"

namespace ptycho {

constexpr double kFix = 4294967296.0;  // 2^32

// Row prefix sums of |ln a| and |phi| in 32.32 fixed point: P(y, x) = sum over x' < x of the value at
// (y, x'), obj_h x (obj_w + 1) each. v * 2^32 is exact in FP32, so llrintf of it is the nearest
// 32.32 value of v.
__device__ __forceinline__ void cc_values(float2 o, long long& l, long long& p) {
  const float f = 4294967296.0f;
  l = llrintf(fabsf(logf(fmaxf(sqrtf(cabs2(o)), 1e-6f))) * f);
  p = llrintf(fabsf(atan2f(o.y, o.x)) * f);
}

__global__ void __launch_bounds__(256) k_cc_rows(const ConstraintArgs c) {
  // one block per object row, warp w scanning segment w of SEG pixels (32 per step, a carry
  // between steps), then every segment adds the totals of the segments before it
  __shared__ long long s_tl[8], s_tp[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int y = blockIdx.x;
  const int W1 = c.obj_w + 1;
  const int SEG = ((c.obj_w + 7) / 8 + 31) / 32 * 32;
  const int x_lo = min(c.obj_w, w * SEG), x_hi = min(c.obj_w, x_lo + SEG);
  long long* pl = c.map_lna + (size_t)y * W1;
  long long* pp = c.map_phi + (size_t)y * W1;
  const float2* Oy = c.O + (size_t)y * c.obj_w;
  if (threadIdx.x == 0) {
    pl[0] = 0;
    pp[0] = 0;
  }
  long long cl = 0, cp = 0;  // this segment's sums so far
  for (int x0 = x_lo; x0 < x_hi; x0 += 32) {
    const int x = x0 + lane;
    long long vl = 0, vp = 0;
    if (x < x_hi) cc_values(Oy[x], vl, vp);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long ul = __shfl_up_sync(0xffffffffu, vl, d);
      const long long up = __shfl_up_sync(0xffffffffu, vp, d);
      if (lane >= d) {
        vl += ul;
        vp += up;
      }
    }
    if (x < x_hi) {
      pl[x + 1] = cl + vl;
      pp[x + 1] = cp + vp;
    }
    cl += __shfl_sync(0xffffffffu, vl, 31);
    cp += __shfl_sync(0xffffffffu, vp, 31);
  }
  if (lane == 0) {
    s_tl[w] = cl;
    s_tp[w] = cp;
  }
  __syncthreads();
  long long ol = 0, op = 0;
  for (int q = 0; q < w; ++q) {
    ol += s_tl[q];
    op += s_tp[q];
  }
  if (w > 0)
    for (int x = x_lo + lane; x < x_hi; x += 32) {
      pl[x + 1] += ol;
      pp[x + 1] += op;
    }
}

// one warp per box: the two box sums (exact) from M row differences each, C_n clamped, C_n in fixed
// point
__global__ void __launch_bounds__(256) k_cc_cbar(const ConstraintArgs c) {
  const int lane = threadIdx.x & 31;
  const int n = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (n >= c.N) return;
  const int2 pn = c.pos[n];
  const int M = c.M, W1 = c.obj_w + 1;
  long long a = 0, b = 0;
  for (int i = lane; i < M; i += 32) {
    const size_t r = (size_t)(pn.x + i) * W1;
    a += c.map_lna[r + pn.y + M] - c.map_lna[r + pn.y];
    b += c.map_phi[r + pn.y + M] - c.map_phi[r + pn.y];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    const double sl = (double)a / kFix;
    const double sp = (double)b / kFix;
    const double r = sl / fmax(sp, 1e-30);
    const float cb = (float)fmin(fmax(r, (double)c.cbar_min), (double)c.cbar_max);
    c.cbar[n] = cb;
    c.cbar_q[n] = llrint((double)cb * kFix);
  }
}

// grid (tiles_x, tiles_y), block 32 x 8. Per tile: every box clipped to the tile adds its fixed-point
// C_n (and 1) at the four corners of a (T + 1)^2 difference array in shared memory (integer atomics:
// exact, order-independent); 2-D prefix sums give each pixel the sum over the boxes that contain it
// and their count; then Eqs. 9-10. Thread (tx, ty) owns pixels (Y0 + ty + 8 i, X0 + tx), i < 4.
__global__ void __launch_bounds__(256) k_cc_apply(const ConstraintArgs c) {
  constexpr int T = kObjTile, T1 = kObjTile + 1;
  __shared__ long long dq[T1 * T1];
  __shared__ int dn[T1 * T1];
  const int tile = blockIdx.y * c.tiles_x + blockIdx.x;
  const int ty0 = blockIdx.y * T, tx0 = blockIdx.x * T;
  const int lt = threadIdx.y * 32 + threadIdx.x;
  const int M = c.M;
  for (int i = lt; i < T1 * T1; i += 256) {
    dq[i] = 0;
    dn[i] = 0;
  }
  __syncthreads();
  // Corners on row or column T lie outside the tile and reach no pixel: skipped. Boxes that cover
  // the tile's first corner all clip to (0, 0): those add up per thread and per warp first.
  unsigned long long* uq = reinterpret_cast<unsigned long long*>(dq);
  unsigned long long q00 = 0;
  int n00 = 0;
  const int e0 = c.tile_start[tile], e1 = c.tile_start[tile + 1];
  for (int e = e0 + lt; e < e1; e += 256) {
    const int4 ent = c.tile_pos[e];  // (n, row, col)
    const int r0 = max(ent.y - ty0, 0), r1 = min(ent.y + M - ty0, T);
    const int c0 = max(ent.z - tx0, 0), c1 = min(ent.z + M - tx0, T);
    if (r0 >= r1 || c0 >= c1) continue;
    const unsigned long long q = (unsigned long long)c.cbar_q[ent.x];
    if (r0 == 0 && c0 == 0) {
      q00 += q;
      n00 += 1;
    } else {
      atomicAdd(&uq[r0 * T1 + c0], q);
      atomicAdd(&dn[r0 * T1 + c0], 1);
    }
    if (c1 < T) {
      atomicAdd(&uq[r0 * T1 + c1], 0ull - q);
      atomicAdd(&dn[r0 * T1 + c1], -1);
    }
    if (r1 < T) {
      atomicAdd(&uq[r1 * T1 + c0], 0ull - q);
      atomicAdd(&dn[r1 * T1 + c0], -1);
    }
    if (r1 < T && c1 < T) {
      atomicAdd(&uq[r1 * T1 + c1], q);
      atomicAdd(&dn[r1 * T1 + c1], 1);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    q00 += __shfl_xor_sync(0xffffffffu, q00, o);
    n00 += __shfl_xor_sync(0xffffffffu, n00, o);
  }
  if ((lt & 31) == 0 && n00 > 0) {
    atomicAdd(&uq[0], q00);
    atomicAdd(&dn[0], n00);
  }
  __syncthreads();
  // prefix sums along the rows, then along the columns: warp scans, each warp T / 8 lines
  static_assert(T == 32, "one lane per tile column");
  const int wl = lt & 31, wi = lt >> 5;
  for (int ln = wi; ln < T; ln += 8) {
    long long q = dq[ln * T1 + wl];
    int m = dn[ln * T1 + wl];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long uq = __shfl_up_sync(0xffffffffu, q, d);
      const int um = __shfl_up_sync(0xffffffffu, m, d);
      if (wl >= d) {
        q += uq;
        m += um;
      }
    }
    dq[ln * T1 + wl] = q;
    dn[ln * T1 + wl] = m;
  }
  __syncthreads();
  for (int ln = wi; ln < T; ln += 8) {
    long long q = dq[wl * T1 + ln];
    int m = dn[wl * T1 + ln];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long uq = __shfl_up_sync(0xffffffffu, q, d);
      const int um = __shfl_up_sync(0xffffffffu, m, d);
      if (wl >= d) {
        q += uq;
        m += um;
      }
    }
    dq[wl * T1 + ln] = q;
    dn[wl * T1 + ln] = m;
  }
  __syncthreads();
  const int X = tx0 + threadIdx.x;
  if (X >= c.obj_w) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int ly = threadIdx.y + 8 * i;
    const int Y = ty0 + ly;
    const int cnt = dn[ly * T1 + threadIdx.x];
    if (Y >= c.obj_h || cnt == 0) continue;
    const size_t q = (size_t)Y * c.obj_w + X;
    const float C = (float)((double)dq[ly * T1 + threadIdx.x] / kFix / (double)cnt);
    const float2 o = c.O[q];
    const float lna = logf(fmaxf(sqrtf(cabs2(o)), 1e-6f));
    const float phi = atan2f(o.y, o.x);
    const float ac = expf((1.f - c.alpha1) * lna + c.alpha1 * C * phi);
    const float pc = (1.f - c.alpha2) * phi + c.alpha2 * lna / C;
    float sn, cs;
    sincosf(pc, &sn, &cs);
    c.O[q] = make_float2(ac * cs, ac * sn);
  }
}

cudaError_t launch_constraint(const ConstraintArgs& c, cudaStream_t s) {
  if (c.N == 0) return cudaSuccess;
  k_cc_rows<<<c.obj_h, 256, 0, s>>>(c);
  k_cc_cbar<<<(c.N + 7) / 8, 256, 0, s>>>(c);
  k_cc_apply<<<dim3(c.tiles_x, c.tiles_y), dim3(32, 8), 0, s>>>(c);
  return cudaGetLastError();
}

}  // namespace ptycho
