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
//   (1) |ln a| and |phi| of every object pixel, in 32.32 fixed point;
//   (2) one block per box sums both maps over the box with integer adds -> C_n, and C_n in
//       fixed point;
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

// |ln a| and |phi| of every object pixel in 32.32 fixed point (obj_h x obj_w each)
__global__ void __launch_bounds__(256) k_cc_maps(const ConstraintArgs c) {
  const size_t n = (size_t)c.obj_h * c.obj_w;
  for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (size_t)gridDim.x * 256) {
    const float2 o = c.O[i];
    c.map_lna[i] = llrint((double)fabsf(logf(fmaxf(sqrtf(cabs2(o)), 1e-6f))) * kFix);
    c.map_phi[i] = llrint((double)fabsf(atan2f(o.y, o.x)) * kFix);
  }
}

// one block of 256 threads per box: the two box sums (exact), C_n clamped, C_n in fixed point
__global__ void __launch_bounds__(256) k_cc_cbar(const ConstraintArgs c) {
  __shared__ long long s1[256], s2[256];
  const int n = blockIdx.x;
  const int2 pn = c.pos[n];
  const int M = c.M;
  const int lg = __ffs(M) - 1;  // M is a power of two
  long long a = 0, b = 0;
  for (int p = threadIdx.x; p < M * M; p += 256) {
    const size_t q = (size_t)(pn.x + (p >> lg)) * c.obj_w + pn.y + (p & (M - 1));
    a += c.map_lna[q];
    b += c.map_phi[q];
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] += s2[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double sl = (double)s1[0] / kFix;
    const double sp = (double)s2[0] / kFix;
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
  // prefix sums along the rows (one thread per row), then along the columns (one per column)
  if (lt < T) {
    long long sq = 0;
    int sn = 0;
    for (int x = 0; x < T; ++x) {
      sq += dq[lt * T1 + x];
      sn += dn[lt * T1 + x];
      dq[lt * T1 + x] = sq;
      dn[lt * T1 + x] = sn;
    }
  }
  __syncthreads();
  if (lt < T) {
    long long sq = 0;
    int sn = 0;
    for (int y = 0; y < T; ++y) {
      sq += dq[y * T1 + lt];
      sn += dn[y * T1 + lt];
      dq[y * T1 + lt] = sq;
      dn[y * T1 + lt] = sn;
    }
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
  const size_t n = (size_t)c.obj_h * c.obj_w;
  const int nb = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_cc_maps<<<nb, 256, 0, s>>>(c);
  k_cc_cbar<<<c.N, 256, 0, s>>>(c);
  k_cc_apply<<<dim3(c.tiles_x, c.tiles_y), dim3(32, 8), 0, s>>>(c);
  return cudaGetLastError();
}

}  // namespace ptycho
