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
#include <cuda_runtime.h>
#include <math.h>

#include "engine.h"
#include "fft.cuh"

namespace ptycho {

// one block per position: box sums in FP32, fixed-order tree
__global__ void __launch_bounds__(256) k_cc_cbar(const ConstraintArgs c) {
  const int n = blockIdx.x;
  const int2 pn = c.pos[n];
  const int M = c.M;
  __shared__ float sl[256], sp[256];
  float a_l = 0.f, a_p = 0.f;
  for (int p = threadIdx.x; p < M * M; p += 256) {
    const int y = p / M, x = p % M;
    const float2 o = c.O[(size_t)(pn.x + y) * c.obj_w + pn.y + x];
    const float amp = fmaxf(sqrtf(cabs2(o)), 1e-6f);
    a_l += fabsf(logf(amp));
    a_p += fabsf(atan2f(o.y, o.x));
  }
  sl[threadIdx.x] = a_l;
  sp[threadIdx.x] = a_p;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sl[threadIdx.x] += sl[threadIdx.x + w];
      sp[threadIdx.x] += sp[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float r = sl[0] / fmaxf(sp[0], 1e-30f);
    c.cbar[n] = fminf(fmaxf(r, c.cbar_min), c.cbar_max);
  }
}

// per object tile (same tiles and position lists as the object gather)
__global__ void __launch_bounds__(256) k_cc_apply(const ConstraintArgs c) {
  const int tile = blockIdx.y * c.tiles_x + blockIdx.x;
  const int X = blockIdx.x * kObjTile + threadIdx.x;
  const int Y0 = blockIdx.y * kObjTile + threadIdx.y;
  const int M = c.M;
  float sum[4] = {0.f, 0.f, 0.f, 0.f};
  int cnt[4] = {0, 0, 0, 0};
  const int s0 = c.tile_start[tile], s1 = c.tile_start[tile + 1];
  for (int idx = s0; idx < s1; ++idx) {
    const int n = c.tile_pos[idx];
    const int2 pn = c.pos[n];
    const int cx = X - pn.y;
    if (cx < 0 || cx >= M) continue;
    const float cb = c.cbar[n];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int cy = Y0 + 8 * i - pn.x;
      if (cy >= 0 && cy < M) {
        sum[i] += cb;
        cnt[i] += 1;
      }
    }
  }
  if (X >= c.obj_w) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int Y = Y0 + 8 * i;
    if (Y >= c.obj_h || cnt[i] == 0) continue;
    const float C = sum[i] / (float)cnt[i];
    const size_t q = (size_t)Y * c.obj_w + X;
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
  k_cc_cbar<<<c.N, 256, 0, s>>>(c);
  k_cc_apply<<<dim3(c.tiles_x, c.tiles_y), dim3(32, 8), 0, s>>>(c);
  return cudaGetLastError();
}

}  // namespace ptycho
