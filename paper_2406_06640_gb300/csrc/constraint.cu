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
//   (1) |ln a| and |phi| of every object pixel into two summed-area tables
//       (prefix sums along rows, then columns);
//   (2) per box, its two sums from four table entries each -> C_n; C_n is
//       added at the four corners of the box in a difference array (integer
//       atomics, order-independent);
//   (3) prefix sums of the difference array give sum_n C_n 1_box(r);
//   (4) divide by the coverage count (fixed per plan), apply Eqs. 9-10.
#include <cuda_runtime.h>
#include <math.h>

#include "engine.h"
#include "fft.cuh"

namespace ptycho {

constexpr double kFix = 4294967296.0;  // 2^32

// (obj_h + 1) x (obj_w + 1) tables, row 0 and column 0 zero: T[y + 1][x + 1] = value(y, x)
__global__ void __launch_bounds__(256) k_cc_maps(const ConstraintArgs c) {
  const size_t n = (size_t)c.obj_h * c.obj_w;
  const int W1 = c.obj_w + 1;
  for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (size_t)gridDim.x * 256) {
    const float2 o = c.O[i];
    const size_t q = (i / c.obj_w + 1) * (size_t)W1 + i % c.obj_w + 1;
    c.sat_lna[q] = llrint((double)fabsf(logf(fmaxf(sqrtf(cabs2(o)), 1e-6f))) * kFix);
    c.sat_phi[q] = llrint((double)fabsf(atan2f(o.y, o.x)) * kFix);
  }
}

// inclusive prefix sums of int64 lines: element i of line l sits at A[l * lstride + i * estride].
// Block (8, 128): threadIdx.x picks one of 8 lines, threadIdx.y one of 128 chunks
// of the line; chunk totals are combined in shared memory (exact integer sums).
// blockIdx.y selects the array (A0 or A1), so two tables scan in one launch.
constexpr int kScanLines = 8, kScanChunks = 128;
__global__ void __launch_bounds__(kScanLines * kScanChunks) k_scan_lines(long long* A0, long long* A1, int lines,
                                                                         int len, size_t lstride, size_t estride) {
  __shared__ long long tot[kScanChunks][kScanLines + 1];
  long long* A = blockIdx.y == 0 ? A0 : A1;
  const int l = blockIdx.x * kScanLines + threadIdx.x;
  const int chunk = (len + kScanChunks - 1) / kScanChunks;
  const int i0 = threadIdx.y * chunk, i1 = min(len, i0 + chunk);
  long long* p = A + (size_t)l * lstride;
  long long s = 0;
  if (l < lines)
    for (int i = i0; i < i1; ++i) s += p[(size_t)i * estride];
  tot[threadIdx.y][threadIdx.x] = s;
  __syncthreads();
  long long off = 0;
  for (int y = 0; y < (int)threadIdx.y; ++y) off += tot[y][threadIdx.x];
  if (l < lines)
    for (int i = i0; i < i1; ++i) {
      off += p[(size_t)i * estride];
      p[(size_t)i * estride] = off;
    }
}

// summed-area tables of one or two int64 rows x cols arrays (row-major): prefix along rows, then columns
static void sat_inplace(long long* A0, long long* A1, int rows, int cols, cudaStream_t s) {
  const dim3 b(kScanLines, kScanChunks);
  const unsigned na = A1 ? 2u : 1u;
  k_scan_lines<<<dim3((rows + kScanLines - 1) / kScanLines, na), b, 0, s>>>(A0, A1, rows, cols, (size_t)cols, 1);
  k_scan_lines<<<dim3((cols + kScanLines - 1) / kScanLines, na), b, 0, s>>>(A0, A1, cols, rows, 1, (size_t)cols);
}

__device__ __forceinline__ long long box_sum(const long long* T, int W1, int y0, int x0, int M) {
  return T[(size_t)(y0 + M) * W1 + x0 + M] - T[(size_t)y0 * W1 + x0 + M] - T[(size_t)(y0 + M) * W1 + x0] +
         T[(size_t)y0 * W1 + x0];
}

// one thread per position: C_n from the tables, corner updates of the difference array
__global__ void k_cc_cbar(const ConstraintArgs c) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= c.N) return;
  const int2 pn = c.pos[n];
  const int W1 = c.obj_w + 1;
  const double sl = (double)box_sum(c.sat_lna, W1, pn.x, pn.y, c.M) / kFix;
  const double sp = (double)box_sum(c.sat_phi, W1, pn.x, pn.y, c.M) / kFix;
  const double r = sl / fmax(sp, 1e-30);
  const float cb = (float)fmin(fmax(r, (double)c.cbar_min), (double)c.cbar_max);
  c.cbar[n] = cb;
  const unsigned long long qv = (unsigned long long)llrint((double)cb * kFix);
  unsigned long long* D = reinterpret_cast<unsigned long long*>(c.diff);
  const int M = c.M;
  atomicAdd(&D[(size_t)pn.x * W1 + pn.y], qv);
  atomicAdd(&D[(size_t)pn.x * W1 + pn.y + M], 0ull - qv);
  atomicAdd(&D[(size_t)(pn.x + M) * W1 + pn.y], 0ull - qv);
  atomicAdd(&D[(size_t)(pn.x + M) * W1 + pn.y + M], qv);
}

__global__ void __launch_bounds__(256) k_cc_apply(const ConstraintArgs c) {
  const size_t n = (size_t)c.obj_h * c.obj_w;
  const int W1 = c.obj_w + 1;
  for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (size_t)gridDim.x * 256) {
    const int cnt = c.cover[i];
    if (cnt == 0) continue;
    const int y = (int)(i / c.obj_w), x = (int)(i % c.obj_w);
    const long long s = c.diff[(size_t)y * W1 + x];
    const float C = (float)((double)s / kFix / (double)cnt);
    const float2 o = c.O[i];
    const float lna = logf(fmaxf(sqrtf(cabs2(o)), 1e-6f));
    const float phi = atan2f(o.y, o.x);
    const float ac = expf((1.f - c.alpha1) * lna + c.alpha1 * C * phi);
    const float pc = (1.f - c.alpha2) * phi + c.alpha2 * lna / C;
    float sn, cs;
    sincosf(pc, &sn, &cs);
    c.O[i] = make_float2(ac * cs, ac * sn);
  }
}

cudaError_t launch_constraint(const ConstraintArgs& c, cudaStream_t s) {
  const int H1 = c.obj_h + 1, W1 = c.obj_w + 1;
  const size_t tbytes = sizeof(long long) * (size_t)H1 * W1;
  const size_t n = (size_t)c.obj_h * c.obj_w;
  const int nb = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  cudaError_t e;
  if ((e = cudaMemsetAsync(c.sat_lna, 0, tbytes, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c.sat_phi, 0, tbytes, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(c.diff, 0, tbytes, s)) != cudaSuccess) return e;
  k_cc_maps<<<nb, 256, 0, s>>>(c);
  sat_inplace(c.sat_lna, c.sat_phi, H1, W1, s);
  k_cc_cbar<<<(c.N + 127) / 128, 128, 0, s>>>(c);
  sat_inplace(c.diff, nullptr, H1, W1, s);
  k_cc_apply<<<nb, 256, 0, s>>>(c);
  return cudaGetLastError();
}

}  // namespace ptycho
