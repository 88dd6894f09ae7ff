// Line transforms of the staged passes (big.cu): a 256- or 512-point DFT held by the 16 threads of one
// line, in registers plus a warp-local swap through shared memory.
//   256 = 16 x 16: DFT-16 in registers over x = t + 16 j, twiddle W_256^(t k2), swap, DFT-16 over t:
//                  thread t holds frequencies t + 16 k1
//   512 = 32 x 16: DFT-32 over j, twiddle W_512^(t k2), swap, two DFT-16 over t:
//                  thread t holds frequencies 2t + i2 + 32 k1 in register 16 i2 + k1
// The inverse consumes the forward's layout and returns x = t + 16 j.
#pragma once
#include <cuda_runtime.h>

#include "fft.cuh"

namespace ptycho {

constexpr int BT = 16;   // threads per line
constexpr int BS = BT + 1;

// per line length: registers per thread (E), lines per CTA in the row passes (LROW) and columns per CTA
// in the column passes (LINES), the swap buffer of one line (SWN float2) and the twiddle table (TWN)
template <int BL>
struct BigShape;
template <>
struct BigShape<256> {
  static constexpr int E = 16, LROW = 16, LINES = 32, SWN = BT * BS, TWS = BS, TWN = BT * BS;
};
template <>
struct BigShape<512> {
  static constexpr int E = 32, LROW = 8, LINES = 16, SWN = 2 * BT * BS, TWS = 33, TWN = BT * 33;
};

// frequency held in register r by thread t after the forward line transform (the inverse expects it)
template <int BL>
__device__ __forceinline__ int line_freq(int t, int r) {
  if constexpr (BL == 256) return t + 16 * r;
  else return 2 * t + (r >> 4) + 32 * (r & 15);
}

// forward: thread t holds x[t + 16 j] in a[j]; returns X[line_freq(t, r)] in a[r] (unscaled). The inverse
// consumes that layout and returns x[t + 16 j] * BL in a[j].
//   256 = 16 x 16: DFT-16 over j, twiddle W_256^(t k2), swap, DFT-16 over t for k2 = t: X[t + 16 k1]
//   512 = 32 x 16: DFT-32 over j, twiddle W_512^(t k2), swap (k2 = 2 t' + i2 to thread t'), DFT-16 over t
//                  for k2 = 2t and 2t + 1: X[2t + i2 + 32 k1] in a[16 i2 + k1]
template <int BL, bool INV>
__device__ __forceinline__ void line_fft(float2 (&a)[BigShape<BL>::E], float2* sw, const float2* tw, int t) {
  constexpr int TWS = BigShape<BL>::TWS;
  if constexpr (BL == 256) {
    if constexpr (!INV) {
      dft<16, false>(a);  // a[k2] = Y[t][k2]
#pragma unroll
      for (int k2 = 1; k2 < 16; ++k2) a[k2] = cmul(a[k2], tw[t * TWS + k2]);
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) sw[k2 * BS + t] = a[k2];
      __syncwarp();
#pragma unroll
      for (int tt = 0; tt < 16; ++tt) a[tt] = sw[t * BS + tt];  // Y[tt][k2 = t]
      __syncwarp();
      dft<16, false>(a);  // a[k1] = X[t + 16 k1]
    } else {
      dft<16, true>(a);  // a[tt] = Y[tt][k2 = t]
#pragma unroll
      for (int tt = 0; tt < 16; ++tt) sw[t * BS + tt] = a[tt];
      __syncwarp();
#pragma unroll
      for (int k2 = 0; k2 < 16; ++k2) a[k2] = sw[k2 * BS + t];  // Y[t][k2]
      __syncwarp();
#pragma unroll
      for (int k2 = 1; k2 < 16; ++k2) a[k2] = cmulc(a[k2], tw[t * TWS + k2]);
      dft<16, true>(a);  // a[j] = x[t + 16 j] * 256
    }
  } else {
    // swap layout: Y[t][k2] at (k2 & 1) * 16 BS + (k2 >> 1) * BS + t (conflict-free both ways)
    if constexpr (!INV) {
      dft<32, false>(a);  // a[k2] = Y[t][k2], k2 < 32
#pragma unroll
      for (int k2 = 1; k2 < 32; ++k2) a[k2] = cmul(a[k2], tw[t * TWS + k2]);
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) sw[(k2 & 1) * 16 * BS + (k2 >> 1) * BS + t] = a[k2];
      __syncwarp();
#pragma unroll
      for (int i2 = 0; i2 < 2; ++i2)
#pragma unroll
        for (int tt = 0; tt < 16; ++tt) a[16 * i2 + tt] = sw[i2 * 16 * BS + t * BS + tt];  // Y[tt][2t + i2]
      __syncwarp();
      dft<16, false>(&a[0]);
      dft<16, false>(&a[16]);  // a[16 i2 + k1] = X[2t + i2 + 32 k1]
    } else {
      dft<16, true>(&a[0]);
      dft<16, true>(&a[16]);  // a[16 i2 + tt] = Z[tt][2t + i2]
#pragma unroll
      for (int i2 = 0; i2 < 2; ++i2)
#pragma unroll
        for (int tt = 0; tt < 16; ++tt) sw[i2 * 16 * BS + t * BS + tt] = a[16 * i2 + tt];
      __syncwarp();
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) a[k2] = sw[(k2 & 1) * 16 * BS + (k2 >> 1) * BS + t];  // Z[t][k2]
      __syncwarp();
#pragma unroll
      for (int k2 = 1; k2 < 32; ++k2) a[k2] = cmulc(a[k2], tw[t * TWS + k2]);
      dft<32, true>(a);  // a[j] = x[t + 16 j] * 512
    }
  }
}

}  // namespace ptycho
