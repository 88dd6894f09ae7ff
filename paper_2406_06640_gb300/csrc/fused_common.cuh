// Device helpers shared by the fused per-position kernels (pc_fused_kernel.cuh: a cluster of K CTAs
// per position; pc_fused_seq.cuh: one CTA per position, modes in sequence): mbarrier and bulk-copy
// wrappers, tensor memory (TMEM) used as per-thread storage, the detector coordinates of the FFT
// register layouts and the zero-padded separable blur of Eqs. 6-7.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"
#include "fft.cuh"

namespace ptycho {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// global -> own shared memory, `bytes` a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// ---- tensor memory (TMEM) used as per-thread storage: each thread owns a
// column range in the 32-lane quarter of its warp (warp w accesses lanes
// 32 (w % 4) .. 32 (w % 4) + 31; address = lane << 16 | column)
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// 16 consecutive 32-bit columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15},"
      " [%16];"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]),
        "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7])
               : "r"(taddr)
               : "memory");
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&r)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]), "f"(r[6]), "f"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14,"
      " %15, %16};" ::"r"(taddr),
      "f"(r[0]), "f"(r[1]), "f"(r[2]), "f"(r[3]), "f"(r[4]), "f"(r[5]), "f"(r[6]), "f"(r[7]), "f"(r[8]),
      "f"(r[9]), "f"(r[10]), "f"(r[11]), "f"(r[12]), "f"(r[13]), "f"(r[14]), "f"(r[15])
      : "memory");
}

// detector (row, col) of register r: the near field ends the propagation in
// the ROW layout (line, t) = (vt / G, vt % G), the far field in the COLUMN
// layout (c, t) = (vt / G, vt % G) holding frequencies (u, c)
template <int M, bool NEAR>
__device__ __forceinline__ void det_coords(int vt, int r, int& row, int& col) {
  if constexpr (NEAR) {
    row = vt / Tile<M>::G;
    col = vt % Tile<M>::G + Tile<M>::G * r;
  } else {
    row = col_freq<M>(vt % Tile<M>::G, r);
    col = vt / Tile<M>::G;
  }
}

// NO consecutive outputs of a zero-padded correlation along a line of a f32
// buffer: out[o] = sum_d g[d] in[c0 + o + d - KH], samples outside [lo, hi)
// read as zero; `stride` steps between consecutive samples.
template <int NO, int KH>
__device__ __forceinline__ void blur_strip(const float* in, int base, int stride, int c0, int lo, int hi,
                                           const float* g, float (&out)[NO]) {
  constexpr int E = NO;
  constexpr int W = E + 2 * KH;
  float win[W];
#pragma unroll
  for (int i = 0; i < W; ++i) {
    const int c = c0 - KH + i;
    win[i] = (c >= lo && c < hi) ? in[base + c * stride] : 0.f;
  }
  if constexpr (KH <= 7) {
    float gr[2 * KH + 1];
#pragma unroll
    for (int d = 0; d < 2 * KH + 1; ++d) gr[d] = g[d];
#pragma unroll
    for (int o = 0; o < E; ++o) {
      float acc = 0.f;
#pragma unroll
      for (int d = 0; d < 2 * KH + 1; ++d) acc = fmaf(gr[d], win[o + d], acc);
      out[o] = acc;
    }
  } else {
#pragma unroll
    for (int o = 0; o < E; ++o) out[o] = 0.f;
#pragma unroll
    for (int d = 0; d < 2 * KH + 1; ++d) {
      const float gd = g[d];
#pragma unroll
      for (int o = 0; o < E; ++o) out[o] = fmaf(gd, win[o + d], out[o]);
    }
  }
}

template <int X>
struct IntC {
  static constexpr int value = X;
};

}  // namespace ptycho
