// Fused per-position pc-engine kernel: one cluster of K CTAs per scan position,
// CTA rank k owns probe mode k. Everything between the object gather and the
// scatter contributions stays on chip:
//
//   psi_k   = P_k o_n                                       (Eq. 1, Fig. 1)
//   Psi_k   = centred FFT2 (far field, checkerboard trick)  (Eq. 1)
//           | IFFT2(FFT2(psi_k) H)  (near field, Fresnel transfer function)
//   S       = sum_k |Psi_k|^2   -- summed across the cluster through DSMEM
//   A^G     = sqrt(S) (x) g  (Eq. 6)  or  I_m = S (x) g (Eq. 2), separable,
//             zero padded, g of Eq. 7 normalised
//   R       = sqrt(I_n) / (A^G + eps)   or   sqrt(I_n) / sqrt(I_m + eps^2)
//   Psi'_k  = R Psi_k;  psi'_k = inverse propagation;  dpsi_k = psi'_k - psi_k
//   c_n     = sum_k conj(P_k) dpsi_k -- summed across the cluster through DSMEM,
//             written once per position (the object update gathers it per tile)
//   pacc    += conj(o_n) dpsi_k, dacc += |o_n|^2  (per-slot partials, no atomics)
//   errpart += sum (Ihat - I_n)^2 in FP64  (rank 0)
//
// Persistent: cluster `slot` handles positions slot, slot + slots, ... so the
// per-slot partials are written in a fixed order and the iteration is
// bitwise reproducible.
#include <cuda_runtime.h>

#include "engine.h"
#include "fft.cuh"

namespace ptycho {

__device__ __forceinline__ unsigned cluster_ctarank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t map_rank(uint32_t addr, unsigned rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ float ld_cluster_f32(uint32_t addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ float2 ld_cluster_f2(uint32_t addr) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}

template <int M>
struct FusedSmem {
  static constexpr int LD = M + 1;  // padded row stride of the f32 detector buffers
  static constexpr size_t kC = (size_t)M * M * 8 > (size_t)2 * M * LD * 4 ? (size_t)M * M * 8 : (size_t)2 * M * LD * 4;
  static constexpr size_t CBUF = (kC + 15) / 16 * 16;
  static constexpr size_t IBUF = ((size_t)M * LD * 4 + 15) / 16 * 16;
  static constexpr size_t TW = (size_t)M * 8;
  static constexpr size_t TAPS = 2 * kMaxTaps * 4 + 8;
  static constexpr size_t BYTES = CBUF + IBUF + 2 * TW + TAPS;
};

// detector (row, col) of register r
template <int M, bool NEAR>
__device__ __forceinline__ void det_coords(int line, int t, int r, int& row, int& col) {
  if constexpr (NEAR) {
    row = line;
    col = t + Tile<M>::G * r;
  } else {
    row = col_freq<M>(t, r);
    col = line;
  }
}

template <int M, bool NEAR>
__global__ void __launch_bounds__(Tile<M>::T, 1) pc_fused_kernel(const FusedArgs a) {
  using TL = Tile<M>;
  using SM = FusedSmem<M>;
  constexpr int E = TL::E, G = TL::G, T = TL::T, LD = SM::LD;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* cbuf = reinterpret_cast<float2*>(smem);
  float* fA = reinterpret_cast<float*>(smem);
  float* fB = fA + M * LD;
  float* ibuf = reinterpret_cast<float*>(smem + SM::CBUF);
  float2* s_tw = reinterpret_cast<float2*>(smem + SM::CBUF + SM::IBUF);
  float2* s_h = s_tw + M;
  float* s_gx = reinterpret_cast<float*>(s_h + M);
  float* s_gy = s_gx + kMaxTaps;

  const int tid = threadIdx.x;
  const int K = a.K;
  const unsigned rank = cluster_ctarank();
  const int slot = blockIdx.x / K;
  const int nslots = gridDim.x / K;
  const int kh = a.kh;

  for (int i = tid; i < M; i += T) {
    s_tw[i] = a.tw[i];
    if constexpr (NEAR) s_h[i] = a.hq[i];
  }
  for (int i = tid; i < 2 * kh + 1; i += T) {
    s_gx[i] = a.gx[i];
    s_gy[i] = a.gy[i];
  }
  __syncthreads();

  const int line = tid / G, t = tid % G;
  const float2* Pk = a.P + (size_t)rank * M * M;
  float2* pacc = a.pacc + ((size_t)slot * K + rank) * M * M;
  float* dacc = a.dacc + (size_t)slot * M * M;
  const int r0 = (int)rank * M / K, r1 = ((int)rank + 1) * M / K;
  const float inv_m2 = 1.0f / (float)(M * M);
  const uint32_t ibuf_s = smem_addr(ibuf), cbuf_s = smem_addr(cbuf);
  const float eps = a.eps;
  double err = 0.0;

  for (int n = slot; n < a.N; n += nslots) {
    const bool first = (n == slot);
    const int2 pn = a.pos[n];
    const float2* On = a.O + (size_t)pn.x * a.obj_w + pn.y;
    float2 v[E];
    // ---- exit wave in ROW layout
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int x = t + G * j;
      float2 psi = cmul(Pk[line * M + x], On[(size_t)line * a.obj_w + x]);
      if (!NEAR && ((line + x) & 1)) psi = make_float2(-psi.x, -psi.y);
      v[j] = psi;
    }
    // ---- forward propagation
    fft2_forward<M>(v, cbuf, s_tw, tid);  // COL layout
    if constexpr (NEAR) {
#pragma unroll
      for (int r = 0; r < E; ++r) v[r] = cmul(v[r], cmul(s_h[col_freq<M>(t, r)], s_h[line]));
      fft2_inverse<M>(v, cbuf, s_tw, tid);  // ROW layout, times M^2
#pragma unroll
      for (int j = 0; j < E; ++j) v[j] = cscale(v[j], inv_m2);
    }
    // ---- |Psi_k|^2 of this mode, then the cluster-wide mode sum
#pragma unroll
    for (int r = 0; r < E; ++r) {
      int row, col;
      det_coords<M, NEAR>(line, t, r, row, col);
      ibuf[row * LD + col] = cabs2(v[r]);
    }
    cluster_sync_all();
#pragma unroll 4
    for (int i = 0; i < E; ++i) {
      const int p = tid + T * i;
      const int row = p / M, col = p % M;
      const uint32_t off = (uint32_t)(row * LD + col) * 4u;
      float s = 0.f;
      for (int q = 0; q < K; ++q) s += ld_cluster_f32(map_rank(ibuf_s + off, (unsigned)q));
      fA[row * LD + col] = a.blur_intensity ? s : sqrtf(s);
    }
    __syncthreads();
    // ---- separable blur, x (columns, sigma_1): thread (row, column strip)
    {
      const int row = tid % M, c0 = (tid / M) * E;
      for (int c = c0; c < c0 + E; ++c) {
        float acc = 0.f;
        for (int d = -kh; d <= kh; ++d) {
          const int cc = c + d;
          if (cc >= 0 && cc < M) acc = fmaf(s_gx[d + kh], fA[row * LD + cc], acc);
        }
        fB[row * LD + c] = acc;
      }
    }
    __syncthreads();
    // ---- blur y (rows, sigma_2), modulus ratio and FP64 error: thread (column, row strip)
    {
      const int col = tid % M, rs = (tid / M) * E;
      const float* In = a.I + (size_t)n * M * M;
      for (int row = rs; row < rs + E; ++row) {
        float acc = 0.f;
        for (int d = -kh; d <= kh; ++d) {
          const int rr = row + d;
          if (rr >= 0 && rr < M) acc = fmaf(s_gy[d + kh], fB[rr * LD + col], acc);
        }
        const float Im = In[row * M + col];
        float ihat, R;
        if (a.blur_intensity) {
          ihat = acc;
          R = sqrtf(Im) / sqrtf(acc + eps * eps);
        } else {
          ihat = acc * acc;
          R = sqrtf(Im) / (acc + eps);
        }
        if (rank == 0) {
          const double d = (double)ihat - (double)Im;
          err += d * d;
        }
        fA[row * LD + col] = R;
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < E; ++r) {
      int row, col;
      det_coords<M, NEAR>(line, t, r, row, col);
      v[r] = cscale(v[r], fA[row * LD + col]);
    }
    __syncthreads();  // fA overlaps cbuf
    // ---- back-propagation to ROW layout
    if constexpr (NEAR) {
      fft2_forward<M>(v, cbuf, s_tw, tid);
#pragma unroll
      for (int r = 0; r < E; ++r) v[r] = cmulc(v[r], cmul(s_h[col_freq<M>(t, r)], s_h[line]));
    }
    fft2_inverse<M>(v, cbuf, s_tw, tid);
    // ---- dpsi, contributions
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int x = t + G * j;
      float2 psi_new = cscale(v[j], inv_m2);
      if (!NEAR && ((line + x) & 1)) psi_new = make_float2(-psi_new.x, -psi_new.y);
      const float2 p = Pk[line * M + x];
      const float2 o = On[(size_t)line * a.obj_w + x];
      const float2 dpsi = csub(psi_new, cmul(p, o));
      cbuf[TL::idxN(line, x)] = cconjmul(p, dpsi);
      const int q = line * M + x;
      const float2 pc = cconjmul(o, dpsi);
      pacc[q] = first ? pc : cadd(pacc[q], pc);
      if (line >= r0 && line < r1) dacc[q] = first ? cabs2(o) : dacc[q] + cabs2(o);
    }
    cluster_sync_all();
    {
      float2* cn = a.cn + (size_t)n * M * M;
      for (int p = r0 * M + tid; p < r1 * M; p += T) {
        const int row = p / M, col = p % M;
        const uint32_t off = (uint32_t)TL::idxN(row, col) * 8u;
        float2 s = make_float2(0.f, 0.f);
        for (int q = 0; q < K; ++q) s = cadd(s, ld_cluster_f2(map_rank(cbuf_s + off, (unsigned)q)));
        cn[p] = s;
      }
    }
    cluster_sync_all();
  }
  // ---- per-slot FP64 error numerator, summed in thread order
  if (rank == 0) {
    double* red = reinterpret_cast<double*>(smem);
    red[tid] = err;
    __syncthreads();
    for (int w = T / 2; w > 0; w >>= 1) {
      if (tid < w) red[tid] += red[tid + w];
      __syncthreads();
    }
    if (tid == 0) a.errpart[slot] = red[0];
  }
}

size_t fused_smem_bytes(int M) {
  switch (M) {
    case 8: return FusedSmem<8>::BYTES;
    case 16: return FusedSmem<16>::BYTES;
    case 32: return FusedSmem<32>::BYTES;
    case 64: return FusedSmem<64>::BYTES;
    case 128: return FusedSmem<128>::BYTES;
    default: return 0;
  }
}

template <int M, bool NEAR>
static cudaLaunchConfig_t fused_config(const FusedArgs& a, int slots, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(slots * a.K));
  cfg.blockDim = dim3(Tile<M>::T);
  cfg.dynamicSmemBytes = FusedSmem<M>::BYTES;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.K;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <int M, bool NEAR>
static cudaError_t launch_t(const FusedArgs& a, int slots, cudaStream_t s) {
  auto kern = pc_fused_kernel<M, NEAR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FusedSmem<M>::BYTES);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = fused_config<M, NEAR>(a, slots, s, attr);
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int M>
static cudaError_t max_slots_t(int K, int* slots) {
  auto kern = pc_fused_kernel<M, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FusedSmem<M>::BYTES);
  if (e != cudaSuccess) return e;
  FusedArgs a = {};
  a.K = K;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = fused_config<M, false>(a, 1, 0, attr);
  int n = 0;
  e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
  *slots = n;
  return e;
}

cudaError_t launch_fused(int M, const FusedArgs& a, int slots, cudaStream_t s) {
  const bool nf = a.near_field != 0;
  switch (M) {
    case 8: return nf ? launch_t<8, true>(a, slots, s) : launch_t<8, false>(a, slots, s);
    case 16: return nf ? launch_t<16, true>(a, slots, s) : launch_t<16, false>(a, slots, s);
    case 32: return nf ? launch_t<32, true>(a, slots, s) : launch_t<32, false>(a, slots, s);
    case 64: return nf ? launch_t<64, true>(a, slots, s) : launch_t<64, false>(a, slots, s);
    case 128: return nf ? launch_t<128, true>(a, slots, s) : launch_t<128, false>(a, slots, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t fused_max_slots(int M, int K, int* slots) {
  switch (M) {
    case 8: return max_slots_t<8>(K, slots);
    case 16: return max_slots_t<16>(K, slots);
    case 32: return max_slots_t<32>(K, slots);
    case 64: return max_slots_t<64>(K, slots);
    case 128: return max_slots_t<128>(K, slots);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ptycho
