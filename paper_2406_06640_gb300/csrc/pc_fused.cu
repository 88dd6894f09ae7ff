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
//             (sqrt(I_n) precomputed once per plan; fast 2-ulp divide / rsqrt)
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
  static constexpr size_t kX = (size_t)Tile<M>::SMEM * 8;  // FFT exchange buffer
  static constexpr size_t kF = (size_t)2 * M * LD * 4;     // two f32 detector buffers (aliases the exchange buffer)
  static constexpr size_t CBUF = ((kX > kF ? kX : kF) + 15) / 16 * 16;
  static constexpr size_t IBUF = ((size_t)M * LD * 4 + 15) / 16 * 16;
  static constexpr size_t TWT = ((size_t)Tile<M>::G * Tile<M>::LDW * 8 + 15) / 16 * 16;  // twiddle table
  static constexpr size_t HQ = (size_t)M * 8;                                             // Fresnel factors
  static constexpr size_t TAPS = 2 * kMaxTaps * 4 + 8;
  static constexpr size_t BYTES = CBUF + IBUF + TWT + HQ + TAPS;
  static_assert(BYTES <= 232448, "shared memory budget of one CTA");
};

// lines per thread: the 128 x 128 tile runs on 512 threads with two lines each
// (128 registers per thread instead of 64 at 1024 threads)
template <int M>
struct FusedShape {
  static constexpr int V = M == 128 ? 2 : 1;
  static constexpr int TR = Tile<M>::T / V;
};

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

// E consecutive outputs of a zero-padded correlation along a line of the
// padded f32 buffer: out[o] = sum_d g[d] in[c0 + o + d - KH]; `stride` steps
// between consecutive samples (1 along a row, LD along a column).
template <int M, int KH>
__device__ __forceinline__ void blur_strip(const float* in, int base, int stride, int c0, const float* g,
                                           float (&out)[Tile<M>::E]) {
  constexpr int E = Tile<M>::E;
  constexpr int W = E + 2 * KH;
  float win[W];
#pragma unroll
  for (int i = 0; i < W; ++i) {
    const int c = c0 - KH + i;
    win[i] = (c >= 0 && c < M) ? in[base + c * stride] : 0.f;
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

template <int M, bool NEAR, int KH>
__global__ void __launch_bounds__(FusedShape<M>::TR, 1) pc_fused_kernel(const FusedArgs a) {
  using TL = Tile<M>;
  using SM = FusedSmem<M>;
  constexpr int E = TL::E, G = TL::G, LD = SM::LD;
  constexpr int V = FusedShape<M>::V, TR = FusedShape<M>::TR;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* cbuf = reinterpret_cast<float2*>(smem);
  float* fA = reinterpret_cast<float*>(smem);
  float* fB = fA + M * LD;
  float* ibuf = reinterpret_cast<float*>(smem + SM::CBUF);
  float2* s_tw = reinterpret_cast<float2*>(smem + SM::CBUF + SM::IBUF);
  float2* s_h = reinterpret_cast<float2*>(smem + SM::CBUF + SM::IBUF + SM::TWT);
  float* s_gx = reinterpret_cast<float*>(smem + SM::CBUF + SM::IBUF + SM::TWT + SM::HQ);
  float* s_gy = s_gx + kMaxTaps;

  const int tid = threadIdx.x;
  const int K = a.K;
  const unsigned rank = cluster_ctarank();
  const int slot = blockIdx.x / K;
  const int nslots = gridDim.x / K;

  // twiddle table s_tw[t * (E + 1) + k2] = W_M^(t k2), t < G, from the host table W_M^m
  for (int i = tid; i < G * TL::LDW; i += TR) {
    const int t = i / TL::LDW, k2 = i % TL::LDW;
    s_tw[i] = k2 < E ? a.tw[(t * k2) % M] : make_float2(0.f, 0.f);
  }
  if constexpr (NEAR)
    for (int i = tid; i < M; i += TR) s_h[i] = a.hq[i];
  // taps centred at index KH; zero outside the requested kernel
  for (int i = tid; i < 2 * KH + 1; i += TR) {
    const int d = i - KH;
    const bool in = d >= -a.kh && d <= a.kh;
    s_gx[i] = in ? a.gx[d + a.kh] : 0.f;
    s_gy[i] = in ? a.gy[d + a.kh] : 0.f;
  }
  __syncthreads();

  int line[V], tp[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    line[v] = (tid + v * TR) / G;
    tp[v] = (tid + v * TR) % G;
  }
  const float2* Pk = a.P + (size_t)rank * M * M;
  float2* pacc = a.pacc + ((size_t)slot * K + rank) * M * M;
  float* dacc = a.dacc + (size_t)slot * M * M;
  const int r0 = (int)rank * M / K, r1 = ((int)rank + 1) * M / K;
  const float inv_m2 = 1.0f / (float)(M * M);
  const uint32_t ibuf_s = smem_addr(ibuf), cbuf_s = smem_addr(cbuf);
  const float eps = a.eps;
  float err_s = 0.f, err_c = 0.f;  // compensated per-thread sum of (Ihat - I)^2

  for (int n = slot; n < a.N; n += nslots) {
    const bool first = (n == slot);
    const int2 pn = a.pos[n];
    const float2* On = a.O + (size_t)pn.x * a.obj_w + pn.y;
    float2 v[V][E];
    // ---- exit wave in ROW layout
#pragma unroll
    for (int q = 0; q < V; ++q)
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int x = tp[q] + G * j;
        float2 psi = cmul(Pk[line[q] * M + x], On[(size_t)line[q] * a.obj_w + x]);
        if (!NEAR && ((line[q] + x) & 1)) psi = make_float2(-psi.x, -psi.y);
        v[q][j] = psi;
      }
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
    // ---- |Psi_k|^2 of this mode, then the cluster-wide mode sum
#pragma unroll
    for (int q = 0; q < V; ++q)
#pragma unroll
      for (int r = 0; r < E; ++r) {
        int row, col;
        det_coords<M, NEAR>(tid + q * TR, r, row, col);
        ibuf[row * LD + col] = cabs2(v[q][r]);
      }
    cluster_sync_all();
#pragma unroll 4
    for (int i = 0; i < V * E; ++i) {
      const int p = tid + TR * i;
      const int row = p / M, col = p % M;
      const uint32_t off = (uint32_t)(row * LD + col) * 4u;
      float s = 0.f;
      for (int q = 0; q < K; ++q) s += ld_cluster_f32(map_rank(ibuf_s + off, (unsigned)q));
      fA[row * LD + col] = a.blur_intensity ? s : sqrtf(s);
    }
    __syncthreads();
    // ---- separable blur, x (columns, sigma_1): virtual thread (row, column strip)
#pragma unroll
    for (int q = 0; q < V; ++q) {
      const int vt = tid + q * TR;
      const int row = vt % M, c0 = (vt / M) * E;
      float out[E];
      blur_strip<M, KH>(fA, row * LD, 1, c0, s_gx, out);
#pragma unroll
      for (int o = 0; o < E; ++o) fB[row * LD + c0 + o] = out[o];
    }
    __syncthreads();
    // ---- blur y (rows, sigma_2), modulus ratio and error: virtual thread (column, row strip)
    {
      const float* In = a.I + (size_t)n * M * M;
      const float* Sn = a.sqrtI + (size_t)n * M * M;
#pragma unroll
      for (int q = 0; q < V; ++q) {
        const int vt = tid + q * TR;
        const int col = vt % M, rs = (vt / M) * E;
        float out[E];
        blur_strip<M, KH>(fB, col, LD, rs, s_gy, out);
#pragma unroll
        for (int o = 0; o < E; ++o) {
          const int row = rs + o;
          const float acc = out[o];
          const float sq = Sn[row * M + col];
          float ihat, R;
          if (a.blur_intensity) {
            ihat = acc;
            R = sq * rsqrtf(acc + eps * eps);
          } else {
            ihat = acc * acc;
            R = __fdividef(sq, acc + eps);
          }
          if (rank == 0) {
            const float d = ihat - In[row * M + col];
            const float y = fmaf(d, d, -err_c);
            const float tt = err_s + y;
            err_c = (tt - err_s) - y;
            err_s = tt;
          }
          fA[row * LD + col] = R;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < V; ++q)
#pragma unroll
      for (int r = 0; r < E; ++r) {
        int row, col;
        det_coords<M, NEAR>(tid + q * TR, r, row, col);
        v[q][r] = cscale(v[q][r], fA[row * LD + col]);
      }
    __syncthreads();  // fA overlaps cbuf
    // ---- back-propagation to ROW layout
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
    // ---- dpsi, contributions
#pragma unroll
    for (int q = 0; q < V; ++q)
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int ln = line[q];
        const int x = tp[q] + G * j;
        float2 psi_new = cscale(v[q][j], inv_m2);
        if (!NEAR && ((ln + x) & 1)) psi_new = make_float2(-psi_new.x, -psi_new.y);
        const float2 p = Pk[ln * M + x];
        const float2 o = On[(size_t)ln * a.obj_w + x];
        const float2 dpsi = csub(psi_new, cmul(p, o));
        cbuf[TL::idxN(ln, x)] = cconjmul(p, dpsi);
        const int qi = ln * M + x;
        const float2 pc = cconjmul(o, dpsi);
        pacc[qi] = first ? pc : cadd(pacc[qi], pc);
        if (ln >= r0 && ln < r1) dacc[qi] = first ? cabs2(o) : dacc[qi] + cabs2(o);
      }
    cluster_sync_all();
    {
      float2* cn = a.cn + (size_t)n * M * M;
      for (int p = r0 * M + tid; p < r1 * M; p += TR) {
        const int row = p / M, col = p % M;
        const uint32_t off = (uint32_t)TL::idxN(row, col) * 8u;
        float2 s = make_float2(0.f, 0.f);
        for (int q = 0; q < K; ++q) s = cadd(s, ld_cluster_f2(map_rank(cbuf_s + off, (unsigned)q)));
        cn[p] = s;
      }
    }
    cluster_sync_all();
  }
  // ---- per-slot FP64 error numerator: the compensated FP32 thread sums, added in thread order
  if (rank == 0) {
    double* red = reinterpret_cast<double*>(smem);
    red[tid] = (double)err_s - (double)err_c;
    __syncthreads();
    for (int w = TR / 2; w > 0; w >>= 1) {
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

template <int M>
static cudaLaunchConfig_t fused_config(const FusedArgs& a, int slots, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(slots * a.K));
  cfg.blockDim = dim3(FusedShape<M>::TR);
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

template <int M, bool NEAR, int KH>
static cudaError_t launch_kh(const FusedArgs& a, int slots, cudaStream_t s) {
  auto kern = pc_fused_kernel<M, NEAR, KH>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FusedSmem<M>::BYTES);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = fused_config<M>(a, slots, s, attr);
  return cudaLaunchKernelEx(&cfg, kern, a);
}

// the paper's 11 x 11 kernel (Sec. 3.1) has its own instantiation; any other
// odd size up to 31 runs with the taps zero-padded to 31
template <int M, bool NEAR>
static cudaError_t launch_t(const FusedArgs& a, int slots, cudaStream_t s) {
  return a.kh == 5 ? launch_kh<M, NEAR, 5>(a, slots, s) : launch_kh<M, NEAR, 15>(a, slots, s);
}

template <int M>
static cudaError_t max_slots_t(int K, int* slots) {
  auto kern = pc_fused_kernel<M, false, 5>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FusedSmem<M>::BYTES);
  if (e != cudaSuccess) return e;
  FusedArgs a = {};
  a.K = K;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = fused_config<M>(a, 1, 0, attr);
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
