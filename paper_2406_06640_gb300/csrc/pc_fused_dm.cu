// pc-DM launches of the fused kernel: the difference map of Thibault et al. with the pc intensity
// model in its modulus projection. Per position and mode, the kernel propagates the estimate P o_n
// through the FFT / blur path for the error E only, then the reflected wave chi = 2 P o_n - psi_n
// through the same path for the modulus ratio, and sets psi_n <- psi_n + Pi_F(chi) - P o_n (the
// exit-wave state lives in global memory). The overlap projection alternates: the object step of
// the single-problem path with dpsi = psi_n - P o_n, then (update.cu) the probe step from the new
// object and the state.
#include <cuda_runtime.h>

#include "pc_fused_kernel.cuh"

namespace ptycho {

template <int M, bool NEAR, int KH>
static cudaError_t launch_dm_kh(const FusedArgs& a, int slots, cudaStream_t s) {
  auto kern = pc_fused_kernel<M, NEAR, KH, false, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FusedSmem<M, KH>::BYTES);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(slots * a.K));
  cfg.blockDim = dim3(FusedShape<M>::TR);
  cfg.dynamicSmemBytes = FusedSmem<M, KH>::BYTES;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.K;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int M, bool NEAR>
static cudaError_t launch_dm_t(const FusedArgs& a, int slots, cudaStream_t s) {
  return a.kh == 5 ? launch_dm_kh<M, NEAR, 5>(a, slots, s) : launch_dm_kh<M, NEAR, 15>(a, slots, s);
}

cudaError_t launch_fused_dm(int M, const FusedArgs& a, int slots, cudaStream_t s) {
  if (!a.psi) return cudaErrorInvalidValue;
  const bool nf = a.near_field != 0;
  switch (M) {
    case 8: return nf ? launch_dm_t<8, true>(a, slots, s) : launch_dm_t<8, false>(a, slots, s);
    case 16: return nf ? launch_dm_t<16, true>(a, slots, s) : launch_dm_t<16, false>(a, slots, s);
    case 32: return nf ? launch_dm_t<32, true>(a, slots, s) : launch_dm_t<32, false>(a, slots, s);
    case 64: return nf ? launch_dm_t<64, true>(a, slots, s) : launch_dm_t<64, false>(a, slots, s);
    case 128: return nf ? launch_dm_t<128, true>(a, slots, s) : launch_dm_t<128, false>(a, slots, s);
    default: return cudaErrorInvalidValue;
  }
}

// co-resident clusters of K CTAs of the pc-DM kernel, taken for its largest shared-memory variant
template <int M>
static cudaError_t dm_slots_t(int K, int* slots) {
  auto kern = pc_fused_kernel<M, false, 15, false, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FusedSmem<M, 15>::BYTES);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)K);
  cfg.blockDim = dim3(FusedShape<M>::TR);
  cfg.dynamicSmemBytes = FusedSmem<M, 15>::BYTES;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)K;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
  *slots = n;
  return e;
}

cudaError_t fused_dm_max_slots(int M, int K, int* slots) {
  switch (M) {
    case 8: return dm_slots_t<8>(K, slots);
    case 16: return dm_slots_t<16>(K, slots);
    case 32: return dm_slots_t<32>(K, slots);
    case 64: return dm_slots_t<64>(K, slots);
    case 128: return dm_slots_t<128>(K, slots);
    default: return cudaErrorInvalidValue;
  }
}

// this translation unit's bounded-wait flag (read and cleared)
cudaError_t fused_dm_timed_out(bool* out) {
  int h = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&h, g_fused_timeout, sizeof(int));
  if (e != cudaSuccess) return e;
  *out = h != 0;
  if (h) {
    const int z = 0;
    e = cudaMemcpyToSymbol(g_fused_timeout, &z, sizeof(int));
  }
  return e;
}

}  // namespace ptycho
