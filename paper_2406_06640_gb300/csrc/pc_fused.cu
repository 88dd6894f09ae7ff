// Fused per-position pc-engine kernel in its cluster form, used by the work-queue launches of
// batch plans and by mini-batches too small to fill the GPU with one CTA per position (the
// single-problem launch runs the one-CTA-per-position kernel of pc_fused_seq.cu):
// one cluster of K CTAs per scan position,
// CTA rank k owns probe mode k and rows [k R, (k + 1) R) of the detector
// (R = ceil(M / K)). Everything between the object gather and the per-position
// contributions stays on chip:
//
//   psi_k   = P_k o_n                                       (Eq. 1, Fig. 1)
//   Psi_k   = centred FFT2 (far field, checkerboard trick)  (Eq. 1)
//           | IFFT2(FFT2(psi_k) H)  (near field, Fresnel transfer function)
//   |Psi_k|^2 is pushed (DSMEM stores) to the rank owning its row; the owner
//   sums the K modes in rank order:  S = sum_k |Psi_k|^2
//   A^G     = sqrt(S) (x) g  (Eq. 6)  or  I_m = S (x) g (Eq. 2), separable and
//             zero padded, g of Eq. 7 normalised; each owner blurs its own
//             rows and receives the x-blurred halo rows it needs from the others
//   R       = sqrt(I_n) / (A^G + eps)   or   sqrt(I_n) / sqrt(I_m + eps^2)
//             (sqrt(I_n) precomputed once per plan; fast 2-ulp divide / rsqrt),
//             pushed by its owner to every rank
//   Psi'_k  = R Psi_k;  psi'_k = inverse propagation;  dpsi_k = psi'_k - psi_k
//   c_n     = sum_k conj(P_k) dpsi_k: pushed to the row owner, summed in rank
//             order, written once per position (the object update gathers it)
//   pacc    += conj(o_n) dpsi_k, dacc += |o_n|^2  (per-slot partials, no atomics)
//   error   : compensated FP32 per thread of sum (Ihat - I_n)^2 over own rows,
//             FP64 across threads, ranks and slots
//
// Persistent: cluster `slot` handles positions slot, slot + slots, ... so the
// per-slot partials are written in a fixed order and the iteration is
// bitwise reproducible. Five cluster barriers per position order the pushes.
#include <cuda_runtime.h>

#include "pc_fused_kernel.cuh"

namespace ptycho {

// Self-test of the bounded wait above (the one the cluster kernels use on their copy barriers):
// one thread waits for phase 0 of a fresh mbarrier with the given budget. With `signal` it arrives
// first and the wait succeeds at once; otherwise nothing ever arrives, the wait gives up after
// `budget_ns` and sets the flag fused_timed_out reads, exactly as a fused kernel does.
__global__ void k_wait_selftest(unsigned long long budget_ns, int signal) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  const uint32_t b = smem_addr(&bar);
  mbar_init(b, 1);
  if (signal) mbar_arrive_expect_tx(b, 0u);  // the one expected arrival, no transaction bytes
  if (!mbar_wait_bounded(b, 0u, budget_ns)) atomicExch(&g_fused_timeout, 1);
}

cudaError_t launch_wait_selftest(unsigned long long budget_ns, bool signal, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(budget_ns, signal ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t fused_timed_out(bool* out) {
  int h = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&h, g_fused_timeout, sizeof(int));
  if (e != cudaSuccess) return e;
  if (h) {
    const int z = 0;
    e = cudaMemcpyToSymbol(g_fused_timeout, &z, sizeof(int));
    if (e != cudaSuccess) return e;
  }
  bool dm = false;
  e = fused_dm_timed_out(&dm);  // the pc-DM instantiations keep their own flag
  *out = h != 0 || dm;
  return e;
}

size_t fused_smem_bytes(int M) {
  switch (M) {
    case 8: return FusedSmem<8, 15>::BYTES;
    case 16: return FusedSmem<16, 15>::BYTES;
    case 32: return FusedSmem<32, 15>::BYTES;
    case 64: return FusedSmem<64, 15>::BYTES;
    case 128: return FusedSmem<128, 15>::BYTES;
    default: return 0;
  }
}

template <int M, int KH, bool QUEUED = false>
static cudaLaunchConfig_t fused_config(const FusedArgs& a, int slots, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(slots * a.K));
  cfg.blockDim = dim3(FusedShape<M>::TR);
  cfg.dynamicSmemBytes = FusedSmem<M, KH>::BYTES + (QUEUED ? FusedSmem<M, KH>::DESC : 0);
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.K;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <int M, bool NEAR, int KH, bool QUEUED = false>
static cudaError_t launch_kh(const FusedArgs& a, int slots, cudaStream_t s) {
  auto kern = pc_fused_kernel<M, NEAR, KH, QUEUED>;
  const size_t bytes = FusedSmem<M, KH>::BYTES + (QUEUED ? FusedSmem<M, KH>::DESC : 0);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = fused_config<M, KH, QUEUED>(a, slots, s, attr);
  return cudaLaunchKernelEx(&cfg, kern, a);
}

// ---- single-problem launches of the cluster form: the mini-batch engine takes them for batches
// with fewer positions than the one-CTA form has slots (K CTAs per position then fill more SMs)
template <int M, bool NEAR>
static cudaError_t launch_cluster_t(const FusedArgs& a, int slots, cudaStream_t s) {
  return a.kh == 5 ? launch_kh<M, NEAR, 5>(a, slots, s) : launch_kh<M, NEAR, 15>(a, slots, s);
}

cudaError_t launch_fused_cluster(int M, const FusedArgs& a, int slots, cudaStream_t s) {
  const bool nf = a.near_field != 0;
  switch (M) {
    case 8: return nf ? launch_cluster_t<8, true>(a, slots, s) : launch_cluster_t<8, false>(a, slots, s);
    case 16: return nf ? launch_cluster_t<16, true>(a, slots, s) : launch_cluster_t<16, false>(a, slots, s);
    case 32: return nf ? launch_cluster_t<32, true>(a, slots, s) : launch_cluster_t<32, false>(a, slots, s);
    case 64: return nf ? launch_cluster_t<64, true>(a, slots, s) : launch_cluster_t<64, false>(a, slots, s);
    case 128: return nf ? launch_cluster_t<128, true>(a, slots, s) : launch_cluster_t<128, false>(a, slots, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int M>
static cudaError_t cluster_slots_t(int K, int* slots) {
  auto kern = pc_fused_kernel<M, false, 15, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FusedSmem<M, 15>::BYTES);
  if (e != cudaSuccess) return e;
  FusedArgs a = {};
  a.K = K;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = fused_config<M, 15>(a, 1, 0, attr);
  int n = 0;
  e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
  *slots = n;
  return e;
}

cudaError_t fused_cluster_max_slots(int M, int K, int* slots) {
  switch (M) {
    case 8: return cluster_slots_t<8>(K, slots);
    case 16: return cluster_slots_t<16>(K, slots);
    case 32: return cluster_slots_t<32>(K, slots);
    case 64: return cluster_slots_t<64>(K, slots);
    case 128: return cluster_slots_t<128>(K, slots);
    default: return cudaErrorInvalidValue;
  }
}

// ---- work-queue launches (batches of problems sharing M, K, geometry and kernel width class)
template <int M, bool NEAR>
static cudaError_t launch_queue_t(const FusedArgs& a, int slots, cudaStream_t s) {
  return a.kh == 5 ? launch_kh<M, NEAR, 5, true>(a, slots, s) : launch_kh<M, NEAR, 15, true>(a, slots, s);
}

bool fused_queue_supported(int M) { return M == 8 || M == 16 || M == 32 || M == 64 || M == 128; }

cudaError_t launch_fused_queue(int M, const FusedArgs& a, int slots, cudaStream_t s) {
  if (!a.probs || !a.chunks || !a.queue || a.nchunks < 0) return cudaErrorInvalidValue;
  const bool nf = a.near_field != 0;
  switch (M) {
    case 8: return nf ? launch_queue_t<8, true>(a, slots, s) : launch_queue_t<8, false>(a, slots, s);
    case 16: return nf ? launch_queue_t<16, true>(a, slots, s) : launch_queue_t<16, false>(a, slots, s);
    case 32: return nf ? launch_queue_t<32, true>(a, slots, s) : launch_queue_t<32, false>(a, slots, s);
    case 64: return nf ? launch_queue_t<64, true>(a, slots, s) : launch_queue_t<64, false>(a, slots, s);
    case 128: return nf ? launch_queue_t<128, true>(a, slots, s) : launch_queue_t<128, false>(a, slots, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int M>
static cudaError_t queue_slots_t(int K, int* slots) {
  auto kern = pc_fused_kernel<M, false, 15, true>;
  const size_t bytes = FusedSmem<M, 15>::BYTES + FusedSmem<M, 15>::DESC;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  FusedArgs a = {};
  a.K = K;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = fused_config<M, 15, true>(a, 1, 0, attr);
  int n = 0;
  e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
  *slots = n;
  return e;
}

cudaError_t fused_queue_max_slots(int M, int K, int* slots) {
  switch (M) {
    case 8: return queue_slots_t<8>(K, slots);
    case 16: return queue_slots_t<16>(K, slots);
    case 32: return queue_slots_t<32>(K, slots);
    case 64: return queue_slots_t<64>(K, slots);
    case 128: return queue_slots_t<128>(K, slots);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ptycho
