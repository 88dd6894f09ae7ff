// BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a) with FP32
// accumulation in tensor memory: the contraction under every 3x3 convolution
// of the warm-start network (forward, data gradient and weight gradient are
// all D = A B^T with K-contiguous operands).
//
//   D[M x N] (+)= A[M x K] . B[N x K]^T      A, B bf16 row-major (K contiguous)
//   M % 128 == 0, N % 16 == 0 and 16 <= N <= 256, K % 64 == 0
//   (optionally split along K over blockIdx.z into separate partial products)
//
// One CTA (128 threads) owns a 128 x N tile of D. K is walked in chunks of 64:
// the chunk of A (128 x 64) and of B (N x 64) is copied into shared memory in
// the no-swizzle K-major core-matrix layout (a core matrix = 8 rows x 16 bytes;
// core matrix (row group g, k group q) at byte (g * 8 + q) * 128, so the
// K-direction stride is 128 B and the row-group stride 1024 B); one thread
// issues four tcgen05.mma.kind::f16 (K = 16 each) into the TMEM accumulator and
// commits them to an mbarrier, which the CTA waits on before the next chunk
// overwrites shared memory. The epilogue reads TMEM (each warp its 32 lanes =
// 32 rows) and applies bias / ReLU / bf16 conversion as requested.
//
// Every mbarrier wait is bounded (wall-clock limit via %globaltimer): on
// timeout the kernel raises *status, waits once more (bounded), frees TMEM and
// returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"

namespace ptycho {

namespace {

constexpr int KC = 64;             // K chunk (elements)
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P1;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// bounded wait; returns false on timeout
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, phase))
    if (globaltimer() - t0 > kWaitNs) return false;
  return true;
}

// shared-memory matrix descriptor: start >> 4 in bits [0,14), leading-dimension
// byte offset >> 4 in [16,30), stride-dimension byte offset >> 4 in [32,46),
// the fixed value 0b001 in [46,49), no swizzle (bits [61,64) = 0)
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor for kind::f16: D f32 (bits [4,6) = 1), A and B bf16
// (bits [7,10) = 1, [10,13) = 1), both K-major, N >> 3 in [17,23), M >> 4 in [24,29)
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tm_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tm_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tm_ld16(uint32_t taddr, float (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15},"
      " [%16];"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]),
        "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// copy rows x 64 bf16 from a K-contiguous matrix into the core-matrix layout
__device__ __forceinline__ void stage(uint8_t* dst, const __nv_bfloat16* src, int rows, int ld, int k0) {
  for (int i = threadIdx.x; i < rows * 8; i += blockDim.x) {
    const int r = i >> 3, q = i & 7;
    const uint4 v = *reinterpret_cast<const uint4*>(src + (size_t)r * ld + k0 + q * 8);
    *reinterpret_cast<uint4*>(dst + (size_t)(((r >> 3) * 8 + q) * 128 + (r & 7) * 16)) = v;
  }
}

// implicit-GEMM operand: 128 rows (pixels m0 ..) x 64 columns of the 3x3
// neighbourhood matrix of an NHWC tensor, gathered 8 channels (16 bytes) at a time
__device__ __forceinline__ void stage_conv(uint8_t* dst, const __nv_bfloat16* X, int m0, int k0, int H, int W,
                                           int Cin) {
  for (int i = threadIdx.x; i < 128 * 8; i += blockDim.x) {
    const int r = i >> 3, q = i & 7;
    const int k = k0 + q * 8;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (k < 9 * Cin) {
      const int tap = k / Cin, c = k - tap * Cin;
      const int p = m0 + r;
      const int x = p % W, y = (p / W) % H, b = p / (W * H);
      const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
      if (yy >= 0 && yy < H && xx >= 0 && xx < W)
        v = *reinterpret_cast<const uint4*>(X + (((size_t)b * H + yy) * W + xx) * Cin + c);
    }
    *reinterpret_cast<uint4*>(dst + (size_t)(((r >> 3) * 8 + q) * 128 + (r & 7) * 16)) = v;
  }
}

}  // namespace

// epilogue modes: 0 = store fp32 D; 1 = accumulate into fp32 D (D += A B^T);
// 2 = bf16 out = act(D + bias[n]) with act = ReLU when `relu`
template <int N>
__global__ void __launch_bounds__(128, 1) k_gemm_bf16(const GemmArgs g) {
  constexpr uint32_t NCOLS = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint8_t* sA = smem;                  // 128 x 64 bf16 = 16 KB
  uint8_t* sB = smem + 128 * KC * 2;   // N x 64 bf16
  __shared__ uint64_t bar;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128;
  const int n0 = blockIdx.y * N;

  if (warp == 0) tm_alloc(&s_tmem, NCOLS);
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = make_idesc(128, N);
  const __nv_bfloat16* A = reinterpret_cast<const __nv_bfloat16*>(g.A) + (g.conv ? 0 : (size_t)m0 * g.K);
  const __nv_bfloat16* B = reinterpret_cast<const __nv_bfloat16*>(g.B) + (size_t)n0 * g.K;
  uint32_t phase = 0;
  bool ok = true;
  const int kbeg = g.ksplit > 1 ? (int)blockIdx.z * g.kc : 0;
  const int kend = g.ksplit > 1 ? min(g.K, kbeg + g.kc) : g.K;
  for (int k0 = kbeg; k0 < kend && ok; k0 += KC) {
    if (g.conv) stage_conv(sA, A, m0, k0, g.H, g.W, g.Cin);
    else stage(sA, A, 128, g.K, k0);
    stage(sB, B, N, g.K, k0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int s = 0; s < KC / 16; ++s) {
        const uint64_t ad = make_desc(smem_u32(sA) + s * 256, 128, 1024);
        const uint64_t bd = make_desc(smem_u32(sB) + s * 256, 128, 1024);
        mma_bf16(tmem, ad, bd, idesc, (k0 > kbeg || s > 0) ? 1u : 0u);
      }
      mma_commit(&bar);
    }
    ok = __syncthreads_and(mbar_wait_bounded(&bar, phase) ? 1 : 0) != 0;  // CTA-uniform outcome
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (!ok) {
    if (tid == 0) atomicExch(g.status, 1);
    mbar_wait_bounded(&bar, phase ^ 1u);  // give the MMAs in flight a bounded chance to finish
  } else {
    // epilogue: warp w owns rows 32 w .. 32 w + 31 (TMEM lanes), 16 columns per load
    const int row = m0 + warp * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 16) {
      float v[16];
      tm_ld16(tl + c0, v);
      if (g.mode == 2) {
        __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(g.Dh) + (size_t)row * g.ldd + n0 + c0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float x = v[j] + (g.bias ? g.bias[n0 + c0 + j] : 0.f);
          if (g.relu) x = fmaxf(x, 0.f);
          out[j] = __float2bfloat16(x);
        }
      } else {
        float* out = g.D + (g.ksplit > 1 ? (size_t)blockIdx.z * g.dsplit : 0) + (size_t)row * g.ldd + n0 + c0;
#pragma unroll
        for (int j = 0; j < 16; ++j) out[j] = g.mode == 1 ? out[j] + v[j] : v[j];
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) tm_dealloc(tmem, NCOLS);
}

template <int N>
static cudaError_t launch_n(const GemmArgs& g, cudaStream_t s) {
  const size_t smem = 128 * KC * 2 + (size_t)N * KC * 2;
  cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gemm_bf16<N><<<dim3(g.M / 128, g.Ntot / N, g.ksplit > 1 ? g.ksplit : 1), 128, smem, s>>>(g);
  return cudaGetLastError();
}

// N tile chosen from the output width: the widest of 256/128/64/32/16 dividing it
cudaError_t launch_gemm_bf16(const GemmArgs& g, cudaStream_t s) {
  if (g.M % 128 || g.K % KC || g.Ntot % 16 || g.M <= 0 || g.K <= 0 || g.Ntot <= 0) return cudaErrorInvalidValue;
  if (g.ksplit > 1 && (g.mode != 0 || g.kc % KC || g.kc <= 0 || (long long)(g.ksplit - 1) * g.kc >= g.K ||
                       (long long)g.ksplit * g.kc < g.K || g.ksplit > 65535))
    return cudaErrorInvalidValue;  // every split must own at least one chunk
  if (g.Ntot % 256 == 0) return launch_n<256>(g, s);
  if (g.Ntot % 128 == 0) return launch_n<128>(g, s);
  if (g.Ntot % 64 == 0) return launch_n<64>(g, s);
  if (g.Ntot % 32 == 0) return launch_n<32>(g, s);
  return launch_n<16>(g, s);
}

}  // namespace ptycho

// ---- C ABI: the tensor-core building block, exposed for callers and tests
namespace {
__device__ int g_gemm_status;
}

extern "C" int ptycho_gemm_bf16(const uint16_t* A, const uint16_t* B, float* D, int M, int N, int K, int accumulate,
                                void* stream) {
  using namespace ptycho;
  if (!A || !B || !D || M <= 0 || N <= 0 || K <= 0 || M % 128 || N % 16 || K % 64) return 1;  // PTYCHO_EINVAL
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* status = nullptr;
  if (cudaGetSymbolAddress((void**)&status, g_gemm_status) != cudaSuccess) return 3;
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return 3;
  GemmArgs g{};
  g.A = A;
  g.B = B;
  g.D = D;
  g.M = M;
  g.Ntot = N;
  g.K = K;
  g.ldd = N;
  g.mode = accumulate ? 1 : 0;
  g.status = status;
  if (launch_gemm_bf16(g, s) != cudaSuccess) return 3;
  int h = 0;
  if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return 3;
  if (cudaStreamSynchronize(s) != cudaSuccess) return 3;
  return h ? 6 : 0;  // PTYCHO_ETIMEOUT
}
