// BF16 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a) with FP32
// accumulation in tensor memory: the contraction under every 3x3 convolution
// of the warm-start network (forward, data gradient and weight gradient are
// all D = A B^T with K-contiguous operands).
//
//   D[M x N] (+)= A[M x K] . B[N x K]^T      A, B bf16 row-major (K contiguous)
//   M % 128 == 0, N % 16 == 0 and 16 <= N <= 256, K % 64 == 0
//   (optionally split along K over blockIdx.z into separate partial products)
//
// One CTA (256 threads) owns a 128 x N tile of D. K is walked in chunks of 64,
// each copied by cp.async (16 bytes per copy) into one of S pipeline stages in
// the no-swizzle K-major core-matrix layout (a core matrix = 8 rows x 16 bytes;
// core matrix (row group g, k group q) at byte (g * 8 + q) * 128, so the
// K-direction stride is 128 B and the row-group stride 1024 B). One thread
// issues four tcgen05.mma.kind::f16 (K = 16 each) per chunk into the TMEM
// accumulator and commits them to that stage's mbarrier; the copies of the next
// S - 1 chunks are in flight meanwhile, and a stage is refilled only after its
// mbarrier reports the MMAs reading it done. The epilogue reads TMEM (each warp
// a 32-lane quarter and every other group of 16 columns) and applies bias /
// ReLU / bf16 conversion as requested.
//
// Every mbarrier wait is bounded (wall-clock limit via %globaltimer): on
// timeout the kernel raises *status, waits once more (bounded), frees TMEM and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
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

// arrive (release at CTA scope) on a barrier counting producer threads
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// shared-memory matrix descriptor of the 128-byte swizzled K-major layout: rows of 128 bytes (64 bf16),
// the 16-byte chunk c of the row at shared address r * 128 (from a 1024-byte aligned base) stored at chunk
// c ^ (r % 8), 8-row groups 1024 bytes apart (SBO); the leading offset is unused (16); layout type 2 in
// [61,64). The swizzle follows the absolute address bits, so a start moved by whole rows (a tap's shift)
// or by 32 bytes along K keeps the base offset field at 0 (checked on the device for shifts of 1, 5, 8,
// 13 and 100 rows)
__device__ __forceinline__ uint64_t make_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// the same for the 64-byte swizzled K-major layout: rows of 64 bytes (32 bf16), chunk c of row r at
// c ^ ((r >> 1) % 4), 8-row groups 512 bytes apart (SBO); layout type 4 in [61,64)
__device__ __forceinline__ uint64_t make_desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
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

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

constexpr int kThreads = 256;                       // 8 warps: copies shared by all, epilogue by column halves
constexpr int kRowsPerThread = 128 * 8 / kThreads;  // A rows each thread copies per chunk (fixed q)

// rows x 64 bf16 of a K-contiguous matrix into the core-matrix layout, 16 bytes per async copy
__device__ __forceinline__ void stage(uint32_t dst, const __nv_bfloat16* src, int rows, int ld, int k0) {
  for (int i = threadIdx.x; i < rows * 8; i += blockDim.x) {
    const int r = i >> 3, q = i & 7;
    cp_async16(dst + (uint32_t)(((r >> 3) * 8 + q) * 128 + (r & 7) * 16), src + (size_t)r * ld + k0 + q * 8, 16u);
  }
}

// pixel coordinates of the A rows this thread copies: row r_t = (tid >> 3) + 32 t
struct ConvRows {
  int off[kRowsPerThread];  // ((b H + y) W + x) Cin
  int y[kRowsPerThread], x[kRowsPerThread];
};
__device__ __forceinline__ ConvRows conv_rows(int m0, int H, int W, int Cin) {
  ConvRows c;
#pragma unroll
  for (int t = 0; t < kRowsPerThread; ++t) {
    const int p = m0 + (threadIdx.x >> 3) + (kThreads / 8) * t;
    const int x = p % W, y = (p / W) % H, b = p / (W * H);
    c.y[t] = y;
    c.x[t] = x;
    c.off[t] = ((b * H + y) * W + x) * Cin;
  }
  return c;
}

// implicit-GEMM operand: 128 rows (pixels m0 ..) x 64 columns of the 3x3
// neighbourhood matrix of an NHWC tensor, gathered 8 channels (16 bytes) at a
// time; taps outside the image and columns beyond 9 Cin are zero-filled
__device__ __forceinline__ void stage_conv(uint32_t dst, const __nv_bfloat16* X, const ConvRows& cr, int k0, int H,
                                           int W, int Cin) {
  const int q = threadIdx.x & 7;
  const int k = k0 + q * 8;
  const bool inK = k < 9 * Cin;
  const int tap = inK ? k / Cin : 0;
  const int c = k - tap * Cin;
  const int dy = tap / 3 - 1, dx = tap % 3 - 1;
  const int shift = (dy * W + dx) * Cin + c;
#pragma unroll
  for (int t = 0; t < kRowsPerThread; ++t) {
    const int r = (threadIdx.x >> 3) + (kThreads / 8) * t;
    const int yy = cr.y[t] + dy, xx = cr.x[t] + dx;
    const bool in = inK && yy >= 0 && yy < H && xx >= 0 && xx < W;
    cp_async16(dst + (uint32_t)(((r >> 3) * 8 + q) * 128 + (r & 7) * 16), in ? X + cr.off[t] + shift : X,
               in ? 16u : 0u);
  }
}

// rows of the transposed operand this thread copies (fixed across the K loop over pixels)
struct ConvTRows {
  size_t off[kRowsPerThread];  // ((dx + 1) Cin + c) Mpix
  int dy[kRowsPerThread];
  bool valid[kRowsPerThread];
};
__device__ __forceinline__ ConvTRows convT_rows(int m0, int Cin, int Mpix) {
  ConvTRows c;
#pragma unroll
  for (int t = 0; t < kRowsPerThread; ++t) {
    const int k = m0 + (threadIdx.x >> 3) + (kThreads / 8) * t;
    c.valid[t] = k < 9 * Cin;
    const int tap = c.valid[t] ? k / Cin : 4, ch = k - tap * Cin;
    c.dy[t] = tap / 3 - 1;
    c.off[t] = ((size_t)(tap % 3) * Cin + (c.valid[t] ? ch : 0)) * Mpix;
  }
  return c;
}
// 128 rows (k) x 64 pixels (p0 ..) of the transposed operand; the 8 pixels of one 16-byte
// copy share an image row because W % 8 == 0
__device__ __forceinline__ void stage_convT(uint32_t dst, const __nv_bfloat16* XT3, const ConvTRows& cr, int p0,
                                            int H, int W) {
  const int q = threadIdx.x & 7;
  const int p = p0 + q * 8;
  const int y = (p / W) % H;
#pragma unroll
  for (int t = 0; t < kRowsPerThread; ++t) {
    const int r = (threadIdx.x >> 3) + (kThreads / 8) * t;
    const int yy = y + cr.dy[t];
    const bool in = cr.valid[t] && yy >= 0 && yy < H;
    cp_async16(dst + (uint32_t)(((r >> 3) * 8 + q) * 128 + (r & 7) * 16),
               in ? XT3 + cr.off[t] + p + (ptrdiff_t)cr.dy[t] * W : XT3, in ? 16u : 0u);
  }
}

}  // namespace

// pipeline depth: stages of (A chunk, B chunk) in shared memory
template <int N>
struct GemmStages {
  static constexpr int S = N >= 128 ? 3 : 4;  // <= 96 KB below N = 256: two CTAs per SM
  static constexpr size_t A_BYTES = 128 * KC * 2, B_BYTES = (size_t)N * KC * 2;
  static constexpr size_t STAGE = A_BYTES + B_BYTES;
  static constexpr size_t SMEM = S * STAGE;
};

// epilogue modes: 0 = store fp32 D; 1 = accumulate into fp32 D (D += A B^T);
// 2 = bf16 out = act(D + bias[n]) with act = ReLU when `relu`
//
// K pipeline: chunk i is copied (cp.async) into stage i % S while the MMAs of
// the chunks before it run; before stage s is refilled, the CTA waits on the
// mbarrier that the MMAs reading it committed to (bounded). One thread issues
// the MMAs after a CTA barrier that follows every thread's wait for its own
// copies of that chunk.
template <int N>
__global__ void __launch_bounds__(kThreads, 2) k_gemm_bf16(const GemmArgs g) {
  using ST = GemmStages<N>;
  constexpr int S = ST::S;
  constexpr uint32_t NCOLS = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar[S];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128;
  const int n0 = blockIdx.y * N;

  if (warp == 0) tm_alloc(&s_tmem, NCOLS);
  if (tid == 0) {
    for (int i = 0; i < S; ++i) mbar_init(&bar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = make_idesc(128, N);
  const __nv_bfloat16* A =
      reinterpret_cast<const __nv_bfloat16*>(g.A) + ((g.conv || g.convT) ? 0 : (size_t)m0 * g.K);
  const __nv_bfloat16* B = reinterpret_cast<const __nv_bfloat16*>(g.B) + (size_t)n0 * g.K;
  const int kbeg = g.ksplit > 1 ? (int)blockIdx.z * g.kc : 0;
  const int kend = g.ksplit > 1 ? min(g.K, kbeg + g.kc) : g.K;
  const int nk = (kend - kbeg) / KC;
  const uint32_t base = smem_u32(smem);
  ConvRows cr{};
  if (g.conv) cr = conv_rows(m0, g.H, g.W, g.Cin);
  ConvTRows ctr{};
  if (g.convT) ctr = convT_rows(m0, g.Cin, g.Mpix);
  bool ok = true;
  for (int i = 0; i < nk + S - 1 && ok; ++i) {
    if (i < nk) {
      const int st = i % S;
      if (i >= S)  // the MMAs of chunk i - S read this stage
        ok = __syncthreads_and(mbar_wait_bounded(&bar[st], (uint32_t)((i / S - 1) & 1)) ? 1 : 0) != 0;
      if (ok) {
        const uint32_t sa = base + (uint32_t)(st * ST::STAGE), sb = sa + (uint32_t)ST::A_BYTES;
        const int k0 = kbeg + i * KC;
        if (g.conv) stage_conv(sa, A, cr, k0, g.H, g.W, g.Cin);
        else if (g.convT) stage_convT(sa, A, ctr, k0, g.H, g.W);
        else stage(sa, A, 128, g.K, k0);
        stage(sb, B, N, g.K, k0);
      }
    }
    cp_async_commit();  // one group per step (possibly empty) keeps the group count aligned
    const int j = i - (S - 1);
    if (j >= 0 && ok) {
      cp_async_wait<S - 1>();  // this thread's copies of chunk j have landed
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int st = j % S;
        const uint32_t sa = base + (uint32_t)(st * ST::STAGE), sb = sa + (uint32_t)ST::A_BYTES;
#pragma unroll
        for (int s = 0; s < KC / 16; ++s) {
          const uint64_t ad = make_desc(sa + s * 256, 128, 1024);
          const uint64_t bd = make_desc(sb + s * 256, 128, 1024);
          mma_bf16(tmem, ad, bd, idesc, (j > 0 || s > 0) ? 1u : 0u);
        }
        mma_commit(&bar[st]);
      }
    }
  }
  cp_async_wait<0>();
  // the last chunk's commit covers every MMA issued before it
  if (ok && nk > 0)
    ok = __syncthreads_and(mbar_wait_bounded(&bar[(nk - 1) % S], (uint32_t)(((nk - 1) / S) & 1)) ? 1 : 0) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok) {
    if (tid == 0) atomicExch(g.status, 1);
    // give the MMAs in flight a bounded chance to finish before TMEM is released
    for (int st = 0; st < S; ++st) mbar_wait_bounded(&bar[st], 0u), mbar_wait_bounded(&bar[st], 1u);
  } else {
    // epilogue: warp w owns rows 32 (w % 4) .. + 31 (its TMEM lane quarter) and every other
    // group of 16 columns, starting at 16 (w / 4)
    const int row = m0 + (warp & 3) * 32 + lane;
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll 1
    for (int c0 = (warp >> 2) * 16; c0 < N; c0 += 32) {
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
        if (g.bias)  // mode 0 / 1 with a bias: the bias added to the product (one add per element)
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] += g.bias[n0 + c0 + j];
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

// ------------------------------------------------------------------ 3x3 convolution on a halo slab
// The implicit GEMM of a 'same' 3x3 convolution, D[p, n] = sum_{tap, c} X[p + tap offset, c] W[n, tap Cin + c],
// with the operand A read from one slab per chunk of up to 64 input channels instead of one gather per
// tap. Output positions are indexed over a zero-padded grid whose rows hold Wp = (W + 2) rounded up to a
// multiple of 8 positions, P = (b (H + 2) + y + 1) Wp + x + 1, so that tap (dy, dx) of every output lies
// at the fixed offset dy Wp + dx: a tile of positions [P0, P0 + 128 T) (T accumulators of 128 rows in
// TMEM) reads the whole padded rows holding positions [P0 - Wp - 1, P0 + 128 T + Wp + 1) of its channel
// chunk once (zero outside the image, so the border needs no masking) and every tap's MMA reads that
// slab through a descriptor shifted by the tap's offset. Positions on the padding are computed and
// dropped by the epilogue. The weights of each (chunk, tap) step feed all T accumulators.
//
// Every copy is done by the tensor-memory-access engine: a slab is one box of all its padded rows
// when they lie in one image, else one box per padded row (Wp positions x the chunk's channels, from
// a 4-D view (C, W, H, batch) of the NHWC input; the padding columns and rows read as out-of-bounds
// zeros, and every box starts on a 1024-byte boundary of the slab, rows being a multiple of 8
// positions long). The weights arrive packed in step order
// (halo_pack), one bulk copy per step. Each copy instruction costs its issuing thread a few hundred
// cycles, so the slabs and the weights have a thread each and the boxes are as large as a row.
//
// Shared-memory layouts (canonical K-major):
//   64-channel chunks: rows of 128 bytes, 16-byte chunk q of row j at q ^ (j % 8) (128-byte swizzle,
//     written so by the copy engine), slab and weights alike
//   narrower chunks (8, 16, 32 channels), no swizzle, a core matrix = 8 rows x 16 bytes:
//     slab  [k group g][row j]  16 bytes each: LBO (next k group) = R * 16, SBO (next 8 rows) = 128
//     B     [k group g][n]      16 bytes each: LBO = N * 16, SBO = 128
// Cin = 8 (the network's input, one channel padded to 8) holds one k group per tap: an MMA then takes
// taps t and t + 1 as its two k groups (LBO = the distance between their offsets), and the ninth tap
// is paired with zero weight columns.
namespace {
// roles: warp 0 lane 0 copies the slabs (and warp 0 owns the TMEM allocation), warp 1 lane 0 issues
// the MMAs, warps 2-5 drain the accumulators (warp w reads TMEM lanes 32 (w % 4) .. + 31), warp 6
// lane 0 copies the weights
constexpr int kHaloThreads = 224;
constexpr int kHaloLoader = 0;
constexpr int kHaloIssuer = 32;
constexpr int kHaloEpi0 = 64;
constexpr int kHaloWeights = 192;
constexpr int kHaloSMax = 8;  // weight stages at most
constexpr int kHaloBufMax = 3;  // slab buffers at most

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> own shared memory by the bulk-copy engine; both addresses 16-byte aligned, bytes % 16 == 0
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// one box of a 4-D tensor map into shared memory (coordinates innermost first; out-of-range elements
// read as zero)
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

template <int N, int T>
struct HaloCfg {
  static constexpr uint32_t NCOLS = N < 32 ? 32 : N;                 // TMEM columns per accumulator
  static constexpr uint32_t ACC = NCOLS * T;                          // one accumulator set (a tile)
  static constexpr uint32_t TMEM_COLS = 2 * ACC < 32 ? 32 : 2 * ACC;  // two sets: fill one, drain the other
  static_assert(TMEM_COLS <= 512 && (TMEM_COLS & (TMEM_COLS - 1)) == 0, "TMEM allocation");
  static constexpr size_t B_STAGE = (size_t)N * 64 * 2;  // N rows x 64 k (the widest chunk)
  __host__ __device__ static int wp(int W) { return (W + 2 + 7) / 8 * 8; }
  // whole padded rows covering positions [P0 - Wp - 1, P0 + 128 T + Wp + 2) for any P0 (a multiple of 8;
  // the row holding P0 - Wp - 1 starts at P0 - 2 Wp at the earliest, and the ninth tap's pair partner
  // reads one position past the last output's tap)
  __host__ __device__ static int rows(int W) {
    const int w = wp(W);
    return ((128 * T + 3 * w + 2 + w - 1) / w) * w;
  }
  // KG k groups (8 channels each) of 16 bytes per row
  __host__ __device__ static size_t slab_bytes(int W, int KG) { return (size_t)rows(W) * 16 * KG; }
  // weight stages S and slab buffers nbuf within `budget` bytes: three buffers (the slab copies run two
  // chunks ahead of the MMAs) when six weight stages still fit beside them (the weights' copies must
  // run five steps ahead to hide their latency), else two
  static bool plan(int W, int KG, size_t budget, int& S, int& nbuf) {
    for (nbuf = kHaloBufMax; nbuf >= 2; --nbuf) {
      const size_t sb = nbuf * slab_bytes(W, KG);
      if (sb >= budget) continue;
      const size_t n = (budget - sb) / B_STAGE;
      S = n > (size_t)kHaloSMax ? kHaloSMax : (int)n;
      if (S >= (nbuf == 3 ? 6 : 2)) return true;
    }
    return false;
  }
};

__device__ __forceinline__ void mma_bf16_acc(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accumulate) {
  mma_bf16(tmem_d, adesc, bdesc, idesc, accumulate);
}
}  // namespace

// PN (pixels as the MMA's N): for outputs of 128 channels per column block and 64-channel chunks the
// operands swap, D^T[channel][position] = W . X^T: the packed weights are A (M = 128 channels) and the
// slab is B (N = 256 positions), so that one instruction computes 128 x 256 x 16 (a 128 x 128 x 16
// instruction issues at about half the FLOP rate of a 128 x 256 x 16 one). The tile geometry is that of
// N = 128, T = 2 (256 positions, 256 TMEM columns); TMEM lane = channel, column = position.
//
// Persistent: CTA b takes tiles b, b + grid, ... (a tile = 128 T padded positions x N output channels;
// consecutive tiles share the positions, so a slab is read from HBM once and from L2 by the other
// column blocks). Steps (chunk, tap) run back to back across tiles; the copies of the next chunk's slab
// (also when it is the next tile's first) overlap the current chunk's MMAs, and the MMAs of tile l + 1
// fill one TMEM accumulator set while the epilogue warps drain tile l's.
// SW: the operands' row layout: 0 unswizzled core matrices (k-group planes), 1 rows of 128 bytes with the
// 128-byte swizzle (64-channel chunks), 2 rows of 64 bytes with the 64-byte swizzle (32-channel inputs)
template <int N, int T, int SW, bool PN>
__global__ void __launch_bounds__(kHaloThreads, 1)
    k_conv3x3_halo(const GemmArgs g, const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmr,
                   int ntiles_px, int S, int nbuf, int whole) {
  using HC = HaloCfg<N, T>;
  static_assert(!PN || (N == 128 && T == 2 && SW == 1), "swapped operands: 128 channels x 256 positions, 64-channel chunks");
  extern __shared__ __align__(1024) unsigned char smem[];
  // bfull[st]: the weights of the step in stage st landed (transaction bytes); sfull[b]: the slab in
  // buffer b landed; bar[st]: the MMAs reading stage st are done (tcgen05.commit); sbar[b]: those of
  // slab buffer b; accf[a]: accumulator set a holds a finished tile; acce[a]: the epilogue has read
  // set a; drain: every MMA issued has completed
  __shared__ uint64_t bar[kHaloSMax], bfull[kHaloSMax], sfull[kHaloBufMax], sbar[kHaloBufMax], accf[2], acce[2],
      drain;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int H = g.H, W = g.W, Cin = g.Cin;
  const int Wp = HC::wp(W), HWp = (H + 2) * Wp;
  const int nb = g.M / (H * W);
  const int Mpi = nb * HWp;  // padded positions fit in 32 bits (checked at launch)
  const int R = HC::rows(W);
  const int CC = Cin < 64 ? Cin : 64;   // channels per chunk
  const int KG = CC / 8;                // k groups per chunk
  const uint32_t slab_bytes = (uint32_t)HC::slab_bytes(W, KG);
  const int nchunks = Cin / CC;
  const bool pairs = Cin == 8 && !g.taps1;  // two taps per MMA
  const int taps = g.taps1 ? 1 : pairs ? 5 : 9;  // steps per chunk
  const int nsteps = nchunks * taps;    // steps per tile
  const int nblk = g.Ntot / N;
  const int ntiles = ntiles_px * nblk;
  const int L = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int total = L * nsteps;         // steps of this CTA
  auto tile_of = [&](int l) { return (int)blockIdx.x + l * (int)gridDim.x; };

  if (warp == 0) tm_alloc(&s_tmem, HC::TMEM_COLS);
  if (tid == 0) {
    for (int i = 0; i < kHaloSMax; ++i) {
      mbar_init(&bar[i], 1);
      mbar_init(&bfull[i], 1);
    }
    for (int i = 0; i < kHaloBufMax; ++i) {
      mbar_init(&sfull[i], 1);
      mbar_init(&sbar[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&acce[i], 128);
    }
    mbar_init(&drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = PN ? make_idesc(128, 256) : make_idesc(128, N);
  const uint32_t base = smem_u32(smem);
  const uint32_t slab0 = base, bring = base + (uint32_t)nbuf * slab_bytes;
  // slab row j of a tile starting at P0 holds position S0 + j, S0 = the start of the padded row holding
  // P0 - Wp - 1; output row r of accumulator m reads, for tap (dy, dx), slab row
  // (P0 - S0) + 128 m + r + dy Wp + dx
  auto slab_start = [&](int P0) {
    const int P = P0 - Wp - 1;
    return (P >= 0 ? P / Wp : -((-P + Wp - 1) / Wp)) * Wp;  // floor to a row start
  };

  bool ok = true;
  if (tid == kHaloLoader) {
    // the slab of chunk gc of this CTA (tile gc / nchunks, channel chunk gc % nchunks) into buffer
    // gc % nbuf, as soon as the MMAs of chunk gc - nbuf (the buffer's last reader) are done: one box per
    // padded row (image row yp - 1 of image b, columns -1 .. Wp - 2; out of range = zeros)
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmx)) : "memory");
    if (whole) asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmr)) : "memory");
    const int nchunks_all = L * nchunks;
    const int rows_per = R / Wp;
    int nslab = 0;  // slabs issued (chunks 0 .. nslab - 1)
    for (int gc = 0; gc < nchunks_all && ok; ++gc) {
      if (gc >= nbuf) ok = mbar_wait_bounded(&sbar[gc % nbuf], (uint32_t)(((gc - nbuf) / nbuf) & 1));
      if (!ok) break;
      const int l = gc / nchunks, c = gc - l * nchunks;
      const int row0 = slab_start((tile_of(l) / nblk) * 128 * T) / Wp;  // padded row index (may be < 0)
      const uint32_t buf = slab0 + (uint32_t)(gc % nbuf) * slab_bytes;
      uint64_t* fb = &sfull[gc % nbuf];
      mbar_expect_tx(fb, slab_bytes);
      // all rows_per rows inside one image's padded rows (0 .. H + 1): one box of rows_per rows (tmr)
      const int b0 = row0 >= 0 ? row0 / (H + 2) : -1;
      const int yp0 = row0 - b0 * (H + 2);
      if (whole && row0 >= 0 && yp0 + rows_per <= H + 2) {
        if (SW) {
          tma_load_4d(buf, &tmr, c * CC, -1, yp0 - 1, b0, fb);
        } else {
          for (int q = 0; q < KG; ++q) tma_load_4d(buf + (uint32_t)(q * R * 16), &tmr, c * CC + q * 8, -1, yp0 - 1, b0, fb);
        }
        nslab = gc + 1;
        continue;
      }
      for (int r = 0; r < rows_per; ++r) {
        const int pr = row0 + r;
        const int b = pr >= 0 ? pr / (H + 2) : -1;  // before the first image: all zeros
        const int yp = pr >= 0 ? pr - b * (H + 2) : 0;
        if (SW) {
          tma_load_4d(buf + (uint32_t)(r * Wp * CC * 2), &tmx, c * CC, -1, yp - 1, b, fb);
        } else {
          for (int q = 0; q < KG; ++q)
            tma_load_4d(buf + (uint32_t)((q * R + r * Wp) * 16), &tmx, c * CC + q * 8, -1, yp - 1, b, fb);
        }
      }
      nslab = gc + 1;
    }
    // no copy may still be writing shared memory when the CTA ends (normally the MMAs consumed them all)
    for (int gc = nslab - nbuf > 0 ? nslab - nbuf : 0; gc < nslab; ++gc)
      if (!mbar_wait_bounded(&sfull[gc % nbuf], (uint32_t)((gc / nbuf) & 1))) ok = false;
  } else if (tid == kHaloWeights) {
    // weights: step gs's block of the packed weights (column block of its tile, step within the tile)
    // into stage gs % S once the MMAs of step gs - S are done; one bulk copy, completing on bfull
    const int kgb = pairs ? 2 : KG;
    const uint32_t bbytes = (uint32_t)(N * kgb * 16);
    int issued = 0;
    for (int gs = 0; gs < total && ok; ++gs) {
      const int st = gs % S;
      if (gs >= S) ok = mbar_wait_bounded(&bar[st], (uint32_t)((gs / S - 1) & 1));
      if (!ok) break;
      const int l = gs / nsteps, i = gs - l * nsteps;
      const int nbk = tile_of(l) % nblk;
      const unsigned char* src = reinterpret_cast<const unsigned char*>(g.Bp) + ((size_t)nbk * nsteps + i) * bbytes;
      mbar_expect_tx(&bfull[st], bbytes);
      bulk_g2s(bring + (uint32_t)(st * HC::B_STAGE), src, bbytes, &bfull[st]);
      issued = gs + 1;
    }
    for (int gs = issued - S > 0 ? issued - S : 0; gs < issued; ++gs)
      if (!mbar_wait_bounded(&bfull[gs % S], (uint32_t)((gs / S) & 1))) ok = false;
  } else if (tid == kHaloIssuer) {
    // MMA issuer: at a tile's first step waits for the epilogue to have read the accumulator set it is
    // about to overwrite, at a chunk's first step for its slab, at every step for its weights; issues the
    // step's MMAs and commits them to bar (and to sbar / accf at a chunk's / tile's last step)
    for (int gs = 0; gs < total && ok; ++gs) {
      const int l = gs / nsteps, i = gs - l * nsteps;
      const int chunk = i / taps, t = i - chunk * taps;
      const int gc = l * nchunks + chunk;
      const int st = gs % S;
      if (i == 0 && l >= 2) ok = mbar_wait_bounded(&acce[l & 1], (uint32_t)(((l >> 1) - 1) & 1));
      if (ok && t == 0) ok = mbar_wait_bounded(&sfull[gc % nbuf], (uint32_t)((gc / nbuf) & 1));
      if (ok) ok = mbar_wait_bounded(&bfull[st], (uint32_t)((gs / S) & 1));
      if (!ok) break;
      // lean issue: a descriptor is linear in its start address ((start >> 4) in the low bits, no carry
      // below 256 KB), so every MMA's descriptors are a base plus a constant; the issuing thread must
      // keep ahead of the tensor pipe (~64-128 cycles per MMA)
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t slab = slab0 + (uint32_t)(gc % nbuf) * slab_bytes;
      const uint32_t bs = bring + (uint32_t)(st * HC::B_STAGE);
      const uint32_t acc0 = tmem + (uint32_t)(l & 1) * HC::ACC;
      const uint32_t first = i == 0 ? 0u : 1u;  // the first MMA of each accumulator overwrites it
      const int P0 = (tile_of(l) / nblk) * 128 * T;
      const int off0 = P0 - slab_start(P0);
      // (a 1 x 1 contraction reads the centre tap only)
      auto tap_row = [&](int tp) { return g.taps1 ? off0 : off0 + (tp / 3 - 1) * Wp + (tp % 3 - 1); };
      if constexpr (PN) {
        // A = the weights (128 channel rows), B = 256 slab rows from the tap's offset; K in steps of 16
        const uint64_t aw = make_desc_sw128(bs);
        const uint64_t bp = make_desc_sw128(slab + (uint32_t)(tap_row(t) * 128));
        mma_bf16_acc(acc0, aw, bp, idesc, first);
        mma_bf16_acc(acc0, aw + 2, bp + 2, idesc, 1u);
        mma_bf16_acc(acc0, aw + 4, bp + 4, idesc, 1u);
        mma_bf16_acc(acc0, aw + 6, bp + 6, idesc, 1u);
      } else if (pairs) {
        // taps 2t and 2t + 1 (the ninth with the row after it, whose weights are zero)
        const int ta = 2 * t, ra = tap_row(ta);
        const int rb = ta + 1 < 9 ? tap_row(ta + 1) : ra + 1;
        const uint64_t ad = make_desc(slab + (uint32_t)(ra * 16), (uint32_t)((rb - ra) * 16), 128);
        const uint64_t bd = make_desc(bs, (uint32_t)(N * 16), 128);
#pragma unroll
        for (int m = 0; m < T; ++m)
          mma_bf16_acc(acc0 + (uint32_t)(m * HC::NCOLS), ad + (uint64_t)(128 * m), bd, idesc, first);
      } else if constexpr (SW == 2) {
        // rows of 64 bytes: two K steps of 16 per tap (32 bytes = 2 descriptor units along each row)
        const uint64_t ad = make_desc_sw64(slab + (uint32_t)(tap_row(t) * 64));
        const uint64_t bd = make_desc_sw64(bs);
#pragma unroll
        for (int m = 0; m < T; ++m) {
          const uint64_t am = ad + (uint64_t)(512 * m);  // 128 rows of 64 bytes, in 16-byte units
          const uint32_t acc = acc0 + (uint32_t)(m * HC::NCOLS);
          mma_bf16_acc(acc, am, bd, idesc, first);
          mma_bf16_acc(acc, am + 2, bd + 2, idesc, 1u);
        }
      } else if constexpr (SW == 1) {
        // rows X .. X + 127 of the slab, K in steps of 16 (32 bytes = 2 descriptor units along each row)
        const uint64_t ad = make_desc_sw128(slab + (uint32_t)(tap_row(t) * 128));
        const uint64_t bd = make_desc_sw128(bs);
#pragma unroll
        for (int m = 0; m < T; ++m) {
          const uint64_t am = ad + (uint64_t)(1024 * m);  // 128 rows of 128 bytes, in 16-byte units
          const uint32_t acc = acc0 + (uint32_t)(m * HC::NCOLS);
          mma_bf16_acc(acc, am, bd, idesc, first);
          mma_bf16_acc(acc, am + 2, bd + 2, idesc, 1u);
          mma_bf16_acc(acc, am + 4, bd + 4, idesc, 1u);
          mma_bf16_acc(acc, am + 6, bd + 6, idesc, 1u);
        }
      } else {
        const uint64_t ad = make_desc(slab + (uint32_t)(tap_row(t) * 16), (uint32_t)(R * 16), 128);
        const uint64_t bd = make_desc(bs, (uint32_t)(N * 16), 128);
#pragma unroll
        for (int m = 0; m < T; ++m) {
          const uint32_t acc = acc0 + (uint32_t)(m * HC::NCOLS);
          const uint64_t am = ad + (uint64_t)(128 * m);  // 128 rows of 16 bytes
#pragma unroll 1
          for (int q = 0; q < KG; q += 2)  // k groups q, q + 1: R rows of 16 bytes each further
            mma_bf16_acc(acc, am + (uint64_t)(q * R), bd + (uint64_t)(q * N), idesc, q > 0 ? 1u : first);
        }
      }
      mma_commit(&bar[st]);
      if (t == taps - 1) mma_commit(&sbar[gc % nbuf]);
      if (i == nsteps - 1) mma_commit(&accf[l & 1]);
    }
    mma_commit(&drain);  // completes once every MMA this thread issued has
    if (!mbar_wait_bounded(&drain, 0u)) ok = false;
  } else if (tid >= kHaloEpi0 && tid < kHaloEpi0 + 128) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 of every accumulator of the finished tile;
    // positions on the padding are dropped
    const int eq = warp & 3;
    const uint32_t tl = tmem + ((uint32_t)(eq * 32) << 16);
    for (int l = 0; l < L && ok; ++l) {
      // one decision per warp: the TMEM loads below are warp-collective
      ok = __all_sync(0xffffffffu, mbar_wait_bounded(&accf[l & 1], (uint32_t)((l >> 1) & 1)));
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int tile = tile_of(l);
      const int P0i = (tile / nblk) * 128 * T, n0 = (tile % nblk) * N;
      const uint32_t ta = tl + (uint32_t)(l & 1) * HC::ACC;
      if constexpr (PN) {
        // lane = channel n0 + 32 eq + lane, column = position P0i + column; 32 columns at a time, lane j
        // decoding the position of column j for the warp
        const int n = n0 + eq * 32 + lane;
        const float bn = g.bias ? g.bias[n] : 0.f;
#pragma unroll 1
        for (int cb = 0; cb < 256; cb += 32) {
          long long mypix = -1;
          const int P = P0i + cb + lane;
          if (P < Mpi) {
            const int b = P / HWp, r = P - b * HWp;
            const int yp = r / Wp, xp = r - yp * Wp;
            if (yp >= 1 && yp <= H && xp >= 1 && xp <= W) mypix = ((long long)b * H + (yp - 1)) * W + (xp - 1);
          }
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float v[16];
            tm_ld16(ta + (uint32_t)(cb + 16 * h), v);
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
              const long long pix = __shfl_sync(0xffffffffu, mypix, 16 * h + jj);
              if (pix < 0) continue;
              if (g.mode == 2) {
                const float x = v[jj] + bn;
                reinterpret_cast<__nv_bfloat16*>(g.Dh)[(size_t)pix * g.ldd + n] = __float2bfloat16(g.relu ? fmaxf(x, 0.f) : x);
              } else {
                float* o = g.D + (size_t)pix * g.ldd + n;
                const float x = g.bias ? v[jj] + bn : v[jj];
                *o = g.mode == 1 ? *o + x : x;
              }
            }
          }
        }
      } else {
        long long pix[T];
#pragma unroll
        for (int m = 0; m < T; ++m) {
          const int P = P0i + 128 * m + eq * 32 + lane;
          pix[m] = -1;
          if (P < Mpi) {
            const int b = P / HWp, r = P - b * HWp;
            const int yp = r / Wp, xp = r - yp * Wp;
            if (yp >= 1 && yp <= H && xp >= 1 && xp <= W) pix[m] = ((long long)b * H + (yp - 1)) * W + (xp - 1);
          }
        }
  #pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 16) {
          float bias[16];
#pragma unroll
          for (int jj = 0; jj < 16; ++jj) bias[jj] = g.bias ? g.bias[n0 + c0 + jj] : 0.f;
#pragma unroll
          for (int m = 0; m < T; ++m) {
            float v[16];
            tm_ld16(ta + (uint32_t)(m * HC::NCOLS + c0), v);
            if (pix[m] < 0) continue;
            if (g.mode == 2) {
              float o[16];
#pragma unroll
              for (int jj = 0; jj < 16; ++jj) {
                const float x = v[jj] + bias[jj];
                o[jj] = g.relu ? fmaxf(x, 0.f) : x;
              }
              uint4 w0, w1;
              __nv_bfloat162* h0 = reinterpret_cast<__nv_bfloat162*>(&w0);
              __nv_bfloat162* h1 = reinterpret_cast<__nv_bfloat162*>(&w1);
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) {
                h0[jj] = __floats2bfloat162_rn(o[2 * jj], o[2 * jj + 1]);
                h1[jj] = __floats2bfloat162_rn(o[8 + 2 * jj], o[8 + 2 * jj + 1]);
              }
              uint4* out = reinterpret_cast<uint4*>(g.Dh + (size_t)pix[m] * g.ldd + n0 + c0);
              out[0] = w0;
              out[1] = w1;
            } else {
              float4* out = reinterpret_cast<float4*>(g.D + (size_t)pix[m] * g.ldd + n0 + c0);
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) {
                float4 o = make_float4(v[4 * jj], v[4 * jj + 1], v[4 * jj + 2], v[4 * jj + 3]);
                if (g.bias) {  // the bias added to the product (one add per element)
                  o.x += bias[4 * jj], o.y += bias[4 * jj + 1], o.z += bias[4 * jj + 2], o.w += bias[4 * jj + 3];
                }
                if (g.mode == 1) {
                  const float4 d = out[jj];
                  o.x += d.x, o.y += d.y, o.z += d.z, o.w += d.w;
                }
                out[jj] = o;
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&acce[l & 1]);  // this set may be overwritten
    }
  }
  ok = __syncthreads_and(ok ? 1 : 0) != 0;
  if (!ok && tid == 0) atomicExch(g.status, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) tm_dealloc(tmem, HC::TMEM_COLS);
}

// The weights of a halo convolution in the order the kernel consumes them: for column block nb and
// step st (chunk, tap) one block of N rows x kgb k groups of 16 bytes, laid out as the B stage in
// shared memory (swizzled rows of 128 bytes, or [k group][n]), so that a step's weights arrive by one
// bulk copy. Redone only when the weights change.
template <int N, int SW>
__global__ void k_halo_pack(const GemmArgs g, uint16_t* dst) {
  const int Cin = g.Cin, CC = Cin < 64 ? Cin : 64, KG = CC / 8;
  const bool pairs = Cin == 8 && !g.taps1;
  const int taps = g.taps1 ? 1 : pairs ? 5 : 9, nsteps = (Cin / CC) * taps, kgb = pairs ? 2 : KG;
  const size_t per_blk = (size_t)N * kgb;  // 16-byte units per block
  const size_t total = (size_t)(g.Ntot / N) * nsteps * per_blk;
  for (size_t u = (size_t)blockIdx.x * blockDim.x + threadIdx.x; u < total; u += (size_t)gridDim.x * blockDim.x) {
    const size_t b = u / per_blk;
    const int r = (int)(u - b * per_blk);
    const int nbk = (int)(b / nsteps), st = (int)(b % nsteps);
    const int n = r / kgb, q = r - n * kgb;
    const int chunk = st / taps, t = st % taps;
    const int k0 = pairs ? 16 * t : t * Cin + chunk * CC;
    const uint4 v = *reinterpret_cast<const uint4*>(g.B + (size_t)(nbk * N + n) * g.K + k0 + q * 8);
    const size_t off = SW == 1   ? (size_t)n * 128 + (size_t)((q ^ (n & 7)) << 4)
                       : SW == 2 ? (size_t)n * 64 + (size_t)((q ^ ((n >> 1) & 3)) << 4)
                                 : (size_t)(q * N + n) * 16;
    *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(dst) + b * per_blk * 16 + off) = v;
  }
}

// the CUDA driver API's tensor-map encoder, looked up once through the runtime (no link-time libcuda dependence)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

template <int N, int T, int SW, bool PN = false>
static cudaError_t launch_halo_sw(const GemmArgs& g, cudaStream_t s) {
  using HC = HaloCfg<N, T>;
  const int CC = g.Cin < 64 ? g.Cin : 64, KG = CC / 8;
  int S = 0, nbuf = 0;
  if (!HC::plan(g.W, KG, 232448 - 1024, S, nbuf)) return cudaErrorInvalidValue;  // + the static barriers
  const size_t smem = nbuf * HC::slab_bytes(g.W, KG) + S * HC::B_STAGE;
  auto kern = k_conv3x3_halo<N, T, SW, PN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nb = g.M / (g.H * g.W);
  const long long Mp = (long long)nb * (g.H + 2) * HC::wp(g.W);
  if (Mp + 128LL * T + 2LL * HC::wp(g.W) + 64 >= (1LL << 31)) return cudaErrorInvalidValue;  // 32-bit positions
  // the NHWC input as a 4-D tensor (C, W, H, batch); a box = the chunk's channels (a k group without the
  // swizzle) x the Wp columns -1 .. Wp - 2 of one row of one image
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode) return cudaErrorNotSupported;
  // and a second map whose box is a whole slab (rows_per rows) for slabs inside one image
  alignas(64) CUtensorMap map, mapr;
  const int rows_per = HC::rows(g.W) / HC::wp(g.W);
  const cuuint64_t dims[4] = {(cuuint64_t)g.Cin, (cuuint64_t)g.W, (cuuint64_t)g.H, (cuuint64_t)nb};
  const cuuint64_t strides[3] = {(cuuint64_t)g.Cin * 2, (cuuint64_t)g.W * g.Cin * 2, (cuuint64_t)g.H * g.W * g.Cin * 2};
  const cuuint32_t cb = SW == 1 ? 64 : SW == 2 ? 32 : 8;  // channels per box row
  const cuuint32_t box[4] = {cb, (cuuint32_t)HC::wp(g.W), 1, 1};
  const cuuint32_t boxr[4] = {cb, (cuuint32_t)HC::wp(g.W), (cuuint32_t)rows_per, 1};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUtensorMapSwizzle swz = SW == 1 ? CU_TENSOR_MAP_SWIZZLE_128B : SW == 2 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                                                : CU_TENSOR_MAP_SWIZZLE_NONE;
  if (encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<uint16_t*>(g.A), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  int whole = rows_per <= g.H && rows_per <= 256;
  if (!whole || encode(&mapr, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<uint16_t*>(g.A), dims, strides, boxr, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
    whole = 0;
    mapr = map;
  }
  const long long ntp = (Mp + 128LL * T - 1) / (128LL * T);
  const long long ntiles = ntp * (g.Ntot / N);
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int grid = (int)(ntiles < sms ? ntiles : sms);  // one persistent CTA per SM
  kern<<<grid, kHaloThreads, smem, s>>>(g, map, mapr, (int)ntp, S, nbuf, whole);
  return cudaGetLastError();
}

// chunks of 64 channels use the 128-byte swizzled layouts, 32-channel inputs the 64-byte swizzled ones;
// narrower inputs (8, 16 channels) the unswizzled core-matrix layout
static int halo_swizzle(const GemmArgs& g) { return g.Cin % 64 == 0 ? 1 : g.Cin == 32 && !g.taps1 ? 2 : 0; }

template <int N, int T>
static cudaError_t launch_halo(const GemmArgs& g, cudaStream_t s) {
  switch (halo_swizzle(g)) {
    case 1: return launch_halo_sw<N, T, 1>(g, s);
    case 2: return launch_halo_sw<N, T, 2>(g, s);
    default: return launch_halo_sw<N, T, 0>(g, s);
  }
}

// halo path: Cin in {8, 16, 32} or a multiple of 64; K = the weights' row length (>= 9 Cin, and >= 80 for Cin =
// 8, whose ninth tap pairs with zero columns; >= Cin for the 1 x 1 form); images of at most 254 columns (a
// padded row is one box)
bool halo_conv_supported(const GemmArgs& g) {
  const bool cin_ok = g.Cin == 8 || g.Cin == 16 || g.Cin == 32 || (g.Cin % 64 == 0 && g.Cin > 0);
  const bool k_ok = g.taps1 ? g.K >= g.Cin : g.K >= 9 * g.Cin && (g.Cin != 8 || g.K >= 80);
  return g.conv && cin_ok && g.W <= 254 && k_ok && g.ksplit <= 1 &&
         g.M % (g.H * g.W) == 0 && g.ldd % 16 == 0 && g.K % 8 == 0;
}

// the column block of the halo kernel: 128 channels with swapped operands (PN) where the output width
// is an odd multiple of 128 and the input has at least two 64-channel chunks (the transposed epilogue
// costs about one 64-channel chunk of MMAs per tile), else the widest of 256/128/64/32/16 dividing it
// (0 stands for PN)
static int halo_n(const GemmArgs& g) {
  const int Ntot = g.Ntot;
  if (Ntot % 128 == 0 && Ntot % 256 != 0 && g.Cin % 64 == 0 && g.Cin >= 128) return 0;
  return Ntot % 256 == 0 ? 256 : Ntot % 128 == 0 ? 128 : Ntot % 64 == 0 ? 64 : Ntot % 32 == 0 ? 32 : 16;
}

static cudaError_t launch_halo_n(const GemmArgs& g, cudaStream_t s) {
  switch (halo_n(g)) {
    case 0: return launch_halo_sw<128, 2, 1, true>(g, s);
    case 256: return launch_halo<256, 1>(g, s);
    case 128: return launch_halo<128, 2>(g, s);
    case 64: return launch_halo<64, 4>(g, s);
    case 32: return launch_halo<32, 4>(g, s);
    default: return launch_halo<16, 4>(g, s);
  }
}

// whether the slab buffers and weight stages of the halo kernel for g fit in shared memory
template <int N, int T>
static bool halo_fits(const GemmArgs& g) {
  int S = 0, nbuf = 0;
  return HaloCfg<N, T>::plan(g.W, (g.Cin < 64 ? g.Cin : 64) / 8, 232448 - 1024, S, nbuf);
}
static bool halo_fits_n(const GemmArgs& g) {
  switch (halo_n(g)) {
    case 0: return halo_fits<128, 2>(g);
    case 256: return halo_fits<256, 1>(g);
    case 128: return halo_fits<128, 2>(g);
    case 64: return halo_fits<64, 4>(g);
    case 32: return halo_fits<32, 4>(g);
    default: return halo_fits<16, 4>(g);
  }
}

template <int N>
static cudaError_t pack_n(const GemmArgs& g, uint16_t* dst, cudaStream_t s) {
  switch (halo_swizzle(g)) {
    case 1: k_halo_pack<N, 1><<<304, 256, 0, s>>>(g, dst); break;
    case 2: k_halo_pack<N, 2><<<304, 256, 0, s>>>(g, dst); break;
    default: k_halo_pack<N, 0><<<304, 256, 0, s>>>(g, dst); break;
  }
  return cudaGetLastError();
}

size_t halo_pack_elems(const GemmArgs& g) {
  return (size_t)g.Ntot * (g.taps1 ? g.Cin : g.Cin == 8 ? 80 : 9 * g.Cin);
}

cudaError_t halo_pack(const GemmArgs& g, uint16_t* dst, cudaStream_t s) {
  if (!halo_conv_supported(g) || !dst) return cudaErrorInvalidValue;
  switch (halo_n(g)) {
    case 0: return pack_n<128>(g, dst, s);  // 128-row blocks, the A operand's layout is the same
    case 256: return pack_n<256>(g, dst, s);
    case 128: return pack_n<128>(g, dst, s);
    case 64: return pack_n<64>(g, dst, s);
    case 32: return pack_n<32>(g, dst, s);
    default: return pack_n<16>(g, dst, s);
  }
}

template <int N>
static cudaError_t launch_n(const GemmArgs& g, cudaStream_t s) {
  const size_t smem = GemmStages<N>::SMEM;
  cudaError_t e = cudaFuncSetAttribute(k_gemm_bf16<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gemm_bf16<N><<<dim3(g.M / 128, g.Ntot / N, g.ksplit > 1 ? g.ksplit : 1), kThreads, smem, s>>>(g);
  return cudaGetLastError();
}

// N tile chosen from the output width: the widest of 256/128/64/32/16 dividing it
cudaError_t launch_gemm_bf16(const GemmArgs& g, cudaStream_t s) {
  if (g.M <= 0 || g.K <= 0 || g.Ntot <= 0 || g.Ntot % 16) return cudaErrorInvalidValue;
  if (g.taps1) {  // the 1 x 1 form exists on the halo kernel only
    if (!(g.Bp && halo_conv_supported(g) && halo_fits_n(g))) return cudaErrorInvalidValue;
    return launch_halo_n(g, s);
  }
  if (g.M % 128 || g.K % KC) return cudaErrorInvalidValue;
  if (g.convT && (g.W % 8 || g.Mpix != g.K || g.conv)) return cudaErrorInvalidValue;
  if (g.ksplit > 1 && g.bias) return cudaErrorInvalidValue;  // a bias would be added once per split
  if (g.ksplit > 1 && (g.mode != 0 || g.kc % KC || g.kc <= 0 || (long long)(g.ksplit - 1) * g.kc >= g.K ||
                       (long long)g.ksplit * g.kc < g.K || g.ksplit > 65535))
    return cudaErrorInvalidValue;  // every split must own at least one chunk
  if (g.Bp && halo_conv_supported(g) && halo_fits_n(g)) return launch_halo_n(g, s);
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
