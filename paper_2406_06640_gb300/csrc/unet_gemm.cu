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
// tap. Output positions are indexed over the zero-padded grid, P = (b (H + 2) + y + 1) (W + 2) + x + 1,
// so that tap (dy, dx) of every output lies at the fixed offset dy (W + 2) + dx: a CTA owning the
// positions [P0, P0 + 128 T) (T accumulators of 128 rows in TMEM) copies the padded rows
// [P0 - (W + 3), P0 + 128 T + W + 3] of its channel chunk once (zero outside the image, so the border
// needs no masking) and every tap's MMA reads that slab through a descriptor shifted by the tap's
// offset. Positions on the padding are computed and dropped by the epilogue (3 % of the work at
// 128 x 128, 21 % at 16 x 16). The weights of each (chunk, tap) step feed all T accumulators.
//
// Shared-memory layouts (canonical K-major, no swizzle; a core matrix = 8 rows x 16 bytes):
//   slab  [k group g][row j]  16 bytes each: LBO (next k group) = R * 16, SBO (next 8 rows) = 128
//   B     [k group g][n]      16 bytes each: LBO = N * 16, SBO = 128
// Cin = 8 (the network's input, one channel padded to 8) holds one k group per tap: an MMA then takes
// taps t and t + 1 as its two k groups (LBO = the distance between their offsets), and the ninth tap
// is paired with zero weight columns.
namespace {
constexpr int kHaloProducers = kThreads - 32;  // warps 0-6 copy, warp 7 issues the MMAs

template <int N, int T>
struct HaloCfg {
  // B ring: S stages; the copies of a step are issued D - 1 steps before its MMAs, so D - 1 steps of
  // copies and S - D + 1 steps of MMAs are in flight at once (two of each at N >= 128, where one step is
  // ~0.6 us of tensor work; three steps of copies below, where a step is shorter)
  static constexpr int S = N >= 128 ? 4 : 6;
  static constexpr int D = N >= 128 ? 3 : 4;
  static constexpr uint32_t NCOLS = N < 32 ? 32 : N;           // TMEM columns per accumulator
  static constexpr size_t B_STAGE = (size_t)N * 64 * 2;         // N rows x 64 k (the widest chunk)
  __host__ __device__ static size_t rows(int W) { return (size_t)(128 * T + 2 * W + 8 + 7) / 8 * 8; }
  // KG k groups (8 channels each) of 16 bytes per row
  __host__ __device__ static size_t slab_bytes(int W, int KG) { return rows(W) * 16 * KG; }
  __host__ __device__ static size_t smem(int W, int KG) { return 2 * slab_bytes(W, KG) + S * B_STAGE; }
};

__device__ __forceinline__ void mma_bf16_acc(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                             uint32_t accumulate) {
  mma_bf16(tmem_d, adesc, bdesc, idesc, accumulate);
}
}  // namespace

template <int N, int T, bool SW>
__global__ void __launch_bounds__(kThreads, 1) k_conv3x3_halo(const GemmArgs g) {
  using HC = HaloCfg<N, T>;
  constexpr int S = HC::S, D = HC::D;
  extern __shared__ __align__(1024) unsigned char smem[];
  // full[st]: the producers' copies of the step in stage st landed (one arrival per producer thread);
  // bar[st]: the MMAs reading stage st are done (tcgen05.commit); sbar[b]: those of slab buffer b
  __shared__ uint64_t bar[S], full[S], sbar[2];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int H = g.H, W = g.W, Cin = g.Cin;
  const int Wp = W + 2, HWp = (H + 2) * Wp;
  const int nb = g.M / (H * W);
  const long long Mp = (long long)nb * HWp;
  const long long P0 = (long long)blockIdx.x * 128 * T;
  const int n0 = blockIdx.y * N;
  const int R = (int)HC::rows(W);
  const int CC = Cin < 64 ? Cin : 64;   // channels per chunk
  const int KG = CC / 8;                // k groups per chunk
  const uint32_t slab_bytes = (uint32_t)HC::slab_bytes(W, KG);
  const int nchunks = Cin / CC;
  const bool pairs = Cin == 8;          // two taps per MMA
  const int taps = pairs ? 5 : 9;       // steps per chunk
  const int nsteps = nchunks * taps;
  const int Kw = g.K;                   // row length of the weights
  constexpr uint32_t NCOLS_ALL = HC::NCOLS * T < 32 ? 32 : HC::NCOLS * T;

  if (warp == 0) tm_alloc(&s_tmem, NCOLS_ALL);
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&bar[i], 1);
      mbar_init(&full[i], kHaloProducers);
    }
    mbar_init(&sbar[0], 1);
    mbar_init(&sbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = make_idesc(128, N);
  const uint32_t base = smem_u32(smem);
  const uint32_t slab0 = base, bring = base + 2 * slab_bytes;
  const __nv_bfloat16* X = reinterpret_cast<const __nv_bfloat16*>(g.A);
  const __nv_bfloat16* B = reinterpret_cast<const __nv_bfloat16*>(g.B) + (size_t)n0 * Kw;

  // slab row j, k group q: [q][j] (no swizzle) or row j of 128 bytes with chunk q at q ^ (j % 8) (swizzled)
  auto slab_at = [&](uint32_t buf, int j, int q) {
    return SW ? buf + (uint32_t)(j * 128 + ((q ^ (j & 7)) << 4)) : buf + (uint32_t)((q * R + j) * 16);
  };
  // element offset in X of slab row j's pixel, or -1 on the padding / outside the tensor
  const int P0i = (int)P0, Mpi = (int)Mp;  // padded positions fit in 32 bits (checked at launch)
  auto row_off = [&](int j) -> long long {
    const int P = P0i - (W + 3) + j;
    if (P < 0 || P >= Mpi) return -1;
    const int b = P / HWp, r = P - b * HWp;
    const int yp = r / Wp, xp = r - yp * Wp;
    if (yp < 1 || yp > H || xp < 1 || xp > W) return -1;
    return (((long long)b * H + (yp - 1)) * W + (xp - 1)) * Cin;
  };
  // copies: the k groups of one row are adjacent threads (a warp reads whole 16 KG-byte pixel chunks)
  auto stage_slab = [&](int chunk, uint32_t dst) {
    const int c0 = chunk * CC;
    for (int i = tid; i < R * KG; i += kHaloProducers) {
      const int j = i / KG, q = i % KG;
      const long long o = row_off(j);
      cp_async16(slab_at(dst, j, q), o >= 0 ? X + o + c0 + q * 8 : X, o >= 0 ? 16u : 0u);
    }
  };
  // weights of step st: k columns [k0, k0 + 8 KGB) -> [k group][n] (no swizzle) or swizzled rows of n
  auto stage_b = [&](int st, uint32_t dst) {
    const int chunk = st / taps, t = st % taps;
    const int kgb = pairs ? 2 : KG;
    const int k0 = pairs ? 16 * t : t * Cin + chunk * CC;
    for (int i = tid; i < N * kgb; i += kHaloProducers) {
      const int n = i / kgb, q = i % kgb;
      const uint32_t d = SW ? dst + (uint32_t)(n * 128 + ((q ^ (n & 7)) << 4)) : dst + (uint32_t)((q * N + n) * 16);
      cp_async16(d, B + (size_t)n * Kw + k0 + q * 8, 16u);
    }
  };
  auto tap_off = [&](int t) { return (t / 3 - 1) * Wp + (t % 3 - 1); };

  // warp-specialised main loop, no CTA-wide barrier inside:
  //   producers (warps 0-6): copies of step i into stage i % S once the MMAs of step i - S are done
  //     (bar), then, D - 1 steps later, wait for their own copies of that step, make them visible to
  //     the tensor core's (async) proxy and arrive on full[stage];
  //   MMA issuer (warp 7, lane 0): waits on full[stage] of step j, issues its MMAs, commits to bar.
  bool ok = true;
  if (tid < kHaloProducers) {
    for (int i = 0; i < nsteps + D - 1 && ok; ++i) {
      if (i < nsteps) {
        const int st = i % S;
        if (i >= S) ok = mbar_wait_bounded(&bar[st], (uint32_t)((i / S - 1) & 1));
        const int chunk = i / taps;
        if (ok && i % taps == 0 && chunk >= 2)  // the MMAs of chunk - 2 read this slab buffer
          ok = mbar_wait_bounded(&sbar[chunk & 1], (uint32_t)(((chunk - 2) >> 1) & 1));
        if (ok) {
          if (i % taps == 0) stage_slab(chunk, slab0 + (uint32_t)(chunk & 1) * slab_bytes);
          stage_b(i, bring + (uint32_t)(st * HC::B_STAGE));
        }
      }
      cp_async_commit();  // one group per iteration (possibly empty) keeps the group count aligned
      const int j = i - (D - 1);
      if (ok && j >= 0 && j < nsteps) {
        cp_async_wait<D - 1>();  // this thread's copies of step j (groups up to i are committed)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&full[j % S]);
      }
    }
    cp_async_wait<0>();
  } else if (tid == kHaloProducers) {
    for (int j = 0; j < nsteps && ok; ++j) {
      ok = mbar_wait_bounded(&full[j % S], (uint32_t)((j / S) & 1));
      if (!ok) break;
      // lean issue: a descriptor is linear in its start address ((start >> 4) in the low bits, no carry
      // below 256 KB), so every MMA's descriptors are a base plus a constant; the issuing thread must
      // keep ahead of the tensor pipe (~64-128 cycles per MMA)
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int st = j % S, chunk = j / taps, t = j % taps;
      const uint32_t slab = slab0 + (uint32_t)(chunk & 1) * slab_bytes;
      const uint32_t bs = bring + (uint32_t)(st * HC::B_STAGE);
      const uint32_t first = j == 0 ? 0u : 1u;  // the first MMA of each accumulator overwrites it
      if (pairs) {
        // taps 2t and 2t + 1 (the ninth with the row after it, whose weights are zero)
        const int ta = 2 * t, oa = tap_off(ta);
        const int ob = ta + 1 < 9 ? tap_off(ta + 1) : oa + 1;
        const uint64_t ad = make_desc(slab + (uint32_t)((W + 3 + oa) * 16), (uint32_t)((ob - oa) * 16), 128);
        const uint64_t bd = make_desc(bs, (uint32_t)(N * 16), 128);
#pragma unroll
        for (int m = 0; m < T; ++m)
          mma_bf16_acc(tmem + (uint32_t)(m * HC::NCOLS), ad + (uint64_t)(128 * m), bd, idesc, first);
      } else if constexpr (SW) {
        // rows X .. X + 127 of the slab, K in steps of 16 (32 bytes = 2 descriptor units along each row)
        const uint64_t ad = make_desc_sw128(slab + (uint32_t)((W + 3 + tap_off(t)) * 128));
        const uint64_t bd = make_desc_sw128(bs);
#pragma unroll
        for (int m = 0; m < T; ++m) {
          const uint64_t am = ad + (uint64_t)(1024 * m);  // 128 rows of 128 bytes, in 16-byte units
          const uint32_t acc = tmem + (uint32_t)(m * HC::NCOLS);
          mma_bf16_acc(acc, am, bd, idesc, first);
          mma_bf16_acc(acc, am + 2, bd + 2, idesc, 1u);
          mma_bf16_acc(acc, am + 4, bd + 4, idesc, 1u);
          mma_bf16_acc(acc, am + 6, bd + 6, idesc, 1u);
        }
      } else {
        const uint64_t ad = make_desc(slab + (uint32_t)((W + 3 + tap_off(t)) * 16), (uint32_t)(R * 16), 128);
        const uint64_t bd = make_desc(bs, (uint32_t)(N * 16), 128);
#pragma unroll
        for (int m = 0; m < T; ++m) {
          const uint32_t acc = tmem + (uint32_t)(m * HC::NCOLS);
          const uint64_t am = ad + (uint64_t)(128 * m);  // 128 rows of 16 bytes
#pragma unroll 1
          for (int q = 0; q < KG; q += 2)  // k groups q, q + 1: R rows of 16 bytes each further
            mma_bf16_acc(acc, am + (uint64_t)(q * R), bd + (uint64_t)(q * N), idesc, q > 0 ? 1u : first);
        }
      }
      mma_commit(&bar[st]);
      if (t == taps - 1) mma_commit(&sbar[chunk & 1]);
    }
  }
  ok = __syncthreads_and(ok ? 1 : 0) != 0;
  if (ok && nsteps > 0)  // the last step's commit covers every MMA issued before it
    ok = __syncthreads_and(mbar_wait_bounded(&bar[(nsteps - 1) % S], (uint32_t)(((nsteps - 1) / S) & 1)) ? 1 : 0) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok) {
    if (tid == 0) atomicExch(g.status, 1);
    for (int st = 0; st < S; ++st) mbar_wait_bounded(&bar[st], 0u), mbar_wait_bounded(&bar[st], 1u);
    for (int b2 = 0; b2 < 2; ++b2) mbar_wait_bounded(&sbar[b2], 0u), mbar_wait_bounded(&sbar[b2], 1u);
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 of every accumulator, every other group of 16
    // columns starting at 16 (w / 4); positions on the padding are dropped
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    long long pix[T];
#pragma unroll
    for (int m = 0; m < T; ++m) {
      const int P = P0i + 128 * m + (warp & 3) * 32 + lane;
      pix[m] = -1;
      if (P < Mpi) {
        const int b = P / HWp, r = P - b * HWp;
        const int yp = r / Wp, xp = r - yp * Wp;
        if (yp >= 1 && yp <= H && xp >= 1 && xp <= W) pix[m] = ((long long)b * H + (yp - 1)) * W + (xp - 1);
      }
    }
#pragma unroll 1
    for (int c0 = (warp >> 2) * 16; c0 < N; c0 += 32) {
      float bias[16];
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) bias[jj] = (g.mode == 2 && g.bias) ? g.bias[n0 + c0 + jj] : 0.f;
#pragma unroll
      for (int m = 0; m < T; ++m) {
        float v[16];
        tm_ld16(tl + (uint32_t)(m * HC::NCOLS + c0), v);
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
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) tm_dealloc(tmem, NCOLS_ALL);
}

template <int N, int T, bool SW>
static cudaError_t launch_halo_sw(const GemmArgs& g, cudaStream_t s) {
  using HC = HaloCfg<N, T>;
  const size_t smem = HC::smem(g.W, (g.Cin < 64 ? g.Cin : 64) / 8);
  if (smem + 1024 > 232448) return cudaErrorInvalidValue;  // dynamic + the static barriers (1 KB aligned)
  auto kern = k_conv3x3_halo<N, T, SW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long Mp = (long long)(g.M / (g.H * g.W)) * (g.H + 2) * (g.W + 2);
  if (Mp + 128LL * T + 2LL * g.W + 16 >= (1LL << 31)) return cudaErrorInvalidValue;  // 32-bit positions
  const long long grid = (Mp + 128LL * T - 1) / (128LL * T);
  kern<<<dim3((unsigned)grid, g.Ntot / N), kThreads, smem, s>>>(g);
  return cudaGetLastError();
}

// chunks of 64 channels use the 128-byte swizzled layouts; narrower inputs (8, 16, 32 channels) the
// unswizzled core-matrix layout
template <int N, int T>
static cudaError_t launch_halo(const GemmArgs& g, cudaStream_t s) {
  return g.Cin % 64 == 0 ? launch_halo_sw<N, T, true>(g, s) : launch_halo_sw<N, T, false>(g, s);
}

// halo path: Cin in {8, 16, 32} or a multiple of 64; K = the weights' row length (>= 9 Cin, and >= 80 for Cin =
// 8, whose ninth tap pairs with zero columns); images of at most 256 columns
static bool halo_supported(const GemmArgs& g) {
  const bool cin_ok = g.Cin == 8 || g.Cin == 16 || g.Cin == 32 || (g.Cin % 64 == 0 && g.Cin > 0);
  return g.conv && cin_ok && g.W <= 256 && g.K >= 9 * g.Cin && (g.Cin != 8 || g.K >= 80) && g.ksplit <= 1 &&
         g.M % (g.H * g.W) == 0 && g.ldd % 16 == 0;
}

static cudaError_t launch_halo_n(const GemmArgs& g, cudaStream_t s) {
  if (g.Ntot % 256 == 0) return launch_halo<256, 2>(g, s);
  if (g.Ntot % 128 == 0) return launch_halo<128, 4>(g, s);
  if (g.Ntot % 64 == 0) return launch_halo<64, 4>(g, s);
  if (g.Ntot % 32 == 0) return launch_halo<32, 4>(g, s);
  return launch_halo<16, 4>(g, s);
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
  if (g.M % 128 || g.K % KC || g.Ntot % 16 || g.M <= 0 || g.K <= 0 || g.Ntot <= 0) return cudaErrorInvalidValue;
  if (g.convT && (g.W % 8 || g.Mpix != g.K || g.conv)) return cudaErrorInvalidValue;
  if (g.ksplit > 1 && (g.mode != 0 || g.kc % KC || g.kc <= 0 || (long long)(g.ksplit - 1) * g.kc >= g.K ||
                       (long long)g.ksplit * g.kc < g.K || g.ksplit > 65535))
    return cudaErrorInvalidValue;  // every split must own at least one chunk
  if (halo_supported(g)) return launch_halo_n(g, s);
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
