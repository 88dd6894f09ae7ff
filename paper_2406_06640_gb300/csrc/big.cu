// Staged path for probe sizes whose M x M complex tile exceeds one SM's
// shared memory (M = 256). Same iteration as the fused kernel (Eqs. 1, 2, 6, 7,
// Fig. 1 box 1), split into passes over an L2-sized scratch W that holds a
// chunk of C positions x K modes:
//
//   far field:  rows(exit wave, DFT) -> cols(DFT) -> modulus (R) -> cols(R x, IDFT)
//               -> rows(IDFT, dpsi, contributions)
//   near field: rows(exit wave, DFT) -> cols(DFT, x H, IDFT) -> rows(IDFT)
//               -> modulus (R) -> rows(R x, DFT) -> cols(DFT, x conj H, IDFT)
//               -> rows(IDFT, dpsi, contributions)
//
// A length-256 line is transformed by 16 threads: a radix-16 pass in
// registers over x = t + 16 j, the twiddle W_256^(t k2), a warp-local swap in
// shared memory, and a second radix-16 pass; thread t then holds frequencies
// t + 16 k1. The inverse consumes that layout and returns x = t + 16 j.
// All sums that cross CTAs are written to per-(slot, mode) or per-(position,
// row-block) partials and added in a fixed order, as on the fused path.
#include <cuda_runtime.h>

#include "big_line.cuh"
#include "engine.h"
#include "fft.cuh"

namespace ptycho {

namespace {

constexpr int RB = 16;   // rows per modulus block

// twiddles W_BL^(t k2) for t < 16 and the k2 of the first pass, from the host table W_BL^m
template <int BL>
__device__ __forceinline__ void load_tw(float2* s_tw, const float2* tw) {
  constexpr int TWS = BigShape<BL>::TWS, K2 = BigShape<BL>::E;
  for (int i = threadIdx.x; i < BigShape<BL>::TWN; i += blockDim.x) {
    const int t = i / TWS, k2 = i % TWS;
    s_tw[i] = k2 < K2 ? tw[(t * k2) % BL] : make_float2(0.f, 0.f);
  }
}

}  // namespace

// ---- row passes. mode 0: exit wave + forward DFT; 1: R x (row) then forward DFT in place;
// 2: inverse DFT in place, / M^2
template <int BL, int MODE, bool NEAR>
__global__ void __launch_bounds__(BigShape<BL>::LROW * BT) k_big_rows(const BigArgs b) {
  constexpr int E = BigShape<BL>::E, LROW = BigShape<BL>::LROW;
  __shared__ float2 s_tw[BigShape<BL>::TWN];
  __shared__ float2 s_sw[LROW][BigShape<BL>::SWN];
  load_tw<BL>(s_tw, b.tw);
  __syncthreads();
  const int li = threadIdx.x / BT, t = threadIdx.x % BT;
  const int y = blockIdx.x * LROW + li;
  const int k = blockIdx.y, c = blockIdx.z;
  const int n = b.n0 + c;
  const size_t MM = (size_t)BL * BL;
  float2* row = b.W + ((size_t)c * b.K + k) * MM + (size_t)y * BL;
  float2 a[E];
  if constexpr (MODE == 0) {
    const int2 pn = b.pos[n];
    const float2* Pk = b.P + (size_t)k * MM + (size_t)y * BL;
    const float2* On = b.O + (size_t)(pn.x + y) * b.obj_w + pn.y;
    // pc-DM second sweep: the reflected wave chi = 2 P o_n - psi_n
    const float2* St = b.dm_pass == 2 ? b.psi + ((size_t)n * b.K + k) * MM + (size_t)y * BL : nullptr;
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int x = t + 16 * j;
      float2 psi = cmul(Pk[x], On[x]);
      if (St) {
        const float2 st = b.dm_init ? psi : St[x];
        psi = make_float2(2.f * psi.x - st.x, 2.f * psi.y - st.y);
      }
      if (!NEAR && ((y + x) & 1)) psi = make_float2(-psi.x, -psi.y);
      a[j] = psi;
    }
  } else if constexpr (MODE == 1) {
    // Psi' = R Psi (the modulus ratio of this position) on the way in
    const float* Rr = b.R + (size_t)c * MM + (size_t)y * BL;
#pragma unroll
    for (int j = 0; j < E; ++j) a[j] = cscale(row[t + 16 * j], Rr[t + 16 * j]);
  } else {
#pragma unroll
    for (int r = 0; r < E; ++r) a[r] = row[line_freq<BL>(t, r)];
  }
  if constexpr (MODE == 2) {
    line_fft<BL, true>(a, s_sw[li], s_tw, t);
    const float s = 1.0f / (float)(BL * BL);
#pragma unroll
    for (int j = 0; j < E; ++j) row[t + 16 * j] = cscale(a[j], s);
  } else {
    line_fft<BL, false>(a, s_sw[li], s_tw, t);
#pragma unroll
    for (int r = 0; r < E; ++r) row[line_freq<BL>(t, r)] = a[r];
  }
}

// ---- column passes on a BL x LINES tile staged through shared memory.
// op 0: forward DFT; 1: R x (tile), inverse DFT (far backward); 2: DFT, x H, IDFT (near forward);
// 3: DFT, x conj H, IDFT (near backward)
template <int BL, int OP>
__global__ void __launch_bounds__(BigShape<BL>::LINES * BT) k_big_cols(const BigArgs b) {
  constexpr int E = BigShape<BL>::E, LINES = BigShape<BL>::LINES;
  constexpr int TP = LINES + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tile = reinterpret_cast<float2*>(smem_raw);  // [BL][TP]
  float2* s_tw = tile + BL * TP;
  float2* s_sw = s_tw + BigShape<BL>::TWN;  // [LINES][SWN]
  float2* s_h = s_sw + LINES * BigShape<BL>::SWN;
  load_tw<BL>(s_tw, b.tw);
  if constexpr (OP >= 2)
    for (int i = threadIdx.x; i < BL; i += blockDim.x) s_h[i] = b.hq[i];
  const int x0 = blockIdx.x * LINES, k = blockIdx.y, c = blockIdx.z;
  const size_t MM = (size_t)BL * BL;
  float2* Wk = b.W + ((size_t)c * b.K + k) * MM;
  // coalesced tile load: LINES consecutive columns per row; the far-field inverse pass applies
  // Psi' = R Psi (the modulus ratio of this position) on the way in
  const float* Rc = b.R + (size_t)c * MM;
  for (int i = threadIdx.x; i < BL * LINES; i += blockDim.x) {
    const int yy = i / LINES, xx = i % LINES;
    const float2 w = Wk[(size_t)yy * BL + x0 + xx];
    tile[yy * TP + xx] = OP == 1 ? cscale(w, Rc[(size_t)yy * BL + x0 + xx]) : w;
  }
  __syncthreads();
  const int cl = threadIdx.x / BT, t = threadIdx.x % BT;
  float2* sw = s_sw + cl * BigShape<BL>::SWN;
  float2 a[E];
  if constexpr (OP == 1) {
#pragma unroll
    for (int r = 0; r < E; ++r) a[r] = tile[line_freq<BL>(t, r) * TP + cl];
    line_fft<BL, true>(a, sw, s_tw, t);
  } else {
#pragma unroll
    for (int j = 0; j < E; ++j) a[j] = tile[(t + 16 * j) * TP + cl];
    line_fft<BL, false>(a, sw, s_tw, t);  // a[r] = column spectrum at u = line_freq(t, r)
    if constexpr (OP >= 2) {
      const float2 hv = s_h[x0 + cl];  // H(u, v) = h[u] h[v], v = this column's frequency
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const float2 hh = cmul(s_h[line_freq<BL>(t, r)], hv);
        a[r] = OP == 2 ? cmul(a[r], hh) : cmulc(a[r], hh);
      }
      line_fft<BL, true>(a, sw, s_tw, t);
    }
  }
  __syncthreads();
  if constexpr (OP == 0) {
#pragma unroll
    for (int r = 0; r < E; ++r) tile[line_freq<BL>(t, r) * TP + cl] = a[r];
  } else {
#pragma unroll
    for (int j = 0; j < E; ++j) tile[(t + 16 * j) * TP + cl] = a[j];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < BL * LINES; i += blockDim.x) {
    const int yy = i / LINES, xx = i % LINES;
    Wk[(size_t)yy * BL + x0 + xx] = tile[yy * TP + xx];
  }
}

// ---- modulus: rows [y0, y0 + RB) of one position, with KH halo rows for the y blur.
// Writes the ratio R to its own buffer (W is still read by the neighbouring
// blocks' halos); the next pass applies Psi' = R Psi as it loads W.
template <int BL, int KH>
__global__ void __launch_bounds__(256) k_big_modulus(const BigArgs b) {
  constexpr int HR = RB + 2 * KH;  // rows held
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sA = reinterpret_cast<float*>(smem_raw);  // HR x BL
  float* sB = sA + HR * BL;                          // HR x BL
  __shared__ float s_gx[2 * KH + 1], s_gy[2 * KH + 1];
  __shared__ double s_red[256];
  for (int i = threadIdx.x; i < 2 * KH + 1; i += blockDim.x) {
    const int d = i - KH;
    const bool in = d >= -b.kh && d <= b.kh;
    s_gx[i] = in ? b.gx[d + b.kh] : 0.f;
    s_gy[i] = in ? b.gy[d + b.kh] : 0.f;
  }
  const int y0 = blockIdx.x * RB, c = blockIdx.y;
  const int n = b.n0 + c;
  const size_t MM = (size_t)BL * BL;
  const float2* Wc = b.W + (size_t)c * b.K * MM;
  // mode sum (rank order k = 0..K-1), amplitude or intensity
  for (int i = threadIdx.x; i < HR * BL; i += blockDim.x) {
    const int yy = y0 - KH + i / BL, x = i % BL;
    float s = 0.f;
    if (yy >= 0 && yy < BL)
      for (int k = 0; k < b.K; ++k) s += cabs2(Wc[(size_t)k * MM + (size_t)yy * BL + x]);
    sA[i] = b.blur_intensity ? s : sqrtf(s);
  }
  __syncthreads();
  // blur along x (columns, sigma_1), zero padded
  for (int i = threadIdx.x; i < HR * BL; i += blockDim.x) {
    const int r = i / BL, x = i % BL;
    float acc = 0.f;
#pragma unroll
    for (int d = -KH; d <= KH; ++d) {
      const int xx = x + d;
      if (xx >= 0 && xx < BL) acc = fmaf(s_gx[d + KH], sA[r * BL + xx], acc);
    }
    sB[i] = acc;
  }
  __syncthreads();
  // blur along y (rows, sigma_2) for the own rows, ratio, error; Psi' = R Psi for every mode
  const float eps = b.eps;
  float es = 0.f, ec = 0.f;
  const float* In = b.I + (size_t)n * MM;
  const float* Sn = b.sqrtI + (size_t)n * MM;
  for (int i = threadIdx.x; i < RB * BL; i += blockDim.x) {
    const int r = i / BL, x = i % BL, y = y0 + r;
    float acc = 0.f;
#pragma unroll
    for (int d = -KH; d <= KH; ++d) acc = fmaf(s_gy[d + KH], sB[(r + KH + d) * BL + x], acc);
    const float sq = Sn[(size_t)y * BL + x];
    float ihat, R;
    if (b.blur_intensity) {
      ihat = acc;
      R = sq * rsqrtf(acc + eps * eps);
    } else {
      ihat = acc * acc;
      R = __fdividef(sq, acc + eps);
    }
    const float dd = ihat - In[(size_t)y * BL + x];
    const float yv = fmaf(dd, dd, -ec);
    const float tt = es + yv;
    ec = (tt - es) - yv;
    es = tt;
    if (b.dm_pass != 1) b.R[(size_t)c * MM + (size_t)y * BL + x] = R;  // pc-DM: R of chi only
  }
  if (b.dm_pass == 2) return;  // pc-DM: the error is the estimate's (first sweep); uniform per block
  s_red[threadIdx.x] = (double)es - (double)ec;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s_red[threadIdx.x] += s_red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) b.errpart[(size_t)n * (BL / RB) + blockIdx.x] = s_red[0];
}

// fire-and-forget adds at L2 for the probe partials: within one launch every element is added to by
// one thread only, and launches are ordered, so each sum keeps its position order (bitwise
// reproducible) while no thread waits for the old value
__device__ __forceinline__ void red_add(float2* a, float2 v) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(a), "f"(v.x), "f"(v.y));
}
__device__ __forceinline__ void red_add(float* a, float v) {
  asm volatile("red.global.add.f32 [%0], %1;" ::"l"(a), "f"(v));
}

// ---- final inverse row DFT of every mode, dpsi, contributions
template <int BL, bool NEAR>
__global__ void __launch_bounds__(BigShape<BL>::LROW * BT) k_big_final(const BigArgs b) {
  constexpr int E = BigShape<BL>::E, LROW = BigShape<BL>::LROW;
  __shared__ float2 s_tw[BigShape<BL>::TWN];
  __shared__ float2 s_sw[LROW][BigShape<BL>::SWN];
  load_tw<BL>(s_tw, b.tw);
  __syncthreads();
  const int li = threadIdx.x / BT, t = threadIdx.x % BT;
  const int y = blockIdx.x * LROW + li;
  const int c = blockIdx.y;
  const int n = b.n0 + c;
  const bool first = b.n0 == b.n_first;
  const size_t MM = (size_t)BL * BL;
  const int2 pn = b.pos[n];
  const float2* On = b.O + (size_t)(pn.x + y) * b.obj_w + pn.y;
  const float s = 1.0f / (float)(BL * BL);
  float2 cacc[E];
#pragma unroll
  for (int j = 0; j < E; ++j) cacc[j] = make_float2(0.f, 0.f);
  for (int k = 0; k < b.K; ++k) {
    const float2* row = b.W + ((size_t)c * b.K + k) * MM + (size_t)y * BL;
    float2 a[E];
#pragma unroll
    for (int r = 0; r < E; ++r) a[r] = row[line_freq<BL>(t, r)];
    line_fft<BL, true>(a, s_sw[li], s_tw, t);
    const float2* Pk = b.P + (size_t)k * MM + (size_t)y * BL;
    float2* pacc = b.pacc + ((size_t)c * b.K + k) * MM + (size_t)y * BL;
    // pc-DM: psi_n <- psi_n + Pi_F(chi) - P o_n, the overlap step takes psi_n - P o_n (its probe
    // sums follow the object step)
    float2* St = b.psi ? b.psi + ((size_t)n * b.K + k) * MM + (size_t)y * BL : nullptr;
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int x = t + 16 * j;
      float2 psi_new = cscale(a[j], s);
      if (!NEAR && ((y + x) & 1)) psi_new = make_float2(-psi_new.x, -psi_new.y);
      const float2 p = Pk[x], o = On[x];
      float2 dpsi = csub(psi_new, cmul(p, o));
      if (St) {
        const float2 ov = cmul(p, o);
        const float2 st = cadd(b.dm_init ? ov : St[x], dpsi);
        St[x] = st;
        dpsi = csub(st, ov);
      }
      cacc[j] = cadd(cacc[j], cconjmul(p, dpsi));
      if (!St) {
        const float2 pc = cconjmul(o, dpsi);
        if (first) pacc[x] = pc;
        else red_add(&pacc[x], pc);
      }
    }
  }
  float2* cn = b.cn + (size_t)n * MM + (size_t)y * BL;
  float* dacc = b.dacc + (size_t)c * MM + (size_t)y * BL;
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int x = t + 16 * j;
    cn[x] = cacc[j];
    const float o2 = cabs2(On[x]);
    if (first) dacc[x] = o2;
    else red_add(&dacc[x], o2);
  }
}

template <int BL>
static size_t big_cols_smem() {
  constexpr int LINES = BigShape<BL>::LINES;
  return sizeof(float2) * ((size_t)BL * (LINES + 1) + BigShape<BL>::TWN + (size_t)LINES * BigShape<BL>::SWN + BL);
}

int big_row_blocks(int M) { return M / RB; }

template <int BL, int KH>
constexpr size_t big_mod_smem() { return sizeof(float) * 2 * (size_t)(RB + 2 * KH) * BL; }

// the passes of one chunk; `full` false stops after the modulus pass (pc-DM first sweep)
template <int BL>
static cudaError_t big_passes(const BigArgs& b, int nc, bool full, cudaStream_t s) {
  constexpr int LINES = BigShape<BL>::LINES, LROW = BigShape<BL>::LROW;
  const dim3 blk(LINES * BT), rblk(LROW * BT);
  const dim3 grow(BL / LROW, b.K, nc), gcol(BL / LINES, b.K, nc), gfin(BL / LROW, nc), gmod(BL / RB, nc);
  const size_t cs = big_cols_smem<BL>();
  cudaError_t e;
  for (auto kern : {k_big_cols<BL, 0>, k_big_cols<BL, 1>, k_big_cols<BL, 2>, k_big_cols<BL, 3>})
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs)) != cudaSuccess)
      return e;
  if ((e = cudaFuncSetAttribute(k_big_modulus<BL, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)big_mod_smem<BL, 5>())) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(k_big_modulus<BL, 15>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)big_mod_smem<BL, 15>())) != cudaSuccess)
    return e;
  if (b.near_field) {
    k_big_rows<BL, 0, true><<<grow, rblk, 0, s>>>(b);
    k_big_cols<BL, 2><<<gcol, blk, cs, s>>>(b);
    k_big_rows<BL, 2, true><<<grow, rblk, 0, s>>>(b);
  } else {
    k_big_rows<BL, 0, false><<<grow, rblk, 0, s>>>(b);
    k_big_cols<BL, 0><<<gcol, blk, cs, s>>>(b);
  }
  if (b.kh == 5) k_big_modulus<BL, 5><<<gmod, 256, big_mod_smem<BL, 5>(), s>>>(b);
  else k_big_modulus<BL, 15><<<gmod, 256, big_mod_smem<BL, 15>(), s>>>(b);
  if (!full) return cudaGetLastError();
  if (b.near_field) {
    k_big_rows<BL, 1, true><<<grow, rblk, 0, s>>>(b);
    k_big_cols<BL, 3><<<gcol, blk, cs, s>>>(b);
    k_big_final<BL, true><<<gfin, rblk, 0, s>>>(b);
  } else {
    k_big_cols<BL, 1><<<gcol, blk, cs, s>>>(b);
    k_big_final<BL, false><<<gfin, rblk, 0, s>>>(b);
  }
  return cudaGetLastError();
}

static cudaError_t big_dispatch(const BigArgs& b, int nc, bool full, cudaStream_t s) {
  if (b.M == 256) return big_passes<256>(b, nc, full, s);
  if (b.M == 512) return big_passes<512>(b, nc, full, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_big_chunk(const BigArgs& b, int nc, cudaStream_t s) { return big_dispatch(b, nc, true, s); }

cudaError_t launch_big_chunk_dm(const BigArgs& b, int nc, cudaStream_t s) {
  if (!b.psi) return cudaErrorInvalidValue;
  BigArgs e = b;
  e.dm_pass = 1;  // the estimate P o_n through the propagation and the model, for the error only
  cudaError_t err = big_dispatch(e, nc, false, s);
  if (err != cudaSuccess) return err;
  e.dm_pass = 2;  // chi = 2 P o_n - psi_n: its modulus ratio, back-propagation, state update
  return big_dispatch(e, nc, true, s);
}

}  // namespace ptycho
