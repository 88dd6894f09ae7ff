// Warm-start network: a 4-level U-Net on the tcgen05 BF16 GEMM (unet_gemm.cu).
// The paper has no learned component; this network seeds the engine with an
// estimate of the object patch (amplitude, phase) and of the coherence blur
// width sigma from each measured pattern.
//
//   a0 = relu(conv(x, 1 -> C))          S      p0 = avgpool2(a0)
//   a1 = relu(conv(p0, C -> 2C))        S/2    p1 = avgpool2(a1)
//   a2 = relu(conv(p1, 2C -> 4C))       S/4    p2 = avgpool2(a2)
//   a3 = relu(conv(p2, 4C -> 8C))       S/8
//   a4 = relu(conv([up2(a3), a2], 12C -> 4C))  S/4
//   a5 = relu(conv([up2(a4), a1], 6C -> 2C))   S/2
//   out = conv(a5, 2C -> 2)             S/2    sigma = mean_hw(a3) . w7 + b7
//   loss = mean((out - target)^2) + lam mean((sigma - sigma_t)^2)
//
// Convolutions are 'same' 3x3 correlations, NHWC bf16 activations, FP32
// accumulation. Forward and data-gradient contractions gather their operand
// straight from the activation tensor (implicit GEMM; the data gradient is the
// convolution of dY with the tap-flipped, transposed weights); the weight
// gradient contracts a transposed neighbourhood matrix (with a row of ones,
// which yields the bias gradient) with the transposed dY. Master weights and
// Adam moments are FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "engine.h"
#include "ptycho.h"

namespace ptycho {
ptycho_status capi_fail(ptycho_status s, const std::string& msg);
ptycho_status capi_cuda_fail(cudaError_t e, const char* what);
bool capi_is_device_pointer(const void* p);
}  // namespace ptycho

using namespace ptycho;

namespace {

using bf16 = __nv_bfloat16;

constexpr int pad_to(int v, int m) { return (v + m - 1) / m * m; }
constexpr int kMaxBatch = 1024;  // samples per call (the sigma head keeps one value per sample in shared memory)

// ---------------------------------------------------------------- elementwise kernels
// the explicit 3x3 neighbourhood of the network's input for the first layer's 1 x 1 form: channel t of
// pixel (b, y, x) = x(b, y + dy, x + dx), t = 3 (dy + 1) + dx + 1, zero outside the image; channels 9 .. 15
// zero (the same bf16 rounding as the 8-channel copy)
__global__ void k_input_nbhd(const float* x, bf16* out, int n, int S) {
  const size_t npix = (size_t)n * S * S;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < npix; i += (size_t)gridDim.x * blockDim.x) {
    const int xx = (int)(i % S), yy = (int)((i / S) % S);
    const size_t img = i - (size_t)yy * S - xx;
    __nv_bfloat16 v[16];
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int y2 = yy + t / 3 - 1, x2 = xx + t % 3 - 1;
      const bool in = t < 9 && y2 >= 0 && y2 < S && x2 >= 0 && x2 < S;
      v[t] = __float2bfloat16(in ? x[img + (size_t)y2 * S + x2] : 0.f);
    }
    uint4* o = reinterpret_cast<uint4*>(out + i * 16);
    o[0] = *reinterpret_cast<const uint4*>(&v[0]);
    o[1] = *reinterpret_cast<const uint4*>(&v[8]);
  }
}

// the first layer's weights for the 1 x 1 form: w0n[o][t] = wb[o][8 t] (channel 0 of tap t), t < 9
__global__ void k_w0_nbhd(const bf16* wb, bf16* w0n, int Cp, int Kf) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Cp * 16; i += gridDim.x * blockDim.x) {
    const int o = i / 16, t = i % 16;
    w0n[i] = t < 9 ? wb[(size_t)o * Kf + 8 * t] : __float2bfloat16(0.f);
  }
}

__global__ void k_input(const float* x, bf16* out, size_t npix) {
  // x (n, S, S) -> (n, S, S, 8) with the value in channel 0; one pixel (16 bytes) per thread
  uint4* out4 = reinterpret_cast<uint4*>(out);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < npix; i += (size_t)gridDim.x * blockDim.x) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x[i], 0.f);
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    v.x = *reinterpret_cast<const uint32_t*>(&h);
    out4[i] = v;
  }
}

// 8 bf16 <-> 8 floats
__device__ __forceinline__ void bf8_to_f(const uint4& v, float (&f)[8]) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 t = __bfloat1622float2(h[i]);
    f[2 * i] = t.x;
    f[2 * i + 1] = t.y;
  }
}
__device__ __forceinline__ uint4 f_to_bf8(const float (&f)[8]) {
  uint4 v;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
  return v;
}

// 2 x 2 average pooling, 8 channels (16 bytes) per thread; C % 8 == 0
__global__ void k_avgpool2(const bf16* in, bf16* out, int n, int H, int W, int C) {
  const int C8 = C / 8;
  const size_t total = (size_t)n * (H / 2) * (W / 2) * C8;
  const uint4* in4 = reinterpret_cast<const uint4*>(in);
  uint4* out4 = reinterpret_cast<uint4*>(out);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int c = i % C8;
    size_t r = i / C8;
    const int x = r % (W / 2);
    r /= (W / 2);
    const int y = r % (H / 2);
    const int b = r / (H / 2);
    const size_t base = (((size_t)b * H + 2 * y) * W + 2 * x) * C8 + c;
    float a[8], t[8];
    bf8_to_f(in4[base], a);
    bf8_to_f(in4[base + C8], t);
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] += t[k];
    bf8_to_f(in4[base + (size_t)W * C8], t);
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] += t[k];
    bf8_to_f(in4[base + (size_t)W * C8 + C8], t);
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = 0.25f * (a[k] + t[k]);
    out4[i] = f_to_bf8(a);
  }
}

// q = [up2(a), skip]: a (n, H/2, W/2, Ca), skip (n, H, W, Cs) -> q (n, H, W, Ca + Cs); 8 channels per thread
__global__ void k_up2_concat(const bf16* a, const bf16* skip, bf16* q, int n, int H, int W, int Ca, int Cs) {
  const int A8 = Ca / 8, S8 = Cs / 8, Q8 = A8 + S8;
  const size_t total = (size_t)n * H * W * Q8;
  const uint4* a4 = reinterpret_cast<const uint4*>(a);
  const uint4* s4 = reinterpret_cast<const uint4*>(skip);
  uint4* q4 = reinterpret_cast<uint4*>(q);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int c = i % Q8;
    const size_t p = i / Q8;
    const int x = p % W, y = (p / W) % H, b = p / ((size_t)W * H);
    q4[i] = c < A8 ? a4[(((size_t)b * (H / 2) + y / 2) * (W / 2) + x / 2) * A8 + c] : s4[p * S8 + (c - A8)];
  }
}

// out (n, h, w, Ca) = bf16( (sum of the 2x2 children of dq[..., :Ca]) + extra[b][c] ) * (act > 0);
// skip (n, 2h, 2w, Cq - Ca) = dq[..., Ca:]  (FP32 copy, if skip != nullptr)
__global__ void k_up2_bwd_mask(const float* dq, int Cq, int Ca, const float* extra, const bf16* act, bf16* out,
                               float* skip, int n, int h, int w) {
  const size_t total = (size_t)n * h * w * Ca;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int c = i % Ca;
    const size_t p = i / Ca;
    const int x = p % w, y = (p / w) % h, b = p / ((size_t)w * h);
    const size_t f = (((size_t)b * 2 * h + 2 * y) * 2 * w + 2 * x) * Cq + c;
    float s = dq[f] + dq[f + Cq] + dq[f + (size_t)2 * w * Cq] + dq[f + (size_t)2 * w * Cq + Cq];
    if (extra) s += extra[(size_t)b * Ca + c];
    out[i] = __float2bfloat16(__bfloat162float(act[i]) > 0.f ? s : 0.f);
  }
  const int Cs = Cq - Ca;
  if (skip) {
    const size_t ts = (size_t)n * 2 * h * 2 * w * Cs;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < ts; i += (size_t)gridDim.x * blockDim.x)
      skip[i] = dq[(i / Cs) * Cq + Ca + i % Cs];
  }
}

// out (n, H, W, C) = bf16( (dp[b][y/2][x/2][c] / 4 + skip) * (act > 0) )
__global__ void k_pool_bwd_mask(const float* dp, const float* skip, const bf16* act, bf16* out, int n, int H, int W,
                                int C) {
  const size_t total = (size_t)n * H * W * C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int c = i % C;
    const size_t p = i / C;
    const int x = p % W, y = (p / W) % H, b = p / ((size_t)W * H);
    float s = 0.25f * dp[(((size_t)b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c];
    if (skip) s += skip[i];
    out[i] = __float2bfloat16(__bfloat162float(act[i]) > 0.f ? s : 0.f);
  }
}

// out = bf16(d * (act > 0)), d with row stride ld (first C channels)
__global__ void k_mask(const float* d, const bf16* act, bf16* out, size_t npix, int C) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < npix * C; i += (size_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16(__bfloat162float(act[i]) > 0.f ? d[i] : 0.f);
}

// colT[k][p] of the zero-padded 3x3 neighbourhoods of X (n, H, W, Cin): k = tap * Cin + c < 9 Cin,
// a row of ones at k = 9 Cin, zeros above. 32 x 32 tiles through shared memory.
__global__ void k_im2colT(const bf16* X, bf16* colT, int n, int H, int W, int Cin, int Kw) {
  __shared__ bf16 tile[32][33];
  const int M = n * H * W;
  const int p0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // (32, 8)
  // load: tile[pixel][k]
  for (int r = ty; r < 32; r += 8) {
    const int p = p0 + r, k = k0 + tx;
    float v = 0.f;
    if (p < M) {
      if (k < 9 * Cin) {
        const int tap = k / Cin, c = k - tap * Cin;
        const int x = p % W, y = (p / W) % H, b = p / (W * H);
        const int yy = y + tap / 3 - 1, xx = x + tap % 3 - 1;
        if (yy >= 0 && yy < H && xx >= 0 && xx < W) v = __bfloat162float(X[(((size_t)b * H + yy) * W + xx) * Cin + c]);
      } else if (k == 9 * Cin) {
        v = 1.f;
      }
    }
    tile[r][tx] = __float2bfloat16(v);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int k = k0 + r, p = p0 + tx;
    if (k < Kw && p < M) colT[(size_t)k * M + p] = tile[tx][r];
  }
}

// XT3[d][c][p] = X[p + d - 1][c] when pixel x + d - 1 lies in [0, W), else 0 (d = 0, 1, 2);
// X (Mpix, Cin) NHWC; 32 pixels x 32 channels per block through shared memory
__global__ void k_shift3T(const bf16* X, bf16* XT3, int Mpix, int W, int Cin) {
  __shared__ bf16 tile[34][33];
  const int p0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int i = threadIdx.y * 32 + threadIdx.x; i < 34 * 32; i += 256) {
    const int j = i / 32, c = c0 + i % 32, p = p0 - 1 + j;
    tile[j][i % 32] = (p >= 0 && p < Mpix && c < Cin) ? X[(size_t)p * Cin + c] : __float2bfloat16(0.f);
  }
  __syncthreads();
  const int j = threadIdx.x, p = p0 + j, x = p % W;
  for (int cc = threadIdx.y; cc < 32; cc += 8) {
    const int c = c0 + cc;
    if (c >= Cin || p >= Mpix) continue;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int xx = x + d - 1;
      XT3[((size_t)d * Cin + c) * Mpix + p] = (xx >= 0 && xx < W) ? tile[j + d][cc] : __float2bfloat16(0.f);
    }
  }
}

// out[o] = sum over p of dYT[o][p] in a fixed order (one block per output channel)
__global__ void k_bias_grad(const bf16* dYT, int M, float* out) {
  __shared__ float red[256];
  const int o = blockIdx.x;
  float s = 0.f;
  for (int p = threadIdx.x; p < M; p += 256) s += __bfloat162float(dYT[(size_t)o * M + p]);
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[(size_t)o] = red[0];
}

// dst[c][r] = src[r][c], bf16, R x C
__global__ void k_transpose(const bf16* src, bf16* dst, int R, int C) {
  __shared__ bf16 tile[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int rr = r0 + r, cc = c0 + threadIdx.x;
    tile[r][threadIdx.x] = (rr < R && cc < C) ? src[(size_t)rr * C + cc] : __float2bfloat16(0.f);
  }
  __syncthreads();
  for (int c = threadIdx.y; c < 32; c += 8) {
    const int cc = c0 + c, rr = r0 + threadIdx.x;
    if (rr < R && cc < C) dst[(size_t)cc * R + rr] = tile[threadIdx.x][c];
  }
}

// master weights -> forward operand wb [Cp][Kf] and data-gradient operand wr [Cin][Kd]:
// wr[c][t * Cp + o] = w[o][(8 - t) Cin + c]
__global__ void k_weights_bf16(const float* w, bf16* wb, bf16* wr, int Cp, int Cin, int Kw, int Kf, int Kd) {
  const int total_b = Cp * Kf, total_r = Cin * Kd;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total_b + total_r; i += gridDim.x * blockDim.x) {
    if (i < total_b) {
      const int o = i / Kf, k = i % Kf;
      wb[i] = __float2bfloat16(k < 9 * Cin ? w[(size_t)o * Kw + k] : 0.f);
    } else if (wr) {
      const int j = i - total_b;
      const int c = j / Kd, kk = j % Kd;
      float v = 0.f;
      if (kk < 9 * Cp) {
        const int t = kk / Cp, o = kk % Cp;
        v = w[(size_t)o * Kw + (8 - t) * Cin + c];
      }
      wr[j] = __float2bfloat16(v);
    }
  }
}

// out (Mo, 16) fp32, first 2 channels used; target (Mo, 2). d_out bf16 (Mo, 16); per-block loss partials
__global__ void k_loss(const float* out, const float* target, bf16* d_out, float* partial, int Mo) {
  __shared__ float red[256];
  float s = 0.f;
  const float inv = 1.0f / (2.0f * Mo);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Mo * 16; i += gridDim.x * blockDim.x) {
    const int p = i / 16, c = i % 16;
    float g = 0.f;
    if (c < 2) {
      const float d = out[i] - target[p * 2 + c];
      s += d * d;
      g = 2.f * d * inv;
    }
    d_out[i] = __float2bfloat16(g);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0] * inv;
}

// g[b][c] = mean over the hw pixels of a3[b, :, :, c]; one block per sample
// mean over the pixels of each sample's channels: block b, thread (phase, c) sums the pixels p = phase (mod 4)
// with four independent accumulators; the four phases are added in order (a fixed summation order)
constexpr int kPoolPhases = 4;
__global__ void __launch_bounds__(1024) k_sigma_pool(const bf16* a3, float* g, int hw, int C8) {
  __shared__ float part[kPoolPhases][256];
  const int b = blockIdx.x;
  const int phase = threadIdx.x / 256, c0 = threadIdx.x % 256;
  for (int cb = 0; cb < C8; cb += 256) {  // the same trip count in every thread (barriers inside)
    const int c = cb + c0;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    int u = 0;
    if (c < C8)
      for (int p = phase; p < hw; p += kPoolPhases, u = (u + 1) & 3)
        s[u] += __bfloat162float(a3[((size_t)b * hw + p) * C8 + c]);
    part[phase][c0] = (s[0] + s[1]) + (s[2] + s[3]);
    __syncthreads();
    if (phase == 0 && c < C8)
      g[(size_t)b * C8 + c] = (((part[0][c0] + part[1][c0]) + part[2][c0]) + part[3][c0]) / hw;
    __syncthreads();
  }
}

// sigma head, forward and backward, one block (g from k_sigma_pool): sigma = g . w7 + b7
__global__ void k_sigma_head(const float* w7, const float* b7, const float* sigma_t, float lam, float* sigma,
                             const float* g, float* extra, float* gw7, float* gb7, float* loss_s, int n, int hw,
                             int C8, int backward) {
  __shared__ float ds[kMaxBatch];
  for (int b = threadIdx.x; b < n; b += blockDim.x) {
    // the sum in channel order; 16-byte loads (C8 % 4 == 0), several in flight
    float s = b7[0];
    const float4* gr = reinterpret_cast<const float4*>(g + (size_t)b * C8);
    const float4* wr = reinterpret_cast<const float4*>(w7);
#pragma unroll 8
    for (int c4 = 0; c4 < C8 / 4; ++c4) {
      const float4 gv = gr[c4], wv = wr[c4];
      s += gv.x * wv.x;
      s += gv.y * wv.y;
      s += gv.z * wv.z;
      s += gv.w * wv.w;
    }
    sigma[b] = s;
    ds[b] = sigma_t ? 2.f * lam * (s - sigma_t[b]) / n : 0.f;
  }
  __syncthreads();
  if (!backward) return;
  if (threadIdx.x == 0) {
    float l = 0.f, gb = 0.f;
    for (int b = 0; b < n; ++b) {
      const float d = sigma[b] - sigma_t[b];
      l += lam * d * d / n;
      gb += ds[b];
    }
    *loss_s = l;
    gb7[0] = gb;
  }
  for (int c = threadIdx.x; c < C8; c += blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < n; ++b) s += ds[b] * g[b * C8 + c];
    gw7[c] = s;
  }
  for (int bc = threadIdx.x; bc < n * C8; bc += blockDim.x) extra[bc] = ds[bc / C8] * w7[bc % C8] / hw;
}

// Adam on a weight tensor whose gradient is stored transposed: grad(o, k) = gT[k * Cp + o];
// the bias gradient is row 9 Cin of gT
__global__ void k_adam_conv(float* w, float* b, float* mw, float* vw, float* mb, float* vb, const float* gT, int Cp,
                            int Cout, int Cin, int Kw, float lr, float c1, float c2) {
  const int nk = 9 * Cin;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Cout * (nk + 1); i += gridDim.x * blockDim.x) {
    const int o = i / (nk + 1), k = i % (nk + 1);
    const float gr = gT[(size_t)k * Cp + o];
    float* pw = k < nk ? &w[(size_t)o * Kw + k] : &b[o];
    float* pm = k < nk ? &mw[(size_t)o * Kw + k] : &mb[o];
    float* pv = k < nk ? &vw[(size_t)o * Kw + k] : &vb[o];
    const float m = 0.9f * *pm + 0.1f * gr, v = 0.999f * *pv + 0.001f * gr * gr;
    *pm = m;
    *pv = v;
    *pw -= lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
  }
}

__global__ void k_adam_plain(float* w, float* m, float* v, const float* g, int n, float lr, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float mm = 0.9f * m[i] + 0.1f * g[i], vv = 0.999f * v[i] + 0.001f * g[i] * g[i];
    m[i] = mm;
    v[i] = vv;
    w[i] -= lr * (mm / c1) / (sqrtf(vv / c2) + 1e-8f);
  }
}

// out (Mo, 16) fp32 -> (Mo, 2)
__global__ void k_extract2(const float* out, float* dst, int Mo) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Mo * 2; i += gridDim.x * blockDim.x)
    dst[i] = out[(i / 2) * 16 + i % 2];
}

// out[i] = sum over z (in order) of part[z count + i]
__global__ void k_sum_splits(const float* part, int ks, size_t count, float* out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < ks; ++z) s += part[(size_t)z * count + i];
    out[i] = s;
  }
}

int grid_for(size_t n) { return (int)std::min<size_t>(4096, (n + 255) / 256); }

// split-K plan of a weight-gradient contraction (output Kw x Cp, contraction over npx pixels):
// enough CTAs to fill the GPU about four times over, at least 4 chunks of 64 per split
struct Split {
  int ks, kc;
};
Split wgrad_split(int Kw, int Cp, int npx) {
  int nt = 16;
  for (int c : {256, 128, 64, 32}) {
    if (Cp % c == 0) {
      nt = c;
      break;
    }
  }
  const int tiles = (Kw / 128) * (Cp / nt);
  const int chunks = npx / 64;
  int ks = std::max(1, std::min((4 * 152 + tiles - 1) / tiles, chunks / 4));
  const int per = (chunks + ks - 1) / ks;
  Split sp;
  sp.kc = per * 64;
  sp.ks = (chunks + per - 1) / per;
  return sp;
}

struct Conv {
  int Cin, Cout, Cp, H, W;  // stored input channels, output channels, stored output channels, spatial size
  int Kf, Kw, Kd;
  bool relu;
  float *w, *b, *mw, *vw, *mb, *vb, *gT;
  bf16 *wb, *wr;
  bf16 *wbp, *wrp;  // wb and wr in the halo kernel's step order (forward and data-gradient convolutions)
};

}  // namespace

struct ptycho_unet_s {
  int S, C, n;
  int nrun;  // samples the next forward / backward runs on (<= n)
  int device;
  cudaStream_t stream;
  std::vector<void*> allocs;
  Conv L[7];
  float *w7, *b7, *gw7, *gb7, *mw7, *vw7, *mb7, *vb7;
  // activations (bf16) and buffers
  bf16 *x, *a0, *p0, *a1, *p1, *a2, *p2, *a3, *q2, *a4, *q1, *a5;
  // the first layer as a 1 x 1 contraction over the explicit neighbourhood: input (n, S, S, 16), weights
  // (Cp, 16) and their packed copy
  bf16 *xn, *w0n, *w0np;
  float *out, *g, *sigma, *extra, *loss_part, *loss_s;
  bf16 *d_out, *dY, *dYT, *colT, *xt3;
  float *dX, *skip1, *skip2;
  float* wpart;  // split-K partial weight gradients
  int* status;
  bool wb_fresh = false;  // the bf16 weight copies match the FP32 masters
  // the warm start's scratch (patches, sigmas, inputs, tile lists): grown on demand, kept across calls so
  // that a warmed-up estimate allocates nothing (an allocation synchronises the device)
  void* ws_buf = nullptr;
  size_t ws_bytes = 0;
  long long step = 0;

  template <class T>
  cudaError_t alloc(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) {
      allocs.push_back(q);
      cudaMemsetAsync(q, 0, std::max<size_t>(count, 1) * sizeof(T), stream);
    }
    *p = static_cast<T*>(q);
    return e;
  }
  ~ptycho_unet_s() {
    for (void* q : allocs) cudaFree(q);
    if (ws_buf) cudaFree(ws_buf);
  }
};

namespace {

#define UN_CUDA(call, what)                                  \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return capi_cuda_fail(e_, what);  \
  } while (0)

GemmArgs gemm_args(ptycho_unet_s* u, const void* A, const void* B, void* D, int M, int N, int K, int ldd, int mode,
                   const float* bias, int relu, const Conv* conv, Split sp = Split{1, 0}, const bf16* Bp = nullptr) {
  GemmArgs g{};
  g.ksplit = sp.ks;
  g.kc = sp.kc;
  g.dsplit = (size_t)M * ldd;
  g.A = static_cast<const uint16_t*>(A);
  g.B = static_cast<const uint16_t*>(B);
  if (mode == 2) g.Dh = static_cast<uint16_t*>(D);
  else g.D = static_cast<float*>(D);
  g.bias = bias;
  g.M = M;
  g.Ntot = N;
  g.K = K;
  g.ldd = ldd;
  g.mode = mode;
  g.relu = relu;
  g.status = u->status;
  if (conv) {
    g.conv = 1;
    g.H = conv->H;
    g.W = conv->W;
    g.Cin = conv->Cin;
  }
  g.Bp = reinterpret_cast<const uint16_t*>(Bp);
  return g;
}

cudaError_t gemm(ptycho_unet_s* u, const void* A, const void* B, void* D, int M, int N, int K, int ldd, int mode,
                 const float* bias, int relu, const Conv* conv, Split sp = Split{1, 0}, const bf16* Bp = nullptr) {
  return launch_gemm_bf16(gemm_args(u, A, B, D, M, N, K, ldd, mode, bias, relu, conv, sp, Bp), u->stream);
}

// weight-gradient contraction over the transposed shifted copies (GemmArgs::convT)
cudaError_t gemm_wgrad_T(ptycho_unet_s* u, const Conv& L, const bf16* XT3, const bf16* dYT, float* D, int M, Split sp) {
  GemmArgs g{};
  g.A = reinterpret_cast<const uint16_t*>(XT3);
  g.B = reinterpret_cast<const uint16_t*>(dYT);
  g.D = D;
  g.M = L.Kw;
  g.Ntot = L.Cp;
  g.K = M;
  g.ldd = L.Cp;
  g.mode = 0;
  g.status = u->status;
  g.ksplit = sp.ks;
  g.kc = sp.kc;
  g.dsplit = (size_t)L.Kw * L.Cp;
  g.convT = 1;
  g.Mpix = M;
  g.H = L.H;
  g.W = L.W;
  g.Cin = L.Cin;
  return launch_gemm_bf16(g, u->stream);
}

// forward of one convolution: out (n, H, W, Cp) bf16 with bias and ReLU, or fp32 without bias
// the first layer: the 1 x 1 form over the explicit neighbourhood (bias, ReLU, bf16 out)
GemmArgs input_layer_args(ptycho_unet_s* u, bf16* out) {
  const Conv& L = u->L[0];
  Conv R = L;
  R.Cin = 16;
  GemmArgs g = gemm_args(u, u->xn, u->w0n, out, u->nrun * L.H * L.W, L.Cp, 16, L.Cp, 2, L.b, L.relu ? 1 : 0, &R,
                         Split{1, 0}, u->w0np);
  g.taps1 = 1;
  return g;
}

cudaError_t conv_forward(ptycho_unet_s* u, Conv& L, const bf16* in, bf16* out_bf16, float* out_f32) {
  const int M = u->nrun * L.H * L.W;
  if (out_bf16) return gemm(u, in, L.wb, out_bf16, M, L.Cp, L.Kf, L.Cp, 2, L.b, L.relu ? 1 : 0, &L, Split{1, 0}, L.wbp);
  return gemm(u, in, L.wb, out_f32, M, L.Cp, L.Kf, L.Cp, 0, L.b, 0, &L, Split{1, 0}, L.wbp);  // FP32 + bias
}

// backward of one convolution given dY (n, H, W, Cp) bf16: weight gradient (into L.gT) and, when dX != nullptr,
// the data gradient dX (n, H, W, Cin) fp32
cudaError_t conv_backward(ptycho_unet_s* u, Conv& L, const bf16* in, const bf16* dY, float* dX) {
  const int M = u->nrun * L.H * L.W;
  cudaStream_t s = u->stream;
  k_transpose<<<dim3((M + 31) / 32, (L.Cp + 31) / 32), dim3(32, 8), 0, s>>>(dY, u->dYT, M, L.Cp);
  const Split sp = wgrad_split(L.Kw, L.Cp, M);
  const bool shifted = L.W % 8 == 0;  // transposed shifted copies (else the explicit neighbourhood matrix)
  cudaError_t e;
  if (shifted)
    k_shift3T<<<dim3(M / 32, (L.Cin + 31) / 32), dim3(32, 8), 0, s>>>(in, u->xt3, M, L.W, L.Cin);
  else
    k_im2colT<<<dim3((M + 31) / 32, L.Kw / 32), dim3(32, 8), 0, s>>>(in, u->colT, u->nrun, L.H, L.W, L.Cin, L.Kw);
  float* D = sp.ks > 1 ? u->wpart : L.gT;
  if (shifted) e = gemm_wgrad_T(u, L, u->xt3, u->dYT, D, M, sp);
  else e = gemm(u, u->colT, u->dYT, D, L.Kw, L.Cp, M, L.Cp, 0, nullptr, 0, nullptr, sp);
  if (e != cudaSuccess) return e;
  if (sp.ks > 1) k_sum_splits<<<grid_for((size_t)L.Kw * L.Cp), 256, 0, s>>>(u->wpart, sp.ks, (size_t)L.Kw * L.Cp, L.gT);
  // bias gradient (row 9 Cin of gT); the explicit matrix's row of ones already produced it
  if (shifted) k_bias_grad<<<L.Cp, 256, 0, s>>>(u->dYT, M, L.gT + (size_t)9 * L.Cin * L.Cp);
  if (e != cudaSuccess || !dX) return e;
  Conv R = L;  // the data gradient gathers dY with Cp channels
  R.Cin = L.Cp;
  return gemm(u, dY, L.wr, dX, M, L.Cin, L.Kd, L.Cin, 0, nullptr, 0, &R, Split{1, 0}, L.wrp);
}

}  // namespace


// infer: the first layer as the 1 x 1 form over the explicit neighbourhood (one K = 16 MMA per
// accumulator instead of five tap pairs); training keeps the tap-pair form, so that the trained network
// does not depend on which form inference uses (the two differ in FP32 summation order only)
static cudaError_t unet_forward(ptycho_unet_s* u, const float* x_dev, bool infer) {
  cudaStream_t s = u->stream;
  const int n = u->nrun, S = u->S, C = u->C;
  const size_t npx = (size_t)n * S * S;
  // inference reads only the explicit neighbourhood, training only the 8-channel copy
  if (infer) k_input_nbhd<<<grid_for(npx), 256, 0, s>>>(x_dev, u->xn, n, S);
  else k_input<<<grid_for(npx), 256, 0, s>>>(x_dev, u->x, npx);
  if (!u->wb_fresh) {  // bf16 copies of the FP32 master weights, redone only after the weights changed
    for (int i = 0; i < 7; ++i)
      k_weights_bf16<<<grid_for((size_t)u->L[i].Cp * u->L[i].Kf + (size_t)u->L[i].Cin * u->L[i].Kd), 256, 0, s>>>(
          u->L[i].w, u->L[i].wb, i == 0 ? nullptr : u->L[i].wr, u->L[i].Cp, u->L[i].Cin, u->L[i].Kw, u->L[i].Kf,
          u->L[i].Kd);
    // the first layer's 1 x 1 form over the explicit neighbourhood
    {
      const Conv& L = u->L[0];
      k_w0_nbhd<<<grid_for((size_t)L.Cp * 16), 256, 0, s>>>(L.wb, u->w0n, L.Cp, L.Kf);
      const cudaError_t e = halo_pack(input_layer_args(u, nullptr), reinterpret_cast<uint16_t*>(u->w0np), s);
      if (e != cudaSuccess) return e;
    }
    // and in the halo kernel's step order (forward, and the data gradient's transposed taps)
    for (int i = 0; i < 7; ++i) {
      Conv& L = u->L[i];
      const int M = u->nrun * L.H * L.W;
      const GemmArgs gf = gemm_args(u, nullptr, L.wb, nullptr, M, L.Cp, L.Kf, L.Cp, 2, L.b, 1, &L);
      if (halo_conv_supported(gf)) {
        const cudaError_t e = halo_pack(gf, reinterpret_cast<uint16_t*>(L.wbp), s);
        if (e != cudaSuccess) return e;
      }
      if (i == 0) continue;  // the input's gradient is not needed
      Conv R = L;
      R.Cin = L.Cp;
      const GemmArgs gd = gemm_args(u, nullptr, L.wr, nullptr, M, L.Cin, L.Kd, L.Cin, 0, nullptr, 0, &R);
      if (halo_conv_supported(gd)) {
        const cudaError_t e = halo_pack(gd, reinterpret_cast<uint16_t*>(L.wrp), s);
        if (e != cudaSuccess) return e;
      }
    }
    u->wb_fresh = true;
  }
  cudaError_t e;
  if (infer) {
    if ((e = launch_gemm_bf16(input_layer_args(u, u->a0), u->stream)) != cudaSuccess) return e;
  } else if ((e = conv_forward(u, u->L[0], u->x, u->a0, nullptr)) != cudaSuccess) {
    return e;
  }
  k_avgpool2<<<grid_for(npx * C / 32), 256, 0, s>>>(u->a0, u->p0, n, S, S, C);
  if ((e = conv_forward(u, u->L[1], u->p0, u->a1, nullptr)) != cudaSuccess) return e;
  k_avgpool2<<<grid_for(npx * C / 64), 256, 0, s>>>(u->a1, u->p1, n, S / 2, S / 2, 2 * C);
  if ((e = conv_forward(u, u->L[2], u->p1, u->a2, nullptr)) != cudaSuccess) return e;
  k_avgpool2<<<grid_for(npx * C / 128), 256, 0, s>>>(u->a2, u->p2, n, S / 4, S / 4, 4 * C);
  if ((e = conv_forward(u, u->L[3], u->p2, u->a3, nullptr)) != cudaSuccess) return e;
  k_up2_concat<<<grid_for(npx * 12 * C / 128), 256, 0, s>>>(u->a3, u->a2, u->q2, n, S / 4, S / 4, 8 * C, 4 * C);
  if ((e = conv_forward(u, u->L[4], u->q2, u->a4, nullptr)) != cudaSuccess) return e;
  k_up2_concat<<<grid_for(npx * 6 * C / 32), 256, 0, s>>>(u->a4, u->a1, u->q1, n, S / 2, S / 2, 4 * C, 2 * C);
  if ((e = conv_forward(u, u->L[5], u->q1, u->a5, nullptr)) != cudaSuccess) return e;
  if ((e = conv_forward(u, u->L[6], u->a5, nullptr, u->out)) != cudaSuccess) return e;  // bias in its epilogue
  return cudaGetLastError();
}

// loss and every gradient for one batch (after unet_forward)
static cudaError_t unet_backward(ptycho_unet_s* u, const float* target, const float* sigma_t, float lam) {
  cudaStream_t s = u->stream;
  const int n = u->nrun, S = u->S, C = u->C;
  const int Mo = n * (S / 2) * (S / 2);
  k_loss<<<64, 256, 0, s>>>(u->out, target, u->d_out, u->loss_part, Mo);
  k_sigma_pool<<<n, 1024, 0, s>>>(u->a3, u->g, (S / 8) * (S / 8), 8 * C);
  k_sigma_head<<<1, kMaxBatch, 0, s>>>(u->w7, u->b7, sigma_t, lam, u->sigma, u->g, u->extra, u->gw7, u->gb7,
                                  u->loss_s, n, (S / 8) * (S / 8), 8 * C, 1);
  cudaError_t e;
  // head and a5
  if ((e = conv_backward(u, u->L[6], u->a5, u->d_out, u->dX)) != cudaSuccess) return e;
  k_mask<<<grid_for((size_t)Mo * 2 * C), 256, 0, s>>>(u->dX, u->a5, u->dY, (size_t)Mo, 2 * C);
  if ((e = conv_backward(u, u->L[5], u->q1, u->dY, u->dX)) != cudaSuccess) return e;  // dX = d q1 (6C)
  k_up2_bwd_mask<<<grid_for((size_t)n * (S / 4) * (S / 4) * 4 * C), 256, 0, s>>>(
      u->dX, 6 * C, 4 * C, nullptr, u->a4, u->dY, u->skip1, n, S / 4, S / 4);
  if ((e = conv_backward(u, u->L[4], u->q2, u->dY, u->dX)) != cudaSuccess) return e;  // dX = d q2 (12C)
  k_up2_bwd_mask<<<grid_for((size_t)n * (S / 8) * (S / 8) * 8 * C), 256, 0, s>>>(
      u->dX, 12 * C, 8 * C, u->extra, u->a3, u->dY, u->skip2, n, S / 8, S / 8);
  if ((e = conv_backward(u, u->L[3], u->p2, u->dY, u->dX)) != cudaSuccess) return e;  // d p2 (4C)
  k_pool_bwd_mask<<<grid_for((size_t)n * (S / 4) * (S / 4) * 4 * C), 256, 0, s>>>(u->dX, u->skip2, u->a2, u->dY, n,
                                                                                   S / 4, S / 4, 4 * C);
  if ((e = conv_backward(u, u->L[2], u->p1, u->dY, u->dX)) != cudaSuccess) return e;  // d p1 (2C)
  k_pool_bwd_mask<<<grid_for((size_t)n * (S / 2) * (S / 2) * 2 * C), 256, 0, s>>>(u->dX, u->skip1, u->a1, u->dY, n,
                                                                                   S / 2, S / 2, 2 * C);
  if ((e = conv_backward(u, u->L[1], u->p0, u->dY, u->dX)) != cudaSuccess) return e;  // d p0 (C)
  k_pool_bwd_mask<<<grid_for((size_t)n * S * S * C), 256, 0, s>>>(u->dX, nullptr, u->a0, u->dY, n, S, S, C);
  if ((e = conv_backward(u, u->L[0], u->x, u->dY, nullptr)) != cudaSuccess) return e;
  return cudaGetLastError();
}

// forward pass and heads without synchronising: out2 (first nvalid samples) and sigma (nvalid) on the device
static cudaError_t unet_infer(ptycho_unet_s* u, const float* x, float* out2, float* sigma, int nvalid) {
  cudaError_t e = unet_forward(u, x, true);
  if (e != cudaSuccess) return e;
  k_sigma_pool<<<u->nrun, 1024, 0, u->stream>>>(u->a3, u->g, (u->S / 8) * (u->S / 8), 8 * u->C);
  k_sigma_head<<<1, kMaxBatch, 0, u->stream>>>(u->w7, u->b7, nullptr, 0.f, u->sigma, u->g, u->extra, u->gw7,
                                               u->gb7, u->loss_s, u->nrun, (u->S / 8) * (u->S / 8), 8 * u->C, 0);
  const int Mo = nvalid * (u->S / 2) * (u->S / 2);
  if (out2) k_extract2<<<grid_for((size_t)Mo * 2), 256, 0, u->stream>>>(u->out, out2, Mo);
  if (sigma) {
    e = cudaMemcpyAsync(sigma, u->sigma, sizeof(float) * nvalid, cudaMemcpyDeviceToDevice, u->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

static ptycho_status read_loss(ptycho_unet_s* u, double* loss) {
  float part[64 + 1];
  UN_CUDA(cudaMemcpyAsync(part, u->loss_part, sizeof(float) * 64, cudaMemcpyDeviceToHost, u->stream), "copy loss");
  UN_CUDA(cudaMemcpyAsync(part + 64, u->loss_s, sizeof(float), cudaMemcpyDeviceToHost, u->stream), "copy loss");
  int st = 0;
  UN_CUDA(cudaMemcpyAsync(&st, u->status, sizeof(int), cudaMemcpyDeviceToHost, u->stream), "copy status");
  UN_CUDA(cudaStreamSynchronize(u->stream), "stream sync");
  if (st) return capi_fail(PTYCHO_ETIMEOUT, "a tensor-core wait gave up");
  double l = 0.0;
  for (int i = 0; i < 65; ++i) l += part[i];
  if (loss) *loss = l;
  return PTYCHO_OK;
}

// flat parameter order (oracle layout): for each conv i: w_i (Cout, 9, Cin_true), b_i (Cout); then w7, b7
static size_t param_count(int C) {
  const int ci[7] = {1, C, 2 * C, 4 * C, 12 * C, 6 * C, 2 * C}, co[7] = {C, 2 * C, 4 * C, 8 * C, 4 * C, 2 * C, 2};
  size_t n = 0;
  for (int i = 0; i < 7; ++i) n += (size_t)co[i] * 9 * ci[i] + co[i];
  return n + 8 * C + 1;
}

extern "C" {

ptycho_status ptycho_unet_create(int32_t S, int32_t C, int32_t batch, uint64_t seed, void* stream,
                                 ptycho_unet_t* out) {
  if (!out) return capi_fail(PTYCHO_EINVAL, "out is NULL");
  *out = nullptr;
  if (S < 16 || S % 16 || S > 512 || C < 16 || C % 16 || C > 64 || batch < 1 || batch > kMaxBatch ||
      ((size_t)batch * (S / 8) * (S / 8)) % 128)
    return capi_fail(PTYCHO_EINVAL, "need 16 <= S <= 512, S % 16 == 0, C % 16 == 0, C <= 64, 1 <= batch <= 1024 and "
                                    "batch (S/8)^2 % 128 == 0");
  // the largest activation (batch x S^2 x max(8, 1.5 C) elements) must be indexable by int
  if ((double)batch * S * S * std::max(8.0, 1.5 * C) >= 2147483647.0)
    return capi_fail(PTYCHO_EINVAL, "batch x S^2 x channels exceeds 2^31 elements");
  ptycho_unet_s* u = new (std::nothrow) ptycho_unet_s();
  if (!u) return capi_fail(PTYCHO_ENOMEM, "host allocation failed");
  u->S = S;
  u->C = C;
  u->n = batch;
  u->nrun = batch;
  u->stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&u->device);
  const int ci_s[7] = {8, C, 2 * C, 4 * C, 12 * C, 6 * C, 2 * C};
  const int ci_t[7] = {1, C, 2 * C, 4 * C, 12 * C, 6 * C, 2 * C};
  const int co[7] = {C, 2 * C, 4 * C, 8 * C, 4 * C, 2 * C, 2};
  const int hs[7] = {S, S / 2, S / 4, S / 8, S / 4, S / 2, S / 2};
  size_t colT_max = 0, xt3_max = 0, wpart_max = 0;
  auto fail_alloc = [&](cudaError_t e) {
    const ptycho_status st = capi_cuda_fail(e, "unet allocation");
    delete u;
    return st;
  };
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  for (int i = 0; i < 7; ++i) {
    Conv& L = u->L[i];
    L.Cin = ci_s[i];
    L.Cout = co[i];
    L.Cp = pad_to(co[i], 16);
    L.H = L.W = hs[i];
    L.Kf = pad_to(9 * L.Cin, 64);
    L.Kw = pad_to(9 * L.Cin + 1, 128);
    L.Kd = pad_to(9 * L.Cp, 64);
    L.relu = i < 6;
    cudaError_t e;
    if ((e = u->alloc(&L.w, (size_t)L.Cp * L.Kw)) != cudaSuccess || (e = u->alloc(&L.b, L.Cp)) != cudaSuccess ||
        (e = u->alloc(&L.mw, (size_t)L.Cp * L.Kw)) != cudaSuccess ||
        (e = u->alloc(&L.vw, (size_t)L.Cp * L.Kw)) != cudaSuccess || (e = u->alloc(&L.mb, L.Cp)) != cudaSuccess ||
        (e = u->alloc(&L.vb, L.Cp)) != cudaSuccess || (e = u->alloc(&L.gT, (size_t)L.Kw * L.Cp)) != cudaSuccess ||
        (e = u->alloc(&L.wb, (size_t)L.Cp * L.Kf)) != cudaSuccess ||
        (e = u->alloc(&L.wr, (size_t)L.Cin * L.Kd)) != cudaSuccess ||
        (e = u->alloc(&L.wbp, (size_t)L.Cp * L.Kf)) != cudaSuccess ||
        (e = u->alloc(&L.wrp, (size_t)L.Cin * L.Kd)) != cudaSuccess)
      return fail_alloc(e);
    if (hs[i] % 8) colT_max = std::max(colT_max, (size_t)L.Kw * batch * hs[i] * hs[i]);
    else xt3_max = std::max(xt3_max, (size_t)3 * L.Cin * batch * hs[i] * hs[i]);
    const Split sp = wgrad_split(L.Kw, L.Cp, batch * hs[i] * hs[i]);
    wpart_max = std::max(wpart_max, sp.ks > 1 ? (size_t)sp.ks * L.Kw * L.Cp : (size_t)0);
    // He initialisation of the true weights (channels beyond the true counts stay zero)
    std::vector<float> w((size_t)L.Cp * L.Kw, 0.f);
    const double sd = std::sqrt(2.0 / (9.0 * ci_t[i]));
    for (int o = 0; o < co[i]; ++o)
      for (int t = 0; t < 9; ++t)
        for (int c = 0; c < ci_t[i]; ++c) w[(size_t)o * L.Kw + t * L.Cin + c] = (float)(sd * nd(rng));
    cudaMemcpyAsync(L.w, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, u->stream);
  }
  const size_t n = batch;
  const size_t px = n * S * S;
  cudaError_t e;
#define UA(p, c) \
  if ((e = u->alloc(&u->p, (c))) != cudaSuccess) return fail_alloc(e)
  UA(w7, 8 * C);
  UA(b7, 1);
  UA(gw7, 8 * C);
  UA(gb7, 1);
  UA(mw7, 8 * C);
  UA(vw7, 8 * C);
  UA(mb7, 1);
  UA(vb7, 1);
  UA(x, px * 8);
  UA(xn, px * 16);
  UA(w0n, (size_t)16 * 16 * ((C + 15) / 16));
  UA(w0np, (size_t)16 * 16 * ((C + 15) / 16));
  UA(a0, px * C);
  UA(p0, px * C / 4);
  UA(a1, px * 2 * C / 4);
  UA(p1, px * 2 * C / 16);
  UA(a2, px * 4 * C / 16);
  UA(p2, px * 4 * C / 64);
  UA(a3, px * 8 * C / 64);
  UA(q2, px * 12 * C / 16);
  UA(a4, px * 4 * C / 16);
  UA(q1, px * 6 * C / 4);
  UA(a5, px * 2 * C / 4);
  UA(out, px * 16 / 4);
  UA(g, n * 8 * C);
  UA(sigma, n);
  UA(extra, n * 8 * C);
  UA(loss_part, 64);
  UA(loss_s, 1);
  UA(d_out, px * 16 / 4);
  UA(dY, px * C);
  UA(dYT, px * C);
  UA(colT, colT_max);
  UA(xt3, xt3_max);
  UA(dX, std::max(px * C, px * 6 * C / 4));
  UA(skip1, px * 2 * C / 4);
  UA(skip2, px * 4 * C / 16);
  UA(wpart, wpart_max);
  UA(status, 1);
#undef UA
  {
    std::vector<float> w7(8 * C);
    for (auto& v : w7) v = (float)(std::sqrt(1.0 / (8 * C)) * nd(rng));
    const float b7 = 1.5f;
    cudaMemcpyAsync(u->w7, w7.data(), sizeof(float) * w7.size(), cudaMemcpyHostToDevice, u->stream);
    cudaMemcpyAsync(u->b7, &b7, sizeof(float), cudaMemcpyHostToDevice, u->stream);
  }
  e = cudaStreamSynchronize(u->stream);
  if (e != cudaSuccess) return fail_alloc(e);
  *out = u;
  return PTYCHO_OK;
}

int64_t ptycho_unet_param_count(ptycho_unet_t u) { return u ? (int64_t)param_count(u->C) : 0; }

ptycho_status ptycho_unet_set_params(ptycho_unet_t u, const float* host, int64_t count) {
  if (!u || !host || count != (int64_t)param_count(u->C)) return capi_fail(PTYCHO_EINVAL, "bad parameter vector");
  u->wb_fresh = false;
  const int ci_t[7] = {1, u->C, 2 * u->C, 4 * u->C, 12 * u->C, 6 * u->C, 2 * u->C};
  size_t off = 0;
  for (int i = 0; i < 7; ++i) {
    Conv& L = u->L[i];
    std::vector<float> w((size_t)L.Cp * L.Kw, 0.f), b(L.Cp, 0.f);
    for (int o = 0; o < L.Cout; ++o)
      for (int t = 0; t < 9; ++t)
        for (int c = 0; c < ci_t[i]; ++c) w[(size_t)o * L.Kw + t * L.Cin + c] = host[off++];
    for (int o = 0; o < L.Cout; ++o) b[o] = host[off++];
    UN_CUDA(cudaMemcpyAsync(L.w, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, u->stream), "params");
    UN_CUDA(cudaMemcpyAsync(L.b, b.data(), sizeof(float) * b.size(), cudaMemcpyHostToDevice, u->stream), "params");
    UN_CUDA(cudaStreamSynchronize(u->stream), "sync");
  }
  // the sigma head's weights, ordered after any forward still reading them on the network's stream
  UN_CUDA(cudaMemcpyAsync(u->w7, host + off, sizeof(float) * 8 * u->C, cudaMemcpyHostToDevice, u->stream), "params");
  off += 8 * u->C;
  UN_CUDA(cudaMemcpyAsync(u->b7, host + off, sizeof(float), cudaMemcpyHostToDevice, u->stream), "params");
  UN_CUDA(cudaStreamSynchronize(u->stream), "sync");
  return PTYCHO_OK;
}

ptycho_status ptycho_unet_get_params(ptycho_unet_t u, float* host, int64_t count) {
  if (!u || !host || count != (int64_t)param_count(u->C)) return capi_fail(PTYCHO_EINVAL, "bad parameter vector");
  const int ci_t[7] = {1, u->C, 2 * u->C, 4 * u->C, 12 * u->C, 6 * u->C, 2 * u->C};
  UN_CUDA(cudaStreamSynchronize(u->stream), "sync");
  size_t off = 0;
  for (int i = 0; i < 7; ++i) {
    Conv& L = u->L[i];
    std::vector<float> w((size_t)L.Cp * L.Kw), b(L.Cp);
    UN_CUDA(cudaMemcpy(w.data(), L.w, sizeof(float) * w.size(), cudaMemcpyDeviceToHost), "params");
    UN_CUDA(cudaMemcpy(b.data(), L.b, sizeof(float) * b.size(), cudaMemcpyDeviceToHost), "params");
    for (int o = 0; o < L.Cout; ++o)
      for (int t = 0; t < 9; ++t)
        for (int c = 0; c < ci_t[i]; ++c) host[off++] = w[(size_t)o * L.Kw + t * L.Cin + c];
    for (int o = 0; o < L.Cout; ++o) host[off++] = b[o];
  }
  UN_CUDA(cudaMemcpy(host + off, u->w7, sizeof(float) * 8 * u->C, cudaMemcpyDeviceToHost), "params");
  off += 8 * u->C;
  UN_CUDA(cudaMemcpy(host + off, u->b7, sizeof(float), cudaMemcpyDeviceToHost), "params");
  return PTYCHO_OK;
}

ptycho_status ptycho_unet_forward(ptycho_unet_t u, const float* x, float* out2, float* sigma) {
  if (!u || !x) return capi_fail(PTYCHO_EINVAL, "NULL argument");
  UN_CUDA(cudaMemsetAsync(u->status, 0, sizeof(int), u->stream), "clear status");
  u->nrun = u->n;
  UN_CUDA(unet_infer(u, x, out2, sigma, u->n), "unet forward");
  int st = 0;
  UN_CUDA(cudaMemcpyAsync(&st, u->status, sizeof(int), cudaMemcpyDeviceToHost, u->stream), "copy status");
  UN_CUDA(cudaStreamSynchronize(u->stream), "stream sync");
  if (st) return capi_fail(PTYCHO_ETIMEOUT, "a tensor-core wait gave up");
  return PTYCHO_OK;
}

ptycho_status ptycho_unet_gradients(ptycho_unet_t u, const float* x, const float* target, const float* sigma_t,
                                    float lam, double* loss, float* grads_host) {
  if (!u || !x || !target || !sigma_t) return capi_fail(PTYCHO_EINVAL, "NULL argument");
  UN_CUDA(cudaMemsetAsync(u->status, 0, sizeof(int), u->stream), "clear status");
  u->nrun = u->n;
  UN_CUDA(unet_forward(u, x, false), "unet forward");
  UN_CUDA(unet_backward(u, target, sigma_t, lam), "unet backward");
  ptycho_status st = read_loss(u, loss);
  if (st != PTYCHO_OK || !grads_host) return st;
  const int ci_t[7] = {1, u->C, 2 * u->C, 4 * u->C, 12 * u->C, 6 * u->C, 2 * u->C};
  size_t off = 0;
  for (int i = 0; i < 7; ++i) {
    Conv& L = u->L[i];
    std::vector<float> gT((size_t)L.Kw * L.Cp);
    UN_CUDA(cudaMemcpy(gT.data(), L.gT, sizeof(float) * gT.size(), cudaMemcpyDeviceToHost), "grads");
    for (int o = 0; o < L.Cout; ++o)
      for (int t = 0; t < 9; ++t)
        for (int c = 0; c < ci_t[i]; ++c) grads_host[off++] = gT[(size_t)(t * L.Cin + c) * L.Cp + o];
    for (int o = 0; o < L.Cout; ++o) grads_host[off++] = gT[(size_t)(9 * L.Cin) * L.Cp + o];
  }
  UN_CUDA(cudaMemcpy(grads_host + off, u->gw7, sizeof(float) * 8 * u->C, cudaMemcpyDeviceToHost), "grads");
  off += 8 * u->C;
  UN_CUDA(cudaMemcpy(grads_host + off, u->gb7, sizeof(float), cudaMemcpyDeviceToHost), "grads");
  return PTYCHO_OK;
}

ptycho_status ptycho_unet_train_step(ptycho_unet_t u, const float* x, const float* target, const float* sigma_t,
                                     float lam, float lr, double* loss) {
  if (!u || !x || !target || !sigma_t) return capi_fail(PTYCHO_EINVAL, "NULL argument");
  UN_CUDA(cudaMemsetAsync(u->status, 0, sizeof(int), u->stream), "clear status");
  u->nrun = u->n;
  UN_CUDA(unet_forward(u, x, false), "unet forward");
  UN_CUDA(unet_backward(u, target, sigma_t, lam), "unet backward");
  u->step++;
  u->wb_fresh = false;  // Adam changes the FP32 masters below
  const float c1 = 1.f - std::pow(0.9f, (float)u->step), c2 = 1.f - std::pow(0.999f, (float)u->step);
  for (int i = 0; i < 7; ++i) {
    Conv& L = u->L[i];
    k_adam_conv<<<grid_for((size_t)L.Cout * (9 * L.Cin + 1)), 256, 0, u->stream>>>(
        L.w, L.b, L.mw, L.vw, L.mb, L.vb, L.gT, L.Cp, L.Cout, L.Cin, L.Kw, lr, c1, c2);
  }
  k_adam_plain<<<1, 256, 0, u->stream>>>(u->w7, u->mw7, u->vw7, u->gw7, 8 * u->C, lr, c1, c2);
  k_adam_plain<<<1, 32, 0, u->stream>>>(u->b7, u->mb7, u->vb7, u->gb7, 1, lr, c1, c2);
  UN_CUDA(cudaGetLastError(), "adam");
  if (loss) return read_loss(u, loss);
  return PTYCHO_OK;
}

ptycho_status ptycho_warmstart(ptycho_unet_t u, const float* intensities, const int32_t* positions, int32_t N,
                               int32_t obj_h, int32_t obj_w, double target_scale, void* object_out,
                               double* sigma_out) {
  if (!u || !intensities || !positions || !object_out || !sigma_out)
    return capi_fail(PTYCHO_EINVAL, "NULL argument");
  if (N < 1 || obj_h < 1 || obj_w < 1 || !(target_scale > 0.0) || N > (1 << 20))
    return capi_fail(PTYCHO_EINVAL, "need 1 <= N <= 2^20, obj_h, obj_w >= 1 and target_scale > 0");
  if (!capi_is_device_pointer(intensities) || !capi_is_device_pointer(object_out))
    return capi_fail(PTYCHO_EINVAL, "intensities and object_out must be device pointers");
  const int S = u->S, Q = S / 2;
  cudaStream_t s = u->stream;
  std::vector<int32_t> pos(2 * (size_t)N);
  if (capi_is_device_pointer(positions)) {
    UN_CUDA(cudaMemcpyAsync(pos.data(), positions, sizeof(int32_t) * pos.size(), cudaMemcpyDeviceToHost, s),
            "positions");
    UN_CUDA(cudaStreamSynchronize(s), "stream sync");
  } else {
    std::memcpy(pos.data(), positions, sizeof(int32_t) * pos.size());
  }
  for (int n = 0; n < N; ++n)
    if (pos[2 * n] < 0 || pos[2 * n + 1] < 0 || pos[2 * n] + S > obj_h || pos[2 * n + 1] + S > obj_w)
      return capi_fail(PTYCHO_EINVAL, "box " + std::to_string(n) + " lies outside the object");
  // CSR of patch corners per object tile, increasing n
  const int tx = (obj_w + kObjTile - 1) / kObjTile, ty = (obj_h + kObjTile - 1) / kObjTile;
  std::vector<int> start((size_t)tx * ty + 1, 0);
  std::vector<std::vector<int>> lists((size_t)tx * ty);
  for (int n = 0; n < N; ++n) {
    const int r0 = pos[2 * n] + S / 4, c0 = pos[2 * n + 1] + S / 4;
    for (int a = r0 / kObjTile; a <= (r0 + Q - 1) / kObjTile; ++a)
      for (int b = c0 / kObjTile; b <= (c0 + Q - 1) / kObjTile; ++b) lists[(size_t)a * tx + b].push_back(n);
  }
  std::vector<int4> entries;
  for (size_t t = 0; t < lists.size(); ++t) {
    start[t] = (int)entries.size();
    for (int n : lists[t]) entries.push_back(make_int4(n, pos[2 * n] + S / 4, pos[2 * n + 1] + S / 4, 0));
  }
  start.back() = (int)entries.size();
  int npad = 1;
  while (npad < N) npad <<= 1;
  // scratch carved from the network's kept buffer (256-byte aligned pieces)
  auto al = [](size_t b) { return (std::max<size_t>(b, 1) + 255) / 256 * 256; };
  const size_t b_patches = al(sizeof(float) * (size_t)N * Q * Q * 2), b_sig = al(sizeof(float) * npad),
               b_x = al(sizeof(float) * (size_t)u->n * S * S), b_start = al(sizeof(int) * start.size()),
               b_entries = al(sizeof(int4) * entries.size()), b_med = al(sizeof(double));
  const size_t need = b_patches + b_sig + b_x + b_start + b_entries + b_med;
  if (need > u->ws_bytes) {
    UN_CUDA(cudaStreamSynchronize(s), "stream sync");  // the old buffer may still be read
    if (u->ws_buf) cudaFree(u->ws_buf);
    u->ws_buf = nullptr;
    u->ws_bytes = 0;
    UN_CUDA(cudaMalloc(&u->ws_buf, need), "warm-start scratch");
    u->ws_bytes = need;
  }
  unsigned char* wp = static_cast<unsigned char*>(u->ws_buf);
  float* patches = reinterpret_cast<float*>(wp);
  float* sig = reinterpret_cast<float*>(wp + b_patches);
  float* x = reinterpret_cast<float*>(wp + b_patches + b_sig);
  int* d_start = reinterpret_cast<int*>(wp + b_patches + b_sig + b_x);
  int4* d_entries = reinterpret_cast<int4*>(wp + b_patches + b_sig + b_x + b_start);
  double* d_med = reinterpret_cast<double*>(wp + b_patches + b_sig + b_x + b_start + b_entries);
  UN_CUDA(cudaMemcpyAsync(d_start, start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice, s), "CSR");
  if (!entries.empty())
    UN_CUDA(cudaMemcpyAsync(d_entries, entries.data(), sizeof(int4) * entries.size(), cudaMemcpyHostToDevice, s),
            "CSR");
  UN_CUDA(cudaMemsetAsync(u->status, 0, sizeof(int), s), "clear status");
  // smallest sample count q whose pixel count at the coarsest level, q (S/8)^2, is a multiple of 128
  int q = 1;
  while ((q * (S / 8) * (S / 8)) % 128) ++q;
  for (int n0 = 0; n0 < N; n0 += u->n) {
    const int nb = std::min(u->n, N - n0);
    u->nrun = std::min(u->n, (nb + q - 1) / q * q);  // run only as many samples as this batch needs
    if (nb < u->nrun)
      UN_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * (size_t)u->nrun * S * S, s), "clear input");
    UN_CUDA(launch_log_input(intensities + (size_t)n0 * S * S, x, (size_t)nb * S * S, s), "input transform");
    UN_CUDA(unet_infer(u, x, patches + (size_t)n0 * Q * Q * 2, sig + n0, nb), "network forward");
  }
  u->nrun = u->n;
  StitchArgs sa{};
  sa.patches = patches;
  sa.patch = Q;
  sa.scale = (float)target_scale;
  sa.tile_start = d_start;
  sa.tile_pos = d_entries;
  sa.tiles_x = tx;
  sa.tiles_y = ty;
  sa.obj_h = obj_h;
  sa.obj_w = obj_w;
  sa.O = static_cast<float2*>(object_out);
  UN_CUDA(launch_stitch(sa, s), "stitch");
  UN_CUDA(launch_median(sig, N, npad, d_med, s), "median");
  int st = 0;
  UN_CUDA(cudaMemcpyAsync(sigma_out, d_med, sizeof(double), cudaMemcpyDeviceToHost, s), "copy sigma");
  UN_CUDA(cudaMemcpyAsync(&st, u->status, sizeof(int), cudaMemcpyDeviceToHost, s), "copy status");
  UN_CUDA(cudaStreamSynchronize(s), "stream sync");
  if (st) return capi_fail(PTYCHO_ETIMEOUT, "a tensor-core wait gave up");
  return PTYCHO_OK;
}

ptycho_status ptycho_unet_destroy(ptycho_unet_t u) {
  if (!u) return PTYCHO_OK;
  cudaStreamSynchronize(u->stream);
  delete u;
  return PTYCHO_OK;
}

}  // extern "C"
