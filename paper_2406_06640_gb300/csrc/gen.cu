// Forward-model data generator and warm-start assembly for the learned warm start.
//
// The generator simulates far-field patterns of random 2-D crystals on the GPU,
// one CTA per pattern:
//   phi(r)  = h sum_{sites p not vacant, |r - p| <= cutoff} exp(-|r - p|^2 / (2 s^2)),
//             sites p_ij = origin + i a1 + j a2 of a hexagonal lattice (|a1| = |a2| = a,
//             60 degrees apart, rotated by theta); a site is vacant when the first word of
//             Philox4x32-10((i, j, sample, 1), key) is below floor(vacancy 2^32)
//   psi     = P . exp(i phi),  Psi = centred 2-D DFT of psi (Eq. 1, the far-field propagator)
//   I       = |Psi|^2 (x) g_sigma (Eq. 2, isotropic, taps +-min(ceil(5 sigma), 15), normalised,
//             zero padding), scaled so that sum I = dose
//   counts  ~ Poisson(I) (counter-based: Philox4x32-10((pixel, sample, attempt, 2), key))
//   x       = log1p(counts) / 4,  target = (ln |o|, arg o) / scale on the central S/2 x S/2 box
// Philox4x32-10 follows its published definition (Salmon, Moraes, Dror, Shaw, SC'11).
// Poisson draws use sequential-search inversion below a mean of 10 and Hoermann's
// transformed rejection (PTRS, 1993) above it; both loops are bounded.
//
// The warm start then stitches the network's patches into an object estimate
//   O(r) = sum_n w(r - c_n) patch_n(r) / sum_n w(r - c_n)   (1 where no patch covers r),
// w a separable Hann window over the patch, c_n the patch corner, in a fixed order per
// object tile, and takes the median of the predicted sigma with a bitonic sort.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "engine.h"
#include "fft.cuh"
#include "ptycho.h"

namespace ptycho {

namespace {

// ---------------------------------------------------------------- Philox4x32-10
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// uniform in (0, 1) from the top 24 bits
__device__ __forceinline__ float u01(uint32_t w) { return ((float)(w >> 8) + 0.5f) * (1.0f / 16777216.0f); }

__device__ float poisson_draw(float lam, uint32_t pixel, uint32_t sample, uint2 key) {
  if (!(lam > 0.f)) return 0.f;
  if (lam < 10.f) {
    const uint4 r = philox4x32_10(make_uint4(pixel, sample, 0u, 2u), key);
    const float u = u01(r.x);
    float p = expf(-lam), F = p;
    int k = 0;
    while (u > F && k < 64) {
      ++k;
      p *= lam / (float)k;
      F += p;
    }
    return (float)k;
  }
  // PTRS
  const float slam = sqrtf(lam), loglam = logf(lam);
  const float b = 0.931f + 2.53f * slam;
  const float a = -0.059f + 0.02483f * b;
  const float invalpha = 1.1239f + 1.1328f / (b - 3.4f);
  const float vr = 0.9277f - 3.6224f / (b - 2.f);
  for (uint32_t attempt = 0; attempt < 32; ++attempt) {
    const uint4 r = philox4x32_10(make_uint4(pixel, sample, attempt, 2u), key);
    const float words[4] = {u01(r.x), u01(r.y), u01(r.z), u01(r.w)};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float U = words[2 * h] - 0.5f, V = words[2 * h + 1];
      const float us = 0.5f - fabsf(U);
      const float k = floorf((2.f * a / us + b) * U + lam + 0.43f);
      if (us >= 0.07f && V <= vr) return k;
      if (k < 0.f || (us < 0.013f && V > us)) continue;
      if (logf(V) + logf(invalpha) - logf(a / (us * us) + b) <= -lam + k * loglam - lgammaf(k + 1.f)) return k;
    }
  }
  return rintf(lam);  // not reached in practice (acceptance rate > 0.9 per pair)
}

struct Lattice {
  float oy, ox, a1y, a1x, a2y, a2x;  // origin and basis (row, col)
  float iyu, ixu, iyv, ixv;          // inverse basis: u = iyu dy + ixu dx, v = iyv dy + ixv dx
  float rho;                          // site-index search radius
};

__device__ __forceinline__ Lattice make_lattice(const GenArgs& a, float theta, float oy, float ox) {
  Lattice L;
  L.oy = oy;
  L.ox = ox;
  L.a1y = a.a * cosf(theta);
  L.a1x = a.a * sinf(theta);
  L.a2y = a.a * cosf(theta + 1.04719755f);
  L.a2x = a.a * sinf(theta + 1.04719755f);
  const float det = L.a1y * L.a2x - L.a1x * L.a2y;
  L.iyu = L.a2x / det;
  L.ixu = -L.a2y / det;
  L.iyv = -L.a1x / det;
  L.ixv = L.a1y / det;
  // |du a1 + dv a2|^2 >= a^2 (du^2 + dv^2) / 2 for a 60-degree basis
  L.rho = a.cutoff * 1.41421356f / a.a + 1e-3f;
  return L;
}

__device__ float lattice_phase(const GenArgs& a, const Lattice& L, float y, float x, uint32_t sample) {
  const float dy = y - L.oy, dx = x - L.ox;
  const float u = L.iyu * dy + L.ixu * dx, v = L.iyv * dy + L.ixv * dx;
  if (!(fabsf(u) < 1e6f && fabsf(v) < 1e6f && L.rho < 4.f)) return 0.f;  // non-finite or absurd parameters
  const int i0 = (int)ceilf(u - L.rho), i1 = (int)floorf(u + L.rho);
  const int j0 = (int)ceilf(v - L.rho), j1 = (int)floorf(v + L.rho);
  const float c2 = a.cutoff * a.cutoff, inv2s2 = 1.f / (2.f * a.s_pk * a.s_pk);
  float phi = 0.f;
  for (int i = i0; i <= i1; ++i)
    for (int j = j0; j <= j1; ++j) {
      const float py = L.oy + i * L.a1y + j * L.a2y, px = L.ox + i * L.a1x + j * L.a2x;
      const float d2 = (y - py) * (y - py) + (x - px) * (x - px);
      if (d2 > c2) continue;
      if (philox4x32_10(make_uint4((uint32_t)i, (uint32_t)j, sample, 1u), make_uint2(a.key_lo, a.key_hi)).x < a.vac_thresh)
        continue;
      phi += a.peak * expf(-d2 * inv2s2);
    }
  return phi;
}

template <int S, int V>
__global__ void __launch_bounds__(Tile<S>::T / V) k_gen(const GenArgs a) {
  using TL = Tile<S>;
  constexpr int E = TL::E, G = TL::G, TR = TL::T / V, LD = S + 1;
  extern __shared__ __align__(16) float2 gen_sm[];
  __shared__ float2 s_tw[G * (E + 1)];
  __shared__ float s_g[kMaxTaps];
  __shared__ float s_red[32];
  const int tid = threadIdx.x;
  const int n = blockIdx.x;
  const uint32_t sample = a.first + (uint32_t)n;
  const float4 prm = a.params[n];  // (theta, origin row, origin col, sigma)
  for (int i = tid; i < G * (E + 1); i += TR) {  // W_S^(t k2)
    const int t = i / (E + 1), k2 = i % (E + 1);
    float sn = 0.f, cs = 0.f;
    if (k2 < E) sincospif(-2.f * (float)((t * k2) % S) / (float)S, &sn, &cs);
    s_tw[i] = make_float2(cs, sn);
  }
  const int kh = prm.w > 0.f ? min((int)ceilf(5.f * prm.w), (kMaxTaps - 1) / 2) : 0;
  if (tid == 0) {
    float tot = 0.f;
    for (int d = -kh; d <= kh; ++d) {
      const float gv = prm.w > 0.f ? expf(-(float)(d * d) / (2.f * prm.w * prm.w)) : 1.f;
      s_g[d + kh] = gv;
      tot += gv;
    }
    for (int d = 0; d <= 2 * kh; ++d) s_g[d] /= tot;
  }
  const Lattice L = make_lattice(a, prm.x, prm.y, prm.z);
  float2 v[V][E];
#pragma unroll
  for (int q = 0; q < V; ++q) {
    const int vt = tid + q * TR, y = vt / G, t = vt % G;
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int x = t + G * j;
      const float phi = lattice_phase(a, L, (float)y, (float)x, sample);
      float sn, cs;
      sincosf(phi, &sn, &cs);
      const float2 p = a.probe[y * S + x];
      const float sg = ((x + y) & 1) ? -1.f : 1.f;
      v[q][j] = make_float2(sg * (p.x * cs - p.y * sn), sg * (p.x * sn + p.y * cs));
      if (a.target && y >= S / 4 && y < 3 * S / 4 && x >= S / 4 && x < 3 * S / 4) {
        float* tg = a.target + (((size_t)n * (S / 2) + (y - S / 4)) * (S / 2) + (x - S / 4)) * 2;
        tg[0] = 0.f;  // ln |o| = 0: a pure phase object
        tg[1] = phi / a.target_scale;
      }
    }
  }
  __syncthreads();
  fft2_forward<S, V>(v, gen_sm, s_tw, tid);
  float* A = reinterpret_cast<float*>(gen_sm);
  float* B = A + S * LD;
#pragma unroll
  for (int q = 0; q < V; ++q) {
    const int vt = tid + q * TR;
#pragma unroll
    for (int r = 0; r < E; ++r) A[col_freq<S>(vt % G, r) * LD + vt / G] = cabs2(v[q][r]);
  }
  __syncthreads();
  for (int p = tid; p < S * S; p += TR) {  // along x
    const int row = p / S, col = p % S;
    float s = 0.f;
    for (int d = -kh; d <= kh; ++d) {
      const int c = col + d;
      if (c >= 0 && c < S) s += s_g[d + kh] * A[row * LD + c];
    }
    B[row * LD + col] = s;
  }
  __syncthreads();
  float part = 0.f;
  for (int p = tid; p < S * S; p += TR) {  // along y
    const int row = p / S, col = p % S;
    float s = 0.f;
    for (int d = -kh; d <= kh; ++d) {
      const int rr = row + d;
      if (rr >= 0 && rr < S) s += s_g[d + kh] * B[rr * LD + col];
    }
    A[row * LD + col] = s;
    part += s;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((tid & 31) == 0) s_red[tid >> 5] = part;
  __syncthreads();
  if (tid < 32) {
    float s = tid < TR / 32 ? s_red[tid] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (tid == 0) s_red[0] = s;
  }
  __syncthreads();
  const float scale = s_red[0] > 0.f ? a.dose / s_red[0] : 0.f;
  const uint2 key = make_uint2(a.key_lo, a.key_hi);
  for (int p = tid; p < S * S; p += TR) {
    const float lam = A[(p / S) * LD + p % S] * scale;
    const size_t o = (size_t)n * S * S + p;
    if (a.clean) a.clean[o] = lam;
    if (a.counts || a.x) {
      const float c = a.noise ? poisson_draw(lam, (uint32_t)p, sample, key) : lam;
      if (a.counts) a.counts[o] = c;
      if (a.x) a.x[o] = 0.25f * log1pf(c);
    }
  }
  if (a.sigma && tid == 0) a.sigma[n] = prm.w;
}

__global__ void k_log_input(const float* I, float* x, size_t count) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    x[i] = 0.25f * log1pf(fmaxf(I[i], 0.f));
}

// one block per 32 x 32 object tile; entries (n, corner row, corner col) in increasing n
// blockIdx.y of gridDim.y blocks share a tile's pixels; the window's factors sin(pi (l + 1/2) / Q) come
// from a table (the same values and products as computed per sample)
__global__ void __launch_bounds__(256) k_stitch(const StitchArgs s) {
  __shared__ float s_sin[kStitchMaxQ];
  const int tile = blockIdx.x;
  const int ty = tile / s.tiles_x, tx = tile % s.tiles_x;
  const int beg = s.tile_start[tile], end = s.tile_start[tile + 1];
  const int Q = s.patch;
  const float pi_q = 3.14159265358979f / (float)Q;
  for (int l = threadIdx.x; l < Q; l += blockDim.x) s_sin[l] = __sinf(pi_q * (l + 0.5f));
  __syncthreads();
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < kObjTile * kObjTile; e += blockDim.x * gridDim.y) {
    const int y = ty * kObjTile + e / kObjTile, x = tx * kObjTile + e % kObjTile;
    if (y >= s.obj_h || x >= s.obj_w) continue;
    float ar = 0.f, ai = 0.f, wsum = 0.f;
    for (int i = beg; i < end; ++i) {
      const int4 t = s.tile_pos[i];
      const int ly = y - t.y, lx = x - t.z;
      if (ly < 0 || ly >= Q || lx < 0 || lx >= Q) continue;
      const float sy = s_sin[ly], sx = s_sin[lx];
      const float w = sy * sy * sx * sx;
      const float* pv = s.patches + (((size_t)t.x * Q + ly) * Q + lx) * 2;
      const float amp = expf(s.scale * pv[0]);
      float sn, cs;
      sincosf(s.scale * pv[1], &sn, &cs);
      ar += w * amp * cs;
      ai += w * amp * sn;
      wsum += w;
    }
    s.O[(size_t)y * s.obj_w + x] = wsum > 0.f ? make_float2(ar / wsum, ai / wsum) : make_float2(1.f, 0.f);
  }
}

// bitonic sort of npad (a power of two, <= 2^20) values in place by one block; then the median of the
// first n (the rest padded with +inf)
__global__ void __launch_bounds__(1024) k_median(float* v, int n, int npad, double* out) {
  for (int i = n + threadIdx.x; i < npad; i += blockDim.x) v[i] = INFINITY;
  __syncthreads();
  for (int k = 2; k <= npad; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < npad; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const float a = v[i], b = v[l];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            v[i] = b;
            v[l] = a;
          }
        }
      }
      __syncthreads();
    }
  if (threadIdx.x == 0)
    *out = (n & 1) ? (double)v[n / 2] : 0.5 * ((double)v[n / 2 - 1] + (double)v[n / 2]);
}

}  // namespace

size_t gen_smem_bytes(int S) {
  if (S == 128) return sizeof(float2) * Tile<128>::SMEM > 2 * 128 * 129 * 4 ? sizeof(float2) * Tile<128>::SMEM
                                                                             : 2 * 128 * 129 * 4;
  if (S == 64) return sizeof(float2) * Tile<64>::SMEM > 2 * 64 * 65 * 4 ? sizeof(float2) * Tile<64>::SMEM
                                                                        : 2 * 64 * 65 * 4;
  return 0;
}

template <int S, int V>
static cudaError_t launch_gen_t(const GenArgs& a, cudaStream_t s) {
  const size_t smem = gen_smem_bytes(S);
  cudaError_t e = cudaFuncSetAttribute(k_gen<S, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_gen<S, V><<<a.n, Tile<S>::T / V, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gen(int S, const GenArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  if (S == 128) return launch_gen_t<128, 2>(a, s);
  if (S == 64) return launch_gen_t<64, 1>(a, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_log_input(const float* I, float* x, size_t count, cudaStream_t s) {
  if (!count) return cudaSuccess;
  k_log_input<<<(int)std::min<size_t>(4096, (count + 255) / 256), 256, 0, s>>>(I, x, count);
  return cudaGetLastError();
}

cudaError_t launch_stitch(const StitchArgs& a, cudaStream_t s) {
  if (a.patch < 1 || a.patch > kStitchMaxQ) return cudaErrorInvalidValue;
  k_stitch<<<dim3(a.tiles_x * a.tiles_y, 4), 256, 0, s>>>(a);  // four blocks per tile: 256 pixels each
  return cudaGetLastError();
}

cudaError_t launch_median(float* v, int n, int npad, double* out, cudaStream_t s) {
  k_median<<<1, 1024, 0, s>>>(v, n, npad, out);
  return cudaGetLastError();
}

ptycho_status capi_fail(ptycho_status s, const std::string& msg);
ptycho_status capi_cuda_fail(cudaError_t e, const char* what);
bool capi_is_device_pointer(const void* p);

}  // namespace ptycho

extern "C" ptycho_status ptycho_generate(const ptycho_gen_spec* spec, const void* probe, const float* params,
                                         int32_t n, uint32_t first, float* x, float* counts, float* clean,
                                         float* target, float* sigma, void* stream) {
  using namespace ptycho;
  if (!spec || !probe || !params) return capi_fail(PTYCHO_EINVAL, "spec, probe and params must not be NULL");
  if (spec->S != 64 && spec->S != 128) return capi_fail(PTYCHO_EUNSUPPORTED, "pattern side must be 64 or 128");
  if (n < 0) return capi_fail(PTYCHO_EINVAL, "n < 0");
  if (!(spec->dose > 0.0) || !(spec->lattice_a > 0.0) || !(spec->peak_sd > 0.0) || !(spec->cutoff >= 0.0) ||
      !(spec->cutoff <= 2.0 * spec->lattice_a) ||
      !(spec->vacancy >= 0.0 && spec->vacancy <= 1.0) || !(spec->target_scale > 0.0) ||
      !std::isfinite(spec->peak))
    return capi_fail(PTYCHO_EINVAL, "dose, lattice constant, peak width and target scale must be positive, "
                                    "0 <= cutoff <= 2 lattice_a, vacancy in [0, 1]");
  if (reinterpret_cast<uintptr_t>(params) % 16 || reinterpret_cast<uintptr_t>(probe) % 8)
    return capi_fail(PTYCHO_EINVAL, "params must be 16-byte aligned and probe 8-byte aligned");
  const void* outs[5] = {x, counts, clean, target, sigma};
  for (const void* p : {probe, (const void*)params})
    if (!capi_is_device_pointer(p)) return capi_fail(PTYCHO_EINVAL, "probe and params must be device pointers");
  for (const void* p : outs)
    if (p && !capi_is_device_pointer(p)) return capi_fail(PTYCHO_EINVAL, "outputs must be device pointers");
  GenArgs a{};
  a.probe = static_cast<const float2*>(probe);
  a.params = reinterpret_cast<const float4*>(params);
  a.n = n;
  a.first = first;
  a.key_lo = (uint32_t)(spec->key & 0xffffffffu);
  a.key_hi = (uint32_t)(spec->key >> 32);
  a.dose = (float)spec->dose;
  a.a = (float)spec->lattice_a;
  a.peak = (float)spec->peak;
  a.s_pk = (float)spec->peak_sd;
  a.cutoff = (float)spec->cutoff;
  a.vac_thresh = (uint32_t)std::min(std::floor(spec->vacancy * 4294967296.0), 4294967295.0);
  a.target_scale = (float)spec->target_scale;
  a.noise = spec->noise;
  a.x = x;
  a.counts = counts;
  a.clean = clean;
  a.target = target;
  a.sigma = sigma;
  const cudaError_t e = launch_gen(spec->S, a, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return capi_cuda_fail(e, "generator launch");
  return PTYCHO_OK;
}
