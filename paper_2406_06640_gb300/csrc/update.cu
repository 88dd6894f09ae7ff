// Atomic-free simultaneous object / probe update of the data-parallel engine.
//
//   N_O(r) = sum_n c_n(r - r_n),            c_n = sum_k conj(P_k) dpsi_{n,k}
//   D_O(r) = sum_n sum_k |P_k(r - r_n)|^2
//   O     += beta_O N_O / (D_O + delta_O max D_O)           (pixels with D_O = 0 unchanged)
//   N_P,k  = sum_n conj(o_n) dpsi_{n,k},   D_P = sum_n |o_n|^2
//   P_k   += beta_P N_P,k / (D_P + delta_P max D_P)         (pixels with D_P = 0 unchanged)
//
// The paper's engines (ePIE, rPIE, DM, LSQML; Sec. 1 and Sec. 4.5) all move
// the object and probe with conj(P) dpsi / |P|^2 style steps; this is the
// simultaneous form of that step. Every sum runs in a fixed order (per-tile
// position lists in increasing n, per-slot partials in slot order), so an
// iteration is bitwise reproducible.
//
// The intensity error of Sec. 4.2, E = sqrt(sum (Ihat - I)^2 / sum I^2), is
// finished here in FP64 from the per-slot partials of the fused kernel.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "engine.h"
#include "cluster.cuh"
#include "fft.cuh"

namespace ptycho {

// ------------------------------------------------------------------ plan-time sums: sum I, sum I^2, bad values
__global__ void k_intensity_sums(const float* __restrict__ I, size_t count, double* __restrict__ partials) {
  __shared__ double s1[256], s2[256], s3[256];
  double a = 0.0, b = 0.0, bad = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
    const float v = I[i];
    if (!isfinite(v)) bad += 1e30;
    else if (v < 0.f) bad += 1.0;
    else {
      a += (double)v;
      b += (double)v * (double)v;
    }
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  s3[threadIdx.x] = bad;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s1[threadIdx.x] += s1[threadIdx.x + w];
      s2[threadIdx.x] += s2[threadIdx.x + w];
      s3[threadIdx.x] += s3[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partials[3 * blockIdx.x + 0] = s1[0];
    partials[3 * blockIdx.x + 1] = s2[0];
    partials[3 * blockIdx.x + 2] = s3[0];
  }
}

__global__ void k_finish_sums(const double* __restrict__ partials, int nblocks, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int i = 0; i < nblocks; ++i) {
      a += partials[3 * i];
      b += partials[3 * i + 1];
      c += partials[3 * i + 2];
    }
    out[0] = a;
    out[1] = b;
    out[2] = c;
  }
}

__global__ void k_sqrt(const float* __restrict__ I, float* __restrict__ out, size_t count) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    out[i] = sqrtf(I[i]);
}

cudaError_t launch_sqrt(const float* I, float* out, size_t count, cudaStream_t s) {
  const int nb = (int)std::min<size_t>(4096, (count + 255) / 256);
  k_sqrt<<<nb, 256, 0, s>>>(I, out, count);
  return cudaGetLastError();
}

cudaError_t launch_intensity_sums(const float* I, size_t count, double* partials, int nblocks, cudaStream_t s) {
  k_intensity_sums<<<nblocks, 256, 0, s>>>(I, count, partials);
  return cudaGetLastError();
}
cudaError_t launch_finish_sums(const double* partials, int nblocks, double* out, cudaStream_t s) {
  k_finish_sums<<<1, 32, 0, s>>>(partials, nblocks, out);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ probe: sum the per-slot partials
// grid (ceil(M^2 / 256), K + 1): y < K sums N_P for mode y; y == K sums D_P, |P|^2 map and block max
// thread (pixel p, group g) sums the slots g, g + 4, g + 8, ..., and the four group sums are added
// in group order (a fixed summation order; four loads in flight per pixel instead of one)
constexpr int kProbeGroups = 4;
__global__ void __launch_bounds__(256 * kProbeGroups) k_probe_gather(const UpdateArgs u) {
  const int MM = u.M * u.M;
  const int tx = threadIdx.x % 256, g = threadIdx.x / 256;
  const int p = blockIdx.x * 256 + tx;
  __shared__ float2 part[kProbeGroups][256];
  __shared__ float smax[256];
  if ((int)blockIdx.y < u.K) {
    const int k = blockIdx.y;
    float2 acc = make_float2(0.f, 0.f);
    if (p < MM) {
#pragma unroll 4
      for (int s = g; s < u.slots; s += kProbeGroups) acc = cadd(acc, u.pacc[((size_t)s * u.K + k) * MM + p]);
    }
    part[g][tx] = acc;
    __syncthreads();
    if (g == 0 && p < MM)
      u.np_sum[(size_t)k * MM + p] = cadd(cadd(cadd(part[0][tx], part[1][tx]), part[2][tx]), part[3][tx]);
    return;
  }
  float dp = 0.f;
  if (p < MM) {
#pragma unroll 4
    for (int s = g; s < u.slots; s += kProbeGroups) dp += u.dacc[(size_t)s * MM + p];
  }
  part[g][tx].x = dp;
  __syncthreads();
  if (g != 0) return;
  dp = ((part[0][tx].x + part[1][tx].x) + part[2][tx].x) + part[3][tx].x;
  if (p < MM) {
    float p2 = 0.f;
    for (int k = 0; k < u.K; ++k) p2 += cabs2(u.P[(size_t)k * MM + p]);
    u.dp_sum[p] = dp;
    u.p2[p] = p2;
  }
  smax[tx] = dp;
  // the first 256 threads (whole warps) finish the block maximum
  asm volatile("bar.sync 1, 256;" ::: "memory");
  for (int w = 128; w > 0; w >>= 1) {
    if (tx < w) smax[tx] = fmaxf(smax[tx], smax[tx + w]);
    asm volatile("bar.sync 1, 256;" ::: "memory");
  }
  if (tx == 0) u.blk_max_p[blockIdx.x] = smax[0];
}

// ------------------------------------------------------------------ pc-DM probe partials
// After the object step: slot s sums, over positions n = s, s + slots, ..., conj(o'_n)(psi_n,k - P_k o'_n)
// into pacc[s][k] and |o'_n|^2 into dacc[s] (o'_n: the new object under position n). Inside a
// complex-constraint window the states first move with their boxes, psi_n,k += P_k (o'_n - o''_n),
// o''_n the object before the constraint. grid (ceil(M^2 / 256), slots); one thread per probe pixel
// and every mode, so o'_n is read once
__global__ void k_dm_probe_partials(const UpdateArgs u) {
  const int MM = u.M * u.M;
  const int p = blockIdx.x * 256 + threadIdx.x;
  if (p >= MM) return;
  const int s = blockIdx.y;
  const int row = p / u.M, col = p % u.M;
  float2 pk[kMaxModes], acc[kMaxModes];
#pragma unroll
  for (int k = 0; k < kMaxModes; ++k) {
    pk[k] = k < u.K ? u.P[(size_t)k * MM + p] : make_float2(0.f, 0.f);
    acc[k] = make_float2(0.f, 0.f);
  }
  float d = 0.f;
  for (int n = s; n < u.N; n += u.slots) {
    const int2 r = u.pos[n];
    const size_t q = (size_t)(r.x + row) * u.obj_w + r.y + col;
    const float2 o = u.O[q];
    d += cabs2(o);
    float2* ps = u.dm_psi + (size_t)n * u.K * MM + p;
    if (u.dm_obj_prev) {
      const float2 dlt = csub(o, u.dm_obj_prev[q]);
#pragma unroll
      for (int k = 0; k < kMaxModes; ++k)
        if (k < u.K) {
          const float2 st = cadd(ps[(size_t)k * MM], cmul(pk[k], dlt));
          ps[(size_t)k * MM] = st;
          acc[k] = cadd(acc[k], cconjmul(o, csub(st, cmul(pk[k], o))));
        }
    } else {
#pragma unroll
      for (int k = 0; k < kMaxModes; ++k)
        if (k < u.K) acc[k] = cadd(acc[k], cconjmul(o, csub(ps[(size_t)k * MM], cmul(pk[k], o))));
    }
  }
#pragma unroll
  for (int k = 0; k < kMaxModes; ++k)
    if (k < u.K) const_cast<float2*>(u.pacc)[((size_t)s * u.K + k) * MM + p] = acc[k];
  const_cast<float*>(u.dacc)[(size_t)s * MM + p] = d;
}

// ------------------------------------------------------------------ object: per-tile gather of the contributions
// grid (tiles_x, tiles_y, kObjSplit) in clusters of the kObjSplit blocks of one tile, block 32 x 8;
// thread (tx, ty) owns pixels (Y0 + ty + 8 i, X0 + tx). Block `split` sums positions split,
// split + kObjSplit, ... of the tile's list; the partial tiles meet in distributed shared memory,
// where rank r adds up rows 4r .. 4r + 3 over the ranks in order and writes N_O, D_O; rank 0 also
// takes the tile maximum of D_O.
__global__ void __launch_bounds__(256, 3) k_obj_gather(const UpdateArgs u) {
  constexpr int TT = kObjTile * kObjTile, RPR = TT / kObjSplit;  // pixels finished per rank
  static_assert(RPR <= 256 && RPR % 32 == 0 && kObjTile == 32, "tile split");
  __shared__ float2 s_acc[TT];
  __shared__ float s_den[TT];
  __shared__ float s_max[kObjSplit * (RPR / 32)];
  const int tile = blockIdx.y * u.tiles_x + blockIdx.x;
  const int split = blockIdx.z;
  const unsigned rank = cluster_ctarank();
  const int tx0 = blockIdx.x * kObjTile, ty0 = blockIdx.y * kObjTile;
  const int X = tx0 + threadIdx.x;
  const int Y0 = ty0 + threadIdx.y;
  const int lt = threadIdx.y * 32 + threadIdx.x;
  const int M = u.M;
  const size_t MM = (size_t)M * M;
  float2 acc[4];
  float den[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    acc[i] = make_float2(0.f, 0.f);
    den[i] = 0.f;
  }
  const int s0 = u.tile_start[tile], s1 = u.tile_start[tile + 1];
  // four positions per round: every load of the round is in flight before the sums, which run in
  // list order (a tile in the middle of a dense scan holds hundreds of positions); three blocks
  // per SM
  constexpr int kU = 4;
  for (int base = s0 + split; base < s1; base += kU * kObjSplit) {
    float2 cv[kU][4];
    float dv[kU][4];
#pragma unroll
    for (int r = 0; r < kU; ++r) {
      const int idx = base + r * kObjSplit;
      const int4 ent = idx < s1 ? u.tile_pos[idx] : make_int4(0, 0, -(1 << 20), 0);  // (n, row, col)
      const int cx = X - ent.z;
      const bool inx = cx >= 0 && cx < M;
      const float2* cn = u.cn + (size_t)ent.x * MM;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int cy = Y0 + 8 * i - ent.y;
        const bool in = inx && cy >= 0 && cy < M;
        cv[r][i] = in ? cn[(size_t)cy * M + cx] : make_float2(0.f, 0.f);
        dv[r][i] = in ? u.p2[cy * M + cx] : 0.f;
      }
    }
#pragma unroll
    for (int r = 0; r < kU; ++r)
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        acc[i] = cadd(acc[i], cv[r][i]);
        den[i] += dv[r][i];
      }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    s_acc[(threadIdx.y + 8 * i) * kObjTile + threadIdx.x] = acc[i];
    s_den[(threadIdx.y + 8 * i) * kObjTile + threadIdx.x] = den[i];
  }
  cluster_sync_all();  // every rank's partial tile is complete
  float m = 0.f;
  if (lt < RPR) {
    const int lp = (int)rank * RPR + lt;
    const uint32_t oa = smem_addr(&s_acc[lp]), od = smem_addr(&s_den[lp]);
    float2 a = ld_cluster_f2(map_rank(oa, 0));
    float d = ld_cluster_f32(map_rank(od, 0));
    for (int q = 1; q < kObjSplit; ++q) {
      a = cadd(a, ld_cluster_f2(map_rank(oa, (unsigned)q)));
      d += ld_cluster_f32(map_rank(od, (unsigned)q));
    }
    const int Y = ty0 + lp / kObjTile, Xp = tx0 + lp % kObjTile;
    if (Y < u.obj_h && Xp < u.obj_w) {
      const size_t q = (size_t)Y * u.obj_w + Xp;
      u.no_part[q] = a;
      u.do_part[q] = d;
      m = d;  // D_O >= 0
    }
    const int wm = __reduce_max_sync(0xffffffffu, __float_as_int(m));  // non-negative floats order as ints
    if ((lt & 31) == 0) st_cluster_f32(map_rank(smem_addr(&s_max[rank * (RPR / 32) + lt / 32]), 0), __int_as_float(wm));
  }
  cluster_sync_all();  // remote reads and the maxima are done
  if (rank == 0 && lt == 0) {
    float mm = 0.f;
    for (int i = 0; i < kObjSplit * (RPR / 32); ++i) mm = fmaxf(mm, s_max[i]);
    u.blk_max_o[tile] = mm;
  }
}

__device__ float block_max_of(const float* vals, int n) {
  __shared__ float smax[256];
  float m = 0.f;
  const int lt = threadIdx.y * blockDim.x + threadIdx.x;
  const int nt = blockDim.x * blockDim.y;
  for (int i = lt; i < n; i += nt) m = fmaxf(m, vals[i]);
  smax[lt] = m;
  __syncthreads();
  for (int w = nt / 2; w > 0; w >>= 1) {
    if (lt < w) smax[lt] = fmaxf(smax[lt], smax[lt + w]);
    __syncthreads();
  }
  const float r = smax[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(256) k_obj_apply(const UpdateArgs u) {
  const float maxd = block_max_of(u.blk_max_o, u.tiles_x * u.tiles_y);
  const int X = blockIdx.x * kObjTile + threadIdx.x;
  const int Y0 = blockIdx.y * kObjTile + threadIdx.y;
  if (X >= u.obj_w) return;
  const float floor_d = u.cmax_obj * maxd;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int Y = Y0 + 8 * i;
    if (Y >= u.obj_h) break;
    const size_t q = (size_t)Y * u.obj_w + X;
    const float d = u.do_part[q];
    if (d > 0.f) {
      const float w = u.beta_obj / fmaf(u.cd_obj, d, floor_d);
      const float2 num = u.no_part[q];
      float2 o = u.O[q];
      o.x = fmaf(w, num.x, o.x);
      o.y = fmaf(w, num.y, o.y);
      u.O[q] = o;
    }
  }
}

// grid (ceil(M^2 / 256), K): apply the probe step; block (0, 0) also finishes the FP64 error
__global__ void k_probe_apply(const UpdateArgs u) {
  const float maxd = block_max_of(u.blk_max_p, u.probe_blocks);
  double e = 0.0;
  if (blockIdx.x == 0 && blockIdx.y == 0) {
    // error numerator: strided partial sums, then a fixed tree (every load in flight at once)
    __shared__ double s_e[256];
    for (int s = threadIdx.x; s < u.nerr; s += 256) e += u.errpart[s];
    s_e[threadIdx.x] = e;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) s_e[threadIdx.x] += s_e[threadIdx.x + w];
      __syncthreads();
    }
    e = s_e[0];
  }
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    if (u.err_mode != 0) e += *u.err_acc;
    if (u.err_mode == 1) {
      *u.err_acc = e;
    } else {
      const unsigned long long r = *u.run_counter;
      u.errhist[r % kErrHistory] = sqrt(e / u.errden);
      *u.run_counter = r + 1;
      if (u.err_mode == 2) *u.err_acc = 0.0;
    }
  }
  if (!u.update_probe) return;
  const int MM = u.M * u.M;
  const int p = blockIdx.x * 256 + threadIdx.x;
  if (p >= MM) return;
  const float d = u.dp_sum[p];
  if (d > 0.f) {
    const float w = u.beta_probe / fmaf(u.cd_probe, d, u.cmax_probe * maxd);
    const size_t q = (size_t)blockIdx.y * MM + p;
    const float2 num = u.np_sum[q];
    float2 pr = u.P[q];
    pr.x = fmaf(w, num.x, pr.x);
    pr.y = fmaf(w, num.y, pr.y);
    u.P[q] = pr;
  }
}

cudaError_t launch_update_object(const UpdateArgs& u, cudaStream_t s) {
  const int MM = u.M * u.M;
  const int pb = (MM + 255) / 256;
  if (u.dm_psi) {
    // the |P|^2 map for the object step only (no partials: the probe sums follow the object step)
    UpdateArgs u0 = u;
    u0.slots = 0;
    k_probe_gather<<<dim3(pb, u.K + 1), 256 * kProbeGroups, 0, s>>>(u0);
  } else {
    k_probe_gather<<<dim3(pb, u.K + 1), 256 * kProbeGroups, 0, s>>>(u);
  }
  const dim3 tb(32, 8);
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)u.tiles_x, (unsigned)u.tiles_y, kObjSplit);
    cfg.blockDim = tb;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = kObjSplit;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k_obj_gather, u);
    if (e != cudaSuccess) return e;
  }
  k_obj_apply<<<dim3(u.tiles_x, u.tiles_y), tb, 0, s>>>(u);
  return cudaGetLastError();
}

cudaError_t launch_update_probe(const UpdateArgs& u, cudaStream_t s) {
  const int MM = u.M * u.M;
  const int pb = (MM + 255) / 256;
  if (u.dm_psi && (u.update_probe || u.dm_obj_prev)) {
    k_dm_probe_partials<<<dim3(pb, u.slots), 256, 0, s>>>(u);
    if (u.update_probe) k_probe_gather<<<dim3(pb, u.K + 1), 256 * kProbeGroups, 0, s>>>(u);
  }
  k_probe_apply<<<dim3(pb, u.K), 256, 0, s>>>(u);
  return cudaGetLastError();
}

cudaError_t launch_update(const UpdateArgs& u, cudaStream_t s) {
  cudaError_t e = launch_update_object(u, s);
  return e != cudaSuccess ? e : launch_update_probe(u, s);
}

// E of a mini-batch iteration whose batches all added their partials to *err_acc (err_mode 1): the
// same sum as a last batch in err_mode 2, so the result does not depend on which form ran
__global__ void k_err_finish(const UpdateArgs u) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double e = *u.err_acc;
  const unsigned long long r = *u.run_counter;
  u.errhist[r % kErrHistory] = sqrt(e / u.errden);
  *u.run_counter = r + 1;
  *u.err_acc = 0.0;
}

cudaError_t launch_err_finish(const UpdateArgs& u, cudaStream_t s) {
  if (!u.err_acc) return cudaErrorInvalidValue;
  k_err_finish<<<1, 32, 0, s>>>(u);
  return cudaGetLastError();
}

}  // namespace ptycho
