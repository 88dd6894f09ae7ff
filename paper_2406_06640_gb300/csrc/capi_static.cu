// Allocation-free entry point ptycho_iterate_static (declared in include/ptycho.h).
//
// Some callers cannot call cudaMalloc: code that runs while a device memory
// pool or budget is locked, latency-critical loops where an allocation's
// implicit device synchronisation is not acceptable, or hosts that embed the
// engine and own every byte of device memory themselves. This entry point
// runs the same kernels as ptycho_plan + ptycho_iterate, but every scratch
// buffer they need is carved from one file-scope __device__ array of
// kStaticScratchBytes (32 MiB) that the module holds on each device until the
// process exits. The caller still provides the intensities, the positions,
// the object and the probe.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "engine.h"
#include "ptycho.h"

namespace ptycho {
ptycho_status capi_validate(const ptycho_params* p);
void capi_step_coefficients(const ptycho_params* p, UpdateArgs* u);
ptycho_status capi_fail(ptycho_status s, const std::string& msg);
ptycho_status capi_cuda_fail(cudaError_t e, const char* what);
std::vector<double> capi_taps(double sigma, int h);
void capi_tile_lists(const std::vector<int2>& pos, int M, int tx, int ty, std::vector<int>& start,
                     std::vector<int4>& flat);
bool capi_is_device_pointer(const void* ptr);
void capi_clear_error();
}  // namespace ptycho

using namespace ptycho;

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

// The scratch itself. In host code `g_static_scratch` names a host-side
// stand-in, not device memory: its device address comes from
// cudaGetSymbolAddress, once per device.
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

ptycho_status scratch_for_current_device(char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return capi_cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return capi_fail(PTYCHO_EUNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return capi_cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<char*>(g_scratch_addr[dev]);
  return PTYCHO_OK;
}

// bump allocator over the static scratch (sizes only; never calls cudaMalloc)
struct Carve {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) / 256 * 256;
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += std::max<size_t>(count, 1) * sizeof(T);
    return p;
  }
};

#define PS_CUDA(call, what)                                   \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return capi_cuda_fail(e_, what);   \
  } while (0)

}  // namespace

extern "C" ptycho_status ptycho_iterate_static(const ptycho_params* p, const float* intensities,
                                               const int32_t* positions, void* object, void* probe, int32_t n_iter,
                                               double* errors, void* cuda_stream) {
  ptycho_status st = capi_validate(p);
  if (st != PTYCHO_OK) return st;
  if (!intensities || !positions || !object || !probe) return capi_fail(PTYCHO_EINVAL, "NULL argument");
  if (n_iter < 0 || n_iter > kErrHistory) return capi_fail(PTYCHO_EINVAL, "n_iter must lie in [0, 4096]");
  if ((p->minibatch > 0 && p->minibatch < p->N) || p->engine == PTYCHO_ENGINE_DM)
    return capi_fail(PTYCHO_EUNSUPPORTED, "the mini-batch and pc-DM engines run through ptycho_plan");
  if (!capi_is_device_pointer(intensities)) return capi_fail(PTYCHO_EINVAL, "intensities must be a device pointer");
  // the fused kernel stages each position's rows of I with bulk async copies, which start on 16-byte
  // boundaries (the plan path copies I into its own buffer; this path reads the caller's)
  if (reinterpret_cast<uintptr_t>(intensities) % 16 != 0)
    return capi_fail(PTYCHO_EINVAL, "intensities must be 16-byte aligned (bulk copies of the pattern rows)");
  if (p->M > 128) return capi_fail(PTYCHO_EUNSUPPORTED, "the static entry point handles M <= 128");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int M = p->M, K = p->K, N = p->N;
  const size_t MM = (size_t)M * M;

  // positions: host copy for validation and the tile lists. A device array is read on the caller's
  // stream, after whatever the caller queued there to produce it. The host vectors below are pageable:
  // a host-to-device cudaMemcpyAsync from pageable memory is staged before the call returns, so they
  // may go out of scope while the copies are still queued.
  std::vector<int2> hpos(N);
  if (capi_is_device_pointer(positions)) {
    PS_CUDA(cudaMemcpyAsync(hpos.data(), positions, sizeof(int2) * N, cudaMemcpyDeviceToHost, s), "copy positions");
    PS_CUDA(cudaStreamSynchronize(s), "stream sync");
  } else {
    std::memcpy(hpos.data(), positions, sizeof(int2) * N);
  }
  for (int n = 0; n < N; ++n)
    if (hpos[n].x < 0 || hpos[n].y < 0 || hpos[n].x > p->obj_h - M || hpos[n].y > p->obj_w - M)
      return capi_fail(PTYCHO_EINVAL, "position " + std::to_string(n) + " puts its box outside the object");

  int max_slots = 0;
  PS_CUDA(fused_max_slots(M, K, &max_slots), "occupancy of the fused kernel");
  if (max_slots < 1) return capi_fail(PTYCHO_EUNSUPPORTED, "the fused kernel does not fit on this device");
  const int slots = std::min(max_slots, N);
  const int tx = (p->obj_w + kObjTile - 1) / kObjTile, ty = (p->obj_h + kObjTile - 1) / kObjTile;
  std::vector<int> start;
  std::vector<int4> flat;
  capi_tile_lists(hpos, M, tx, ty, start, flat);
  const size_t count = (size_t)N * MM;
  const int nb = (int)std::min<size_t>(1024, (count + 255) / 256);
  const size_t plane = (size_t)p->obj_h * p->obj_w;
  const int pb = (int)((MM + 255) / 256);

  // ---- size the request against the static scratch before touching it
  Carve c{nullptr};
  auto layout = [&](Carve& cv, FusedArgs& fa, UpdateArgs& ua, ConstraintArgs& ca, double*& part, double*& sums,
                    int2*& dpos, float2*& tw, float2*& hq) {
    dpos = cv.take<int2>(N);
    part = cv.take<double>((size_t)3 * nb);
    sums = cv.take<double>(3);
    tw = cv.take<float2>(M);
    hq = cv.take<float2>(M);
    fa.sqrtI = cv.take<float>(count);
    fa.cn = cv.take<float2>(count);
    fa.pacc = cv.take<float2>((size_t)slots * K * MM);
    fa.dacc = cv.take<float>((size_t)slots * MM);
    fa.errpart = cv.take<double>((size_t)slots * K);
    ua.tile_start = cv.take<int>(start.size());
    ua.tile_pos = cv.take<int4>(flat.size());
    ua.no_part = cv.take<float2>(plane);
    ua.do_part = cv.take<float>(plane);
    ua.blk_max_o = cv.take<float>((size_t)tx * ty);
    ua.np_sum = cv.take<float2>((size_t)K * MM);
    ua.dp_sum = cv.take<float>(MM);
    ua.p2 = cv.take<float>(MM);
    ua.blk_max_p = cv.take<float>((size_t)pb);
    ua.errhist = cv.take<double>((size_t)kErrHistory);
    ua.run_counter = cv.take<unsigned long long>(1);
    ca.cbar = cv.take<float>((size_t)N);
    ca.cbar_q = cv.take<long long>((size_t)N);
    ca.map_lna = cv.take<long long>((size_t)p->obj_h * (p->obj_w + 1));
    ca.map_phi = cv.take<long long>((size_t)p->obj_h * (p->obj_w + 1));
  };
  FusedArgs fa{};
  UpdateArgs ua{};
  ConstraintArgs ca{};
  double *part, *sums;
  int2* dpos;
  float2 *tw_d, *hq_d;
  layout(c, fa, ua, ca, part, sums, dpos, tw_d, hq_d);
  if (c.off > kStaticScratchBytes)
    return capi_fail(PTYCHO_EINVAL, "request needs " + std::to_string(c.off) +
                                        " bytes of scratch; the static scratch holds " +
                                        std::to_string(kStaticScratchBytes) + " bytes (32 MiB)");
  char* base = nullptr;
  st = scratch_for_current_device(&base);
  if (st != PTYCHO_OK) return st;
  Carve cv{base};
  fa = FusedArgs{};
  ua = UpdateArgs{};
  ca = ConstraintArgs{};
  layout(cv, fa, ua, ca, part, sums, dpos, tw_d, hq_d);

  // ---- per-call set-up, all through the scratch
  PS_CUDA(cudaMemcpyAsync(dpos, hpos.data(), sizeof(int2) * N, cudaMemcpyHostToDevice, s), "copy positions");
  PS_CUDA(cudaMemsetAsync(ua.run_counter, 0, sizeof(unsigned long long), s), "clear the run counter");
  PS_CUDA(cudaMemcpyAsync(const_cast<int*>(ua.tile_start), start.data(), sizeof(int) * start.size(), cudaMemcpyHostToDevice, s),
          "copy tile lists");
  if (!flat.empty())
    PS_CUDA(cudaMemcpyAsync(const_cast<int4*>(ua.tile_pos), flat.data(), sizeof(int4) * flat.size(), cudaMemcpyHostToDevice, s),
            "copy tile lists");
  std::vector<float2> tw(M), hq(M);
  for (int m = 0; m < M; ++m) {
    const double a = -2.0 * M_PI * m / M;
    tw[m] = make_float2((float)std::cos(a), (float)std::sin(a));
    const double fu = m < M / 2 ? m : m - M;
    const double ph = p->geometry == PTYCHO_NEARFIELD ? -M_PI * fu * fu / (M * p->fresnel_F) : 0.0;
    hq[m] = make_float2((float)std::cos(ph), (float)std::sin(ph));
  }
  PS_CUDA(cudaMemcpyAsync(tw_d, tw.data(), sizeof(float2) * M, cudaMemcpyHostToDevice, s), "copy twiddles");
  PS_CUDA(cudaMemcpyAsync(hq_d, hq.data(), sizeof(float2) * M, cudaMemcpyHostToDevice, s), "copy fresnel");
  PS_CUDA(launch_intensity_sums(intensities, count, part, nb, s), "intensity sums");
  PS_CUDA(launch_finish_sums(part, nb, sums, s), "intensity sums");
  double h_sums[3];
  PS_CUDA(cudaMemcpyAsync(h_sums, sums, sizeof(h_sums), cudaMemcpyDeviceToHost, s), "copy sums");
  PS_CUDA(cudaStreamSynchronize(s), "stream sync");
  if (h_sums[2] >= 1e30) return capi_fail(PTYCHO_ENUMERIC, "intensities contain non-finite values");
  if (h_sums[2] > 0) return capi_fail(PTYCHO_EINVAL, "intensities contain negative values");
  if (!(h_sums[1] > 0)) return capi_fail(PTYCHO_EINVAL, "intensities are all zero");
  const double eps = p->eps_mod > 0 ? p->eps_mod : 1e-6 * std::sqrt(h_sums[0] / (double)count);
  PS_CUDA(launch_sqrt(intensities, const_cast<float*>(fa.sqrtI), count, s), "sqrt intensities");

  const int kh = p->kernel_size / 2;
  const std::vector<double> gx = capi_taps(p->sigma1, kh), gy = capi_taps(p->sigma2, kh);
  fa.O = static_cast<const float2*>(object);
  fa.P = static_cast<const float2*>(probe);
  fa.I = intensities;
  fa.pos = dpos;
  fa.N = N;
  fa.K = K;
  fa.obj_w = p->obj_w;
  fa.near_field = p->geometry == PTYCHO_NEARFIELD;
  fa.blur_intensity = p->blur_domain == PTYCHO_BLUR_INTENSITY;
  fa.kh = kh;
  fa.eps = (float)eps;
  for (int i = 0; i < 2 * kh + 1; ++i) {
    fa.gx[i] = (float)gx[i];
    fa.gy[i] = (float)gy[i];
  }
  fa.tw = tw_d;
  fa.hq = hq_d;
  ua.O = static_cast<float2*>(object);
  ua.P = static_cast<float2*>(probe);
  ua.pos = dpos;
  ua.N = N;
  ua.K = K;
  ua.M = M;
  ua.obj_h = p->obj_h;
  ua.obj_w = p->obj_w;
  ua.slots = slots;
  ua.cn = fa.cn;
  ua.pacc = fa.pacc;
  ua.dacc = fa.dacc;
  ua.errpart = fa.errpart;
  ua.nerr = slots * K;
  ua.tiles_x = tx;
  ua.tiles_y = ty;
  ua.probe_blocks = pb;
  ua.errden = h_sums[1];
  ua.beta_obj = (float)p->beta_obj;
  ua.beta_probe = (float)p->beta_probe;
  capi_step_coefficients(p, &ua);
  ca.O = static_cast<float2*>(object);
  ca.pos = dpos;
  ca.N = N;
  ca.M = M;
  ca.obj_h = p->obj_h;
  ca.obj_w = p->obj_w;
  ca.alpha1 = (float)p->alpha1;
  ca.alpha2 = (float)p->alpha2;
  ca.cbar_min = (float)p->cbar_min;
  ca.cbar_max = (float)p->cbar_max;
  ca.tile_start = ua.tile_start;
  ca.tile_pos = ua.tile_pos;
  ca.tiles_x = tx;
  ca.tiles_y = ty;

  for (int i = 0; i < n_iter; ++i) {
    const long long t = (long long)p->start_iteration + i;
    PS_CUDA(launch_fused(M, fa, slots, s), "fused kernel launch");
    ua.update_probe = t >= p->probe_update_start;
    PS_CUDA(launch_update(ua, s), "update launch");
    bool win = false;
    for (int w = 0; w < p->n_windows; ++w)
      if (t >= p->windows[2 * w] && t <= p->windows[2 * w + 1]) win = true;
    if (win) PS_CUDA(launch_constraint(ca, s), "constraint launch");
  }
  if (errors && n_iter > 0)
    PS_CUDA(cudaMemcpyAsync(errors, ua.errhist, sizeof(double) * n_iter, cudaMemcpyDeviceToHost, s), "copy errors");
  PS_CUDA(cudaStreamSynchronize(s), "stream sync");
  bool timed_out = false;
  PS_CUDA(fused_timed_out(&timed_out), "read wait status");
  if (timed_out) return capi_fail(PTYCHO_ETIMEOUT, "a bounded device wait gave up; results are not valid");
  capi_clear_error();
  return PTYCHO_OK;
}
