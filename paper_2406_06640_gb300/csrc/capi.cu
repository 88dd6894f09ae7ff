// C ABI of the engine (declared in include/ptycho.h): plan construction,
// validation, the per-iteration launch sequence and error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <array>
#include <vector>

#include "engine.h"
#include "ptycho.h"

using namespace ptycho;

namespace {

thread_local std::string g_last_error;

ptycho_status fail(ptycho_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

ptycho_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky launch error where possible
  const ptycho_status s = (e == cudaErrorMemoryAllocation) ? PTYCHO_ENOMEM : PTYCHO_ECUDA;
  return fail(s, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

#define PT_CUDA(call, what)                       \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// normalised 1-D factor of Eq. 7 (the 2-D kernel is the outer product; its
// normalisation factors into the two 1-D normalisations)
std::vector<double> taps_1d(double sigma, int h) {
  std::vector<double> g(2 * h + 1);
  double s = 0.0;
  for (int d = -h; d <= h; ++d) {
    const double v = sigma > 0 ? std::exp(-(double)d * d / (2.0 * sigma * sigma)) : (d == 0 ? 1.0 : 0.0);
    g[d + h] = v;
    s += v;
  }
  for (double& v : g) v /= s;
  return g;
}

}  // namespace

// positions per chunk of a work-queue launch (each chunk has its own probe / error partials):
// candidates of the autotuner, smallest first (partial buffers are sized for the smallest)
constexpr int kChunkCandidates[] = {8, 16, 32, 64};
constexpr int kQueueChunkMin = 8;

// autotuner cache: chunk length per (device, M, K, geometry, kernel width class), and an optional
// caller-fixed chunk length (0: tune)
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int, int>, int> g_tune_cache;
int g_fixed_chunk = 0;
// staged path (M = 256, 512): positions per chunk of the staged passes, same key, and its fixed value
constexpr int kStagedCandidates[] = {4, 8, 16, 32};
std::map<std::tuple<int, int, int, int, int>, int> g_tune_staged;
int g_fixed_staged = 0;

// Philox4x32-10 on the host (Salmon et al., SC'11) and the Fisher-Yates permutation of 0..n-1 that
// mini-batch plans draw their batches (stream 3, t = 0) and visiting orders (stream 4, t) from:
// for i = n-1 .. 1, j = (w (i + 1)) >> 32 with w the first word of Philox((i, t, stream, 5), seed).
static uint32_t philox_first_word(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t key) {
  uint32_t k0 = (uint32_t)(key & 0xffffffffu), k1 = (uint32_t)(key >> 32);
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0, hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c0;
}

static std::vector<int> philox_permutation(int n, uint64_t seed, uint32_t stream, uint32_t t) {
  std::vector<int> a(std::max(n, 0));
  for (int i = 0; i < n; ++i) a[i] = i;
  for (int i = n - 1; i >= 1; --i) {
    const uint32_t w = philox_first_word((uint32_t)i, t, stream, 5u, seed);
    const int j = (int)(((uint64_t)w * (uint64_t)(i + 1)) >> 32);
    std::swap(a[i], a[j]);
  }
  return a;
}

struct ptycho_plan_s {
  ptycho_params p{};
  std::vector<int32_t> windows;
  cudaStream_t stream = nullptr;
  int device = 0;
  std::vector<void*> allocs;
  std::vector<int2> h_pos;
  double errden = 0.0, eps = 0.0;
  int slots = 0;
  int cluster_slots = 0;  // mini-batch plans: co-resident clusters of the cluster form (small batches)
  long long iter = 1;  // number of the next iteration
  long long runs = 0;  // iterations run so far
  FusedArgs fa{};
  UpdateArgs ua{};
  ConstraintArgs ca{};
  BigArgs ba{};
  bool big = false;  // M = 256, 512: staged passes over a chunk of positions
  // batch plans: independent member plans replayed as one CUDA graph per iteration
  std::vector<ptycho_plan_s*> members;
  std::vector<cudaStream_t> branch;
  std::vector<cudaEvent_t> branch_ev;
  std::vector<std::pair<std::vector<uintptr_t>, cudaGraphExec_t>> graphs;
  std::vector<std::vector<FusedArgs*>> graph_descs;  // per graph: each class's device argument array
  std::vector<int> graph_kernels;                     // per graph: kernel nodes (launches per replay)
  int last_kernels = 0;                               // kernel nodes of the last replayed graph
  cudaStream_t origin = nullptr;          // capture / replay stream of a batch plan
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int chunk = 0;
  // batch member drained by a work-queue launch: number of position chunks (its partial count)
  int parts = 0;
  // mini-batch engine: batch size (0: off), number of batches, per-batch tile lists (nb x (tiles + 1)
  // offsets into one entry array), running FP64 error of the current iteration
  int mb = 0, nb = 1, tiles = 0;
  int* d_starts = nullptr;
  double* d_err_acc = nullptr;
  // pc-DM: exit-wave state, and whether the next iteration starts it at P o_n
  float2* d_psi = nullptr;
  float2* d_obj_prev = nullptr;  // the object before the complex constraint (pc-DM windows)
  bool dm_fresh = true;
  // batch plans: one work-queue launch per shape class (M, K, geometry, kernel width class)
  struct QueueClass {
    int M = 0, K = 0, near = 0, kh = 0;
    std::vector<int> members;  // batch member indices, in order
    int4* d_chunks = nullptr;
    int nchunks = 0;
    int* d_queue = nullptr;
    int slots = 0;
    int chunk_len = 0;
  };
  std::vector<QueueClass> qclasses;
  std::vector<char> queued;  // per member: drained by its class's work-queue launch
  double* d_errhist = nullptr;
  // profiling: event pairs around the fused kernel
  bool profiling = false;
  std::vector<cudaEvent_t> ev;  // 2 * kProfSlots
  int prof_count = 0;
  static constexpr int kProfSlots = 1024;
  // single plans: an iteration's launches replayed as one CUDA graph once the same key (object,
  // probe, probe step on, constraint window, pc-DM state start) has run eagerly kGraphAfter times:
  // capturing costs host time while the stream may be idle, which short runs should not pay. Each key
  // has a ring of kRing graphs, captured together, each recording the fused kernel's start and end as
  // event nodes; with profiling on, a replay's times are read back before its graph replays again.
  struct SingleGraph {
    std::array<uintptr_t, 3> key{};
    int slot = 0;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bool pending = false;
  };
  static constexpr int kGraphAfter = 2, kRing = 4, kMaxGraphKeys = 32;  // beyond: eager
  std::vector<SingleGraph> sgraphs;
  std::vector<std::pair<std::array<uintptr_t, 3>, int>> eager_runs;
  cudaStream_t gstream = nullptr;
  int ring = 0;
  // mini-batch plans: one graph per batch (its fused launch or staged passes and its update), keyed
  // by (batch, probe step on, object, probe) and replayed in each iteration's visiting order
  std::vector<std::pair<std::array<uintptr_t, 4>, cudaGraphExec_t>> bgraphs;
  std::vector<std::pair<std::array<uintptr_t, 4>, int>> beager;
  static constexpr int kMaxBatchGraphs = 1024;
  double prof_graph_ms = 0.0;
  int prof_graph_n = 0;

  template <class T>
  cudaError_t alloc(T** ptr, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) allocs.push_back(q);
    *ptr = static_cast<T*>(q);
    return e;
  }
  ~ptycho_plan_s() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.second);
    for (auto& g : bgraphs) cudaGraphExecDestroy(g.second);
    for (auto& g : sgraphs) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.e0) cudaEventDestroy(g.e0);
      if (g.e1) cudaEventDestroy(g.e1);
    }
    if (gstream) cudaStreamDestroy(gstream);
    for (cudaEvent_t e : branch_ev) cudaEventDestroy(e);
    for (cudaStream_t s : branch) cudaStreamDestroy(s);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (origin) cudaStreamDestroy(origin);
    for (ptycho_plan_s* m : members) delete m;
    for (void* q : allocs) cudaFree(q);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  bool in_window(long long t) const {
    for (size_t i = 0; i + 1 < windows.size(); i += 2)
      if (t >= windows[i] && t <= windows[i + 1]) return true;
    return false;
  }
};

static ptycho_status validate(const ptycho_params* p) {
  if (!p) return fail(PTYCHO_EINVAL, "params is NULL");
  if (!is_pow2(p->M) || p->M < 8 || p->M > 512) return fail(PTYCHO_EINVAL, "M must be a power of two in [8, 512]");
  if (p->K < 1) return fail(PTYCHO_EINVAL, "K must be >= 1");
  if (p->K > kMaxModes) return fail(PTYCHO_EUNSUPPORTED, "K > 8 probe modes is not handled by this build");
  if (p->N < 1) return fail(PTYCHO_EINVAL, "N must be >= 1");
  if (p->obj_h < p->M || p->obj_w < p->M) return fail(PTYCHO_EINVAL, "object must be at least M x M");
  if (p->geometry != PTYCHO_FARFIELD && p->geometry != PTYCHO_NEARFIELD) return fail(PTYCHO_EINVAL, "bad geometry");
  if (p->blur_domain != PTYCHO_BLUR_AMPLITUDE && p->blur_domain != PTYCHO_BLUR_INTENSITY)
    return fail(PTYCHO_EINVAL, "bad blur_domain");
  if (p->geometry == PTYCHO_NEARFIELD && !(std::isfinite(p->fresnel_F) && p->fresnel_F > 0))
    return fail(PTYCHO_EINVAL, "near field needs fresnel_F > 0");
  if (!(std::isfinite(p->sigma1) && p->sigma1 >= 0 && std::isfinite(p->sigma2) && p->sigma2 >= 0))
    return fail(PTYCHO_EINVAL, "sigma1 and sigma2 must be finite and >= 0");
  if (p->kernel_size < 1 || p->kernel_size > kMaxTaps || (p->kernel_size % 2) == 0)
    return fail(PTYCHO_EINVAL, "kernel_size must be odd, 1..31");
  if (!(std::isfinite(p->eps_mod) && p->eps_mod >= 0)) return fail(PTYCHO_EINVAL, "eps_mod must be >= 0");
  if (!(std::isfinite(p->beta_obj) && std::isfinite(p->beta_probe))) return fail(PTYCHO_EINVAL, "beta not finite");
  if (!(std::isfinite(p->delta_obj) && p->delta_obj >= 0 && std::isfinite(p->delta_probe) && p->delta_probe >= 0))
    return fail(PTYCHO_EINVAL, "delta must be finite and >= 0");
  if (!(p->alpha1 >= 0 && p->alpha1 <= 1 && p->alpha2 >= 0 && p->alpha2 <= 1))
    return fail(PTYCHO_EINVAL, "alpha1 and alpha2 must lie in [0, 1]");
  if (!(std::isfinite(p->cbar_min) && std::isfinite(p->cbar_max) && p->cbar_min > 0 && p->cbar_min <= p->cbar_max))
    return fail(PTYCHO_EINVAL, "need 0 < cbar_min <= cbar_max");
  if (p->n_windows < 0 || (p->n_windows > 0 && !p->windows)) return fail(PTYCHO_EINVAL, "bad windows");
  for (int i = 0; i < p->n_windows; ++i)
    if (p->windows[2 * i] < 1 || p->windows[2 * i] > p->windows[2 * i + 1])
      return fail(PTYCHO_EINVAL, "windows must be [first, last] with 1 <= first <= last");
  if (p->start_iteration < 1) return fail(PTYCHO_EINVAL, "start_iteration must be >= 1");
  if (p->minibatch < 0) return fail(PTYCHO_EINVAL, "minibatch must be >= 0");
  if (p->engine != PTYCHO_ENGINE_PIE && p->engine != PTYCHO_ENGINE_DM)
    return fail(PTYCHO_EINVAL, "engine must be PTYCHO_ENGINE_PIE or PTYCHO_ENGINE_DM");
  if (p->engine == PTYCHO_ENGINE_DM && p->minibatch > 0 && p->minibatch < p->N)
    return fail(PTYCHO_EUNSUPPORTED, "pc-DM runs without mini-batches");
  if (p->step_rule != PTYCHO_STEP_NORMALISED && p->step_rule != PTYCHO_STEP_RPIE)
    return fail(PTYCHO_EINVAL, "step_rule must be PTYCHO_STEP_NORMALISED or PTYCHO_STEP_RPIE");
  if (p->step_rule == PTYCHO_STEP_RPIE &&
      !(p->rpie_alpha_obj >= 0 && p->rpie_alpha_obj <= 1 && p->rpie_alpha_probe >= 0 && p->rpie_alpha_probe <= 1))
    return fail(PTYCHO_EINVAL, "rPIE weights must lie in [0, 1]");
  return PTYCHO_OK;
}

// denominator coefficients of the step rule: step = beta num / (cd d + cmax max d)
static void step_coefficients(const ptycho_params& p, UpdateArgs& u) {
  if (p.step_rule == PTYCHO_STEP_RPIE) {
    u.cd_obj = (float)(1.0 - p.rpie_alpha_obj);
    u.cmax_obj = (float)p.rpie_alpha_obj;
    u.cd_probe = (float)(1.0 - p.rpie_alpha_probe);
    u.cmax_probe = (float)p.rpie_alpha_probe;
  } else {
    u.cd_obj = 1.f;
    u.cmax_obj = (float)p.delta_obj;
    u.cd_probe = 1.f;
    u.cmax_probe = (float)p.delta_probe;
  }
}

static bool is_device_pointer(const void* ptr) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Autotuner of the staged path (M = 256, 512): positions per chunk of the staged passes, timed on the
// device for each candidate over one pass of all positions (object and probe from scratch buffers
// of ones -- the passes only read them; they write the scratch, contributions and partials, which
// the first real iteration overwrites), best of two after a warm-up.
// Host vector -> plan buffer: ordered on the plan's stream and complete when it returns (a blocking
// copy on the legacy stream is not ordered against a non-blocking caller stream).
static cudaError_t h2d(cudaStream_t s, void* dst, const void* src, size_t bytes) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
  return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
}

static ptycho_status tune_staged_chunk(ptycho_plan_s* pl, int* best) {
  cudaStream_t s = pl->stream;
  const ptycho_params& p = pl->p;
  const size_t MM = (size_t)p.M * p.M;
  float2 *d_o, *d_p;
  PT_CUDA(pl->alloc(&d_o, (size_t)p.obj_h * p.obj_w), "alloc tuning object");
  PT_CUDA(pl->alloc(&d_p, (size_t)p.K * MM), "alloc tuning probe");
  {
    std::vector<float2> ones(std::max((size_t)p.obj_h * p.obj_w, (size_t)p.K * MM), make_float2(1.f, 0.f));
    PT_CUDA(h2d(pl->stream, d_o, ones.data(), sizeof(float2) * p.obj_h * p.obj_w), "tuning data");
    PT_CUDA(h2d(pl->stream, d_p, ones.data(), sizeof(float2) * p.K * MM), "tuning data");
  }
  BigArgs ba = pl->ba;
  ba.O = d_o;
  ba.P = d_p;
  cudaEvent_t e0, e1;
  PT_CUDA(cudaEventCreate(&e0), "event");
  PT_CUDA(cudaEventCreate(&e1), "event");
  float best_ms = 1e30f;
  *best = std::min(p.N, kStagedCandidates[0]);
  cudaError_t ce = cudaSuccess;
  for (int cand : kStagedCandidates) {
    const int c = std::min(cand, pl->chunk);
    if (cand > kStagedCandidates[0] && c != cand) break;  // larger candidates than N add nothing
    float t_best = 1e30f;
    for (int r = 0; r < 3 && ce == cudaSuccess; ++r) {
      ce = cudaEventRecord(e0, s);
      for (int n0 = 0; n0 < p.N && ce == cudaSuccess; n0 += c) {
        ba.n0 = n0;
        ce = launch_big_chunk(ba, std::min(c, p.N - n0), s);
      }
      if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
      if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce == cudaSuccess && r > 0) t_best = std::min(t_best, ms);
    }
    if (ce != cudaSuccess) break;
    if (t_best < best_ms) {
      best_ms = t_best;
      *best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ce != cudaSuccess) return cuda_fail(ce, "autotuner launch");
  return PTYCHO_OK;
}

// Object-tile position lists (CSR) of positions [n0, n1): for each kObjTile tile, in increasing n,
// (n, row, col, 0) of every position whose box overlaps it; appends tiles + 1 offsets to `start`
// (relative to the whole `flat` array) and the entries to `flat`.
static void append_tile_lists(const std::vector<int2>& pos, int n0, int n1, int M, int tx, int ty,
                              std::vector<int>& start, std::vector<int4>& flat) {
  std::vector<std::vector<int>> lists((size_t)tx * ty);
  for (int n = n0; n < n1; ++n)
    for (int by = pos[n].x / kObjTile; by <= (pos[n].x + M - 1) / kObjTile; ++by)
      for (int bx = pos[n].y / kObjTile; bx <= (pos[n].y + M - 1) / kObjTile; ++bx)
        lists[(size_t)by * tx + bx].push_back(n);
  for (const auto& l : lists) {
    start.push_back((int)flat.size());
    for (int n : l) flat.push_back(make_int4(n, pos[n].x, pos[n].y, 0));
  }
  start.push_back((int)flat.size());
}

static ptycho_status build_plan(ptycho_plan_s* pl, const float* intensities, const int32_t* positions) {
  const ptycho_params& p = pl->p;
  const int M = p.M, K = p.K, N = p.N;
  const size_t MM = (size_t)M * M;
  cudaStream_t s = pl->stream;

  // ---- positions
  pl->h_pos.resize(N);
  if (is_device_pointer(positions)) {
    // read on the plan's stream, after whatever the caller queued there to produce the positions
    PT_CUDA(cudaMemcpyAsync(pl->h_pos.data(), positions, sizeof(int2) * N, cudaMemcpyDeviceToHost, s),
            "copy positions");
    PT_CUDA(cudaStreamSynchronize(s), "stream sync");
  } else {
    std::memcpy(pl->h_pos.data(), positions, sizeof(int2) * N);
  }
  for (int n = 0; n < N; ++n) {
    const int2 q = pl->h_pos[n];
    if (q.x < 0 || q.y < 0 || q.x > p.obj_h - M || q.y > p.obj_w - M)
      return fail(PTYCHO_EINVAL, "position " + std::to_string(n) + " puts its box outside the object");
  }
  if (!is_device_pointer(intensities)) return fail(PTYCHO_EINVAL, "intensities must be a device pointer");
  // ---- mini-batch engine: positions (and below, their patterns) stored in the order of the batch
  // partition, so batch b is the contiguous range [b mb, min(N, (b + 1) mb))
  std::vector<int> order;
  if (p.minibatch > 0 && p.minibatch < N) {
    pl->mb = p.minibatch;
    pl->nb = (N + pl->mb - 1) / pl->mb;
    order = philox_permutation(N, p.order_seed, 3u, 0u);
    std::vector<int2> perm(N);
    for (int i = 0; i < N; ++i) perm[i] = pl->h_pos[order[i]];
    pl->h_pos = perm;
  }

  // ---- slots: co-resident clusters of the fused kernel (M <= 128), or the position chunk of
  // the staged path (M = 256, 512), whose per-slot partials are summed in slot order
  pl->big = M > 128;
  if (pl->big) {
    pl->chunk = std::min(N, kStagedCandidates[3]);  // buffers for the largest candidate; tuned below
    pl->slots = pl->chunk;
  } else {
    int max_slots = 0;
    if (p.engine == PTYCHO_ENGINE_DM) {
      PT_CUDA(fused_dm_max_slots(M, K, &max_slots), "occupancy of the pc-DM kernel");
      if (max_slots < 1) return fail(PTYCHO_EUNSUPPORTED, "a cluster of K CTAs does not fit on this device");
    } else {
      PT_CUDA(fused_max_slots(M, K, &max_slots), "occupancy of the fused kernel");
      if (max_slots < 1) return fail(PTYCHO_EUNSUPPORTED, "the fused kernel does not fit on this device");
    }
    pl->slots = std::min(max_slots, N);
  }
  if (pl->parts > 0) pl->slots = pl->parts;  // partials per position chunk (work-queue batch member)
  if (pl->mb > 0 && !pl->big) {
    PT_CUDA(fused_cluster_max_slots(M, K, &pl->cluster_slots), "occupancy of the cluster form");
    pl->cluster_slots = std::min(pl->cluster_slots, pl->slots);
  }

  // ---- buffers
  FusedArgs& fa = pl->fa;
  UpdateArgs& ua = pl->ua;
  ConstraintArgs& ca = pl->ca;
  float* d_I;
  int2* d_pos;
  PT_CUDA(pl->alloc(&d_I, (size_t)N * MM), "alloc intensities");
  PT_CUDA(pl->alloc(&d_pos, (size_t)N), "alloc positions");
  if (order.empty()) {
    PT_CUDA(cudaMemcpyAsync(d_I, intensities, sizeof(float) * N * MM, cudaMemcpyDeviceToDevice, s),
            "copy intensities");
  } else {
    for (int i = 0; i < N; ++i)
      PT_CUDA(cudaMemcpyAsync(d_I + (size_t)i * MM, intensities + (size_t)order[i] * MM, sizeof(float) * MM,
                              cudaMemcpyDeviceToDevice, s),
              "copy intensities");
  }
  PT_CUDA(cudaMemcpyAsync(d_pos, pl->h_pos.data(), sizeof(int2) * N, cudaMemcpyHostToDevice, s), "copy positions");

  // plan-time FP64 sums: sum I (for eps), sum I^2 (error denominator), bad values
  const size_t count = (size_t)N * MM;
  const int nb = (int)std::min<size_t>(1024, (count + 255) / 256);
  double* d_part;
  double* d_sums;
  PT_CUDA(pl->alloc(&d_part, (size_t)3 * nb), "alloc sums");
  PT_CUDA(pl->alloc(&d_sums, 3), "alloc sums");
  PT_CUDA(launch_intensity_sums(d_I, count, d_part, nb, s), "intensity sums");
  PT_CUDA(launch_finish_sums(d_part, nb, d_sums, s), "intensity sums");
  double h_sums[3];
  PT_CUDA(cudaMemcpyAsync(h_sums, d_sums, sizeof(h_sums), cudaMemcpyDeviceToHost, s), "copy sums");
  PT_CUDA(cudaStreamSynchronize(s), "plan sync");
  if (h_sums[2] >= 1e30) return fail(PTYCHO_ENUMERIC, "intensities contain non-finite values");
  if (h_sums[2] > 0) return fail(PTYCHO_EINVAL, "intensities contain negative values");
  if (!(h_sums[1] > 0)) return fail(PTYCHO_EINVAL, "intensities are all zero");
  pl->errden = h_sums[1];
  float* d_sqrtI;
  PT_CUDA(pl->alloc(&d_sqrtI, count), "alloc sqrt intensities");
  PT_CUDA(launch_sqrt(d_I, d_sqrtI, count, s), "sqrt intensities");
  pl->fa.sqrtI = d_sqrtI;
  pl->eps = p.eps_mod > 0 ? p.eps_mod : 1e-6 * std::sqrt(h_sums[0] / (double)count);

  // twiddles, Fresnel factors, taps (FP64 on the host, rounded once)
  std::vector<float2> tw(M), hq(M);
  for (int m = 0; m < M; ++m) {
    const double a = -2.0 * M_PI * m / M;
    tw[m] = make_float2((float)std::cos(a), (float)std::sin(a));
    const double fu = m < M / 2 ? m : m - M;
    const double ph = p.geometry == PTYCHO_NEARFIELD ? -M_PI * fu * fu / (M * p.fresnel_F) : 0.0;
    hq[m] = make_float2((float)std::cos(ph), (float)std::sin(ph));
  }
  float2 *d_tw, *d_hq;
  PT_CUDA(pl->alloc(&d_tw, M), "alloc twiddles");
  PT_CUDA(pl->alloc(&d_hq, M), "alloc fresnel");
  PT_CUDA(cudaMemcpyAsync(d_tw, tw.data(), sizeof(float2) * M, cudaMemcpyHostToDevice, s), "copy twiddles");
  PT_CUDA(cudaMemcpyAsync(d_hq, hq.data(), sizeof(float2) * M, cudaMemcpyHostToDevice, s), "copy fresnel");
  const int kh = p.kernel_size / 2;
  const std::vector<double> gx = taps_1d(p.sigma1, kh), gy = taps_1d(p.sigma2, kh);

  // per-position and per-slot work buffers
  float2 *d_cn, *d_pacc;
  float* d_dacc;
  double* d_errpart;
  PT_CUDA(pl->alloc(&d_cn, (size_t)N * MM), "alloc contributions");
  PT_CUDA(pl->alloc(&d_pacc, (size_t)pl->slots * K * MM), "alloc probe partials");
  PT_CUDA(pl->alloc(&d_dacc, (size_t)pl->slots * MM), "alloc probe partials");
  const size_t nerr = pl->big ? (size_t)N * big_row_blocks(M) : (size_t)pl->slots * K;
  PT_CUDA(pl->alloc(&d_errpart, nerr), "alloc error partials");
  float2* d_W = nullptr;
  float* d_R = nullptr;
  if (pl->big) {
    PT_CUDA(pl->alloc(&d_W, (size_t)pl->chunk * K * MM), "alloc staged scratch");
    PT_CUDA(pl->alloc(&d_R, (size_t)pl->chunk * MM), "alloc staged ratios");
  }

  // object tiles and their position lists (increasing n)
  const int tx = (p.obj_w + kObjTile - 1) / kObjTile, ty = (p.obj_h + kObjTile - 1) / kObjTile;
  // one list per batch (the whole scan when there are no mini-batches), offsets into one entry array
  pl->tiles = tx * ty;
  const int bsize = pl->mb > 0 ? pl->mb : N;
  std::vector<int> start;
  std::vector<int4> flat;
  for (int b = 0; b < pl->nb; ++b)
    append_tile_lists(pl->h_pos, b * bsize, std::min(N, (b + 1) * bsize), M, tx, ty, start, flat);
  int* d_start;
  int4* d_list;
  PT_CUDA(pl->alloc(&d_start, start.size()), "alloc tile lists");
  PT_CUDA(pl->alloc(&d_list, flat.size()), "alloc tile lists");
  PT_CUDA(h2d(pl->stream, d_start, start.data(), sizeof(int) * start.size()), "copy tiles");
  if (!flat.empty())
    PT_CUDA(h2d(pl->stream, d_list, flat.data(), sizeof(int4) * flat.size()), "copy tiles");
  pl->d_starts = d_start;
  if (p.engine == PTYCHO_ENGINE_DM) {
    PT_CUDA(pl->alloc(&pl->d_psi, (size_t)N * K * MM), "alloc exit-wave state");
    PT_CUDA(pl->alloc(&pl->d_obj_prev, (size_t)p.obj_h * p.obj_w), "alloc object copy");
    pl->ua.dm_psi = pl->d_psi;
  }
  PT_CUDA(pl->alloc(&pl->d_err_acc, 1), "alloc error accumulator");
  PT_CUDA(cudaMemset(pl->d_err_acc, 0, sizeof(double)), "clear error accumulator");

  const size_t plane = (size_t)p.obj_h * p.obj_w;
  float2* d_no;
  float *d_do, *d_bmo;
  PT_CUDA(pl->alloc(&d_no, plane), "alloc object sums");
  PT_CUDA(pl->alloc(&d_do, plane), "alloc object sums");
  PT_CUDA(pl->alloc(&d_bmo, (size_t)tx * ty), "alloc tile maxima");
  const int pb = (int)((MM + 255) / 256);
  float2* d_np;
  float *d_dp, *d_p2, *d_bmp, *d_cbar;
  PT_CUDA(pl->alloc(&d_np, (size_t)K * MM), "alloc probe sums");
  PT_CUDA(pl->alloc(&d_dp, MM), "alloc probe sums");
  PT_CUDA(pl->alloc(&d_p2, MM), "alloc probe sums");
  PT_CUDA(pl->alloc(&d_bmp, (size_t)pb), "alloc probe maxima");
  PT_CUDA(pl->alloc(&d_cbar, (size_t)N), "alloc cbar");
  long long *d_lna, *d_phi, *d_cbar_q;
  PT_CUDA(pl->alloc(&d_lna, (size_t)p.obj_h * (p.obj_w + 1)), "alloc constraint maps");
  PT_CUDA(pl->alloc(&d_phi, (size_t)p.obj_h * (p.obj_w + 1)), "alloc constraint maps");
  PT_CUDA(pl->alloc(&d_cbar_q, (size_t)N), "alloc cbar");
  // the constraint visits every box of a tile: the whole scan's lists (the batch lists when
  // there is one batch)
  const int* d_cstart = d_start;
  const int4* d_clist = d_list;
  if (pl->nb > 1) {
    std::vector<int> cs;
    std::vector<int4> cl;
    append_tile_lists(pl->h_pos, 0, N, M, tx, ty, cs, cl);
    int* ds;
    int4* dl;
    PT_CUDA(pl->alloc(&ds, cs.size()), "alloc constraint tile lists");
    PT_CUDA(pl->alloc(&dl, cl.size()), "alloc constraint tile lists");
    PT_CUDA(h2d(pl->stream, ds, cs.data(), sizeof(int) * cs.size()), "copy tiles");
    PT_CUDA(h2d(pl->stream, dl, cl.data(), sizeof(int4) * cl.size()), "copy tiles");
    d_cstart = ds;
    d_clist = dl;
  }
  PT_CUDA(pl->alloc(&pl->d_errhist, (size_t)kErrHistory), "alloc error history");
  unsigned long long* d_runs;
  PT_CUDA(pl->alloc(&d_runs, 1), "alloc run counter");
  PT_CUDA(cudaMemset(d_runs, 0, sizeof(unsigned long long)), "clear run counter");

  // ---- kernel argument blocks
  fa.I = d_I;
  fa.pos = d_pos;
  fa.N = N;
  fa.K = K;
  fa.obj_w = p.obj_w;
  fa.near_field = p.geometry == PTYCHO_NEARFIELD;
  fa.blur_intensity = p.blur_domain == PTYCHO_BLUR_INTENSITY;
  fa.kh = kh;
  fa.eps = (float)pl->eps;
  for (int i = 0; i < 2 * kh + 1; ++i) {
    fa.gx[i] = (float)gx[i];
    fa.gy[i] = (float)gy[i];
  }
  fa.tw = d_tw;
  fa.hq = d_hq;
  fa.cn = d_cn;
  fa.pacc = d_pacc;
  fa.dacc = d_dacc;
  fa.errpart = d_errpart;

  ua.pos = d_pos;
  ua.N = N;
  ua.K = K;
  ua.M = M;
  ua.obj_h = p.obj_h;
  ua.obj_w = p.obj_w;
  ua.slots = pl->slots;
  ua.cn = d_cn;
  ua.pacc = d_pacc;
  ua.dacc = d_dacc;
  ua.errpart = d_errpart;
  ua.nerr = (int)nerr;
  ua.tile_start = d_start;
  ua.tile_pos = d_list;
  ua.tiles_x = tx;
  ua.tiles_y = ty;
  ua.no_part = d_no;
  ua.do_part = d_do;
  ua.blk_max_o = d_bmo;
  ua.np_sum = d_np;
  ua.dp_sum = d_dp;
  ua.p2 = d_p2;
  ua.blk_max_p = d_bmp;
  ua.probe_blocks = pb;
  ua.errhist = pl->d_errhist;
  ua.run_counter = d_runs;
  ua.errden = pl->errden;
  ua.beta_obj = (float)p.beta_obj;
  ua.beta_probe = (float)p.beta_probe;
  step_coefficients(p, ua);

  ca.pos = d_pos;
  ca.N = N;
  ca.M = M;
  ca.obj_h = p.obj_h;
  ca.obj_w = p.obj_w;
  ca.cbar = d_cbar;
  ca.map_lna = d_lna;
  ca.map_phi = d_phi;
  ca.cbar_q = d_cbar_q;
  ca.tile_start = d_cstart;
  ca.tile_pos = d_clist;
  ca.tiles_x = tx;
  ca.tiles_y = ty;
  ca.alpha1 = (float)p.alpha1;
  ca.alpha2 = (float)p.alpha2;
  ca.cbar_min = (float)p.cbar_min;
  ca.cbar_max = (float)p.cbar_max;

  BigArgs& ba = pl->ba;
  ba.I = d_I;
  ba.sqrtI = fa.sqrtI;
  ba.pos = d_pos;
  ba.M = M;
  ba.N = N;
  ba.K = K;
  ba.obj_w = p.obj_w;
  ba.near_field = fa.near_field;
  ba.blur_intensity = fa.blur_intensity;
  ba.kh = kh;
  ba.eps = fa.eps;
  for (int i = 0; i < kMaxTaps; ++i) {
    ba.gx[i] = fa.gx[i];
    ba.gy[i] = fa.gy[i];
  }
  ba.tw = d_tw;
  ba.hq = d_hq;
  ba.W = d_W;
  ba.R = d_R;
  ba.cn = d_cn;
  ba.pacc = d_pacc;
  ba.dacc = d_dacc;
  ba.errpart = d_errpart;

  PT_CUDA(cudaStreamSynchronize(s), "plan sync");
  if (pl->big) {
    const std::tuple<int, int, int, int, int> key{pl->device, M, K, fa.near_field, kh == 5 ? 5 : 15};
    int c = 0;
    {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      if (g_fixed_staged > 0) c = g_fixed_staged;
      else if (g_tune_staged.count(key)) c = g_tune_staged[key];
    }
    if (c == 0) {
      ptycho_status st = tune_staged_chunk(pl, &c);
      if (st != PTYCHO_OK) return st;
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      g_tune_staged[key] = c;
    }
    pl->chunk = std::min(c, pl->chunk);  // a chunk holds at most N positions; buffers hold the largest
    pl->slots = pl->chunk;
    pl->ua.slots = pl->chunk;
  }
  return PTYCHO_OK;
}

extern "C" {

ptycho_status ptycho_plan(const ptycho_params* p, const float* intensities, const int32_t* positions,
                          void* cuda_stream, ptycho_plan_t* out) {
  if (!out) return fail(PTYCHO_EINVAL, "out is NULL");
  *out = nullptr;
  ptycho_status st = validate(p);
  if (st != PTYCHO_OK) return st;
  if (!intensities || !positions) return fail(PTYCHO_EINVAL, "intensities and positions must be non-NULL");
  ptycho_plan_s* pl = new (std::nothrow) ptycho_plan_s();
  if (!pl) return fail(PTYCHO_ENOMEM, "host allocation failed");
  pl->p = *p;
  pl->windows.assign(p->windows, p->windows + 2 * p->n_windows);
  pl->p.windows = nullptr;
  pl->stream = static_cast<cudaStream_t>(cuda_stream);
  pl->iter = p->start_iteration;
  cudaError_t e = cudaGetDevice(&pl->device);
  if (e != cudaSuccess) {
    delete pl;
    return cuda_fail(e, "cudaGetDevice");
  }
  st = build_plan(pl, intensities, positions);
  if (st != PTYCHO_OK) {
    cudaStreamSynchronize(pl->stream);
    delete pl;
    return st;
  }
  g_last_error.clear();
  *out = pl;
  return PTYCHO_OK;
}

// Enqueue one iteration (number t) of plan pl on stream s.
// batch b of a mini-batch iteration: its fused launch (or staged passes) over its positions and its
// update, the error partials added to the iteration's running sum
static ptycho_status enqueue_batch(ptycho_plan_s* pl, const FusedArgs& fa, const UpdateArgs& ua, int b,
                                   cudaStream_t s) {
  const size_t MM = (size_t)pl->p.M * pl->p.M;
  const int s0 = b * pl->mb, len = std::min(pl->mb, pl->p.N - s0);
  UpdateArgs ub = ua;
  ub.tile_start = pl->d_starts + (size_t)b * (pl->tiles + 1);
  if (pl->big) {
    // staged passes over the batch's positions; the probe partials restart at its first chunk
    BigArgs ba = pl->ba;
    ba.O = fa.O;
    ba.P = fa.P;
    ba.n_first = s0;
    for (int n0 = s0; n0 < s0 + len; n0 += pl->chunk) {
      ba.n0 = n0;
      PT_CUDA(launch_big_chunk(ba, std::min(pl->chunk, s0 + len - n0), s), "staged pass launch");
    }
    ub.slots = std::min(pl->chunk, len);
    ub.errpart = ua.errpart + (size_t)s0 * big_row_blocks(pl->p.M);
    ub.nerr = len * big_row_blocks(pl->p.M);
  } else {
    FusedArgs fb = fa;
    fb.I = fa.I + (size_t)s0 * MM;
    fb.sqrtI = fa.sqrtI + (size_t)s0 * MM;
    fb.pos = fa.pos + s0;
    fb.N = len;
    fb.cn = fa.cn + (size_t)s0 * MM;
    // a batch with fewer positions than one-CTA slots fills more SMs as clusters of K CTAs
    const bool clustered = pl->p.K > 1 && len < pl->slots && pl->cluster_slots > 0;
    const int slots = std::min(clustered ? pl->cluster_slots : pl->slots, len);
    if (clustered) PT_CUDA(launch_fused_cluster(pl->p.M, fb, slots, s), "fused kernel launch");
    else PT_CUDA(launch_fused(pl->p.M, fb, slots, s), "fused kernel launch");
    ub.slots = slots;
    ub.nerr = slots * pl->p.K;
  }
  ub.err_mode = 1;
  ub.err_acc = pl->d_err_acc;
  PT_CUDA(launch_update(ub, s), "update launch");
  return PTYCHO_OK;
}

// batch b as a graph replay once its key has run eagerly kGraphAfter times; *used = false: run it
// eagerly (a failed capture marks the key eager for good)
static ptycho_status batch_graph(ptycho_plan_s* pl, const FusedArgs& fa, const UpdateArgs& ua, void* object,
                                 void* probe, int b, bool* used) {
  *used = false;
  const std::array<uintptr_t, 4> key = {(uintptr_t)b, (uintptr_t)(ua.update_probe ? 1 : 0), (uintptr_t)object,
                                        (uintptr_t)probe};
  for (auto& g : pl->bgraphs)
    if (g.first == key) {
      PT_CUDA(cudaGraphLaunch(g.second, pl->stream), "graph launch");
      *used = true;
      return PTYCHO_OK;
    }
  int* count = nullptr;
  for (auto& e : pl->beager)
    if (e.first == key) count = &e.second;
  if (!count) {
    if (pl->beager.size() >= (size_t)ptycho_plan_s::kMaxBatchGraphs) return PTYCHO_OK;
    pl->beager.emplace_back(key, 0);
    count = &pl->beager.back().second;
  }
  if (*count < 0) return PTYCHO_OK;
  if (*count < ptycho_plan_s::kGraphAfter) {
    ++*count;
    return PTYCHO_OK;
  }
  if (!pl->gstream) PT_CUDA(cudaStreamCreateWithFlags(&pl->gstream, cudaStreamNonBlocking), "graph stream");
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  bool ok = cudaStreamBeginCapture(pl->gstream, cudaStreamCaptureModeRelaxed) == cudaSuccess;
  if (ok) {
    const ptycho_status st = enqueue_batch(pl, fa, ua, b, pl->gstream);
    const cudaError_t ee = cudaStreamEndCapture(pl->gstream, &graph);
    ok = st == PTYCHO_OK && ee == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  }
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    cudaGetLastError();  // nothing was launched: this batch runs eagerly
    if (exec) cudaGraphExecDestroy(exec);
    *count = -1;
    return PTYCHO_OK;
  }
  pl->bgraphs.emplace_back(key, exec);
  PT_CUDA(cudaGraphLaunch(exec, pl->stream), "graph launch");
  *used = true;
  return PTYCHO_OK;
}

// pe0 / pe1 (graph capture with profiling): events recorded as graph nodes around the fused kernel
// instead of the plan's event ring
static ptycho_status enqueue_iteration(ptycho_plan_s* pl, void* object, void* probe, long long t, cudaStream_t s,
                                       cudaEvent_t pe0 = nullptr, cudaEvent_t pe1 = nullptr) {
  FusedArgs fa = pl->fa;
  UpdateArgs ua = pl->ua;
  ConstraintArgs ca = pl->ca;
  fa.O = static_cast<const float2*>(object);
  fa.P = static_cast<const float2*>(probe);
  ua.O = static_cast<float2*>(object);
  ua.P = static_cast<float2*>(probe);
  ca.O = static_cast<float2*>(object);
  const int ps = pl->prof_count % ptycho_plan_s::kProfSlots;
  if (pe0) PT_CUDA(cudaEventRecordWithFlags(pe0, s, cudaEventRecordExternal), "profile event");
  else if (pl->profiling) PT_CUDA(cudaEventRecord(pl->ev[2 * ps], s), "profile event");
  if (pl->mb > 0) {
    // mini-batch engine: the batches in this iteration's order, each a fused launch over its own
    // positions followed by its update (a graph replay once it has run eagerly twice); the error
    // accumulates over the batches and one more launch finishes it
    const std::vector<int> visit = philox_permutation(pl->nb, pl->p.order_seed, 4u, (uint32_t)t);
    ua.update_probe = t >= pl->p.probe_update_start;
    for (int j = 0; j < pl->nb; ++j) {
      bool used = false;
      ptycho_status st = batch_graph(pl, fa, ua, object, probe, visit[j], &used);
      if (st == PTYCHO_OK && !used) st = enqueue_batch(pl, fa, ua, visit[j], s);
      if (st != PTYCHO_OK) return st;
    }
    {
      UpdateArgs uf = ua;
      uf.err_acc = pl->d_err_acc;
      PT_CUDA(launch_err_finish(uf, s), "error launch");
    }
    if (pl->profiling) {
      PT_CUDA(cudaEventRecord(pl->ev[2 * ps + 1], s), "profile event");
      pl->prof_count++;
    }
    if (pl->in_window(t)) PT_CUDA(launch_constraint(ca, s), "constraint launch");
    return PTYCHO_OK;
  } else if (pl->big && pl->d_psi) {
    // pc-DM on the staged path: per chunk, the estimate sweep (error) and the chi sweep
    BigArgs ba = pl->ba;
    ba.O = static_cast<const float2*>(object);
    ba.P = static_cast<const float2*>(probe);
    ba.n_first = 0;
    ba.psi = pl->d_psi;
    ba.dm_init = pl->dm_fresh ? 1 : 0;
    for (int n0 = 0; n0 < pl->p.N; n0 += pl->chunk) {
      ba.n0 = n0;
      PT_CUDA(launch_big_chunk_dm(ba, std::min(pl->chunk, pl->p.N - n0), s), "staged pc-DM launch");
    }
    pl->dm_fresh = false;
  } else if (pl->big) {
    BigArgs ba = pl->ba;
    ba.O = static_cast<const float2*>(object);
    ba.P = static_cast<const float2*>(probe);
    ba.n_first = 0;
    for (int n0 = 0; n0 < pl->p.N; n0 += pl->chunk) {
      ba.n0 = n0;
      PT_CUDA(launch_big_chunk(ba, std::min(pl->chunk, pl->p.N - n0), s), "staged pass launch");
    }
  } else if (pl->d_psi) {
    fa.psi = pl->d_psi;
    fa.dm_init = pl->dm_fresh ? 1 : 0;
    PT_CUDA(launch_fused_dm(pl->p.M, fa, pl->slots, s), "pc-DM kernel launch");
    pl->dm_fresh = false;
  } else {
    PT_CUDA(launch_fused(pl->p.M, fa, pl->slots, s), "fused kernel launch");
  }
  if (pe1) {
    PT_CUDA(cudaEventRecordWithFlags(pe1, s, cudaEventRecordExternal), "profile event");
  } else if (pl->profiling) {
    PT_CUDA(cudaEventRecord(pl->ev[2 * ps + 1], s), "profile event");
    pl->prof_count++;
  }
  ua.update_probe = t >= pl->p.probe_update_start;
  if (pl->d_psi) {
    // pc-DM: the complex constraint acts between the object and the probe step, and the states
    // move with their boxes by P (O constrained - O)
    PT_CUDA(launch_update_object(ua, s), "update launch");
    ua.dm_obj_prev = nullptr;
    if (pl->in_window(t)) {
      PT_CUDA(cudaMemcpyAsync(pl->d_obj_prev, ua.O, (size_t)pl->p.obj_h * pl->p.obj_w * sizeof(float2),
                              cudaMemcpyDeviceToDevice, s),
              "object copy");
      PT_CUDA(launch_constraint(ca, s), "constraint launch");
      ua.dm_obj_prev = pl->d_obj_prev;
    }
    PT_CUDA(launch_update_probe(ua, s), "update launch");
    return PTYCHO_OK;
  }
  PT_CUDA(launch_update(ua, s), "update launch");
  if (pl->in_window(t)) PT_CUDA(launch_constraint(ca, s), "constraint launch");
  return PTYCHO_OK;
}

// The update part of iteration t (object / probe steps, complex constraint) of a batch member whose
// per-position work ran in its class's work-queue launch.
static ptycho_status enqueue_update(ptycho_plan_s* pl, void* object, void* probe, long long t, cudaStream_t s) {
  UpdateArgs ua = pl->ua;
  ConstraintArgs ca = pl->ca;
  ua.O = static_cast<float2*>(object);
  ua.P = static_cast<float2*>(probe);
  ca.O = static_cast<float2*>(object);
  ua.update_probe = t >= pl->p.probe_update_start;
  if (pl->d_psi) {
    // pc-DM: the complex constraint acts between the object and the probe step, and the states
    // move with their boxes by P (O constrained - O)
    PT_CUDA(launch_update_object(ua, s), "update launch");
    ua.dm_obj_prev = nullptr;
    if (pl->in_window(t)) {
      PT_CUDA(cudaMemcpyAsync(pl->d_obj_prev, ua.O, (size_t)pl->p.obj_h * pl->p.obj_w * sizeof(float2),
                              cudaMemcpyDeviceToDevice, s),
              "object copy");
      PT_CUDA(launch_constraint(ca, s), "constraint launch");
      ua.dm_obj_prev = pl->d_obj_prev;
    }
    PT_CUDA(launch_update_probe(ua, s), "update launch");
    return PTYCHO_OK;
  }
  PT_CUDA(launch_update(ua, s), "update launch");
  if (pl->in_window(t)) PT_CUDA(launch_constraint(ca, s), "constraint launch");
  return PTYCHO_OK;
}

// the fused kernel's time of a profiled graph's last replay, once its end event has been reached
static ptycho_status harvest(ptycho_plan_s* pl, ptycho_plan_s::SingleGraph& g) {
  if (!g.pending) return PTYCHO_OK;
  g.pending = false;
  PT_CUDA(cudaEventSynchronize(g.e1), "profile event sync");
  float ms = 0.f;
  PT_CUDA(cudaEventElapsedTime(&ms, g.e0, g.e1), "cudaEventElapsedTime");
  pl->prof_graph_ms += ms;
  pl->prof_graph_n++;
  return PTYCHO_OK;
}

// one iteration of a single plan as a graph replay (capturing the key's graphs first when it qualifies);
// *used = false when the iteration is to run eagerly (the key has not run kGraphAfter times yet, the
// mini-batch engine, or a capture that failed)
static ptycho_status iterate_graph(ptycho_plan_s* pl, void* object, void* probe, bool* used) {
  *used = false;
  if (pl->mb > 0) return PTYCHO_OK;  // the visiting order changes every iteration
  const long long t = pl->iter;
  const uintptr_t flags = (t >= pl->p.probe_update_start ? 1u : 0u) | (pl->in_window(t) ? 2u : 0u) |
                          (pl->d_psi && pl->dm_fresh ? 4u : 0u);
  const std::array<uintptr_t, 3> key = {(uintptr_t)object, (uintptr_t)probe, flags};
  int* count = nullptr;
  for (auto& e : pl->eager_runs)
    if (e.first == key) count = &e.second;
  if (!count) {
    if (pl->eager_runs.size() >= (size_t)ptycho_plan_s::kMaxGraphKeys) return PTYCHO_OK;  // many buffers: eager
    pl->eager_runs.emplace_back(key, 0);
    count = &pl->eager_runs.back().second;
  }
  if (*count < 0) return PTYCHO_OK;  // this key failed to capture: eager from now on
  if (*count < ptycho_plan_s::kGraphAfter) {
    ++*count;
    return PTYCHO_OK;
  }
  const int slot = pl->ring++ % ptycho_plan_s::kRing;
  size_t gi = pl->sgraphs.size();
  for (size_t x = 0; x < pl->sgraphs.size(); ++x)
    if (pl->sgraphs[x].key == key && pl->sgraphs[x].slot == slot) gi = x;
  if (gi == pl->sgraphs.size()) {
    // capture the key's whole ring
    if (!pl->gstream) PT_CUDA(cudaStreamCreateWithFlags(&pl->gstream, cudaStreamNonBlocking), "graph stream");
    const bool fresh = pl->dm_fresh;
    const bool prof = pl->profiling;
    pl->profiling = false;  // the ring's own events, not the eager event ring
    std::vector<ptycho_plan_s::SingleGraph> ring;
    bool ok = true;
    for (int r = 0; r < ptycho_plan_s::kRing && ok; ++r) {
      ptycho_plan_s::SingleGraph ng;
      ng.key = key;
      ng.slot = r;
      ok = cudaEventCreate(&ng.e0) == cudaSuccess && cudaEventCreate(&ng.e1) == cudaSuccess;
      cudaGraph_t graph = nullptr;
      if (ok) ok = cudaStreamBeginCapture(pl->gstream, cudaStreamCaptureModeRelaxed) == cudaSuccess;
      if (ok) {
        const ptycho_status st = enqueue_iteration(pl, object, probe, t, pl->gstream, ng.e0, ng.e1);
        const cudaError_t ee = cudaStreamEndCapture(pl->gstream, &graph);
        ok = st == PTYCHO_OK && ee == cudaSuccess && graph && cudaGraphInstantiate(&ng.exec, graph, 0) == cudaSuccess;
      }
      if (graph) cudaGraphDestroy(graph);
      pl->dm_fresh = fresh;  // a replay starts the state; the caller marks it started
      ring.push_back(ng);
    }
    pl->profiling = prof;
    if (!ok) {
      cudaGetLastError();  // a failed capture launched nothing: this key runs eagerly
      for (auto& g : ring) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.e0) cudaEventDestroy(g.e0);
        if (g.e1) cudaEventDestroy(g.e1);
      }
      *count = -1;
      return PTYCHO_OK;
    }
    gi = pl->sgraphs.size() + (size_t)slot;
    for (auto& g : ring) pl->sgraphs.push_back(g);
  }
  ptycho_plan_s::SingleGraph& g = pl->sgraphs[gi];
  const ptycho_status hs = harvest(pl, g);
  if (hs != PTYCHO_OK) return hs;
  PT_CUDA(cudaGraphLaunch(g.exec, pl->stream), "graph launch");
  g.pending = pl->profiling;
  *used = true;
  return PTYCHO_OK;
}

ptycho_status ptycho_iterate(ptycho_plan_t pl, void* object, void* probe, int32_t n_iter) {
  if (!pl) return fail(PTYCHO_EINVAL, "plan is NULL");
  if (!pl->members.empty()) return fail(PTYCHO_EINVAL, "batch plans run through ptycho_iterate_batch");
  if (!object || !probe) return fail(PTYCHO_EINVAL, "object and probe must be non-NULL");
  if (n_iter < 0) return fail(PTYCHO_EINVAL, "n_iter must be >= 0");
  PT_CUDA(cudaSetDevice(pl->device), "cudaSetDevice");
  for (int i = 0; i < n_iter; ++i) {
    bool graphed = false;
    ptycho_status st = iterate_graph(pl, object, probe, &graphed);
    if (st != PTYCHO_OK) return st;
    if (graphed) {
      if (pl->d_psi) pl->dm_fresh = false;
    } else {
      st = enqueue_iteration(pl, object, probe, pl->iter, pl->stream);
      if (st != PTYCHO_OK) return st;
    }
    pl->iter++;
    pl->runs++;
  }
  return PTYCHO_OK;
}

// Chunk list of a class for chunk length L: (member position in the class, first position, end,
// partial index), members in order; sets each member's partial count (<= what its buffers hold).
static std::vector<int4> chunk_list(ptycho_plan_s* pl, ptycho_plan_s::QueueClass& qc, int L) {
  std::vector<int4> chunks;
  for (size_t j = 0; j < qc.members.size(); ++j) {
    const ptycho_plan_s* m = pl->members[qc.members[j]];
    const int parts = (m->p.N + L - 1) / L;
    for (int c = 0; c < parts; ++c) chunks.push_back(make_int4((int)j, c * L, std::min(m->p.N, (c + 1) * L), c));
  }
  return chunks;
}

static cudaError_t st_apply_chunk_length(ptycho_plan_s* pl, ptycho_plan_s::QueueClass& qc, int L, int max_slots) {
  const std::vector<int4> chunks = chunk_list(pl, qc, L);
  qc.chunk_len = L;
  qc.nchunks = (int)chunks.size();
  qc.slots = std::min(max_slots, qc.nchunks);
  const cudaError_t e = h2d(pl->stream, qc.d_chunks, chunks.data(), sizeof(int4) * chunks.size());
  for (int b : qc.members) {
    ptycho_plan_s* m = pl->members[b];
    m->parts = (m->p.N + L - 1) / L;
    m->slots = m->parts;
    m->ua.slots = m->parts;
    m->ua.nerr = m->parts * m->p.K;
  }
  return e;
}

// Autotuner: time the class's work-queue launch for every candidate chunk length (object and probe
// read from scratch buffers of ones; the launch writes only per-position contributions and
// partials, which the first real iteration overwrites) and keep the fastest. Best of three
// launches after one warm-up, CUDA events on the plan's stream.
static ptycho_status tune_chunk_length(ptycho_plan_s* pl, ptycho_plan_s::QueueClass& qc, int max_slots, int* best) {
  cudaStream_t s = pl->stream;
  size_t obj_max = 1, probe_max = 1;
  for (int b : qc.members) {
    const ptycho_params& p = pl->members[b]->p;
    obj_max = std::max(obj_max, (size_t)p.obj_h * p.obj_w);
    probe_max = std::max(probe_max, (size_t)p.K * p.M * p.M);
  }
  float2 *d_o, *d_p;
  FusedArgs* d_desc;
  PT_CUDA(pl->alloc(&d_o, obj_max), "alloc tuning object");
  PT_CUDA(pl->alloc(&d_p, probe_max), "alloc tuning probe");
  PT_CUDA(pl->alloc(&d_desc, qc.members.size()), "alloc tuning arguments");
  {
    std::vector<float2> ones(std::max(obj_max, probe_max), make_float2(1.f, 0.f));
    PT_CUDA(h2d(pl->stream, d_o, ones.data(), sizeof(float2) * obj_max), "tuning object");
    PT_CUDA(h2d(pl->stream, d_p, ones.data(), sizeof(float2) * probe_max), "tuning probe");
    std::vector<FusedArgs> h;
    for (int b : qc.members) {
      FusedArgs f = pl->members[b]->fa;
      f.O = d_o;
      f.P = d_p;
      h.push_back(f);
    }
    PT_CUDA(h2d(pl->stream, d_desc, h.data(), sizeof(FusedArgs) * h.size()), "tuning arguments");
  }
  cudaEvent_t e0, e1;
  PT_CUDA(cudaEventCreate(&e0), "event");
  PT_CUDA(cudaEventCreate(&e1), "event");
  float best_ms = 1e30f;
  *best = kChunkCandidates[0];
  ptycho_status st = PTYCHO_OK;
  for (int L : kChunkCandidates) {
    const std::vector<int4> chunks = chunk_list(pl, qc, L);
    cudaError_t ce = h2d(pl->stream, qc.d_chunks, chunks.data(), sizeof(int4) * chunks.size());
    FusedArgs fa = pl->members[qc.members[0]]->fa;
    fa.probs = d_desc;
    fa.chunks = qc.d_chunks;
    fa.nchunks = (int)chunks.size();
    fa.queue = qc.d_queue;
    fa.kh = qc.kh;
    const int slots = std::min(max_slots, fa.nchunks);
    float t_best = 1e30f;
    for (int r = 0; r < 4 && ce == cudaSuccess; ++r) {
      ce = cudaMemsetAsync(qc.d_queue, 0, sizeof(int), s);
      if (ce == cudaSuccess) ce = cudaEventRecord(e0, s);
      if (ce == cudaSuccess) ce = launch_fused_queue(qc.M, fa, slots, s);
      if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
      if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
      if (ce == cudaSuccess && r > 0) t_best = std::min(t_best, ms);
    }
    if (ce != cudaSuccess) {
      st = cuda_fail(ce, "autotuner launch");
      break;
    }
    if (t_best < best_ms) {
      best_ms = t_best;
      *best = L;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == PTYCHO_OK) {
    bool timed_out = false;
    PT_CUDA(fused_timed_out(&timed_out), "read wait status");
    if (timed_out) return fail(PTYCHO_ETIMEOUT, "a bounded device wait gave up while tuning");
  }
  return st;
}

ptycho_status ptycho_plan_batch(int32_t B, const ptycho_params* const* params, const float* const* intensities,
                                const int32_t* const* positions, void* cuda_stream, ptycho_plan_t* out) {
  if (!out) return fail(PTYCHO_EINVAL, "out is NULL");
  *out = nullptr;
  if (B < 1 || !params || !intensities || !positions) return fail(PTYCHO_EINVAL, "need B >= 1 and non-NULL arrays");
  for (int b = 0; b < B; ++b) {
    ptycho_status st = validate(params[b]);
    if (st == PTYCHO_OK && (!intensities[b] || !positions[b]))
      st = fail(PTYCHO_EINVAL, "intensities and positions must be non-NULL");
    if (st == PTYCHO_OK && params[b]->minibatch > 0 && params[b]->minibatch < params[b]->N)
      st = fail(PTYCHO_EUNSUPPORTED, "mini-batch problems run through ptycho_plan");
    if (st != PTYCHO_OK) return fail(st, "problem " + std::to_string(b) + ": " + g_last_error);
  }
  ptycho_plan_s* pl = new (std::nothrow) ptycho_plan_s();
  if (!pl) return fail(PTYCHO_ENOMEM, "host allocation failed");
  pl->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&pl->device);
  if (e != cudaSuccess) {
    delete pl;
    return cuda_fail(e, "cudaGetDevice");
  }
  // shape classes of the work-queue launches: members with M in {8, ..., 128} sharing K, geometry
  // and kernel width class are drained together; the others keep their own launches
  std::vector<int> member_class(B, -1);
  for (int b = 0; b < B; ++b) {
    const ptycho_params& q = *params[b];
    // pc-DM members keep their own launches (the work queue runs the simultaneous engine)
    if (!fused_queue_supported(q.M) || q.engine == PTYCHO_ENGINE_DM) continue;
    const int kh = (q.kernel_size - 1) / 2 == 5 ? 5 : 15;
    const int near = q.geometry == PTYCHO_NEARFIELD ? 1 : 0;
    int ci = -1;
    for (size_t c = 0; c < pl->qclasses.size(); ++c) {
      const auto& qc = pl->qclasses[c];
      if (qc.M == q.M && qc.K == q.K && qc.near == near && qc.kh == kh) ci = (int)c;
    }
    if (ci < 0) {
      ptycho_plan_s::QueueClass qc;
      qc.M = q.M;
      qc.K = q.K;
      qc.near = near;
      qc.kh = kh;
      qc.chunk_len = kQueueChunkMin;
      pl->qclasses.push_back(qc);
      ci = (int)pl->qclasses.size() - 1;
    }
    pl->qclasses[ci].members.push_back(b);
    member_class[b] = ci;
  }
  pl->queued.assign(B, 0);
  for (int b = 0; b < B; ++b) {
    ptycho_status st = PTYCHO_OK;
    ptycho_plan_s* m = new (std::nothrow) ptycho_plan_s();
    if (!m) st = fail(PTYCHO_ENOMEM, "host allocation failed");
    if (st == PTYCHO_OK) {
      pl->members.push_back(m);
      m->p = *params[b];
      m->windows.assign(params[b]->windows, params[b]->windows + 2 * params[b]->n_windows);
      m->p.windows = nullptr;
      m->stream = pl->stream;
      m->iter = params[b]->start_iteration;
      m->device = pl->device;
      if (member_class[b] >= 0) {
        const int L = pl->qclasses[member_class[b]].chunk_len;
        m->parts = (m->p.N + L - 1) / L;
        pl->queued[b] = 1;
      }
      st = build_plan(m, intensities[b], positions[b]);
    }
    if (st != PTYCHO_OK) {
      const std::string msg = "problem " + std::to_string(b) + ": " + g_last_error;
      cudaStreamSynchronize(pl->stream);
      delete pl;
      return fail(st, msg);
    }
  }
  // chunk lists, sized for the smallest chunk length (the most chunks); the autotuner then picks the
  // length per class and the lists and partial counts are rebuilt for it
  for (auto& qc : pl->qclasses) {
    int max_chunks = 0;
    for (int b : qc.members) max_chunks += pl->members[b]->parts;
    int max_slots = 0;
    PT_CUDA(pl->alloc(&qc.d_chunks, (size_t)max_chunks), "alloc chunk list");
    PT_CUDA(pl->alloc(&qc.d_queue, 1), "alloc work counter");
    PT_CUDA(fused_queue_max_slots(qc.M, qc.K, &max_slots), "occupancy of the work-queue kernel");
    if (max_slots < 1) return fail(PTYCHO_EUNSUPPORTED, "a cluster of K CTAs does not fit on this device");
    const std::tuple<int, int, int, int, int> key{pl->device, qc.M, qc.K, qc.near, qc.kh};
    int L = 0;
    {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      if (g_fixed_chunk > 0) L = g_fixed_chunk;
      else if (g_tune_cache.count(key)) L = g_tune_cache[key];
    }
    if (L == 0) {
      ptycho_status st = tune_chunk_length(pl, qc, max_slots, &L);
      if (st != PTYCHO_OK) return st;
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      g_tune_cache[key] = L;
    }
    PT_CUDA(st_apply_chunk_length(pl, qc, L, max_slots), "chunk list");
  }
  const int S = std::min(B, 8);
  pl->branch.resize(S);
  pl->branch_ev.resize(S + 1);
  for (int i = 0; i < S; ++i) PT_CUDA(cudaStreamCreateWithFlags(&pl->branch[i], cudaStreamNonBlocking), "branch stream");
  for (auto& ev : pl->branch_ev) PT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "branch event");
  PT_CUDA(cudaStreamCreateWithFlags(&pl->origin, cudaStreamNonBlocking), "origin stream");
  PT_CUDA(cudaEventCreateWithFlags(&pl->ev_in, cudaEventDisableTiming), "event");
  PT_CUDA(cudaEventCreateWithFlags(&pl->ev_out, cudaEventDisableTiming), "event");
  g_last_error.clear();
  *out = pl;
  return PTYCHO_OK;
}

ptycho_status ptycho_iterate_batch(ptycho_plan_t pl, void* const* objects, void* const* probes, int32_t n_iter) {
  if (!pl || pl->members.empty()) return fail(PTYCHO_EINVAL, "not a batch plan");
  if (!objects || !probes || n_iter < 0) return fail(PTYCHO_EINVAL, "bad arguments");
  const int B = (int)pl->members.size();
  for (int b = 0; b < B; ++b)
    if (!objects[b] || !probes[b]) return fail(PTYCHO_EINVAL, "object and probe pointers must be non-NULL");
  PT_CUDA(cudaSetDevice(pl->device), "cudaSetDevice");
  const int S = (int)pl->branch.size();
  for (int i = 0; i < n_iter; ++i) {
    // the graph depends on which members update the probe / apply the constraint this iteration
    std::vector<uintptr_t> key;
    key.reserve(3 * B);
    for (int b = 0; b < B; ++b) {
      const ptycho_plan_s* m = pl->members[b];
      // pc-DM members: whether this iteration starts the exit-wave state (baked into the graph)
      key.push_back((uintptr_t)((m->iter >= m->p.probe_update_start ? 1 : 0) | (m->in_window(m->iter) ? 2 : 0) |
                                (m->d_psi && m->dm_fresh ? 4 : 0)));
      key.push_back((uintptr_t)objects[b]);
      key.push_back((uintptr_t)probes[b]);
    }
    cudaGraphExec_t exec = nullptr;
    int kernels = 0;
    for (size_t gi = 0; gi < pl->graphs.size(); ++gi)
      if (pl->graphs[gi].first == key) {
        exec = pl->graphs[gi].second;
        kernels = pl->graph_kernels[gi];
      }
    if (!exec) {
      // each class's per-problem arguments with this call's object / probe pointers (kept with the graph)
      std::vector<FusedArgs*> descs;
      for (const auto& qc : pl->qclasses) {
        std::vector<FusedArgs> h;
        for (int b : qc.members) {
          FusedArgs f = pl->members[b]->fa;
          f.O = static_cast<const float2*>(objects[b]);
          f.P = static_cast<const float2*>(probes[b]);
          h.push_back(f);
        }
        FusedArgs* d = nullptr;
        PT_CUDA(pl->alloc(&d, h.size()), "alloc work-queue arguments");
        PT_CUDA(h2d(pl->stream, d, h.data(), sizeof(FusedArgs) * h.size()), "copy arguments");
        descs.push_back(d);
      }
      PT_CUDA(cudaStreamBeginCapture(pl->origin, cudaStreamCaptureModeRelaxed), "begin capture");
      ptycho_status st = PTYCHO_OK;
      cudaError_t ce = cudaEventRecord(pl->branch_ev[S], pl->origin);
      for (int j = 0; j < S && ce == cudaSuccess; ++j) ce = cudaStreamWaitEvent(pl->branch[j], pl->branch_ev[S], 0);
      int br = 0;
      // one persistent work-queue launch per class, then its members' updates on the same branch
      for (size_t c = 0; c < pl->qclasses.size() && ce == cudaSuccess && st == PTYCHO_OK; ++c) {
        const auto& qc = pl->qclasses[c];
        cudaStream_t bs = pl->branch[br++ % S];
        ce = cudaMemsetAsync(qc.d_queue, 0, sizeof(int), bs);
        FusedArgs fa = pl->members[qc.members[0]]->fa;
        fa.probs = descs[c];
        fa.chunks = qc.d_chunks;
        fa.nchunks = qc.nchunks;
        fa.queue = qc.d_queue;
        fa.kh = qc.kh;
        if (ce == cudaSuccess) ce = launch_fused_queue(qc.M, fa, qc.slots, bs);
        for (size_t j = 0; j < qc.members.size() && ce == cudaSuccess && st == PTYCHO_OK; ++j) {
          const int b = qc.members[j];
          st = enqueue_update(pl->members[b], objects[b], probes[b], pl->members[b]->iter, bs);
        }
      }
      for (int b = 0; b < B && ce == cudaSuccess && st == PTYCHO_OK; ++b)
        if (!pl->queued[b])
          st = enqueue_iteration(pl->members[b], objects[b], probes[b], pl->members[b]->iter, pl->branch[br++ % S]);
      for (int j = 0; j < S && ce == cudaSuccess && st == PTYCHO_OK; ++j) {
        ce = cudaEventRecord(pl->branch_ev[j], pl->branch[j]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(pl->origin, pl->branch_ev[j], 0);
      }
      cudaGraph_t graph = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(pl->origin, &graph);
      if (st != PTYCHO_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
      }
      if (ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(ce, "capture of the batch iteration");
      }
      PT_CUDA(ee, "end capture");
      {
        size_t nn = 0;
        cudaError_t ge = cudaGraphGetNodes(graph, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (ge == cudaSuccess && nn) ge = cudaGraphGetNodes(graph, nodes.data(), &nn);
        for (size_t q = 0; q < nn && ge == cudaSuccess; ++q) {
          cudaGraphNodeType ty;
          ge = cudaGraphNodeGetType(nodes[q], &ty);
          if (ge == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
        }
        if (ge != cudaSuccess) {
          cudaGraphDestroy(graph);
          return cuda_fail(ge, "count the batch graph's kernels");
        }
      }
      const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      PT_CUDA(ie, "instantiate the batch graph");
      pl->graphs.emplace_back(key, exec);
      pl->graph_descs.push_back(descs);
      pl->graph_kernels.push_back(kernels);
    }
    pl->last_kernels = kernels;
    PT_CUDA(cudaEventRecord(pl->ev_in, pl->stream), "event");
    PT_CUDA(cudaStreamWaitEvent(pl->origin, pl->ev_in, 0), "wait");
    PT_CUDA(cudaGraphLaunch(exec, pl->origin), "graph launch");
    PT_CUDA(cudaEventRecord(pl->ev_out, pl->origin), "event");
    PT_CUDA(cudaStreamWaitEvent(pl->stream, pl->ev_out, 0), "wait");
    for (ptycho_plan_s* m : pl->members) {
      m->iter++;
      m->runs++;
      m->dm_fresh = false;  // a replayed graph started every pc-DM state it holds
    }
  }
  return PTYCHO_OK;
}

ptycho_status ptycho_set_batch_chunk(int32_t chunk_len) {
  if (chunk_len != 0 && chunk_len != 8 && chunk_len != 16 && chunk_len != 32 && chunk_len != 64)
    return fail(PTYCHO_EINVAL, "chunk length must be 0 (autotune), 8, 16, 32 or 64");
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_fixed_chunk = chunk_len;
  return PTYCHO_OK;
}

ptycho_status ptycho_set_staged_chunk(int32_t chunk) {
  if (chunk != 0 && chunk != 4 && chunk != 8 && chunk != 16 && chunk != 32)
    return fail(PTYCHO_EINVAL, "staged chunk must be 0 (autotune), 4, 8, 16 or 32");
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_fixed_staged = chunk;
  return PTYCHO_OK;
}

int32_t ptycho_staged_chunk(ptycho_plan_t pl) { return (pl && pl->big) ? pl->chunk : 0; }

ptycho_status ptycho_batch_launches(ptycho_plan_t pl, int32_t* kernels) {
  if (!pl || pl->members.empty() || !kernels) return fail(PTYCHO_EINVAL, "not a batch plan or bad output");
  *kernels = pl->last_kernels;
  return PTYCHO_OK;
}

ptycho_status ptycho_batch_classes(ptycho_plan_t pl, int32_t max_classes, int32_t* out, int32_t* count) {
  if (!pl || pl->members.empty() || !count || max_classes < 0 || (max_classes > 0 && !out))
    return fail(PTYCHO_EINVAL, "not a batch plan or bad output");
  *count = (int32_t)pl->qclasses.size();
  for (int c = 0; c < std::min<int>(max_classes, *count); ++c) {
    const auto& qc = pl->qclasses[c];
    const int32_t v[8] = {qc.M, qc.K, qc.near, qc.kh, (int32_t)qc.members.size(), qc.chunk_len, qc.nchunks, qc.slots};
    std::memcpy(out + 8 * c, v, sizeof(v));
  }
  return PTYCHO_OK;
}

ptycho_status ptycho_error_batch(ptycho_plan_t pl, double* nrmse_last) {
  if (!pl || pl->members.empty() || !nrmse_last) return fail(PTYCHO_EINVAL, "not a batch plan or NULL output");
  PT_CUDA(cudaStreamSynchronize(pl->stream), "stream sync");
  bool timed_out = false;
  PT_CUDA(fused_timed_out(&timed_out), "read wait status");
  if (timed_out) return fail(PTYCHO_ETIMEOUT, "a bounded device wait gave up; results are not valid");
  bool finite = true;
  for (size_t b = 0; b < pl->members.size(); ++b) {
    const ptycho_plan_s* m = pl->members[b];
    if (m->runs == 0) return fail(PTYCHO_EINVAL, "no iteration has run");
    PT_CUDA(cudaMemcpy(&nrmse_last[b], m->d_errhist + (m->runs - 1) % kErrHistory, sizeof(double),
                       cudaMemcpyDeviceToHost),
            "copy error");
    finite = finite && std::isfinite(nrmse_last[b]);
  }
  if (!finite) return fail(PTYCHO_ENUMERIC, "an error metric is not finite");
  return PTYCHO_OK;
}

ptycho_status ptycho_error(ptycho_plan_t pl, double* nrmse_last) {
  if (!pl || !nrmse_last) return fail(PTYCHO_EINVAL, "NULL argument");
  if (!pl->members.empty()) return fail(PTYCHO_EINVAL, "batch plans report through ptycho_error_batch");
  PT_CUDA(cudaStreamSynchronize(pl->stream), "stream sync");
  if (pl->runs == 0) return fail(PTYCHO_EINVAL, "no iteration has run");
  bool timed_out = false;
  PT_CUDA(fused_timed_out(&timed_out), "read wait status");
  if (timed_out) return fail(PTYCHO_ETIMEOUT, "a bounded device wait gave up; results are not valid");
  double e = 0.0;
  PT_CUDA(cudaMemcpy(&e, pl->d_errhist + (pl->runs - 1) % kErrHistory, sizeof(double), cudaMemcpyDeviceToHost),
          "copy error");
  *nrmse_last = e;
  if (!std::isfinite(e)) return fail(PTYCHO_ENUMERIC, "error metric is not finite");
  return PTYCHO_OK;
}

ptycho_status ptycho_error_history(ptycho_plan_t pl, double* out, int32_t n, int32_t* count) {
  if (!pl || !out || !count || n < 0) return fail(PTYCHO_EINVAL, "bad argument");
  if (!pl->members.empty()) return fail(PTYCHO_EINVAL, "batch plans report through ptycho_error_batch");
  PT_CUDA(cudaStreamSynchronize(pl->stream), "stream sync");
  const long long c = std::min<long long>({(long long)n, pl->runs, (long long)kErrHistory});
  std::vector<double> ring(kErrHistory);
  PT_CUDA(cudaMemcpy(ring.data(), pl->d_errhist, sizeof(double) * kErrHistory, cudaMemcpyDeviceToHost),
          "copy error history");
  for (long long i = 0; i < c; ++i) out[i] = ring[(pl->runs - c + i) % kErrHistory];
  *count = (int32_t)c;
  return PTYCHO_OK;
}

ptycho_status ptycho_destroy(ptycho_plan_t pl) {
  if (!pl) return PTYCHO_OK;
  cudaSetDevice(pl->device);
  cudaStreamSynchronize(pl->stream);
  if (pl->origin) cudaStreamSynchronize(pl->origin);
  delete pl;
  return PTYCHO_OK;
}

ptycho_status ptycho_profile(ptycho_plan_t pl, int32_t enable) {
  if (!pl) return fail(PTYCHO_EINVAL, "plan is NULL");
  if (!pl->members.empty()) return fail(PTYCHO_EINVAL, "profiling applies to single plans");
  if (enable && pl->ev.empty()) {
    pl->ev.resize(2 * ptycho_plan_s::kProfSlots);
    for (cudaEvent_t& e : pl->ev) PT_CUDA(cudaEventCreate(&e), "cudaEventCreate");
  }
  pl->profiling = enable != 0;
  pl->prof_count = 0;
  for (auto& g : pl->sgraphs) g.pending = false;  // earlier replays' times are dropped
  pl->prof_graph_ms = 0.0;
  pl->prof_graph_n = 0;
  return PTYCHO_OK;
}

ptycho_status ptycho_profile_read(ptycho_plan_t pl, double* fused_ms, int32_t* launches) {
  if (!pl || !fused_ms || !launches) return fail(PTYCHO_EINVAL, "NULL argument");
  PT_CUDA(cudaStreamSynchronize(pl->stream), "stream sync");
  const int c = std::min(pl->prof_count, ptycho_plan_s::kProfSlots);
  double tot = 0.0;
  for (int i = 0; i < c; ++i) {
    float ms = 0.f;
    PT_CUDA(cudaEventElapsedTime(&ms, pl->ev[2 * i], pl->ev[2 * i + 1]), "cudaEventElapsedTime");
    tot += ms;
  }
  // and the iterations that ran as graph replays
  for (auto& g : pl->sgraphs) {
    const ptycho_status hs = harvest(pl, g);
    if (hs != PTYCHO_OK) return hs;
  }
  *fused_ms = tot + pl->prof_graph_ms;
  *launches = c + pl->prof_graph_n;
  pl->prof_count = 0;
  pl->prof_graph_ms = 0.0;
  pl->prof_graph_n = 0;
  return PTYCHO_OK;
}

int32_t ptycho_launches_per_iteration(ptycho_plan_t pl, int32_t in_window) {
  if (!pl) return 0;
  const int passes = pl->p.geometry == PTYCHO_NEARFIELD ? 7 : 5;  // staged passes per chunk
  int fft = 1;
  // pc-DM: the estimate sweep stops after the modulus pass (3 far, 4 near)
  const int dm_extra = pl->p.geometry == PTYCHO_NEARFIELD ? 4 : 3;
  if (pl->big) fft = (pl->p.N + pl->chunk - 1) / pl->chunk * (pl->d_psi ? passes + dm_extra : passes);
  if (pl->mb > 0) {  // per batch: its fused launch or staged passes, and the 4 update kernels; the error
    fft = -4 + 1;    // finish after the batches
    for (int b = 0; b < pl->nb; ++b) {
      const int len = std::min(pl->mb, pl->p.N - b * pl->mb);
      fft += (pl->big ? (len + pl->chunk - 1) / pl->chunk * passes : 1) + 4;
    }
  }
  if (pl->d_psi) fft += 2;                // pc-DM probe partials and their gather (probe step on)
  // update: probe gather, object gather (one clustered launch), object step, probe step;
  // constraint: row prefix sums, box sums, tile apply
  return fft + 4 + (in_window ? 3 : 0);
}

ptycho_status ptycho_permutation(int32_t n, uint64_t seed, int32_t stream, int32_t t, int32_t* out) {
  if (n < 0 || (n > 0 && !out)) return fail(PTYCHO_EINVAL, "need n >= 0 and an output array");
  const std::vector<int> a = philox_permutation(n, seed, (uint32_t)stream, (uint32_t)t);
  for (int i = 0; i < n; ++i) out[i] = a[i];
  return PTYCHO_OK;
}

ptycho_status ptycho_monochromatise(int32_t M, int32_t J, const double* scale, const double* weight, int32_t N,
                                    int32_t k, const float* b, float* x, double* resid, int32_t clamp,
                                    void* cuda_stream) {
  if (M <= 0 || N < 0 || k < 0 || J <= 0) return fail(PTYCHO_EINVAL, "need M > 0, J > 0, N >= 0, k >= 0");
  if (M != 8 && M != 16 && M != 32 && M != 64 && M != 128 && M != 256)
    return fail(PTYCHO_EUNSUPPORTED, "monochromatisation handles M = 8, 16, 32, 64, 128, 256");
  if (J > kMonoMaxJ) return fail(PTYCHO_EUNSUPPORTED, "more than 64 spectral samples");
  if (!scale || !weight) return fail(PTYCHO_EINVAL, "scale and weight must be non-NULL");
  if (N > 0 && (!b || !x)) return fail(PTYCHO_EINVAL, "b and x must be non-NULL");
  if (clamp != 0 && clamp != 1) return fail(PTYCHO_EINVAL, "clamp must be 0 or 1");
  MonoArgs a{};
  double wsum = 0.0;
  for (int j = 0; j < J; ++j) {
    if (!(scale[j] > 0.0 && scale[j] <= 2.5)) return fail(PTYCHO_EINVAL, "scale values must lie in (0, 2.5]");
    if (!(weight[j] >= 0.0 && std::isfinite(weight[j]))) return fail(PTYCHO_EINVAL, "weights must be finite, >= 0");
    wsum += weight[j];
    a.a[j] = (float)scale[j];
    a.inv_a[j] = (float)(1.0 / scale[j]);
    a.w[j] = (float)(weight[j] / (scale[j] * scale[j]));
  }
  if (!(wsum > 0.0)) return fail(PTYCHO_EINVAL, "weights are all zero");
  a.b = b;
  a.x = x;
  a.resid = resid;
  a.N = N;
  a.M = M;
  a.J = J;
  a.k = k;
  a.clamp = clamp;
  PT_CUDA(launch_mono(a, static_cast<cudaStream_t>(cuda_stream)), "monochromatisation launch");
  g_last_error.clear();
  return PTYCHO_OK;
}

const char* ptycho_last_error(void) { return g_last_error.c_str(); }

ptycho_status ptycho_wait_selftest(int64_t budget_ns, int32_t signal, void* cuda_stream) {
  if (budget_ns < 0 || budget_ns > 2000000000LL) return fail(PTYCHO_EINVAL, "budget_ns must be in [0, 2e9]");
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  bool pending = false;
  PT_CUDA(fused_timed_out(&pending), "read wait status");
  if (pending) return fail(PTYCHO_ETIMEOUT, "a bounded device wait of an earlier launch had given up");
  PT_CUDA(launch_wait_selftest((unsigned long long)budget_ns, signal != 0, s), "self-test launch");
  PT_CUDA(cudaStreamSynchronize(s), "stream sync");
  bool timed_out = false;
  PT_CUDA(fused_timed_out(&timed_out), "read wait status");
  if (timed_out) return fail(PTYCHO_ETIMEOUT, "the self-test wait gave up after its budget");
  return PTYCHO_OK;
}

const char* ptycho_version(void) { return "ptycho-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// ---- helpers shared with the allocation-free entry point (capi_static.cu)
namespace ptycho {
ptycho_status capi_validate(const ptycho_params* p) { return validate(p); }
void capi_step_coefficients(const ptycho_params* p, UpdateArgs* u) { step_coefficients(*p, *u); }
ptycho_status capi_fail(ptycho_status s, const std::string& msg) { return fail(s, msg); }
void capi_tile_lists(const std::vector<int2>& pos, int M, int tx, int ty, std::vector<int>& start,
                     std::vector<int4>& flat) {
  append_tile_lists(pos, 0, (int)pos.size(), M, tx, ty, start, flat);
}
ptycho_status capi_cuda_fail(cudaError_t e, const char* what) { return cuda_fail(e, what); }
std::vector<double> capi_taps(double sigma, int h) { return taps_1d(sigma, h); }
bool capi_is_device_pointer(const void* ptr) { return is_device_pointer(ptr); }
void capi_clear_error() { g_last_error.clear(); }
}  // namespace ptycho
