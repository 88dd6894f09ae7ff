// Internal declarations shared by the engine's translation units (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace ptycho {

constexpr int kMaxTaps = 31;        // largest odd Gaussian kernel side accepted (Eq. 7 support)
constexpr int kObjTile = 32;        // object tile side of the gather kernels
constexpr int kMaxModes = 8;        // probe modes K handled (one cluster rank per mode)
constexpr int kObjSplit = 8;        // position groups per object tile (one cluster, fixed order)
constexpr int kErrHistory = 4096;   // ring of per-iteration errors kept on the device

// Arguments of the fused per-position kernel (one cluster of K CTAs per position).
struct FusedArgs {
  const float2* O;      // object, obj_h x obj_w, row-major
  const float2* P;      // probe modes, K x M x M
  const float* I;       // measured intensities, N x M x M (far field: DC at (M/2, M/2))
  const float* sqrtI;   // sqrt of the measured intensities (computed once per plan)
  const int2* pos;      // top-left (row, col) of each box
  int N, K, obj_w;
  int near_field;       // 0: centred FFT; 1: Fresnel transfer function
  int blur_intensity;   // 0: blur the amplitude (Eq. 6); 1: blur the intensity (Eq. 2)
  int kh;               // kernel half-width, taps in [-kh, kh]
  float eps;            // modulus guard
  float gx[kMaxTaps];   // taps along x (columns, sigma_1)
  float gy[kMaxTaps];   // taps along y (rows, sigma_2)
  const float2* tw;     // W_M^m, m in [0, M)
  const float2* hq;     // near field: h[u] = exp(-i pi fu^2 / (M F)), H[u, v] = h[u] h[v]
  float2* cn;           // out: per-position object numerator contributions, N x M x M
  float2* pacc;         // out: per-slot probe numerator partials, slots x K x M x M (accumulated)
  float* dacc;          // out: per-slot probe denominator partials, slots x M x M (accumulated)
  double* errpart;      // out: per-CTA FP64 error numerators, slots x K
  // work-queue launches over several problems of one shape (M, K, geometry, blur kernel width):
  // chunk c = (problem index into probs, first position, end position, partial index); partials
  // (pacc, dacc, errpart) are indexed by the chunk's partial index instead of the slot
  const FusedArgs* probs;  // device, one entry per problem; unused by single-problem launches
  const int4* chunks;
  int nchunks;
  int* queue;  // device counter, zero before the launch
  // pc-DM launches: exit-wave state N x K x M x M (updated in place); dm_init: start it at P o_n
  float2* psi;
  int dm_init;
};

// single-problem fused launch (pc_fused_seq.cu: one CTA per position, modes in sequence) over
// `slots` persistent CTAs; fused_max_slots gives the co-resident CTAs of the GPU. Partials: pacc
// slots x K x M x M, dacc slots x M x M, errpart slots x K (the slot's error in entry 0)
cudaError_t launch_fused(int M, const FusedArgs& a, int slots, cudaStream_t s);
cudaError_t fused_max_slots(int M, int K, int* slots);
// cluster form for a single problem (one cluster of K CTAs per position, `slots` clusters); partials
// as launch_fused (errpart slots x K, one entry per rank)
cudaError_t launch_fused_cluster(int M, const FusedArgs& a, int slots, cudaStream_t s);
cudaError_t fused_cluster_max_slots(int M, int K, int* slots);
// work-queue launch (M = 32, 64, 128): `slots` persistent clusters drain a.chunks through a.queue;
// a.K, a.near_field, a.kh (kernel width class) and a.tw are those of every problem in a.probs
cudaError_t launch_fused_queue(int M, const FusedArgs& a, int slots, cudaStream_t s);
cudaError_t fused_queue_max_slots(int M, int K, int* slots);
// pc-DM launch (single problem, M <= 128): as launch_fused with the exit-wave state a.psi
cudaError_t launch_fused_dm(int M, const FusedArgs& a, int slots, cudaStream_t s);
cudaError_t fused_dm_max_slots(int M, int K, int* slots);
cudaError_t fused_dm_timed_out(bool* out);
bool fused_queue_supported(int M);
size_t fused_smem_bytes(int M);
// true if a bounded device wait of the fused kernel gave up since the last call (clears the flag; synchronous)
cudaError_t fused_timed_out(bool* out);
// one bounded mbarrier wait of the fused kernels' kind on a barrier that `signal` completes (or
// nothing does), giving up after budget_ns; its timeout shows in fused_timed_out
cudaError_t launch_wait_selftest(unsigned long long budget_ns, bool signal, cudaStream_t s);

// staged path for M = 256 and 512 (big.cu): a chunk of C positions x K modes in the scratch W
struct BigArgs {
  const float2* O; const float2* P; const float* I; const float* sqrtI; const int2* pos;
  int M;              // 256 or 512
  int N, K, obj_w;
  int near_field, blur_intensity, kh;
  float eps;
  float gx[kMaxTaps], gy[kMaxTaps];
  const float2* tw;   // W_M^m, m in [0, M)
  const float2* hq;   // near field: h[u]
  float2* W;          // C x K x M x M scratch
  float* R;           // C x M x M modulus ratios
  int n0;             // first position of the chunk
  int n_first;        // first position of the current accumulation (its chunk restarts the partials)
  float2* cn;         // N x M x M contributions
  float2* pacc;       // C x K x M x M probe partials (slot = position within the chunk)
  float* dacc;        // C x M x M
  double* errpart;    // N x big_row_blocks(M) error partials
  // pc-DM: exit-wave state (N x K x M x M) or null; dm_init: the state starts at P o_n this pass
  float2* psi;
  int dm_init;
  int dm_pass;        // pc-DM: 1 propagates P o_n for the error only, 2 propagates chi = 2 P o_n - psi_n
};
// the staged passes of one chunk; launch_big_chunk_dm: the two pc-DM sweeps (b.psi set)
cudaError_t launch_big_chunk(const BigArgs& b, int nc, cudaStream_t s);
cudaError_t launch_big_chunk_dm(const BigArgs& b, int nc, cudaStream_t s);
int big_row_blocks(int M);  // error partials per position (row blocks of the modulus pass)

// tcgen05 BF16 GEMM (unet_gemm.cu): D[M x Ntot] (+)= A[M x K] . B[Ntot x K]^T, bf16 operands
// stored as raw 16-bit words, K contiguous
struct GemmArgs {
  const uint16_t* A; const uint16_t* B;
  float* D; uint16_t* Dh; const float* bias;
  int M, Ntot, K, ldd;
  int mode;   // 0: D = AB^T (+ bias) (fp32); 1: D += AB^T (+ bias) (fp32); 2: Dh = act(AB^T + bias) (bf16);
              // bias optional (null: none), not with split-K
  int relu;
  int* status;  // set to 1 when a bounded wait gave up
  // implicit 3x3 convolution: row p of A is the zero-padded 3x3 neighbourhood of
  // pixel p of the NHWC tensor A (batch x H x W x Cin), k = tap * Cin + c,
  // tap = 3 (dy + 1) + (dx + 1); K may exceed 9 Cin (zero columns)
  int conv, H, W, Cin;
  // with conv: a 1 x 1 contraction over the Cin channels of each pixel instead of the 3x3 neighbourhood
  // (the input is an explicit neighbourhood already; halo kernel only)
  int taps1;
  // transposed implicit operand of a weight gradient: row k = tap * Cin + c of A over pixels p is
  // XT3[dx + 1][c][p + dy W] (zero where row y + dy leaves the image; zero for k >= 9 Cin), XT3 the
  // three x-shifted channel-major copies of the NHWC activation (Mpix pixels, W % 8 == 0)
  int convT, Mpix;
  // split-K (mode 0 only): blockIdx.z walks K columns [z kc, min(K, (z + 1) kc)) and stores
  // its partial product at D + z dsplit; 1 = no split
  int ksplit, kc;
  size_t dsplit;
  // implicit convolutions: B packed by halo_pack (then the halo kernel runs), or null
  const uint16_t* Bp;
};
cudaError_t launch_gemm_bf16(const GemmArgs& g, cudaStream_t s);
// the halo kernel's weight order for convolution g (g.B packed into halo_pack_elems(g) bf16 at dst)
bool halo_conv_supported(const GemmArgs& g);
size_t halo_pack_elems(const GemmArgs& g);
cudaError_t halo_pack(const GemmArgs& g, uint16_t* dst, cudaStream_t s);

// update / reduction kernels (update.cu)
struct UpdateArgs {
  float2* O; float2* P;
  const int2* pos;
  int N, K, M, obj_h, obj_w, slots;
  const float2* cn; const float2* pacc; const float* dacc; const double* errpart;
  int nerr;  // entries of errpart
  // object gather
  const int* tile_start;  // (tiles_y * tiles_x + 1) CSR offsets into tile_pos
  const int4* tile_pos;   // per tile, (n, row, col, 0) of each overlapping position, increasing n
  int tiles_x, tiles_y;
  float2* no_part; float* do_part;  // N_O and D_O, obj_h x obj_w each
  float* blk_max_o;                  // per object tile
  // probe gather
  float2* np_sum; float* dp_sum; float* p2;  // K x M x M, M x M, M x M
  float* blk_max_p;
  int probe_blocks;
  double* errhist; double errden;
  unsigned long long* run_counter;  // device: iterations finished; E goes to errhist[counter % kErrHistory]
  // error of a launch: 0 finishes E from this launch's partials; 1 adds them to *err_acc (a batch
  // of a mini-batch iteration); 2 adds them and finishes E from the total, clearing *err_acc
  int err_mode;
  double* err_acc;
  // step = beta num / (c_d d + c_max max d): normalised rule (1, delta), rPIE rule (1 - a, a)
  float beta_obj, beta_probe, cd_obj, cmax_obj, cd_probe, cmax_probe;
  int update_probe;
  // pc-DM: exit-wave state (N x K x M x M). When set, the probe step follows the object step and is
  // taken from the new object and this state (alternating overlap projection)
  float2* dm_psi;
  // pc-DM inside a complex-constraint window: the object before the constraint (the states move by
  // P (O - dm_obj_prev) under their boxes); null otherwise
  const float2* dm_obj_prev;
};
// launch_update = launch_update_object then launch_update_probe (pc-DM runs the complex constraint
// between the two)
cudaError_t launch_update(const UpdateArgs& u, cudaStream_t s);
cudaError_t launch_update_object(const UpdateArgs& u, cudaStream_t s);
cudaError_t launch_update_probe(const UpdateArgs& u, cudaStream_t s);
// finishes E of a mini-batch iteration from *err_acc (every batch ran with err_mode 1)
cudaError_t launch_err_finish(const UpdateArgs& u, cudaStream_t s);

// numerical monochromatisation by CGLS (mono.cu): x_n = k CGLS steps on min ||C x - b_n|| from 0,
// C = sum_j w[j] T_j, T_j sampling at c + (i - c) inv_a[j] (c = M / 2) with linear interpolation and
// zero outside; one CTA per pattern
constexpr int kMonoMaxJ = 64;
struct MonoArgs {
  const float* b; float* x;  // N x M x M each (x may be b)
  double* resid;             // N x (k + 1) residual norms ||b - C x_i||, or null
  int N, M, J, k, clamp;
  float inv_a[kMonoMaxJ], a[kMonoMaxJ], w[kMonoMaxJ];  // 1 / a_j, a_j, weight_j / a_j^2
};
cudaError_t launch_mono(const MonoArgs& a, cudaStream_t s);

// complex constraint (constraint.cu)
struct ConstraintArgs {
  float2* O; const int2* pos; int N, M, obj_h, obj_w;
  float* cbar; float alpha1, alpha2, cbar_min, cbar_max;
  long long* map_lna; long long* map_phi;  // row prefix sums of |ln a|, |phi|: obj_h x (obj_w + 1), 32.32
  long long* cbar_q;                       // C_n in 32.32 fixed point (N)
  const int* tile_start;  // (tiles_y * tiles_x + 1) CSR offsets into tile_pos, kObjTile tiles
  const int4* tile_pos;   // per tile, (n, row, col, 0) of every position whose box overlaps it
  int tiles_x, tiles_y;
};
cudaError_t launch_constraint(const ConstraintArgs& c, cudaStream_t s);

// plan-time helpers (update.cu)
cudaError_t launch_intensity_sums(const float* I, size_t count, double* partials, int nblocks, cudaStream_t s);
cudaError_t launch_finish_sums(const double* partials, int nblocks, double* out2, cudaStream_t s);
cudaError_t launch_sqrt(const float* I, float* out, size_t count, cudaStream_t s);

// warm-start data generator and assembly (gen.cu)
struct GenArgs {
  const float2* probe;   // S x S probe
  const float4* params;  // per pattern: (lattice rotation, origin row, origin col, blur sigma)
  int n;                 // patterns
  uint32_t first;        // sample index of the first pattern (Philox counter word)
  uint32_t key_lo, key_hi;
  float dose;            // photons / electrons per pattern
  float a, peak, s_pk, cutoff;  // lattice constant (px), peak phase (rad), peak sd (px), peak radius (px)
  uint32_t vac_thresh;           // a site is vacant when its Philox word is below this
  float target_scale;    // targets are (ln |o|, arg o) / target_scale
  int noise;             // 0: counts = the noise-free intensities
  float* x;              // n x S x S network input log1p(counts) / 4, or nullptr
  float* counts;         // n x S x S, or nullptr
  float* clean;          // n x S x S dose-scaled noise-free intensities, or nullptr
  float* target;         // n x (S/2) x (S/2) x 2, or nullptr
  float* sigma;          // n, or nullptr
};
cudaError_t launch_gen(int S, const GenArgs& a, cudaStream_t s);
size_t gen_smem_bytes(int S);
cudaError_t launch_log_input(const float* I, float* x, size_t count, cudaStream_t s);
constexpr int kStitchMaxQ = 256;  // stitch: patch side at most
struct StitchArgs {
  const float* patches;   // N x patch x patch x 2 network outputs
  int patch;              // patch side (<= kStitchMaxQ)
  float scale;            // patch value = exp(scale (out0 + i out1))
  const int* tile_start;  // CSR over kObjTile x kObjTile object tiles
  const int4* tile_pos;   // (n, corner row, corner col, 0), increasing n
  int tiles_x, tiles_y, obj_h, obj_w;
  float2* O;              // out: obj_h x obj_w
};
cudaError_t launch_stitch(const StitchArgs& a, cudaStream_t s);
cudaError_t launch_median(float* v, int n, int npad, double* out, cudaStream_t s);

}  // namespace ptycho
