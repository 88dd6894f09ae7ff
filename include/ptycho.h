/*
 * ptycho.h -- C ABI of the GB300 data-parallel partially coherent ptychographic engine.
 *
 * The engine runs the paper's partially coherent ptychographic iteration
 * (Xu, Ning et al., "A high-performance reconstruction method for partially
 * coherent ptychography", arXiv 2406.06640) in its simultaneous form: every
 * scan position n uses the same object O and probe modes P_k, and the object
 * and probe move by a normalised scatter-add of all positions' corrections.
 *
 * One iteration t (1-based):
 *   psi_{n,k} = P_k . o_n,  o_n the M x M box of O at positions[n]   (Eq. 1, Fig. 1)
 *   Psi_{n,k} = far field: centred 2-D DFT of psi (Eq. 1);
 *               near field: IDFT(DFT(psi) H), H = exp(-i pi (u^2 + v^2) / (M F)),
 *               u, v the signed integer frequencies (Sec. 3.1, near-field setup)
 *   amplitude blur (default, Eq. 6):  A^G = sqrt(sum_k |Psi_k|^2) (x) g,
 *       Ihat = (A^G)^2, R = sqrt(I_n) / (A^G + eps)
 *   intensity blur (Eq. 2):           I_m = (sum_k |Psi_k|^2) (x) g,
 *       Ihat = I_m, R = sqrt(I_n) / sqrt(I_m + eps^2)
 *       g: Eq. 7, kernel_size x kernel_size, sigma1 along x (columns),
 *       sigma2 along y (rows), normalised to sum 1, zero padding; sigma = 0
 *       makes that axis a delta (the coherent engine)
 *   Psi' = R Psi (Fig. 1 box 1), psi' = inverse propagation, dpsi = psi' - psi
 *   O   += beta_obj   sum_n conj(P) dpsi / (D_O + delta_obj   max D_O),  D_O = sum_n sum_k |P_k|^2
 *   P_k += beta_probe sum_n conj(o_n) dpsi_k / (D_P + delta_probe max D_P), D_P = sum_n |o_n|^2
 *       (pixels with a zero denominator are left unchanged; the probe moves
 *        from iteration probe_update_start on)
 *   inside a complex-constraint window: Eqs. 9-11 on the new object, C_n
 *       clamped to [cbar_min, cbar_max] (Sec. 4.8) and averaged per pixel
 *       over the covering boxes
 *   E_t = sqrt(sum (Ihat - I)^2 / sum I^2) in FP64 (the NRMSE of Sec. 4.2),
 *       evaluated on the state before the update of iteration t.
 *
 * Layouts: complex values are interleaved float pairs (re, im) = complex64.
 * Object: obj_h x obj_w, row-major. Probe: K x M x M, row-major per mode.
 * Intensities: N x M x M float32; far field in the detector-centred frame
 * (zero frequency at (M/2, M/2)); near field in the detector plane.
 * Positions: N pairs (row, col) of int32, the top-left corner of each box;
 * every box must lie inside the object.
 *
 * Errors: every call returns a ptycho_status; no C++ exception crosses the
 * ABI. ptycho_last_error() returns a message for the calling thread's last
 * failure. Calls on one plan must not run concurrently from several threads.
 */
#ifndef PTYCHO_H_
#define PTYCHO_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ptycho_plan_s* ptycho_plan_t; /* opaque, owned by the library */

typedef enum {
  PTYCHO_OK = 0,
  PTYCHO_EINVAL = 1,       /* invalid parameter, size or position */
  PTYCHO_ENOMEM = 2,       /* device allocation failed */
  PTYCHO_ECUDA = 3,        /* a CUDA call failed (message in ptycho_last_error) */
  PTYCHO_EUNSUPPORTED = 4, /* valid request this build does not handle */
  PTYCHO_ENUMERIC = 5,     /* non-finite input or non-finite error metric */
  PTYCHO_ETIMEOUT = 6      /* a bounded device-side wait gave up */
} ptycho_status;

enum { PTYCHO_FARFIELD = 0, PTYCHO_NEARFIELD = 1 };
enum { PTYCHO_BLUR_AMPLITUDE = 0 /* Eq. 6 */, PTYCHO_BLUR_INTENSITY = 1 /* Eq. 2 */ };
enum { PTYCHO_STEP_NORMALISED = 0, PTYCHO_STEP_RPIE = 1 };
enum { PTYCHO_ENGINE_PIE = 0, PTYCHO_ENGINE_DM = 1 };

typedef struct {
  int32_t M;            /* probe = box = detector side, power of two, 8..512 */
  int32_t K;            /* probe modes (mixed state, Sec. 4.4), 1..8 */
  int32_t N;            /* scan positions, >= 1 */
  int32_t obj_h, obj_w; /* object size, >= M */
  int32_t geometry;     /* PTYCHO_FARFIELD or PTYCHO_NEARFIELD */
  int32_t blur_domain;  /* PTYCHO_BLUR_AMPLITUDE (default) or PTYCHO_BLUR_INTENSITY */
  double fresnel_F;     /* near field: F = M dx^2 / (lambda z) > 0; ignored in the far field */
  double sigma1;        /* Eq. 7 blur width along x (columns), pixels, >= 0 */
  double sigma2;        /* Eq. 7 blur width along y (rows), pixels, >= 0 */
  int32_t kernel_size;  /* odd, 1..31; the paper uses 11 (Sec. 3.1) */
  double eps_mod;       /* modulus guard in amplitude units; 0 => 1e-6 sqrt(mean I) */
  double beta_obj, beta_probe;   /* step sizes, typically 1 */
  double delta_obj, delta_probe; /* relative denominator floors, >= 0, typically 1e-3 */
  int32_t probe_update_start;    /* first iteration (1-based) that moves the probe */
  double alpha1, alpha2;         /* Eqs. 9-10 weights in [0, 1] */
  double cbar_min, cbar_max;     /* Sec. 4.8 clamp of C_n, 0 < cbar_min <= cbar_max */
  int32_t n_windows;             /* number of complex-constraint windows */
  const int32_t* windows;        /* host, 2 * n_windows: [first, last], 1-based inclusive */
  int32_t start_iteration;       /* number of the first iteration (resume), >= 1 */
  /* Step rule of the object / probe update (zero-initialised: the normalised rule above).
   * PTYCHO_STEP_RPIE uses the regularised denominator of the rPIE family (Sec. 5, Fig. 11c)
   *   O   += beta_obj   N_O / ((1 - a_O) D_O + a_O max D_O),
   *   P_k += beta_probe N_P / ((1 - a_P) D_P + a_P max D_P),  a in [0, 1];
   * a = 1 is the ePIE-style max-normalised step, a = 0 the plain normalised step without a
   * floor. Pixels with a zero denominator are left unchanged under both rules. */
  int32_t step_rule;             /* PTYCHO_STEP_NORMALISED (0) or PTYCHO_STEP_RPIE (1) */
  double rpie_alpha_obj, rpie_alpha_probe;
  /* Mini-batch (sequential) engine, the paper's pc-ePIE of Fig. 1 for minibatch = 1: 0 (default)
   * or >= N runs every position in one simultaneous step. Otherwise the positions are split into
   * batches of `minibatch` by a Philox4x32-10 permutation keyed by order_seed (ptycho_permutation
   * with stream 3, t = 0, consecutive groups), and iteration t visits the batches in the order of
   * ptycho_permutation(batches, order_seed, 4, t); each batch takes one step of the rule above over
   * its own positions, from the object and probe the previous batch left. The complex constraint
   * (inside its windows) follows the last batch; E_t sums every position's error numerator at the
   * state its batch saw. Every M (M = 256 and 512 run each batch through the staged passes); not available
   * in batch plans or ptycho_iterate_static. */
  int32_t minibatch;
  uint64_t order_seed;
  /* Engine: PTYCHO_ENGINE_PIE (0, default) takes the steps above from dpsi = Pi_F(P o_n) - P o_n;
   * PTYCHO_ENGINE_DM (1) is pc-DM (Sec. 4.5, the difference map with the pc intensity model): the
   * plan keeps an exit wave psi_{n,k} per position and mode (N K M^2 complex, started at P_k o_n
   * when the plan first iterates), each position forms chi = 2 P_k o_n - psi_{n,k}, runs it through
   * the propagation and the pc modulus step, sets psi_{n,k} <- psi_{n,k} + Pi_F(chi) - P_k o_n,
   * and the overlap projection alternates: O takes the step of the chosen rule with
   * dpsi = psi_{n,k} - P_k o_n; inside a complex-constraint window the constraint acts on O next
   * and every psi_{n,k} moves by P_k (o_n after - o_n before); then P takes its step from the new
   * object, sum conj(o'_n) (psi_{n,k} - P_k o'_n) over sum |o'_n|^2. E_t is the pc model error
   * of the estimate P_k o_n. Every M (M = 256 and 512 sweep the staged passes twice per chunk, the
   * estimate for the error and chi to the state update); without mini-batches; in single and
   * batch plans (a batch member keeps its own launches), not in ptycho_iterate_static. */
  int32_t engine;
} ptycho_params;

/* Build a plan on the current CUDA device.
 *   p           parameters (copied; `windows` may be freed on return)
 *   intensities device pointer, N * M * M float32 measured intensities; copied
 *               into the plan, so the caller may free them on return. Negative
 *               values give PTYCHO_EINVAL, non-finite ones PTYCHO_ENUMERIC.
 *   positions   host or device pointer, N * 2 int32 (row, col) top-left corners;
 *               a box outside the object gives PTYCHO_EINVAL
 *   cuda_stream cudaStream_t the plan launches on (NULL: the legacy default stream)
 *   out         receives the plan; the caller releases it with ptycho_destroy
 * Blocks until the plan-time reductions are done. */
ptycho_status ptycho_plan(const ptycho_params* p, const float* intensities, const int32_t* positions,
                          void* cuda_stream, ptycho_plan_t* out);

/* Run n_iter >= 0 iterations in place, asynchronously on the plan's stream.
 *   object  device, obj_h * obj_w complex64, read and written
 *   probe   device, K * M * M complex64, read and written
 * The iteration counter continues across calls (windows and
 * probe_update_start refer to it). Do not touch object or probe until the
 * stream has been synchronised (ptycho_error does that).
 * Launch path: an iteration whose key (object and probe pointers, probe step on,
 * constraint window active, pc-DM state start) has run twice is captured once
 * as CUDA graphs (a ring of four) and replayed from then on, one graph launch
 * per iteration (mini-batch plans: one graph per batch); the results are those
 * of the eager launches. The first capture of a key costs host time in that
 * call. Up to 32 keys are kept per plan; further keys run eagerly. */
ptycho_status ptycho_iterate(ptycho_plan_t plan, void* object, void* probe, int32_t n_iter);

/* Synchronise the plan's stream and return E of the last iteration run
 * (host double). PTYCHO_EINVAL if no iteration has run yet; PTYCHO_ENUMERIC
 * if E is not finite. */
ptycho_status ptycho_error(ptycho_plan_t plan, double* nrmse_last);

/* Synchronise and copy the errors of the last min(n, runs, 4096) iterations,
 * oldest first, into out (host, n doubles); *count receives how many. */
ptycho_status ptycho_error_history(ptycho_plan_t plan, double* out, int32_t n, int32_t* count);

/* Release every device resource of the plan (synchronises its stream). */
ptycho_status ptycho_destroy(ptycho_plan_t plan);

/* Batched reconstructions: B independent problems (each with its own sizes,
 * geometry, blur and schedule), built once and iterated together. One
 * iteration of every problem is captured into a CUDA graph whose branches run
 * the problems concurrently on up to 8 streams; every later iteration with
 * the same pattern of probe updates and constraint windows (and the same
 * object / probe pointers) replays that graph with a single launch.
 *   params, intensities, positions  arrays of B entries, as for ptycho_plan
 *   cuda_stream  the caller's stream; each iteration waits for it and it
 *                waits for the iteration (events), so ordering is preserved
 * ptycho_plan_batch fails with the status of the first invalid problem and a
 * message naming it. ptycho_iterate_batch takes B object and B probe device
 * pointers (updated in place); ptycho_error_batch synchronises and writes the
 * last E of every problem (host, B doubles). ptycho_destroy releases a batch
 * plan and all its problems. Single-plan calls reject batch plans. pc-DM problems are
 * members with their own launches (the first iteration, which starts their exit-wave state, is a
 * graph of its own); mini-batch problems are rejected (PTYCHO_EUNSUPPORTED). */
ptycho_status ptycho_plan_batch(int32_t B, const ptycho_params* const* params, const float* const* intensities,
                                const int32_t* const* positions, void* cuda_stream, ptycho_plan_t* out);
ptycho_status ptycho_iterate_batch(ptycho_plan_t plan, void* const* objects, void* const* probes, int32_t n_iter);
ptycho_status ptycho_error_batch(ptycho_plan_t plan, double* nrmse_last);

/* Work-queue batching: problems with M in {32, 64, 128} sharing K, geometry and
 * kernel width class (11 x 11 or any other size) are drained by one persistent
 * launch per class; each chunk of L consecutive positions keeps its own probe and
 * error partials, summed in chunk order (results do not depend on which cluster
 * took a chunk). L is chosen per class by an autotuner the first time a batch
 * plan of that class is built on a device in the process: it times the class's
 * launch for L = 8, 16, 32, 64 on the device and keeps the fastest (cached per
 * device, M, K, geometry and kernel width class).
 * ptycho_set_batch_chunk fixes L for every later ptycho_plan_batch (8, 16, 32 or
 * 64; 0 restores tuning), e.g. for bitwise-reproducible runs across processes:
 * different L give the same result up to the FP32 order of the partial sums. */
ptycho_status ptycho_set_batch_chunk(int32_t chunk_len);
/* Staged path (M = 256, 512): positions per chunk of the staged passes (their scratch
 * holds chunk x K x M^2 complex values, so the chunk decides how much of it stays
 * in L2). Chosen per (device, M, K, geometry, kernel width class) by timing one
 * pass over all positions for 4, 8, 16 and 32 when the first such plan is built
 * in the process, then cached. ptycho_set_staged_chunk fixes it for later plans
 * (4, 8, 16 or 32; 0 restores tuning); the probe partials are per position of a
 * chunk, so different chunks change only the FP32 order of their sums.
 * ptycho_staged_chunk returns a plan's chunk (0 for M <= 128). */
ptycho_status ptycho_set_staged_chunk(int32_t chunk);
int32_t ptycho_staged_chunk(ptycho_plan_t plan);
/* Describe the work-queue classes of a batch plan: for each of the first
 * max_classes classes, 8 int32 (M, K, near field, kernel width class 5 or 15,
 * members, chunk length, chunks, persistent clusters) into out; *count = the
 * number of classes. */
ptycho_status ptycho_batch_classes(ptycho_plan_t plan, int32_t max_classes, int32_t* out, int32_t* count);

/* Kernel launches of one iteration of a batch plan: the kernel nodes of the CUDA graph that the last
 * ptycho_iterate_batch replayed per iteration (0 before the first call). kernels: host. EINVAL if
 * plan is not a batch plan or kernels is NULL. */
ptycho_status ptycho_batch_launches(ptycho_plan_t plan, int32_t* kernels);

/* Tensor-core GEMM used by the warm-start network (the paper has no learned
 * component; this is the contraction under its 3x3 convolutions):
 *   D[M x N] = A[M x K] . B[N x K]^T      (accumulate != 0: D += A . B^T)
 * A, B: device, bf16 bit patterns, row-major with K contiguous; D: device fp32,
 * row-major N x ... (leading dimension N). BF16 products, FP32 accumulation in
 * tensor memory (tcgen05). Requires M % 128 == 0, N % 16 == 0, K % 64 == 0,
 * 16-byte aligned A and B (PTYCHO_EINVAL otherwise). Synchronises `stream`;
 * PTYCHO_ETIMEOUT if a bounded device-side wait gave up. */
int ptycho_gemm_bf16(const uint16_t* A, const uint16_t* B, float* D, int M, int N, int K, int accumulate,
                     void* stream);

/* Per-kernel timing for roofline reports. While enabled, ptycho_iterate records
 * a CUDA event pair on the plan's stream around every launch of the fused
 * per-position kernel (the dominant kernel of an iteration); for M = 256 and 512 the
 * pair brackets the staged FFT / modulus passes of the iteration.
 * Graph replays record the pair as graph nodes; their times are read back
 * before a graph replays again and at ptycho_profile_read. For mini-batch
 * plans the pair brackets all batches of the iteration with their updates.
 * ptycho_profile_read synchronises the stream, returns the summed device time
 * of those launches in milliseconds and their count, and resets both. At most
 * 1024 eager launches are kept between reads (older ones are dropped from the sum). */
ptycho_status ptycho_profile(ptycho_plan_t plan, int32_t enable);
ptycho_status ptycho_profile_read(ptycho_plan_t plan, double* fused_ms, int32_t* launches);

/* Kernel launches one iteration issues: the fused kernel (M <= 128) or 5 (far)
 * / 7 (near) staged passes per chunk of positions (M = 256, 512; pc-DM 8 / 11), 4 update kernels
 * (2 more for pc-DM), per batch for the mini-batch engine, and 3 complex-constraint
 * kernels when `in_window` is non-zero (copies not counted). */
int32_t ptycho_launches_per_iteration(ptycho_plan_t plan, int32_t in_window);

/* Allocation-free one-shot run (this entry point has no counterpart in the paper).
 * For callers that must not call cudaMalloc -- e.g. code running while a
 * device memory pool or budget is locked, latency-critical loops that cannot
 * afford an allocation's implicit synchronisation, or hosts that own all
 * device memory -- it runs n_iter iterations exactly like ptycho_plan +
 * ptycho_iterate, but takes every scratch buffer from one file-scope device
 * array of 32 MiB that the library holds on each device until the process
 * exits. It calls no cudaMalloc, cudaFree or other allocating routine.
 *   p, intensities, positions  as for ptycho_plan (intensities: device, 16-byte aligned -- the
 *                              kernels read them in place; a misaligned pointer gives PTYCHO_EINVAL;
 *                              device positions are read on cuda_stream)
 *   object, probe              device, updated in place as by ptycho_iterate
 *   n_iter                     0..4096 (M <= 128; larger M gives PTYCHO_EUNSUPPORTED)
 *   errors                     host, n_iter doubles (E of each iteration), or NULL
 *   cuda_stream                stream to run on (NULL: the legacy default stream)
 * The scratch needed is about N M^2 (4 + 8) bytes + slots K M^2 8 bytes
 * + obj_h obj_w (8 x 12 + 28) bytes + small tables; a request larger than 32 MiB is
 * rejected with PTYCHO_EINVAL and a message giving the bytes it needs.
 * The call synchronises the stream before returning. The first call on a
 * device looks up the scratch's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture. Every call shares the one
 * scratch array and overwrites it (the call clears the one counter in it that
 * has to start at zero), so
 * calls that overlap on the GPU -- from several host threads or streams --
 * race and must be serialised by the caller. */
ptycho_status ptycho_iterate_static(const ptycho_params* p, const float* intensities, const int32_t* positions,
                                    void* object, void* probe, int32_t n_iter, double* errors, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Learned warm start (the paper has no learned component; it asks for no prior
 * knowledge of the source, so these calls estimate the object and the blur width
 * sigma from the patterns themselves before the iteration starts).
 *
 * A U-Net with 4 levels (base width C) maps log1p(I) / 4 of each S x S pattern to
 * (ln |o|, arg o) / target_scale on the central S/2 x S/2 box of its object patch
 * and to the pattern's sigma. 3x3 convolutions, ReLU, 2x2 average pooling,
 * nearest 2x upsampling with skip concatenation; BF16 activations and weights,
 * FP32 accumulation on the tcgen05 tensor cores, FP32 master weights and Adam.
 * Loss = mean((out - target)^2) + lam mean((sigma - sigma_t)^2).
 * ------------------------------------------------------------------------- */
typedef struct ptycho_unet_s* ptycho_unet_t;

/* Create a network for batches of `batch` patterns of S x S pixels (S % 16 == 0,
 * 16 <= S <= 512; C % 16 == 0, C <= 64; 1 <= batch <= 1024; batch (S/8)^2 a
 * multiple of 128), He-initialised from `seed`, on `cuda_stream`. */
ptycho_status ptycho_unet_create(int32_t S, int32_t C, int32_t batch, uint64_t seed, void* cuda_stream,
                                 ptycho_unet_t* out);
/* Number of floats of the flat parameter vector: for each convolution i = 0..6,
 * w_i (C_out, 9 taps, C_in) then b_i (C_out), tap = 3 (dy + 1) + (dx + 1); then
 * the sigma head w7 (8C) and b7 (1). */
int64_t ptycho_unet_param_count(ptycho_unet_t net);
/* Copy the parameters in (set) or out (get); host float arrays of param_count
 * entries. Both synchronise the network's stream. */
ptycho_status ptycho_unet_set_params(ptycho_unet_t net, const float* params, int64_t count);
ptycho_status ptycho_unet_get_params(ptycho_unet_t net, float* params_out, int64_t count);
/* Forward pass on `batch` inputs x (device, batch x S x S f32). out2: device,
 * batch x (S/2) x (S/2) x 2, or NULL; sigma: device, batch floats, or NULL.
 * Synchronises; PTYCHO_ETIMEOUT if a bounded tensor-core wait gave up. */
ptycho_status ptycho_unet_forward(ptycho_unet_t net, const float* x, float* out2, float* sigma);
/* Loss (host double) and every parameter gradient (host, param_count floats in the
 * flat order, or NULL) for one batch: x as above, target device batch x (S/2)^2 x 2,
 * sigma_t device batch floats. Synchronises. */
ptycho_status ptycho_unet_gradients(ptycho_unet_t net, const float* x, const float* target, const float* sigma_t,
                                    float lam, double* loss, float* grads);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on one batch.
 * With loss != NULL it synchronises and writes the batch loss (before the step);
 * with loss == NULL it only enqueues on the network's stream. */
ptycho_status ptycho_unet_train_step(ptycho_unet_t net, const float* x, const float* target, const float* sigma_t,
                                     float lam, float lr, double* loss);
ptycho_status ptycho_unet_destroy(ptycho_unet_t net);

/* Forward-model training data: far-field patterns of random hexagonal crystals
 * (Gaussian phase peaks of height `peak` rad and sd `peak_sd` px, lattice
 * constant `lattice_a` px, each site vacant with probability `vacancy` by
 * Philox4x32-10((i, j, sample, 1), key)), psi = P exp(i phi), the centred DFT
 * (Eq. 1), |Psi|^2 blurred by an isotropic Gaussian of the pattern's sigma
 * (Eq. 2; taps +-min(ceil(5 sigma), 15)), scaled to sum `dose`, then Poisson
 * counts (Philox4x32-10((pixel, sample, attempt, 2), key)) unless noise == 0. */
typedef struct {
  int32_t S;                /* pattern side: 64 or 128 */
  int32_t noise;            /* 0: counts are the noise-free intensities */
  double dose;              /* counts per pattern */
  double lattice_a, peak, peak_sd, cutoff, vacancy;  /* px, rad, px, px (peak radius, <= 2 lattice_a), probability */
  double target_scale;      /* targets = (ln |o|, arg o) / target_scale */
  uint64_t key;             /* Philox key (low word first) */
} ptycho_gen_spec;
/* params: device, n x 4 floats (lattice rotation rad, origin row px, origin col
 * px, sigma px), 16-byte aligned; probe: device complex64 S x S. Outputs
 * (device, each optional): x (n x S x S, log1p(counts)/4), counts, clean
 * (dose-scaled noise-free intensities), target (n x (S/2)^2 x 2, central box),
 * sigma (n). Pattern i uses sample index first + i. Asynchronous on `stream`. */
ptycho_status ptycho_generate(const ptycho_gen_spec* spec, const void* probe, const float* params, int32_t n,
                              uint32_t first, float* x, float* counts, float* clean, float* target, float* sigma,
                              void* cuda_stream);

/* Warm start: run the network over N measured patterns (device, N x S x S counts,
 * S the network's side), stitch the predicted central boxes (corner = position +
 * (S/4, S/4), side S/2, value exp(target_scale (out0 + i out1))) with a separable
 * Hann window into object_out (device complex64 obj_h x obj_w; 1 where no box
 * covers a pixel) and write the median predicted sigma to *sigma_out (host).
 * positions: host or device, N (row, col) int32 box corners; every box of side S
 * must lie inside the object. Runs on the network's stream and synchronises. Its scratch
 * (patches, sigmas, tile lists) is a buffer kept by the network and grown when a call needs
 * more, so repeated calls of the same size allocate nothing. */
ptycho_status ptycho_warmstart(ptycho_unet_t net, const float* intensities, const int32_t* positions, int32_t N,
                               int32_t obj_h, int32_t obj_w, double target_scale, void* object_out,
                               double* sigma_out);

/* The Philox permutation of 0..n-1 a mini-batch plan uses (Fisher-Yates: for i = n-1 .. 1,
 * j = (w (i + 1)) >> 32 with w the first word of Philox4x32-10((i, t, stream, 5), key = seed
 * as two 32-bit words, low first); out: host, n int32. For reproducing a plan's batches (stream 3,
 * t = 0) and visiting order (stream 4, iteration t). */
ptycho_status ptycho_permutation(int32_t n, uint64_t seed, int32_t stream, int32_t t, int32_t* out);

/* ---- Numerical monochromatisation (Sec. 4.2, Eqs. 12-13) ------------------------------------
 * A broadband far-field pattern is modelled as b = C m: the monochromatic pattern m at the
 * reference wavelength lambda_c, magnified about the detector centre c = M / 2 by each relative
 * wavelength a_j = lambda_j / lambda_c and weighted by weight_j / a_j^2 (the weight's share of the
 * energy):  (C m)(y, x) = sum_j weight_j / a_j^2 m(c + (y - c) / a_j, c + (x - c) / a_j), with linear
 * interpolation and zero outside the grid. For every pattern, x_n = k steps of CGLS on
 * min ||C x - b_n||_2 from x = 0: the least-squares solution over the Krylov subspace
 * span{C^T b, (C^T C) C^T b, ..., (C^T C)^(k-1) C^T b} (Eq. 13); k is the regularisation.
 *   M: 8, 16, 32, 64, 128 or 256 (EUNSUPPORTED otherwise); J: 1..64 spectral samples;
 *   scale: host, J values a_j in (0, 2.5]; weight: host, J finite values >= 0, not all zero;
 *   N >= 0 patterns; k >= 0 steps;
 *   b: device float32, N x M x M, row-major, detector-centred (DC at (M/2, M/2));
 *   x: device float32, N x M x M (x == b is allowed: each pattern is read before it is written);
 *   resid: device float64, N x (k + 1) residual norms ||b_n - C x_i|| for i = 0..k, or NULL;
 *   clamp: 1 sets negative values of x to zero (the pc engine takes non-negative patterns).
 * Enqueued on cuda_stream (NULL: the default stream); returns before the work finishes. The caller
 * owns every buffer. PTYCHO_EINVAL for invalid sizes, values or NULL buffers, PTYCHO_ECUDA for a
 * failed launch. Computed in FP32 with FP64 step sizes and norms. */
ptycho_status ptycho_monochromatise(int32_t M, int32_t J, const double* scale, const double* weight, int32_t N,
                                    int32_t k, const float* b, float* x, double* resid, int32_t clamp,
                                    void* cuda_stream);

/* Measured FP32 FMA throughput of the current device (a measurement utility; the paper has no
 * counterpart): the roofline denominator of the ALU-bound kernels beside the nominal SMs x 128
 * lanes x 2 FLOP x clock. Runs an FFMA loop (8 independent chains per thread, 4 CTAs of 256 threads
 * per SM) six times on cuda_stream and reports the best of the last five: *tflops (host) in
 * TFLOP/s and *ms (host) the duration of that launch. Synchronises the stream; allocates and frees
 * one small device buffer. PTYCHO_EINVAL for NULL outputs, PTYCHO_ENOMEM, PTYCHO_ECUDA. */
ptycho_status ptycho_measure_fp32_peak(double* tflops, double* ms, void* cuda_stream);

/* Failure-detection self-test (no counterpart in the paper): runs, on cuda_stream, one bounded
 * mbarrier wait of the kind the cluster-form fused kernels use on their copy barriers, with a
 * budget of budget_ns nanoseconds (0 ... 2e9, the kernels' own budget being 2 s). With signal != 0
 * the barrier is completed before the wait, which then succeeds (PTYCHO_OK); with signal == 0
 * nothing ever completes it, the wait gives up after the budget and sets the device flag that
 * ptycho_error reads, and this call reports it: PTYCHO_ETIMEOUT, the flag cleared and the context
 * still usable. Synchronises the stream. A timeout left pending by an earlier launch is reported
 * (and cleared) before the test runs, as PTYCHO_ETIMEOUT. PTYCHO_EINVAL for a budget out of
 * range (checked before any device work), PTYCHO_ECUDA. */
ptycho_status ptycho_wait_selftest(int64_t budget_ns, int32_t signal, void* cuda_stream);

/* Message of the calling thread's last failed call ("" if none). */
const char* ptycho_last_error(void);

/* Library version string. */
const char* ptycho_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PTYCHO_H_ */
