/*
 * cgh.h -- C ABI of the GB300 (sm_103a) hot path of complex-valued 2D Gaussian hologram
 * optimisation (arXiv 2511.15022).
 *
 * The problem (Sec. 3, "Problem Definition"): given pre-activation Gaussian parameters
 * G_n = {x~_n, s~_n, theta_n, c_n, phi_n, alpha~_n} (Sec. 3.1), wavelengths, pixel pitch,
 * plane distances d_l and target intensities I^_l in R^{C x H x W}, render the complex
 * field U(0) = H in C^{C x H x W} (Algorithm 2), propagate it to every plane with the
 * band-limited angular spectrum method (Algorithm 3 and Sec. 2: zero-pad, FFT, multiply
 * by H_d, inverse FFT, crop), take the intensity loss L_MSE = 1/L sum_l ||I_l - I^_l||^2
 * with I_l = |U(d_l)|^2 (Sec. 3.2; mean over C*H*W pixels), and run the backward pass
 * through both steps (Suppl. gradients, Suppl. BLASM backward with conj(H)).
 *
 * Conventions shared by every entry point
 *   - Every array argument is a DEVICE pointer owned by the caller, except where a
 *     parameter says "host".  The library never frees caller memory.
 *   - Device work is enqueued on `stream` (a cudaStream_t passed as void*; NULL = the
 *     legacy default stream) and is asynchronous; a return of CGH_OK means the work was
 *     enqueued, not that it finished.  Launch errors are reported as CGH_ERR_CUDA.
 *   - Floating point is FP32.  Complex arrays are interleaved (re, im) float pairs
 *     (CUDA float2, 8-byte aligned).  Field layout [C][H][W] row-major; multi-plane
 *     layout [L][C][H][W].  Gradients w.r.t. a complex array hold (dL/dRe, dL/dIm).
 *   - Parameters are structure-of-arrays in pre-activation form (Sec. 3.1):
 *     xy_raw[N][2], s_raw[N][2], theta[N], amp[N][C], phase[N][C], alpha_raw[N].
 *     Activations (Suppl.): x = (tanh(x~)+1)/2 * (W, H), s = exp(s~) + 0.1,
 *     alpha = sigmoid(alpha~).  Pixel centres are the integers 0..W-1, 0..H-1.
 *   - Errors: every function returns a cgh_status; no exception crosses the ABI.
 *     cgh_last_error_string() gives a human-readable detail for the calling thread.
 *   - A plan is not thread-safe: one plan is driven from one host thread at a time, and
 *     calls that share a plan's workspace must be ordered on one stream.
 */
#ifndef CGH_H
#define CGH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { CGH_LOSS_MSE = 0, CGH_LOSS_RECON = 1 } cgh_loss_kind;

typedef enum {
  CGH_OK = 0,
  CGH_ERR_ARG = 1,              /* invalid argument (null pointer, bad size, ...) */
  CGH_ERR_CUDA = 2,             /* a CUDA runtime call or kernel launch failed */
  CGH_ERR_TIMEOUT = 3,          /* a bounded device-side wait expired */
  CGH_ERR_NONFINITE = 4,        /* non-finite parameter seen (reported by cgh_plan_status) */
  CGH_ERR_UNSUPPORTED_SIZE = 5, /* padded FFT length has a prime factor > 5, or C > 4 */
  CGH_ERR_WORKSPACE = 6,        /* no workspace attached, or it is too small */
  CGH_ERR_CAPACITY = 7          /* N exceeds the plan's max_gaussians */
} cgh_status;

typedef struct cgh_plan cgh_plan;

/* Pre-activation Gaussian parameters (device pointers, layouts above). */
typedef struct {
  int32_t N;
  const float* xy_raw;
  const float* s_raw;
  const float* theta;
  const float* amp;
  const float* phase;
  const float* alpha_raw;
} cgh_params;

/* Gradients of the pre-activation parameters (device pointers, same layouts).  Every
 * array is overwritten (not accumulated). */
typedef struct {
  float* xy_raw;
  float* s_raw;
  float* theta;
  float* amp;
  float* phase;
  float* alpha_raw;
} cgh_grads;

/* Create a plan for one hologram geometry.
 *   H, W           image size in pixels (>= 1)
 *   C              colour channels, 1..4; lambda_m[C] (host) wavelengths in metres
 *   L              target planes (>= 1); z_m[L] (host) propagation distances in metres
 *   pad_factor     zero-pad factor of Alg. 1 "ZeroPad" (the padded grid is
 *                  pad_factor*H x pad_factor*W with the image centred at
 *                  ((pad*H-H)/2, (pad*W-W)/2)); both padded sizes must factor into 2,3,5
 *   pitch_m        pixel pitch in metres
 *   aperture       optional circular aperture radius in frequency-index units
 *                  (Algorithm 3; 0 disables it)
 *   cutoff         effective-opacity skip threshold of Algorithm 2 (1/255 in the paper;
 *                  0 keeps every pair -- "smooth mode")
 *   max_gaussians  largest N the plan will be called with (sizes the workspace)
 * The plan owns only host memory and small device tables (twiddles, transfer-function
 * constants); bulk scratch is the caller-provided workspace (cgh_plan_set_workspace). */
cgh_status cgh_plan_create(int32_t H, int32_t W, int32_t C, int32_t L, int32_t pad_factor,
                           const double* lambda_m, double pitch_m, const double* z_m,
                           double aperture, float cutoff, int32_t max_gaussians,
                           cgh_plan** out_plan);

cgh_status cgh_plan_destroy(cgh_plan* plan);

/* Bytes of device workspace the plan needs (host output). */
cgh_status cgh_plan_workspace_bytes(const cgh_plan* plan, size_t* out_bytes);

/* Attach a caller-owned device workspace (256-byte aligned, >= the size above).  It must
 * stay valid until it is replaced or the plan is destroyed. */
cgh_status cgh_plan_set_workspace(cgh_plan* plan, void* workspace, size_t bytes);

/* Tuning knobs (host input).  Zero fields keep the current value.
 *   col_block    columns per CTA in the column FFT passes (1, 2, 4 or 8)
 *   row_block    rows per CTA in the row FFT passes (1..8)
 *   fft_threads  threads per CTA of the FFT passes (128..1024)
 *   pair_capacity_per_gaussian  (Gaussian, tile) list capacity as a multiple of N
 *   fft_kernels  1: compile-time specialised FFT kernels where one matches the padded
 *                length and block shape (default), 2: generic mixed-radix kernels only
 *   identity_planes  1 (default): in cgh_forward_loss, cgh_step, cgh_step_scaled and the batch
 *                step, planes whose propagation is the identity -- distance exactly 0, no
 *                aperture, every frequency bin inside the band, so H = 1 in Algorithm 3 and
 *                U(d) = U(0) -- take their loss and gradient seed on U(0) in the pixel domain
 *                and skip the FFT passes; 2: propagate every plane through the FFT passes.
 *                Both compute the same loss and gradients (the first without the FFT
 *                round-off of an identity transform).  cgh_blasm_fwd/bwd always propagate
 *                every plane.  A plan that has such planes sizes its workspace for C x H x W
 *                complex values more (their gradient seed, later dL/dU(0)). */
typedef struct {
  int32_t col_block;
  int32_t row_block;
  int32_t fft_threads;
  int32_t pair_capacity_per_gaussian;
  int32_t fft_kernels;
  int32_t identity_planes;
} cgh_tuning;

cgh_status cgh_plan_set_tuning(cgh_plan* plan, const cgh_tuning* tuning);
cgh_status cgh_plan_get_tuning(const cgh_plan* plan, cgh_tuning* out);

/* Per-(channel, plane) band-limit bounds of Algorithm 3 (host outputs [C*L] each): the
 * largest |signed frequency index| that passes |f_x| < f_x^max (resp. y), index c*L + l.
 * Computed on the host in FP64 exactly as the definition reads. */
cgh_status cgh_plan_band_limits(const cgh_plan* plan, int32_t* kx_max, int32_t* ky_max);

/* Planes whose propagation is the identity (host output, bit l set for plane l): distance
 * exactly 0, no aperture and every frequency bin of every channel inside the band of
 * Algorithm 3 (at d = 0 the phase k_z d vanishes and f_max = 1/lambda exceeds the grid's
 * Nyquist frequency whenever lambda < 2 pitch, so H = 1).  With the tuning knob
 * identity_planes = 1 the fused entry points take these planes in the pixel domain. */
cgh_status cgh_plan_identity_planes(const cgh_plan* plan, uint32_t* mask_out);

/* Loss taken by cgh_intensity_loss, cgh_forward_loss, cgh_step and the batch step of this
 * plan (Sec. 3.2).  kind = CGH_LOSS_MSE (default): L_MSE = 1/L sum_l mean_{c,p}
 * (I_l - I^_l)^2.  kind = CGH_LOSS_RECON: the three-term reconstruction loss
 *   L_recon = 1/L sum_l mean_{c,p} [ (I_l - I^_l)^2 + (I_l M_l - I^_l M_l)^2
 *                                    + (I_l I^_l - I^_l I^_l)^2 ]
 * with recon_mask the binary depth masks M_l: DEVICE bytes [L][H][W] (nonzero = 1, shared by
 * the colour channels; NULL means M = 0), owned by the caller and read at every later call
 * until the loss is set again.  A mask with CGH_LOSS_MSE is an argument error. */
cgh_status cgh_plan_set_loss(cgh_plan* plan, int32_t kind, const uint8_t* recon_mask);

/* Synchronous status read of the last raster call on this plan (blocks on `stream`):
 * pairs_needed = (Gaussian, tile) pairs of the last binning, overflow = 1 if that
 * exceeded the list capacity (tiles past it were rendered by the exhaustive path, still
 * exact), nonfinite = 1 if a non-finite parameter was seen (those Gaussians were
 * skipped).  Any output pointer may be NULL. */
cgh_status cgh_plan_status(cgh_plan* plan, int64_t* pairs_needed, int32_t* overflow,
                           int32_t* nonfinite, void* stream);

/* Forward rasterisation, Algorithm 2 with the per-pixel sum of Sec. 3.1:
 *   U_c(p) = sum_n c_{n,c} a_n(p) exp(j phi_{n,c}),  a_n(p) = min(0.99, alpha_n G_n(p)),
 *   G_n(p) = exp(max(-1/2 (p-x_n)^T Sigma_n^{-1} (p-x_n), -50)), pairs with a < cutoff
 *   skipped.  U_out: [C][H][W] complex. */
cgh_status cgh_raster_fwd(cgh_plan* plan, const cgh_params* params, void* U_out,
                          void* stream);

/* Work counters of the two rasteriser sweeps (a diagnostic; the paper has no counterpart):
 * bins `params` as cgh_raster_fwd does, then counts with the kernels' own box geometry, and
 * returns (blocking on `stream`) six int64 in the HOST array counts_out:
 *   [0] lane slots the forward sweep evaluates (32 per 8x4 pixel block per listed Gaussian
 *       whose box touches it),
 *   [1] (pixel, Gaussian) pairs with alpha G >= cutoff (the pairs that contribute),
 *   [2] lane slots the backward sweep evaluates (per Gaussian and 32x32 region, the box's
 *       pixels in the region rounded up to whole warps of 32),
 *   [3] (Gaussian, 32x32 region) pairs of the backward, [4] (Gaussian, 16x16 tile) entries,
 *   [5] tiles whose list overflowed the capacity (not counted in [0]..[4]).
 * Uses the plan's workspace like every other call (its loss partials are overwritten). */
cgh_status cgh_raster_stats(cgh_plan* plan, const cgh_params* params, int64_t* counts_out,
                            void* stream);

/* Forward rasterisation that allocates nothing and needs no plan.  The paper has no
 * counterpart: this exists for callers that may not allocate device memory -- e.g. an
 * application that reserves all device memory at start-up, or a latency-critical loop where
 * cudaMalloc's implicit device-wide synchronisation is not acceptable.  It computes the same
 * field as cgh_raster_fwd (H x W pixels, C channels 1..4, skip threshold `cutoff`; U_out
 * [C][H][W] complex, caller-allocated), keeping its binning scratch in one fixed 16 MiB
 * device array compiled into the library, which every device that loads the library holds
 * until the process exits.  Limits: N <= 65536 Gaussians and at most 16384 16x16 tiles
 * (e.g. 2048 x 2048 pixels); larger inputs return CGH_ERR_CAPACITY or
 * CGH_ERR_UNSUPPORTED_SIZE with a message, and nothing is launched.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress), so make that first
 * call before any stream capture.  All calls share the one array: calls whose GPU work
 * overlaps (different streams, or concurrent host threads) race and corrupt each other's
 * results; order them on one stream.  The call works on the CURRENT device (the caller makes
 * the device that holds params and U_out current).  Having no plan, it has no status to
 * report through cgh_plan_status: Gaussians with a non-finite parameter are skipped without
 * notice, and when the (Gaussian, tile) list outgrows the space left in the array the tiles
 * past it fall back, silently, to the slower exhaustive path (the field stays exact). */
cgh_status cgh_raster_fwd_noalloc(int32_t H, int32_t W, int32_t C, float cutoff,
                                  const cgh_params* params, void* U_out, void* stream);

/* Backward rasterisation (Suppl. "Detailed Gradient Derivation"): given dU = dL/dU
 * [C][H][W] complex, writes the gradients of all pre-activation parameters.  The
 * Gaussian values are recomputed; no forward state is needed. */
cgh_status cgh_raster_bwd(cgh_plan* plan, const cgh_params* params, const void* dU,
                          const cgh_grads* grads, void* stream);

/* BLASM forward (Algorithm 3 inside Alg. 1 "ZeroPad" + "MultiPlanePropagate"):
 *   Ud[l][c] = crop(IFFT2(H_{c,l} . FFT2(pad(U0[c])))) / (Ny*Nx normalisation).
 * U0: [C][H][W] complex;  Ud_out: [L][C][H][W] complex. */
cgh_status cgh_blasm_fwd(cgh_plan* plan, const void* U0, void* Ud_out, void* stream);

/* BLASM backward (Suppl. BLASM "Backward Pass", conj(H) under the same band limit):
 *   dU0[c] = sum_l crop(IFFT2(conj(H_{c,l}) . FFT2(pad(dUd[l][c])))).
 * dUd: [L][C][H][W] complex;  dU0_out: [C][H][W] complex. */
cgh_status cgh_blasm_bwd(cgh_plan* plan, const void* dUd, void* dU0_out, void* stream);

/* Intensity loss (Sec. 3.2 L_MSE): loss = 1/(L*C*H*W) sum (|Ud|^2 - target)^2 written to
 * loss_out (device float[1]); dUd_out (may be NULL) receives dL/dUd = 4 (|Ud|^2 - target)
 * / (L*C*H*W) * Ud.  Ud: [L][C][H][W] complex; target: [L][C][H][W] float. */
cgh_status cgh_intensity_loss(cgh_plan* plan, const void* Ud, const float* target,
                              float* loss_out, void* dUd_out, void* stream);

/* Intensity of the propagated fields (Sec. 3.2, I_l = |U(d_l)|^2):
 *   I_out[i] = Re(Ud[i])^2 + Im(Ud[i])^2 for the L*C*H*W values of the plan's geometry.
 * Ud: [L][C][H][W] complex (e.g. the output of cgh_blasm_fwd); I_out: [L][C][H][W] float.
 * For losses defined by the caller on the intensities. */
cgh_status cgh_intensity(cgh_plan* plan, const void* Ud, float* I_out, void* stream);

/* Adjoint of cgh_intensity (chain rule of I = |U|^2 in the gradient convention of the
 * supplementary, dL/dU = dL/dRe + j dL/dIm):  dUd_out[i] = 2 dI[i] Ud[i].
 * Ud: [L][C][H][W] complex (the same field); dI = dL/dI: [L][C][H][W] float;
 * dUd_out: [L][C][H][W] complex (may be fed to cgh_blasm_bwd). */
cgh_status cgh_intensity_bwd(cgh_plan* plan, const void* Ud, const float* dI, void* dUd_out,
                             void* stream);

/* Forward only: raster -> BLASM -> loss (loss_out: device float[1]).  Nothing but the
 * workspace is written. */
cgh_status cgh_forward_loss(cgh_plan* plan, const cgh_params* params, const float* target,
                            float* loss_out, void* stream);

/* One fused forward + backward pass of the whole path (Algorithm 1 loop body without
 * the optimiser): raster -> pad -> FFT -> x H_{c,l} for all planes -> IFFT -> crop ->
 * |U|^2 -> loss -> dL/dU -> adjoint propagation -> raster backward.  Writes loss_out
 * (device float[1]) and all gradients. */
cgh_status cgh_step(cgh_plan* plan, const cgh_params* params, const float* target,
                    float* loss_out, const cgh_grads* grads, void* stream);

/* cgh_step as the backward pass of an autograd function (forward recomputed, Sec. 3.4):
 *   grad_scale    device pointer to one float multiplying every gradient (the upstream
 *                 gradient of the loss; NULL: 1), applied inside the gradient kernel;
 *   reuse_binning nonzero: the caller guarantees that the parameter values are unchanged
 *                 since the last call on this plan that rasterised them, so the
 *                 per-Gaussian records and per-tile lists left in the workspace are reused
 *                 instead of rebuilt.  If N or a parameter pointer differs from that call
 *                 (or nothing was rasterised yet) they are rebuilt anyway.
 * Everything else, including loss_out, as cgh_step. */
cgh_status cgh_step_scaled(cgh_plan* plan, const cgh_params* params, const float* target,
                           float* loss_out, const cgh_grads* grads, const float* grad_scale,
                           int32_t reuse_binning, void* stream);

/* One Adam step over up to 8 parameter groups in a single launch (PyTorch semantics, no
 * weight decay): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr/(1-b1^t) * m / (sqrt(v)/sqrt(1-b2^t) + eps).  step >= 1.  The paper uses
 * Adan with per-group learning rates (Sec. 4); this is the Adam variant with the same
 * per-group rates. */
typedef struct {
  float* param;
  const float* grad;
  float* exp_avg;
  float* exp_avg_sq;
  int64_t count;
  float lr;
} cgh_adam_group;

cgh_status cgh_adam_step(const cgh_adam_group* groups /* host array */, int32_t num_groups,
                         int32_t step, float beta1, float beta2, float eps, void* stream);

/* Adan (adaptive Nesterov momentum), the optimiser of Sec. 4, restated from its published
 * algorithm with the bias corrections of the authors' release (betas as running-average
 * weights; 0.98, 0.92, 0.99 are the usual values).  Per element, step t >= 1:
 *   d = g - prev_grad (0 when t = 1); m = b1 m + (1-b1) g; v = b2 v + (1-b2) d;
 *   n = b3 n + (1-b3) (g + b2 d)^2;
 *   p = (p - lr (m/(1-b1^t) + b2 v/(1-b2^t)) / (sqrt(n/(1-b3^t)) + eps)) / (1 + lr wd);
 *   prev_grad = g.
 * Up to 8 groups (host array); all state arrays (exp_avg = m, exp_avg_diff = v,
 * exp_avg_sq = n, prev_grad) are device float arrays of `count` elements, zero at t = 1. */
typedef struct {
  float* param;
  const float* grad;
  float* exp_avg;
  float* exp_avg_diff;
  float* exp_avg_sq;
  float* prev_grad;
  int64_t count;
  float lr;
} cgh_adan_group;

cgh_status cgh_adan_step(const cgh_adan_group* groups, int32_t num_groups, int32_t step,
                         float beta1, float beta2, float beta3, float eps, float weight_decay,
                         void* stream);

/* Adam over any number of parameter groups in one launch: groups_dev is a DEVICE array of
 * num_groups cgh_adam_group records, offsets_dev a DEVICE array of num_groups + 1 int64
 * prefix sums of their counts (offsets_dev[num_groups] = total).  Same update as
 * cgh_adam_step with every group's learning rate multiplied by lr_scale >= 0 (a schedule
 * shared by all groups; 0 leaves everything untouched).  Used to step every hologram of a
 * batch at once. */
cgh_status cgh_adam_step_table(const cgh_adam_group* groups_dev, const int64_t* offsets_dev,
                               int32_t num_groups, int64_t total, int32_t step, float beta1,
                               float beta2, float eps, float lr_scale, void* stream);

/* Batches of independent holograms (the paper optimises one hologram at a time; batching
 * many of uneven size is this library's addition).  A batch holds one plan per hologram
 * (the plans keep their own workspaces and must outlive the batch).  cgh_batch_bind fixes
 * hologram i's device pointers (parameters, target, device float loss, gradients).
 * cgh_batch_step runs cgh_step for every hologram: with use_graph = 1 the steps are
 * captured once (on the first call after a bind) into one CUDA graph with one branch per
 * hologram and replayed with a single graph launch on `stream`; with use_graph = 0 they are
 * issued one after another on `stream`.  The bound pointers must stay valid and their
 * contents are read at replay time.  Profiling (cgh_profile_enable) must be off during the
 * capturing call.  cgh_batch_kernels_per_step reports the kernels one replay runs. */
typedef struct cgh_batch cgh_batch;
cgh_status cgh_batch_create(cgh_plan* const* plans /* host array */, int32_t count,
                            cgh_batch** out_batch);
cgh_status cgh_batch_destroy(cgh_batch* batch);
cgh_status cgh_batch_bind(cgh_batch* batch, int32_t index, const cgh_params* params,
                          const float* target, float* loss_out, const cgh_grads* grads);
cgh_status cgh_batch_step(cgh_batch* batch, int32_t use_graph, void* stream);
int64_t cgh_batch_kernels_per_step(const cgh_batch* batch);

/* The same batched step as ONE persistent kernel launch (cooperative: every CTA resident):
 * its phases -- clear, preprocess, tile scan and emit, raster forward, row pass,
 * identity-plane loss, column pass, loss row pass, adjoint column pass, crop row pass, raster
 * backward, gradient finalize and loss -- run for all holograms at once, the CTAs drawing
 * (hologram, Gaussian block / tile / row / column) items from an atomic work queue, with a
 * grid barrier between phases.  Same results as cgh_batch_step (the FFT passes are the
 * generic runtime-length ones, one row or column per item).  The first call after a bind
 * builds the descriptors (a small device allocation owned by the batch).  Each barrier wait is
 * bounded (about one second of clock cycles): if it runs out, the kernel sets an error word
 * and returns instead of hanging, and cgh_batch_persistent_status reports it. */
cgh_status cgh_batch_step_persistent(cgh_batch* batch, void* stream);

/* Synchronous read (blocks on `stream`) of the last persistent step's error word:
 * *timed_out = 1 and CGH_ERR_TIMEOUT if a grid-barrier wait ran out, else 0 and CGH_OK. */
cgh_status cgh_batch_persistent_status(cgh_batch* batch, int32_t* timed_out, void* stream);

/* Test hook of the bounded barrier: with skip_barrier >= 0, CTA 0 of the next persistent
 * steps does not arrive at grid barrier `skip_barrier` (0 = the one after the first phase),
 * so that barrier can never complete and every CTA's wait runs out; timeout_s > 0 sets the
 * wait budget in seconds of SM clock (<= 0: the default of about one second).
 * skip_barrier = -1 restores normal operation. */
cgh_status cgh_batch_persistent_test(cgh_batch* batch, int32_t skip_barrier, double timeout_s);

/* CTAs of the persistent launch (all resident at once), 0 before the first persistent step. */
int32_t cgh_batch_persistent_grid(const cgh_batch* batch);

/* Autotuner: runs cgh_step `iters` times (after one warm-up) for every valid combination of
 * column block {1,2,4,8} x row block {1,2,3,4,8} x FFT kernel family {specialised, generic}
 * on the given data, keeps the fastest on the plan and writes it to best_out (may be NULL).
 * Gradients and loss_out are overwritten. */
cgh_status cgh_autotune(cgh_plan* plan, const cgh_params* params, const float* target,
                        const cgh_grads* grads, float* loss_out, int32_t iters, void* stream,
                        cgh_tuning* best_out);

/* ---- learned initialiser (the paper has no learned part; it lists feed-forward prediction
 * as future work, Sec. 6): a stack of 3x3 convolutions with BF16 weights and activations
 * (16-bit bfloat16 values passed as void*) and FP32 accumulation, run on the tensor cores,
 * and the decode from the last layer to Gaussian parameters.
 *
 * cgh_conv3x3_fwd: y[b][co][oy][ox] = act(bias[co] + sum_{ci,ky,kx} w[co][ci][ky][kx]
 *   x[b][ci][oy*stride+ky-1][ox*stride+kx-1]) (zero outside the image), act = ReLU if relu.
 *   x: [B][CI][Hi][Wi] bf16; w: [CO][CI][3][3] bf16; bias: [CO] f32; y: [B][CO][Ho][Wo] with
 *   Ho = (Hi-1)/stride + 1, bf16 or f32 (y_f32).  stride 1 or 2 (else
 *   CGH_ERR_UNSUPPORTED_SIZE).  The products of the BF16 operands are exact in FP32. */
cgh_status cgh_conv3x3_fwd(int32_t B, int32_t CI, int32_t Hi, int32_t Wi, int32_t CO,
                           int32_t stride, const void* x, const void* w, const float* bias,
                           int32_t relu, void* y, int32_t y_f32, void* stream);

/* Backward of cgh_conv3x3_fwd given dy = dL/dy (f32, same layout as y) and the forward
 * output y (needed for the ReLU mask when relu = 1): dx = dL/dx (f32, may be NULL to skip),
 * dw = dL/dw [CO][CI][3][3] f32 and db = dL/dbias [CO] f32 (both overwritten).  The FP32
 * gradient g = dy [y > 0] enters the tensor-core products as two BF16 parts hi = bf16(g),
 * lo = bf16(g - hi), which represent it to 2^-18 relative; stride 1 or 2. */
cgh_status cgh_conv3x3_bwd(int32_t B, int32_t CI, int32_t Hi, int32_t Wi, int32_t CO,
                           int32_t stride, const void* x, const void* w, int32_t relu,
                           const void* y, int32_t y_f32, const float* dy, float* dx, float* dw,
                           float* db, void* stream);

/* dst[i] = bf16(src[i]) (round to nearest even), n elements. */
cgh_status cgh_cast_bf16(int64_t n, const float* src, void* dst, void* stream);

/* Decode the encoder output out [B][S*P][CY][CX] f32 (P = 6 + 2C channels per slot: dx, dy,
 * sx, sy, theta, amp[C], phase[C], alpha) into pre-activation parameters of B images of
 * N = CY*CX*S Gaussians each (arrays of B*N records, layouts as cgh_params; written through
 * a cgh_grads struct of writable pointers).  Gaussian n = (cy*CX + cx)*S + g sits at slot g
 * of cell (cy, cx), slots on a ceil(sqrt(S))^2 grid inside the cell (cells of W/CX x H/CY
 * pixels); parameter = base + scale * out with base = the slot's centre (pre-activation,
 * atanh(2 x / W - 1)) for the position and log(1.5), 0, 0.5, 0, -0.5 for scale, rotation,
 * amplitude, phase, opacity; scales 0.02 (position), 0.5 (scale), 1, 0.5 (amplitude), 1, 1.
 * Decoding zeros gives the plain structured initialisation. */
cgh_status cgh_encoder_decode(int32_t B, int32_t CY, int32_t CX, int32_t S, int32_t C, int32_t H,
                              int32_t W, const float* out, const cgh_grads* params_out,
                              void* stream);

/* Weighted squared-error term of the encoder's training loss: grad[i] = 2 w (pred[i] -
 * target[i]), added to grad[i] when accumulate = 1 (overwriting it when 0), and, if
 * loss_accum (device float) is not NULL, *loss_accum += w sum_i (pred[i] - target[i])^2. */
cgh_status cgh_mse_grad(int64_t n, const float* pred, const float* target, float weight,
                        int32_t accumulate, float* grad, float* loss_accum, void* stream);

/* Adjoint of the decode: dout = scale * dL/dparameter (dout overwritten). */
cgh_status cgh_encoder_decode_bwd(int32_t B, int32_t CY, int32_t CX, int32_t S, int32_t C,
                                  int32_t H, int32_t W, const cgh_grads* param_grads,
                                  float* dout, void* stream);

/* ---- phase-only hologram (POH) conversion (Sec. 3.3) ----
 *
 * cgh_poh_dpac: smooth POH by checkerboard multiplexing (DPAC).  With A = |U0| and
 *   phi = arg U0 per channel and pixel (row i, column j):
 *   mode 1, double-phase amplitude coding (the method the paper cites): phi_DPAC = phi +
 *     acos(A / max_c A) where i + j is even and phi - acos(A / max_c A) where it is odd
 *     (max over the channel's pixels), so each neighbouring pair averages to U0 / max A;
 *   mode 0, the formula as printed: phi_DPAC = A where i + j is even, phi where odd.
 *   H_out = exp(j phi_DPAC).  U0, H_out: DEVICE complex64 [C][H][W] of the plan's size; uses
 *   the plan's workspace for the per-channel maxima. */
cgh_status cgh_poh_dpac(const cgh_plan* plan, const void* U0, void* H_out, int32_t mode,
                        void* stream);

/* H_out = exp(j phi): the random POH of a phase field phi (DEVICE float [C][H][W]). */
cgh_status cgh_poh_field(const cgh_plan* plan, const float* phi, void* H_out, void* stream);

/* Scratch (caller-owned device memory) needed by cgh_poh_step: (2 L C + C) H W complex64. */
cgh_status cgh_poh_scratch_bytes(const cgh_plan* plan, size_t* bytes);

/* One joint forward + backward pass of the random-POH conversion (Sec. 3.3): the Gaussians'
 * field H and the random POH exp(j phi) are both propagated to the L planes and
 *   L_extract = sum_l [ R_l(I_l) + R_l(I_rand,l) + lambda_comp mean (I_l - I_rand,l)^2
 *               + lambda_field mean (|Re(U(d_l) - U_rand(d_l))| + |Im(U(d_l) - U_rand(d_l))|) ]
 * is written to loss_out (device float[1]), with R_l plane l's part of L_recon (the plan's
 * depth masks, cgh_plan_set_loss; M = 0 without them) and every mean over the C H W values
 * of one plane (the paper uses lambda_comp = 0.1, lambda_field = 0.01).  Gradients of the
 * Gaussian parameters go to grads (overwritten), dL/dphi to dphi (DEVICE float [C][H][W],
 * overwritten).  scratch: at least cgh_poh_scratch_bytes bytes of device memory. */
cgh_status cgh_poh_step(cgh_plan* plan, const cgh_params* params, const float* phi,
                        const float* target, float lambda_comp, float lambda_field,
                        float* loss_out, const cgh_grads* grads, float* dphi, void* scratch,
                        size_t scratch_bytes, void* stream);

/* Measurement utility (no counterpart in the paper): FP32 FMA throughput (flop/s, one FMA
 * = 2 flops) and MUFU throughput (special-function operations/s) of the current device,
 * from two microbenchmark kernels timed with CUDA events on `stream` (synchronous, ~50 ms).
 * These are the denominators of the arithmetic rooflines the benchmark reports. */
cgh_status cgh_measure_peaks(double* fp32_flops_per_s, double* sfu_ops_per_s, void* stream);

/* Number of kernels launched by the library in this process so far, from every thread
 * (host counter; used to report launches per step). */
int64_t cgh_launch_count(void);

/* Per-kernel timing with CUDA events recorded on each kernel's own launch stream.
 * cgh_profile_enable(1) starts recording (at most 65536 launches per window; later ones
 * are not timed); cgh_profile_collect() waits for the recorded events, writes per kernel
 * id the summed milliseconds and launch counts (arrays of cgh_kernel_count() entries,
 * host outputs) and starts a new window.  cgh_kernel_name(id) names a kernel id.
 * Profiling records events and must not be enabled during CUDA-graph capture. */
cgh_status cgh_profile_enable(int32_t enable);
cgh_status cgh_profile_collect(double* total_ms, int64_t* launches);
int32_t cgh_kernel_count(void);
const char* cgh_kernel_name(int32_t id);

const char* cgh_last_error_string(void);

#ifdef __cplusplus
}
#endif

#endif /* CGH_H */
