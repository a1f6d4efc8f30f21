// cgh_internal.h -- plan structure and kernel launch interfaces shared by the
// translation units of libcgh.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cgh.h"

#define CGH_MAX_C 4
#define CGH_MAX_L 16
#define CGH_MAX_PASSES 6
#define CGH_TILE 16
// per-Gaussian raw-gradient slots: 2C (P_c, Q_c) + 6 (SG, Sx, Sy, Sxx, Sxy, Syy)
#define CGH_RAW_STRIDE 16
// per-Gaussian render record: 5 float4 (see raster.cu)
#define CGH_REC_F4 5
// per-tile Gaussian counters (also the emit cursors) sit one per 32-byte sector: their
// atomics then spread over many L2 lines instead of queueing on the few that a dense array
// occupies
#define CGH_COUNT_STRIDE 8
// largest CTA of the FFT passes (their __launch_bounds__)
constexpr int kMaxFFTThreads = 512;
// opt-in dynamic shared memory per CTA on sm_103a (227 KB)
constexpr size_t kMaxSmemBytes = 227 * 1024;

// One 1D transform length: mixed-radix Stockham passes and its twiddle table
// tw[m] = exp(-2 pi i m / n), m in [0, n), computed on the host in FP64.
struct FFTDesc {
  int n;
  int npass;
  int radix[CGH_MAX_PASSES];
  const float2* tw;
};

// Transfer-function constants of one (channel, plane) pair (Algorithm 3), computed on the
// host in FP64 and rounded once to FP32:
//   phase in turns = frac(d/lambda) - (ax*sx^2 + ay*sy^2) / (1 + sqrt(1 - q)),
//   q = qx*sx^2 + qy*sy^2 (= lambda^2 (f_x^2 + f_y^2)), ax = (d/lambda) qx, ay = (d/lambda) qy,
// which equals k_z d / 2pi = (d/lambda) sqrt(1 - q) with the large integer part removed
// exactly on the host.  Bins with |s_x| > kx_max or |s_y| > ky_max are outside the band.
struct TFConst {
  float turns0;
  float qx, qy;
  float ax, ay;
  int kx_max, ky_max;
  int _pad;
};

// Geometry, optics and plane map of the propagation kernels.  The row and column passes loop
// over L planes; plane l of those is plane `plane[l]` of the hologram's Ltot planes, which
// selects its transfer function (tf[c * Ltot + plane[l]]), its target and depth mask.  The
// full map (L = Ltot, plane[l] = l) propagates every plane; the map of the fused step leaves
// out the planes whose propagation is the identity (see cgh_plan::n_ident).
struct BlasmDev {
  int H, W, C, L;
  int Ltot;        // planes of the hologram (loss normalisation 1 / (Ltot C H W))
  int Ny, Nx;      // padded sizes
  int oy, ox;      // offset of the image window inside the padded grid
  float inv_ntot;  // 1 / (Ny * Nx)
  float aperture2; // aperture radius^2 in index units (0 = off)
  int series_ok;   // every bin has q = lambda^2 (fx^2 + fy^2) < 0.04 (see transfer_series)
  int loss_kind;   // 0: intensity MSE; 1: three-term L_recon (Sec. 3.2)
  const unsigned char* recon_mask;  // L_recon depth masks [L][H][W] (NULL: M = 0)
  int plane[CGH_MAX_L];                // kernel plane index -> hologram plane
  TFConst tf[CGH_MAX_C * CGH_MAX_L];  // index c * Ltot + hologram plane
};

// Per-pixel weight of the loss: (I - T)^2 w.  The three-term L_recon of Sec. 3.2 is
// (I - T)^2 + (I M - T M)^2 + (I T - T T)^2 = (I - T)^2 (1 + M + T^2) for binary M.
__device__ __forceinline__ float loss_weight(const BlasmDev& bl, int l, int y, int x, float t) {
  if (bl.loss_kind == 0) return 1.f;
  const float m = bl.recon_mask ? (bl.recon_mask[((size_t)l * bl.H + y) * bl.W + x] ? 1.f : 0.f) : 0.f;
  return 1.f + m + t * t;
}

struct cgh_plan {
  // geometry and optics
  int H, W, C, L, pad;
  double lambda[CGH_MAX_C];
  double z[CGH_MAX_L];
  double pitch, aperture;
  float cutoff;
  int max_gaussians;
  int tiles_x, tiles_y;
  // tuning
  int col_block, row_block, fft_threads, pair_cap_mult;
  int use_spec;  // 1: use compile-time specialised FFT kernels when one matches
  // FFT descriptors (host copies; tw points into tables_dev)
  FFTDesc fx, fy;
  BlasmDev bl;       // every plane propagated
  // Planes at distance 0 with no aperture and every bin inside the band: their transfer
  // function is exactly 1 (Algorithm 3 with d = 0: phase k_z d = 0, f_max = 1/lambda above
  // the Nyquist frequency), so U(d_l) = U(0).  The fused step takes their loss and gradient
  // seed on U(0) in the pixel domain and propagates only the others (bl_prop).
  int n_ident;
  unsigned ident_mask;  // bit l: hologram plane l is such a plane
  int use_ident;        // 1: skip their transforms in the fused step (default); 0: propagate all
  BlasmDev bl_prop;     // plane map of the planes that are propagated
  // device tables owned by the plan (twiddles)
  void* tables_dev;
  size_t tables_bytes;
  // caller workspace
  char* ws;
  size_t ws_bytes;
  // workspace carve-up (byte offsets)
  size_t off_rec, off_rect, off_raw, off_tile_count, off_tile_start, off_tile_cursor,
      off_pairs, off_status, off_loss, off_U0, off_Y, off_V, off_S, ws_needed;
  int64_t pair_capacity;
  int loss_slots;
  // parameters the binning in the workspace was built for (bin_valid = 0: none)
  int bin_valid;
  cgh_params bin_params;
};

// status words in the workspace (int32 each)
// ST_LOSS_TICKET: CTAs of the loss pass that have written their partial (the last one sums
// them all and resets it to 0)
enum { ST_PAIRS_LO = 0, ST_PAIRS_HI = 1, ST_OVERFLOW = 2, ST_NONFINITE = 3, ST_LOSS_TICKET = 4,
       ST_COUNT = 8 };

struct LaunchShape {
  int threads, maxb;
  bool ok;
};
// blasm.cu: shared-memory stride (float2) of one transform of length n in the generic passes
int fft_smem_stride(int n);
// blasm.cu: CTA shape for nb transforms of d held in `buffers` shared-memory buffers
// (ok = false if no shape fits the thread or shared-memory limits)
LaunchShape fft_shape(const cgh_plan* p, const FFTDesc& d, int nb, int buffers);

// ---- launch interfaces (return cudaError_t of the launch) ----
// raster.cu
// rebin = false reuses the binning in the workspace when it was built for these parameter
// pointers and N (the caller vouches for the values); otherwise the Gaussians are binned.
// The identity planes' loss taken in the forward raster's epilogue: for every pixel of U(0),
// channel c and plane l in `mask`, w (|U|^2 - T_l)^2 (w of loss_weight) summed into one
// partial per tile, partials[ty * tiles_x + tx]; with `seed` non-NULL also
// seed = gscale sum_l w (|U|^2 - T_l) U, in the layout of U (C x H x W).
struct IdentLoss {
  const float* target;              // [Ltot][C][H][W]
  float* partials;                  // tiles_x * tiles_y
  float2* seed;                     // NULL: the loss only
  const unsigned char* recon_mask;  // L_recon depth masks [Ltot][H][W] (NULL: M = 0)
  float gscale;                     // 4 / (Ltot C H W)
  unsigned mask;                    // bit l: hologram plane l
  int loss_kind;                    // 0: intensity MSE; 1: three-term L_recon
};
cudaError_t launch_raster_fwd(cgh_plan* p, const cgh_params* prm, float2* U, cudaStream_t s,
                              bool rebin = true, const IdentLoss* ident = nullptr);
// rebin = false reuses the binning left in the workspace by the preceding raster_fwd with
// the same parameters.
// grad_scale: device float multiplying every gradient (NULL: 1).
cudaError_t launch_raster_bwd(cgh_plan* p, const cgh_params* prm, const float2* dU,
                              const cgh_grads* g, cudaStream_t s, bool rebin,
                              const float* grad_scale = nullptr);
// bins `prm` and counts the sweeps' work into out[6] (device, cgh_raster_stats)
cudaError_t launch_raster_stats(cgh_plan* p, const cgh_params* prm, unsigned long long* out,
                                cudaStream_t s);
// blasm.cu
// The column passes and the loss pass take a plane map (NULL: every plane, &p->bl).
cudaError_t launch_rows_pad_fwd(cgh_plan* p, const float2* in, float2* half, int batches,
                                cudaStream_t s);
cudaError_t launch_cols_fwd_planes(cgh_plan* p, const float2* Y, float2* V, cudaStream_t s,
                                   const BlasmDev* planes = nullptr);
// accumulate: out += the cropped rows (instead of out = ...)
cudaError_t launch_rows_inv_crop(cgh_plan* p, const float2* half, float2* out, int batches,
                                 cudaStream_t s, bool accumulate = false);
// ... and the loss itself: loss_out[0] = sum(partials) / (Ltot C H W), summed in FP64 in a
// fixed order (by the pass's last CTA when a specialised kernel runs, else by
// k_loss_finalize); `extra` more partials, written before the launch right after the pass's
// own, are included in the sum.
cudaError_t launch_rows_loss(cgh_plan* p, float2* V, const float* target, float* partials,
                             cudaStream_t s, bool want_grad, float* loss_out,
                             const BlasmDev* planes = nullptr, int extra = 0);
cudaError_t launch_cols_bwd_planes(cgh_plan* p, const float2* G, float2* D, cudaStream_t s,
                                   const BlasmDev* planes = nullptr);
// loss partials of the identity planes' pass (one per tile of the forward raster)
int ident_loss_blocks(const cgh_plan* p);
cudaError_t launch_loss_pointwise(cgh_plan* p, const float2* Ud, const float* target,
                                  float* partials, float2* dUd, cudaStream_t s);
cudaError_t launch_loss_finalize(cgh_plan* p, const float* partials, int count, float* out,
                                 cudaStream_t s);
// sum(partials) * inv (FP64, fixed order) -> out[0]
cudaError_t launch_loss_finalize_scaled(const float* partials, int count, double inv, float* out,
                                        cudaStream_t s);
// I = |U|^2 and its adjoint dU = 2 dI U, element-wise over `total` complex values
cudaError_t launch_intensity(long long total, const float2* U, float* I, cudaStream_t s);
cudaError_t launch_intensity_bwd(long long total, const float2* U, const float* dI, float2* dU,
                                 cudaStream_t s);
// CTAs of the loss pass over the planes of `planes` (NULL: every plane)
int rows_loss_blocks(const cgh_plan* p, const BlasmDev* planes = nullptr);
int pointwise_loss_blocks(const cgh_plan* p);
// conv_tc.cu: tensor-core 3x3 convolutions (strides 1 and 2) of the learned initialiser
cudaError_t conv3x3_fwd_tc(int B, int CI, int Hi, int Wi, int CO, int stride, const void* x,
                           const void* w, const float* bias, int relu, void* y, int y_f32,
                           cudaStream_t s);
cudaError_t conv3x3_dgrad_tc(int B, int CI, int Hi, int Wi, int CO, int stride, const void* w,
                             int relu, const void* y, int y_f32, const float* dy, float* dx,
                             cudaStream_t s);
// adds into dw [CO][CI][9] and db [CO] (zero them first)
cudaError_t conv3x3_wgrad_tc(int B, int CI, int Hi, int Wi, int CO, int stride, const void* x,
                             int relu, const void* y, int y_f32, const float* dy, float* dw,
                             float* db, cudaStream_t s);
// persist.cu: the persistent batched step (state owned by a cgh_batch)
struct PersistState;
cgh_status persist_prepare(PersistState** ps, cgh_plan* const* plans, const cgh_params* prm,
                           const cgh_grads* grads, const float* const* targets,
                           float* const* losses, int count);
cgh_status persist_launch(PersistState* ps, cudaStream_t s);
cgh_status persist_status(PersistState* ps, int32_t* timed_out, cudaStream_t s);
void persist_set_test(PersistState* ps, int skip_barrier, long long budget_cycles);
void persist_invalidate(PersistState* ps);
void persist_release(PersistState* ps);
int persist_grid(const PersistState* ps);
// api.cu
cudaError_t launch_adam(const cgh_adam_group* groups, int n, int step, float b1, float b2,
                        float eps, cudaStream_t s);

// host-side launch counter (api.cu)
void cgh_count_launch(int n);
// record a message for cgh_last_error_string() and return st (api.cu)
cgh_status cgh_record_error(cgh_status st, const char* msg);

// kernel ids for the event profiler (profile.cu)
enum KernelId {
  KID_PREPROCESS = 0, KID_SCAN_TILES, KID_EMIT, KID_RASTER_FWD, KID_RASTER_BWD,
  KID_GRAD_FINALIZE, KID_ROWS_PAD_FWD, KID_COLS_FWD_PLANES, KID_ROWS_LOSS,
  KID_COLS_BWD_PLANES, KID_ROWS_INV_CROP, KID_LOSS_POINTWISE, KID_LOSS_FINALIZE, KID_ADAM,
  KID_ENCODER, KID_POH, KID_PERSIST, KID_COUNT
};
// Bracket one kernel launch: records a CUDA event before and after it on its stream when
// profiling is enabled; otherwise only the launch counter moves.
void prof_begin(int kid, cudaStream_t s);
void prof_end(int kid, cudaStream_t s);
