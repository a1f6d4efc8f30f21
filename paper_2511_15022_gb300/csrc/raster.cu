// raster.cu -- tile-binned complex 2D Gaussian rasteriser, forward and backward (sm_103a).
//
// Algorithm 2 of the paper, re-planned for GB300:
//   1. k_preprocess   one thread per Gaussian: activations (Suppl. activation formulas),
//                     covariance and its clamped adjugate inverse (Suppl. 2D covariance /
//                     inversion), per-channel A_c = c cos(phi), B_c = c sin(phi) (hoisted out
//                     of the pixel loop), and the axis-aligned box of the ellipse where
//                     alpha G >= cutoff.  Counts the Gaussian in every 16x16 tile its box
//                     touches.
//   2. k_scan_tiles   exclusive scan of the per-tile counts (one CTA).
//   3. k_emit         scatters Gaussian ids into per-tile lists.  The sum over Gaussians is
//                     order-free, so a counting sort by tile replaces the paper's radix
//                     sort of (tile, depth) keys.
//   4. k_raster_fwd   one CTA per tile, one thread per pixel; the tile's Gaussians are
//                     staged in shared memory 256 at a time; each warp owns an 8x4 pixel
//                     block and visits only the staged Gaussians whose box touches it
//                     (per-warp lists compacted with ballots).  In the fused step it also
//                     takes the loss (and seed) of the planes at distance 0 on the finished
//                     pixels.
//   5. k_raster_bwd_region  one CTA per 32x32 region (2x2 tiles) with the region's dL/dU
//                     in shared memory; every Gaussian is kept once per region (from the
//                     first of its tiles inside it); warps draw the kept Gaussians from a
//                     shared counter and sweep each one's box inside the region,
//                     accumulating the gradient moments in registers, then reduce them
//                     across the warp with shuffles and add them with global atomics.
//   6. k_grad_finalize one thread per Gaussian: chain rule from the accumulated moments to
//                     the pre-activation parameters (Suppl. items 1-7; the
//                     inverse-covariance -> covariance step is the exact derivative of the
//                     adjugate formula, which the paper does not print).
// If the (Gaussian, tile) list outgrows its capacity, tiles past the capacity evaluate
// every Gaussian with the same box test instead: slower, still exact.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <atomic>

#include "raster.cuh"


using namespace cgh;

static RasterConsts make_consts(const cgh_plan* p, int N) {
  RasterConsts rc;
  rc.H = p->H; rc.W = p->W; rc.C = p->C; rc.N = N;
  rc.tiles_x = p->tiles_x; rc.tiles_y = p->tiles_y;
  rc.cutoff = p->cutoff; rc._pad = 0;
  rc.cap = p->pair_capacity;
  return rc;
}

// Binning shared by forward and backward: preprocess, scan, emit.
static cudaError_t bin(cgh_plan* p, const cgh_params* prm, cudaStream_t s) {
  const int T = p->tiles_x * p->tiles_y;
  RasterConsts rc = make_consts(p, prm->N);
  int* tile_count = (int*)(p->ws + p->off_tile_count);
  int* tile_start = (int*)(p->ws + p->off_tile_start);
  int* status = (int*)(p->ws + p->off_status);
  cudaError_t e = cudaMemsetAsync(tile_count, 0, sizeof(int) * CGH_COUNT_STRIDE * (size_t)T, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(status, 0, sizeof(int) * ST_COUNT, s);
  if (e != cudaSuccess) return e;
  p->bin_valid = 1;
  p->bin_params = *prm;
  const int nblk = (prm->N + 255) / 256;
  if (prm->N > 0) {
    prof_begin(KID_PREPROCESS, s);
    float4* rec = (float4*)(p->ws + p->off_rec);
    int4* rect = (int4*)(p->ws + p->off_rect);
    switch (p->C) {
      case 1: k_preprocess<1><<<nblk, 256, 0, s>>>(rc, *prm, rec, rect, tile_count, status); break;
      case 2: k_preprocess<2><<<nblk, 256, 0, s>>>(rc, *prm, rec, rect, tile_count, status); break;
      case 3: k_preprocess<3><<<nblk, 256, 0, s>>>(rc, *prm, rec, rect, tile_count, status); break;
      default: k_preprocess<4><<<nblk, 256, 0, s>>>(rc, *prm, rec, rect, tile_count, status); break;
    }
    prof_end(KID_PREPROCESS, s);
  }
  prof_begin(KID_SCAN_TILES, s);
  const size_t stage_bytes = sizeof(int) * scan_stage_ints(T < kScanChunk ? T : kScanChunk);
  // opt in to more than 48 KB of dynamic shared memory, once per device (the attribute
  // belongs to the function on the current device)
  constexpr int kMaxDev = 64;
  static std::atomic<bool> attr[kMaxDev];
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDev || !attr[dev].load(std::memory_order_acquire)) {
    e = cudaFuncSetAttribute(k_scan_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(int) * scan_stage_ints(kScanChunk)));
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kMaxDev) attr[dev].store(true, std::memory_order_release);
  }
  k_scan_tiles<<<1, 1024, stage_bytes, s>>>(T, p->pair_capacity, tile_count, tile_start, status);
  prof_end(KID_SCAN_TILES, s);
  if (prm->N > 0) {
    prof_begin(KID_EMIT, s);
    k_emit<<<nblk, 256, 0, s>>>(rc, (const int4*)(p->ws + p->off_rect), tile_start, tile_count,
                                (int*)(p->ws + p->off_pairs));
    prof_end(KID_EMIT, s);
  }
  return cudaGetLastError();
}

static bool same_params(const cgh_params* a, const cgh_params* b) {
  return a->N == b->N && a->xy_raw == b->xy_raw && a->s_raw == b->s_raw &&
         a->theta == b->theta && a->amp == b->amp && a->phase == b->phase &&
         a->alpha_raw == b->alpha_raw;
}

template <int C>
static void raster_fwd_c(dim3 grid, cudaStream_t s, const RasterConsts& rc, const float4* rec,
                         const int4* rect, const int* ts, const int* pairs, float2* U,
                         const IdentLoss* ident) {
  if (ident)
    k_raster_fwd<C, true><<<grid, 256, 0, s>>>(rc, rec, rect, ts, pairs, U, *ident);
  else
    k_raster_fwd<C, false><<<grid, 256, 0, s>>>(rc, rec, rect, ts, pairs, U, IdentLoss{});
}

cudaError_t launch_raster_fwd(cgh_plan* p, const cgh_params* prm, float2* U, cudaStream_t s,
                              bool rebin, const IdentLoss* ident) {
  const bool reuse = !rebin && p->bin_valid && same_params(&p->bin_params, prm);
  cudaError_t e = reuse ? cudaSuccess : bin(p, prm, s);
  if (e != cudaSuccess) return e;
  RasterConsts rc = make_consts(p, prm->N);
  dim3 grid(p->tiles_x, p->tiles_y);
  const float4* rec = (const float4*)(p->ws + p->off_rec);
  const int4* rect = (const int4*)(p->ws + p->off_rect);
  const int* ts = (const int*)(p->ws + p->off_tile_start);
  const int* pairs = (const int*)(p->ws + p->off_pairs);
  prof_begin(KID_RASTER_FWD, s);
  switch (p->C) {
    case 1: raster_fwd_c<1>(grid, s, rc, rec, rect, ts, pairs, U, ident); break;
    case 2: raster_fwd_c<2>(grid, s, rc, rec, rect, ts, pairs, U, ident); break;
    case 3: raster_fwd_c<3>(grid, s, rc, rec, rect, ts, pairs, U, ident); break;
    default: raster_fwd_c<4>(grid, s, rc, rec, rect, ts, pairs, U, ident); break;
  }
  prof_end(KID_RASTER_FWD, s);
  return cudaGetLastError();
}

cudaError_t launch_raster_bwd(cgh_plan* p, const cgh_params* prm, const float2* dU,
                              const cgh_grads* g, cudaStream_t s, bool rebin,
                              const float* grad_scale) {
  cudaError_t e = rebin ? bin(p, prm, s) : cudaSuccess;
  if (e != cudaSuccess) return e;
  float* raw = (float*)(p->ws + p->off_raw);
  if (prm->N > 0) {
    e = cudaMemsetAsync(raw, 0, sizeof(float) * CGH_RAW_STRIDE * (size_t)prm->N, s);
    if (e != cudaSuccess) return e;
  }
  RasterConsts rc = make_consts(p, prm->N);
  dim3 grid(p->tiles_x, p->tiles_y);
  const float4* rec = (const float4*)(p->ws + p->off_rec);
  const int4* rect = (const int4*)(p->ws + p->off_rect);
  const int* ts = (const int*)(p->ws + p->off_tile_start);
  const int* pairs = (const int*)(p->ws + p->off_pairs);
  const int nblk = (prm->N + 255) / 256;
  // one CTA per 32 x 32 region of 2 x 2 tiles
  dim3 rgrid((p->tiles_x + 1) / 2, (p->tiles_y + 1) / 2);
  const size_t rsmem = raster_bwd_region_smem(p->C);
  switch (p->C) {
    case 1: e = cudaFuncSetAttribute(k_raster_bwd_region<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem); break;
    case 2: e = cudaFuncSetAttribute(k_raster_bwd_region<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem); break;
    case 3: e = cudaFuncSetAttribute(k_raster_bwd_region<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem); break;
    default: e = cudaFuncSetAttribute(k_raster_bwd_region<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem); break;
  }
  if (e != cudaSuccess) return e;
  prof_begin(KID_RASTER_BWD, s);
  switch (p->C) {
    case 1: k_raster_bwd_region<1><<<rgrid, 256, rsmem, s>>>(rc, rec, rect, ts, pairs, dU, raw); break;
    case 2: k_raster_bwd_region<2><<<rgrid, 256, rsmem, s>>>(rc, rec, rect, ts, pairs, dU, raw); break;
    case 3: k_raster_bwd_region<3><<<rgrid, 256, rsmem, s>>>(rc, rec, rect, ts, pairs, dU, raw); break;
    default: k_raster_bwd_region<4><<<rgrid, 256, rsmem, s>>>(rc, rec, rect, ts, pairs, dU, raw); break;
  }
  prof_end(KID_RASTER_BWD, s);
  (void)grid;
  if (prm->N > 0) {
    prof_begin(KID_GRAD_FINALIZE, s);
    switch (p->C) {
      case 1: k_grad_finalize<1><<<nblk, 256, 0, s>>>(rc, *prm, raw, *g, grad_scale); break;
      case 2: k_grad_finalize<2><<<nblk, 256, 0, s>>>(rc, *prm, raw, *g, grad_scale); break;
      case 3: k_grad_finalize<3><<<nblk, 256, 0, s>>>(rc, *prm, raw, *g, grad_scale); break;
      default: k_grad_finalize<4><<<nblk, 256, 0, s>>>(rc, *prm, raw, *g, grad_scale); break;
    }
    prof_end(KID_GRAD_FINALIZE, s);
  }
  return cudaGetLastError();
}
