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

// ------------------------------------------------------------------ sweep work counters
// Diagnostics of the two sweeps over the binning of `params` (not on the timed path).  One
// CTA per 16x16 tile; each thread takes entries of the tile's list and counts, with the same
// box geometry the kernels use:
//   out[0] forward lane slots: 32 per 8x4 warp block the Gaussian's box touches
//          (raster_fwd_tile visits exactly those (block, Gaussian) pairs);
//   out[1] (pixel, Gaussian) pairs that pass the cutoff (alpha G >= cutoff, the test both
//          sweeps take; tiles partition the pixels, so each pair is counted once);
//   out[2] backward lane slots: for the Gaussian's home tile in its 32x32 region, the box's
//          pixels inside the region rounded up to whole warps (raster_bwd_region sweeps
//          exactly those);
//   out[3] (Gaussian, region) pairs of the backward;  out[4] (Gaussian, tile) list entries.
// Tiles whose list overflowed the capacity are not counted (out[5] = their number).
__global__ void __launch_bounds__(256) k_raster_stats(RasterConsts rc, const float4* __restrict__ rec,
                                                      const int4* __restrict__ rect,
                                                      const int* __restrict__ tile_start,
                                                      const int* __restrict__ pairs,
                                                      unsigned long long* __restrict__ out) {
  const int tx = blockIdx.x, ty = blockIdx.y, tile = ty * rc.tiles_x + tx;
  const int start = tile_start[tile], end = tile_start[tile + 1];
  unsigned long long fwd = 0, hits = 0, bwd = 0, regions = 0, entries = 0;
  if ((long long)end > rc.cap) {
    if (threadIdx.x == 0) atomicAdd(&out[5], 1ull);
    return;  // CTA-uniform: no barrier follows
  }
  const int ox = tx * CGH_TILE, oy = ty * CGH_TILE;
  const int STX = tx / 2, STY = ty / 2;
  for (int i = start + (int)threadIdx.x; i < end; i += blockDim.x) {
    const int gid = pairs[i];
    const float4* g = rec + (size_t)gid * CGH_REC_F4;
    const float4 r0 = g[0], r1 = g[1], bb = g[2];
    const int4 r = rect[gid];
    ++entries;
    // forward: the warp blocks of this tile the box touches
    for (int w = 0; w < 8; ++w) {
      const float x0 = (float)(ox + (w & 1) * 8), y0 = (float)(oy + (w >> 1) * 4);
      if (bb.y >= x0 && bb.x <= x0 + 7.f && bb.w >= y0 && bb.z <= y0 + 3.f) fwd += 32;
    }
    // pairs passing the cutoff inside this tile
    for (int py = oy; py < oy + CGH_TILE && py < rc.H; ++py)
      for (int px = ox; px < ox + CGH_TILE && px < rc.W; ++px) {
        const float p2 = gauss_power(r0, r1, (float)px - r0.x, (float)py - r0.y);
        if (p2 >= r1.y) ++hits;
      }
    // backward: counted once per region, from the Gaussian's home tile
    if (tx == max(r.x, 2 * STX) && ty == max(r.y, 2 * STY)) {
      const int rx = STX * kSuper, ry = STY * kSuper;
      const int x0 = (int)ceilf(fmaxf(bb.x, (float)rx)), x1 = (int)floorf(fminf(bb.y, (float)(rx + kSuper - 1)));
      const int y0 = (int)ceilf(fmaxf(bb.z, (float)ry)), y1 = (int)floorf(fminf(bb.w, (float)(ry + kSuper - 1)));
      if (x0 <= x1 && y0 <= y1) {
        const int npx = (x1 - x0 + 1) * (y1 - y0 + 1);
        bwd += (unsigned long long)((npx + 31) / 32) * 32;
        ++regions;
      }
    }
  }
  unsigned long long v[5] = {fwd, hits, bwd, regions, entries};
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    unsigned long long x = v[k];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&out[k], x);
  }
}

cudaError_t launch_raster_stats(cgh_plan* p, const cgh_params* prm, unsigned long long* out,
                                cudaStream_t s) {
  cudaError_t e = bin(p, prm, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(out, 0, sizeof(unsigned long long) * 6, s);
  if (e != cudaSuccess) return e;
  RasterConsts rc = make_consts(p, prm->N);
  dim3 grid(p->tiles_x, p->tiles_y);
  k_raster_stats<<<grid, 256, 0, s>>>(rc, (const float4*)(p->ws + p->off_rec),
                                      (const int4*)(p->ws + p->off_rect),
                                      (const int*)(p->ws + p->off_tile_start),
                                      (const int*)(p->ws + p->off_pairs), out);
  return cudaGetLastError();
}
