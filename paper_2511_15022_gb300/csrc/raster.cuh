// raster.cuh -- device code of the tile-binned rasteriser (see raster.cu for the
// design): per-Gaussian, per-warp and per-tile item functions, and the kernels that
// launch them one item per thread, warp or CTA.  Included by raster.cu (the planned
// launches) and persist.cu (the persistent batched step).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "cgh_internal.h"

// Loads of data the binning wrote (records, rectangles, lists, tile starts, moments, dL/dU):
// read-only for the whole of a planned kernel, so through the read-only cache; a kernel
// that writes and reads them in one launch (the persistent step) defines CGH_WS_LOAD as an
// L2 load before including this file.
#ifndef CGH_WS_LOAD
#define CGH_WS_LOAD(p) __ldg(p)
#endif
// ... and of data a kernel reads that its own later phases rewrite (the tile counters the scan
// reads and the emit counts down)
#ifndef CGH_RW_LOAD
#define CGH_RW_LOAD(p) (*(p))
#endif

namespace cgh {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kP2Floor = -50.0f * 1.4426950408889634f;  // power clamp -50 in log2 units
constexpr float kAlphaCap = 0.99f;

// 2^max(x, kP2Floor) with the hardware base-2 exponential (PTX ex2.approx.ftz.f32).  The
// argument is clamped at kP2Floor (about -72), so every result is a normal number and the
// flush-to-zero mode never applies; the instruction's relative error (about 2^-22) is far
// inside the field and gradient tolerances.
__device__ __forceinline__ float pow2_clamped(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(fmaxf(x, kP2Floor)));
  return y;
}

// Exponent of one Gaussian (log2 units) at offset (dx, dy) from its mean from the record's
// first two float4s: r0.z dx^2 + r0.w dx dy + r1.x dy^2 (the record holds -log2(e) / 2 times
// the inverse covariance, the cross term doubled).  One form for the forward and both
// backward sweeps, so that they take the same cutoff decisions.
__device__ __forceinline__ float gauss_power(const float4& r0, const float4& r1, float dx,
                                             float dy) {
  return fmaf(dx, fmaf(r0.z, dx, r0.w * dy), r1.x * dy * dy);
}

struct RasterConsts {
  int H, W, C, N, tiles_x, tiles_y;
  float cutoff;
  int _pad;
  long long cap;
};

__device__ __forceinline__ bool finitef(float x) { return isfinite(x); }

// Pre-activation parameters of one Gaussian, loaded together up front (the loads are all
// independent, so they are in flight at the same time).
template <int C>
struct RawParams {
  float x, y, sx, sy, th, al, amp[C], ph[C];
};

template <int C>
__device__ __forceinline__ RawParams<C> load_params(const cgh_params& p, int n) {
  RawParams<C> r;
  r.x = __ldg(&p.xy_raw[2 * n + 0]);
  r.y = __ldg(&p.xy_raw[2 * n + 1]);
  r.sx = __ldg(&p.s_raw[2 * n + 0]);
  r.sy = __ldg(&p.s_raw[2 * n + 1]);
  r.th = __ldg(&p.theta[n]);
  r.al = __ldg(&p.alpha_raw[n]);
#pragma unroll
  for (int c = 0; c < C; ++c) {
    r.amp[c] = __ldg(&p.amp[n * C + c]);
    r.ph[c] = __ldg(&p.phase[n * C + c]);
  }
  return r;
}

// every parameter finite (no short-circuit: nothing waits on one load to decide another)
template <int C>
__device__ __forceinline__ bool all_finite(const RawParams<C>& r) {
  bool ok = finitef(r.x) & finitef(r.y) & finitef(r.sx) & finitef(r.sy) & finitef(r.th) &
            finitef(r.al);
#pragma unroll
  for (int c = 0; c < C; ++c) ok = ok & finitef(r.amp[c]) & finitef(r.ph[c]);
  return ok;
}

// Activated quantities of one Gaussian (shared by preprocess and finalize).
struct Act {
  float tx, ty, mx, my, esx, esy, sx, sy, c, s, S00, S01, S11, det, i00, i01, i11, alpha;
};

template <int C>
__device__ __forceinline__ Act activate(const RawParams<C>& r, int W, int H) {
  Act a;
  a.tx = tanhf(r.x);
  a.ty = tanhf(r.y);
  a.mx = (a.tx + 1.0f) * 0.5f * (float)W;
  a.my = (a.ty + 1.0f) * 0.5f * (float)H;
  a.esx = expf(r.sx);
  a.esy = expf(r.sy);
  a.sx = a.esx + 0.1f;
  a.sy = a.esy + 0.1f;
  sincosf(r.th, &a.s, &a.c);
  float sx2 = a.sx * a.sx, sy2 = a.sy * a.sy;
  a.S00 = sx2 * a.c * a.c + sy2 * a.s * a.s + 0.1f;
  a.S01 = (sx2 - sy2) * a.c * a.s;
  a.S11 = sx2 * a.s * a.s + sy2 * a.c * a.c + 0.1f;
  a.det = a.S00 * a.S11 - a.S01 * a.S01;
  float ds = fmaxf(a.det, 1e-10f);
  a.i00 = a.S11 / ds;
  a.i01 = -a.S01 / ds;
  a.i11 = a.S00 / ds;
  a.alpha = 1.0f / (1.0f + expf(-r.al));
  return a;
}

template <int C>
__device__ __forceinline__ void preprocess_one(const RasterConsts& rc, const cgh_params& p,
                                               float4* __restrict__ rec, int4* __restrict__ rect,
                                               int* __restrict__ tile_count,
                                               int* __restrict__ status, int n) {
  const RawParams<C> q = load_params<C>(p, n);
  const bool ok = all_finite(q);
  float A[CGH_MAX_C] = {0.f, 0.f, 0.f, 0.f}, B[CGH_MAX_C] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int c = 0; c < C; ++c) {
    float sp, cp;
    sincosf(q.ph[c], &sp, &cp);
    A[c] = q.amp[c] * cp;
    B[c] = q.amp[c] * sp;
  }
  if (!ok) atomicExch(&status[ST_NONFINITE], 1);
  Act a = activate(q, rc.W, rc.H);
  const float k = -0.5f * kLog2e;
  float thr = rc.cutoff > 0.f ? log2f(rc.cutoff / a.alpha) : -INFINITY;
  // box of the ellipse m <= m*, m* = 2 ln(alpha / cutoff) (power floor m = 100 in smooth
  // mode); half-widths sqrt(m* S00), sqrt(m* S11), widened slightly for FP32 rounding.
  float mstar = rc.cutoff > 0.f ? 2.0f * logf(a.alpha / rc.cutoff) : 100.0f;
  int4 r = make_int4(1, 1, 0, 0);  // empty
  float bx0 = 1.f, bx1 = 0.f, by0 = 1.f, by1 = 0.f;
  if (ok && a.alpha >= rc.cutoff && mstar >= 0.f && isfinite(a.mx) && isfinite(a.my)) {
    float rx = sqrtf(mstar * a.S00) * 1.0001f + 0.01f;
    float ry = sqrtf(mstar * a.S11) * 1.0001f + 0.01f;
    bx0 = fmaxf(a.mx - rx, 0.f);
    bx1 = fminf(a.mx + rx, (float)(rc.W - 1));
    by0 = fmaxf(a.my - ry, 0.f);
    by1 = fminf(a.my + ry, (float)(rc.H - 1));
    if (bx0 <= bx1 && by0 <= by1 && isfinite(rx) && isfinite(ry)) {
      r.x = (int)floorf(bx0) / CGH_TILE;
      r.z = (int)floorf(bx1) / CGH_TILE;
      r.y = (int)floorf(by0) / CGH_TILE;
      r.w = (int)floorf(by1) / CGH_TILE;
    } else {
      bx0 = 1.f; bx1 = 0.f; by0 = 1.f; by1 = 0.f;
    }
  }
  float4* o = rec + (size_t)n * CGH_REC_F4;
  o[0] = make_float4(a.mx, a.my, k * a.i00, 2.0f * k * a.i01);
  o[1] = make_float4(k * a.i11, thr, a.alpha, 0.f);
  o[2] = make_float4(bx0, bx1, by0, by1);
  o[3] = make_float4(A[0], B[0], A[1], B[1]);
  o[4] = make_float4(A[2], B[2], A[3], B[3]);
  rect[n] = r;
  for (int ty = r.y; ty <= r.w; ++ty)
    for (int tx = r.x; tx <= r.z; ++tx) atomicAdd(&tile_count[(ty * rc.tiles_x + tx) * CGH_COUNT_STRIDE], 1);
}

#ifndef CGH_ITEMS_ONLY
template <int C>
__global__ void k_preprocess(RasterConsts rc, cgh_params p, float4* __restrict__ rec,
                             int4* __restrict__ rect, int* __restrict__ tile_count,
                             int* __restrict__ status) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < rc.N) preprocess_one<C>(rc, p, rec, rect, tile_count, status, n);
}
#endif  // CGH_ITEMS_ONLY

// Exclusive scan of tile counts (one CTA of 1024 threads).  tile_start has T+1 entries;
// tile_count is left as it is: k_emit counts it down to zero as the per-tile cursor.
// The tiles are scanned in chunks of at most kScanChunk, each staged through shared memory
// so that global memory is read and written with coalesced accesses (with one CTA doing the
// whole scan, per-thread chunks read straight from global memory would cost one L1 wavefront
// per thread per element).  Within a chunk each thread owns `per` consecutive tiles; the
// stage holds element i at i + i / 32, which spreads a warp's chunk-wise accesses over all
// 32 banks.  A running carry joins the chunks.
constexpr int kScanChunk = 32768;
__host__ __device__ __forceinline__ int scan_pad(int i) { return i + (i >> 5); }
__host__ __device__ __forceinline__ size_t scan_stage_ints(int n) { return (size_t)scan_pad(n) + 1; }

// The scan by one CTA (any multiple of 32 threads up to 1024): `stage` holds
// scan_stage_ints(chunk) ints of shared memory, `warp_sums` 32.
__device__ __forceinline__ void scan_tiles_cta(int T, long long cap, int* __restrict__ tile_count,
                                               int* __restrict__ tile_start,
                                               int* __restrict__ status, int* stage,
                                               long long* warp_sums, int chunk) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  long long carry = 0;  // pairs of the chunks before this one
  for (int c0 = 0; c0 < T; c0 += chunk) {
    const int n = min(chunk, T - c0);
    __syncthreads();  // the previous chunk's stage has been written out
    // kScanU independent loads in flight per thread before any of them is stored
    constexpr int kScanU = 8;
    for (int i0 = tid; i0 < n; i0 += nt * kScanU) {
      int cv[kScanU];
#pragma unroll
      for (int u = 0; u < kScanU; ++u) {
        const int i = i0 + u * nt;
        cv[u] = i < n ? CGH_RW_LOAD(&tile_count[(size_t)(c0 + i) * CGH_COUNT_STRIDE]) : 0;
      }
#pragma unroll
      for (int u = 0; u < kScanU; ++u) {
        const int i = i0 + u * nt;
        if (i < n) stage[scan_pad(i)] = cv[u];
      }
    }
    __syncthreads();
    const int per = (n + nt - 1) / nt;
    const int beg = min(n, tid * per), end = min(n, beg + per);
    long long local = 0;
    for (int i = beg; i < end; ++i) local += stage[scan_pad(i)];
    // inclusive scan of `local` over the CTA
    long long v = local;
    for (int o = 1; o < 32; o <<= 1) {
      long long u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane == 31) warp_sums[wid] = v;
    __syncthreads();
    if (wid == 0) {
      long long w = (lane < (nt >> 5)) ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        long long u = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += u;
      }
      warp_sums[lane] = w;
    }
    __syncthreads();
    // exclusive starts replace the counts in the stage
    long long excl = carry + v - local + (wid > 0 ? warp_sums[wid - 1] : 0);
    for (int i = beg; i < end; ++i) {
      const int c = stage[scan_pad(i)];
      stage[scan_pad(i)] = (int)min(excl, (long long)0x7fffffff);
      excl += c;
    }
    carry += warp_sums[(nt >> 5) - 1];
    __syncthreads();
    for (int i = tid; i < n; i += nt) tile_start[c0 + i] = stage[scan_pad(i)];
  }
  if (tid == 0) {
    tile_start[T] = (int)min(carry, (long long)0x7fffffff);
    status[ST_PAIRS_LO] = (int)(carry & 0xffffffff);
    status[ST_PAIRS_HI] = (int)(carry >> 32);
    if (carry > cap) status[ST_OVERFLOW] = 1;
  }
}

#ifndef CGH_ITEMS_ONLY
__global__ void __launch_bounds__(1024) k_scan_tiles(int T, long long cap,
                                                     int* __restrict__ tile_count,
                                                     int* __restrict__ tile_start,
                                                     int* __restrict__ status) {
  extern __shared__ int stage[];
  __shared__ long long warp_sums[32];
  scan_tiles_cta(T, cap, tile_count, tile_start, status, stage, warp_sums, kScanChunk);
}
#endif  // CGH_ITEMS_ONLY

// The (Gaussian, tile) slots.  A warp pools the boxes of its 32 Gaussians and deals the
// (Gaussian, tile) items out to its lanes, EMIT_U per lane per round, so that one large box
// (optimised Gaussians can grow to cover a hundred tiles) costs its warp a few rounds instead
// of a long serial loop in one lane; each round's cursor updates are all in flight at once.
constexpr int EMIT_U = 4;
// Called by all 32 lanes of a warp together, Gaussian n per lane (n >= N: no box).
__device__ __forceinline__ void emit_warp(const RasterConsts& rc, const int4* __restrict__ rect,
                                          const int* __restrict__ tile_start,
                                          int* __restrict__ cursor, int* __restrict__ pairs,
                                          int n) {
  const int lane = threadIdx.x & 31;
  int4 r = make_int4(1, 1, 0, 0);
  if (n < rc.N) r = CGH_WS_LOAD(&rect[n]);
  const int bw = r.z - r.x + 1;
  const int cnt = (r.z >= r.x && r.w >= r.y) ? bw * (r.w - r.y + 1) : 0;
  // exclusive prefix of the box sizes over the warp
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  const int excl = incl - cnt;
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  const int warp_n0 = n - lane;
  for (int k0 = 0; k0 < total; k0 += 32 * EMIT_U) {
    int t[EMIT_U], slot[EMIT_U], gid[EMIT_U];
#pragma unroll
    for (int u = 0; u < EMIT_U; ++u) {
      const int k = k0 + u * 32 + lane;
      // owner: the last lane whose exclusive prefix is <= k (it holds item k when k < total)
      int o = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const int e = __shfl_sync(0xffffffffu, excl, o + step);
        if (e <= k) o += step;
      }
      const int j = k - __shfl_sync(0xffffffffu, excl, o);
      const int obw = __shfl_sync(0xffffffffu, bw, o);
      const int ox = __shfl_sync(0xffffffffu, r.x, o), oy = __shfl_sync(0xffffffffu, r.y, o);
      gid[u] = warp_n0 + o;
      t[u] = k < total ? (oy + j / obw) * rc.tiles_x + ox + j % obw : -1;
      // the tile's count, counted down: slots count-1, ..., 0 (it ends at zero)
      slot[u] = t[u] >= 0 ? atomicSub(&cursor[t[u] * CGH_COUNT_STRIDE], 1) - 1 : 0;
    }
#pragma unroll
    for (int u = 0; u < EMIT_U; ++u) {
      if (t[u] < 0) continue;
      const long long pos = (long long)CGH_WS_LOAD(&tile_start[t[u]]) + slot[u];
      if (pos < rc.cap) pairs[pos] = gid[u];
    }
  }
}

#ifndef CGH_ITEMS_ONLY
__global__ void __launch_bounds__(256) k_emit(RasterConsts rc, const int4* __restrict__ rect,
                                              const int* __restrict__ tile_start,
                                              int* __restrict__ cursor, int* __restrict__ pairs) {
  emit_warp(rc, rect, tile_start, cursor, pairs, blockIdx.x * blockDim.x + threadIdx.x);
}
#endif  // CGH_ITEMS_ONLY

// Stage records [base, base + 256) of a tile's list into shared memory.  In exhaustive
// mode (list overflowed) the candidates are all Gaussians and the ones whose tile
// rectangle misses this tile get an empty box.
__device__ __forceinline__ int stage_batch(const RasterConsts& rc, const float4* __restrict__ rec,
                                           const int4* __restrict__ rect,
                                           const int* __restrict__ pairs, int start, int count,
                                           bool exhaustive, int base, int tx, int ty,
                                           float4* srec, int* sgid) {
  const int i = base + threadIdx.x;
  if (i < count) {
    int gid = exhaustive ? i : CGH_WS_LOAD(&pairs[start + i]);
    const float4* g = rec + (size_t)gid * CGH_REC_F4;
#pragma unroll
    for (int k = 0; k < CGH_REC_F4; ++k) srec[threadIdx.x * CGH_REC_F4 + k] = CGH_WS_LOAD(&g[k]);
    if (exhaustive) {
      int4 r = CGH_WS_LOAD(&rect[gid]);
      if (tx < r.x || tx > r.z || ty < r.y || ty > r.w)
        srec[threadIdx.x * CGH_REC_F4 + 2] = make_float4(1.f, 0.f, 1.f, 0.f);
    }
    if (sgid) sgid[threadIdx.x] = gid;
  }
  return min(256, count - base);
}

// Forward: one CTA per tile, one thread per pixel; warp w owns the 8 x 4 block at
// ((w & 1) 8, (w >> 1) 4) of the tile.  When a batch is staged, the thread that staged a
// Gaussian also marks which warp blocks its box touches; each warp then compacts its own
// list with ballots and visits only those Gaussians.

// Pixel of this thread in tile (tx, ty) and the tile's origin.
struct FwdPixel {
  int px, py;
  float fpx, fpy, fox, foy;
  __device__ __forceinline__ FwdPixel(int tx, int ty) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    px = tx * CGH_TILE + (warp & 1) * 8 + (lane & 7);
    py = ty * CGH_TILE + (warp >> 1) * 4 + (lane >> 3);
    fpx = (float)px; fpy = (float)py;
    fox = (float)(tx * CGH_TILE); foy = (float)(ty * CGH_TILE);
  }
};

// One staged batch of nb records in srec (thread i < nb staged record i and may read it back
// without a barrier): warp masks, a barrier, per-warp compaction, then the warp's Gaussians
// accumulated into accr / acci.
template <int C>
__device__ __forceinline__ void fwd_sweep_batch(const FwdPixel& q, const float4* srec, int nb,
                                                unsigned char* smask,
                                                unsigned char (*slist)[256], float (&accr)[C],
                                                float (&acci)[C]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if ((int)threadIdx.x < nb) {
    // warp blocks (2 columns x 4 rows of the tile) the staged box touches
    const float4 bb = srec[threadIdx.x * CGH_REC_F4 + 2];
    unsigned m = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const float x0 = q.fox + (float)((w & 1) * 8), y0 = q.foy + (float)((w >> 1) * 4);
      if (bb.y >= x0 && bb.x <= x0 + 7.f && bb.w >= y0 && bb.z <= y0 + 3.f) m |= 1u << w;
    }
    smask[threadIdx.x] = (unsigned char)m;
  }
  __syncthreads();
  int cnt = 0;
  for (int k = 0; k < nb; k += 32) {
    const int i = k + lane;
    const bool mine = i < nb && ((smask[i] >> warp) & 1u);
    const unsigned b = __ballot_sync(0xffffffffu, mine);
    if (mine) slist[warp][cnt + __popc(b & ((1u << lane) - 1u))] = (unsigned char)i;
    cnt += __popc(b);
  }
  __syncwarp();
  // contribution of the Gaussian whose record starts at srec[j] (power p2 >= its cutoff)
  auto splat = [&](int j, float p2, float alpha) {
    const float a = fminf(kAlphaCap, alpha * pow2_clamped(p2));
    const float4 r3 = srec[j + 3];
    const float4 r4 = srec[j + 4];
    const float Ac[4] = {r3.x, r3.z, r4.x, r4.z};
    const float Bc[4] = {r3.y, r3.w, r4.y, r4.w};
#pragma unroll
    for (int c = 0; c < C; ++c) {
      accr[c] = fmaf(a, Ac[c], accr[c]);
      acci[c] = fmaf(a, Bc[c], acci[c]);
    }
  };
  // the warp's Gaussians two at a time, in list order: both records' geometry is read
  // before either power is tested (more loads in flight, half the loop overhead)
  int t = 0;
  for (; t + 2 <= cnt; t += 2) {
    const int j0 = slist[warp][t] * CGH_REC_F4, j1 = slist[warp][t + 1] * CGH_REC_F4;
    const float4 a0 = srec[j0], b0 = srec[j0 + 1];
    const float4 a1 = srec[j1], b1 = srec[j1 + 1];
    const float p0 = gauss_power(a0, b0, q.fpx - a0.x, q.fpy - a0.y);
    const float p1 = gauss_power(a1, b1, q.fpx - a1.x, q.fpy - a1.y);
    if (p0 >= b0.y) splat(j0, p0, b0.z);
    if (p1 >= b1.y) splat(j1, p1, b1.z);
  }
  if (t < cnt) {
    const int j0 = slist[warp][t] * CGH_REC_F4;
    const float4 a0 = srec[j0], b0 = srec[j0 + 1];
    const float p0 = gauss_power(a0, b0, q.fpx - a0.x, q.fpy - a0.y);
    if (p0 >= b0.y) splat(j0, p0, b0.z);
  }
}

// The finished pixel: U stored and, with LOSS, the identity planes' loss (and seed) of `il`
// on it (U(d_l) = U(0) for those planes): per plane l and channel c, d = |U|^2 - T_l and the
// weight w of the loss (1, or 1 + M + T^2 for L_recon, Sec. 3.2); the tile's sum of w d^2 is
// one loss partial, the seed gscale sum_l w d U the loss row pass would form.  Ends with a
// barrier when LOSS.
template <int C, bool LOSS>
__device__ __forceinline__ void fwd_epilogue(const RasterConsts& rc, const FwdPixel& q, int tile,
                                             const float (&accr)[C], const float (&acci)[C],
                                             float2* __restrict__ U, const IdentLoss* il,
                                             float* red) {
  const int px = q.px, py = q.py;
  const bool inside = px < rc.W && py < rc.H;
  const size_t plane = (size_t)rc.H * rc.W, o = (size_t)py * rc.W + px;
  if (inside) {
#pragma unroll
    for (int c = 0; c < C; ++c) U[c * plane + o] = make_float2(accr[c], acci[c]);
  }
  if constexpr (LOSS) {
    float acc = 0.f;
    if (inside) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const float I = fmaf(accr[c], accr[c], acci[c] * acci[c]);
        float gs = 0.f;
        for (unsigned m = il->mask; m != 0u; m &= m - 1u) {
          const int l = __ffs((int)m) - 1;
          const float t = __ldg(&il->target[((size_t)l * C + c) * plane + o]);
          const float d = I - t;
          float w = 1.f;
          if (il->loss_kind != 0) {
            const float mk =
                (il->recon_mask && il->recon_mask[((size_t)l * rc.H + py) * rc.W + px]) ? 1.f : 0.f;
            w = 1.f + mk + t * t;
          }
          const float wd = w * d;
          acc = fmaf(wd, d, acc);
          gs += wd;
        }
        if (il->seed) {
          const float g = il->gscale * gs;
          il->seed[c * plane + o] = make_float2(accr[c] * g, acci[c] * g);
        }
      }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = 16; k > 0; k >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, k);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float tot = 0.f;
      for (int w = 0; w < 8; ++w) tot += red[w];
      il->partials[tile] = tot;
    }
  }
}

// One tile (tx, ty) by a CTA of 256 threads; shared memory: srec[256 * CGH_REC_F4],
// smask[256], slist[8][256] (+ red[8] with LOSS).  LOSS: the identity planes' loss (and
// seed) of IdentLoss on the finished pixels, whose values are still in registers.
template <int C, bool LOSS = false>
__device__ __forceinline__ void raster_fwd_tile(const RasterConsts& rc,
                                                const float4* __restrict__ rec,
                                                const int4* __restrict__ rect,
                                                const int* __restrict__ tile_start,
                                                const int* __restrict__ pairs,
                                                float2* __restrict__ U, int tx, int ty,
                                                float4* srec, unsigned char* smask,
                                                unsigned char (*slist)[256],
                                                const IdentLoss* il = nullptr,
                                                float* red = nullptr) {
  const int tile = ty * rc.tiles_x + tx;
  const FwdPixel q(tx, ty);
  const int start = CGH_WS_LOAD(&tile_start[tile]), end = CGH_WS_LOAD(&tile_start[tile + 1]);
  const bool exhaustive = (long long)end > rc.cap;
  const int count = exhaustive ? rc.N : end - start;
  float accr[C], acci[C];
#pragma unroll
  for (int c = 0; c < C; ++c) { accr[c] = 0.f; acci[c] = 0.f; }
  for (int base = 0; base < count; base += 256) {
    __syncthreads();
    const int nb = stage_batch(rc, rec, rect, pairs, start, count, exhaustive, base, tx, ty,
                               srec, nullptr);
    fwd_sweep_batch<C>(q, srec, nb, smask, slist, accr, acci);
  }
  fwd_epilogue<C, LOSS>(rc, q, tile, accr, acci, U, il, red);
}

#ifndef CGH_ITEMS_ONLY
// LOSS: with the identity planes' loss of `il` (one partial per tile).
template <int C, bool LOSS>
__global__ void __launch_bounds__(256) k_raster_fwd(RasterConsts rc, const float4* __restrict__ rec,
                                                    const int4* __restrict__ rect,
                                                    const int* __restrict__ tile_start,
                                                    const int* __restrict__ pairs,
                                                    float2* __restrict__ U, IdentLoss il) {
  __shared__ float4 srec[256 * CGH_REC_F4];
  __shared__ unsigned char smask[256];
  __shared__ unsigned char slist[8][256];
  __shared__ float red[8];
  raster_fwd_tile<C, LOSS>(rc, rec, rect, tile_start, pairs, U, blockIdx.x, blockIdx.y, srec,
                           smask, slist, &il, red);
}
#endif  // CGH_ITEMS_ONLY


// Warp reduce-scatter of COUNT values per lane (COUNT a power of two <= 32): at each step
// lanes exchange half of their values with the partner OFF lanes away and keep the sum of
// the other half, so COUNT values cost COUNT - 1 + log2(32 / COUNT) shuffles instead of
// 5 * COUNT.  Afterwards every lane holds the warp total of value `base`; lanes that differ
// only in the bits below log2(32 / COUNT) hold the same value.
template <int COUNT, int OFF>
struct ReduceScatter {
  __device__ __forceinline__ static void run(float* cur, int lane, int& base) {
    constexpr int HALF = COUNT / 2;
    const bool hi = (lane & OFF) != 0;
#pragma unroll
    for (int i = 0; i < HALF; ++i) {
      const float send = hi ? cur[i] : cur[i + HALF];
      const float keep = hi ? cur[i + HALF] : cur[i];
      cur[i] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
    }
    if (hi) base += HALF;
    ReduceScatter<HALF, OFF / 2>::run(cur, lane, base);
  }
};
template <int OFF>
struct ReduceScatter<1, OFF> {
  __device__ __forceinline__ static void run(float* cur, int, int&) {
#pragma unroll
    for (int o = OFF; o >= 1; o >>= 1) cur[0] += __shfl_xor_sync(0xffffffffu, cur[0], o);
  }
};

// The same for exactly 12 values per lane (C = 3): 13 shuffles instead of the 16 of the padded
// 16-value form.  After halving twice (6, then 3 values) the three values split unevenly --
// lanes with bit 2 clear keep values 0 and 1, lanes with bit 2 set keep value 2 -- and one more
// exchange leaves one value per lane.  Lane value index: (lane & 16 ? 6 : 0) + (lane & 8 ? 3 : 0)
// + (lane & 4 ? 2 : lane & 2 ? 1 : 0); it owns the value (adds it out) when bit 0 is clear and
// not both bits 2 and 1 are set.
__device__ __forceinline__ void reduce_scatter_12(float* cur, int lane, int& vidx,
                                                  bool& owner) {
  {  // 12 -> 6
    const bool hi = (lane & 16) != 0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const float send = hi ? cur[i] : cur[i + 6];
      const float keep = hi ? cur[i + 6] : cur[i];
      cur[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
  }
  {  // 6 -> 3
    const bool hi = (lane & 8) != 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float send = hi ? cur[i] : cur[i + 3];
      const float keep = hi ? cur[i + 3] : cur[i];
      cur[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
  }
  const bool b2 = (lane & 4) != 0, b1 = (lane & 2) != 0;
  {  // 3 -> {0, 1} (bit 2 clear) or {2} (bit 2 set)
    const float r0 = __shfl_xor_sync(0xffffffffu, b2 ? cur[0] : cur[2], 4);
    const float r1 = __shfl_xor_sync(0xffffffffu, cur[1], 4);
    if (b2) {
      cur[0] = cur[2] + r0;
    } else {
      cur[0] += r0;
      cur[1] += r1;
    }
  }
  {  // -> one value: {0} / {1} by bit 1 (bit 2 clear), {2} on both partners (bit 2 set)
    const float send = b2 ? cur[0] : (b1 ? cur[0] : cur[1]);
    const float keep = b2 ? cur[0] : (b1 ? cur[1] : cur[0]);
    cur[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  cur[0] += __shfl_xor_sync(0xffffffffu, cur[0], 1);
  vidx = ((lane & 16) ? 6 : 0) + ((lane & 8) ? 3 : 0) + (b2 ? 2 : (b1 ? 1 : 0));
  owner = (lane & 1) == 0 && !(b2 && b1);
}

// Raw accumulated moments per Gaussian (NV = 2C + 6 values):
//   [0, C)      P_c = sum a dL/dRe_c          [C, 2C)  Q_c = sum a dL/dIm_c
//   2C          SG  = sum G S (unclamped pairs), S = sum_c (A_c dRe_c + B_c dIm_c)
//   2C+1..2C+5  sum u dx, u dy, u dx^2, u dx dy, u dy^2 with u = S alpha G (power unclamped)
// One CTA per tile.  The tile's dL/dU is staged in shared memory; each warp takes one staged
// Gaussian at a time and sweeps the pixels of its box inside the tile (flattened, one
// pixel per lane per step), accumulating the moments in registers; one
// reduce-scatter over the warp and NV global atomics per (Gaussian, tile) follow.  Pixels
// outside the box fail the cutoff test anyway (the box bounds the cutoff ellipse with
// margin), so the sum equals that over all pixels of the tile.
// One tile (tx, ty) by a CTA of 256 threads; shared memory: srec[256 * CGH_REC_F4],
// sgid[256], sdu[C][256].
template <int C>
__device__ __forceinline__ void raster_bwd_tile(const RasterConsts& rc,
                                                const float4* __restrict__ rec,
                                                const int4* __restrict__ rect,
                                                const int* __restrict__ tile_start,
                                                const int* __restrict__ pairs,
                                                const float2* __restrict__ dU,
                                                float* __restrict__ raw, int tx, int ty,
                                                float4* srec, int* sgid,
                                                float2 (*sdu)[CGH_TILE * CGH_TILE]) {
  constexpr int NV = 2 * C + 6;
  constexpr int NVP = NV <= 8 ? 8 : 16;  // padded to a power of two for the reduce-scatter
  const int tile = ty * rc.tiles_x + tx;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ox = tx * CGH_TILE, oy = ty * CGH_TILE;
  {
    const int px = ox + (threadIdx.x & (CGH_TILE - 1)), py = oy + (threadIdx.x >> 4);
    const bool inside = px < rc.W && py < rc.H;
    const size_t plane = (size_t)rc.H * rc.W, o = (size_t)py * rc.W + px;
#pragma unroll
    for (int c = 0; c < C; ++c) sdu[c][threadIdx.x] = inside ? CGH_WS_LOAD(&dU[c * plane + o]) : make_float2(0.f, 0.f);
  }
  const int start = CGH_WS_LOAD(&tile_start[tile]), end = CGH_WS_LOAD(&tile_start[tile + 1]);
  const bool exhaustive = (long long)end > rc.cap;
  const int count = exhaustive ? rc.N : end - start;
  const float fox = (float)ox, foy = (float)oy;
  for (int base = 0; base < count; base += 256) {
    __syncthreads();
    const int nb = stage_batch(rc, rec, rect, pairs, start, count, exhaustive, base, tx, ty,
                               srec, sgid);
    __syncthreads();
    for (int j = warp; j < nb; j += 8) {
      const float4 bb = srec[j * CGH_REC_F4 + 2];
      // pixel box of the Gaussian inside this tile (tile coordinates)
      const int x0 = (int)ceilf(fmaxf(bb.x, fox)) - ox;
      const int x1 = (int)floorf(fminf(bb.y, fox + (float)(CGH_TILE - 1))) - ox;
      const int y0 = (int)ceilf(fmaxf(bb.z, foy)) - oy;
      const int y1 = (int)floorf(fminf(bb.w, foy + (float)(CGH_TILE - 1))) - oy;
      if (x0 > x1 || y0 > y1) continue;  // warp-uniform
      const float4 r0 = srec[j * CGH_REC_F4 + 0];
      const float4 r1 = srec[j * CGH_REC_F4 + 1];
      const float4 r3 = srec[j * CGH_REC_F4 + 3];
      const float4 r4 = srec[j * CGH_REC_F4 + 4];
      const float Ac[4] = {r3.x, r3.z, r4.x, r4.z};
      const float Bc[4] = {r3.y, r3.w, r4.y, r4.w};
      // the box's pixels, flattened: lane k takes pixels k, k + 32, ...; floor(k / bw) from
      // one FP32 product, exact here because k < 256 and the fractional part of
      // (k + 1/2) / bw stays at least 1/32 away from an integer
      const int bw = x1 - x0 + 1, npx = bw * (y1 - y0 + 1);
      const float inv_bw = 1.f / (float)bw;
      float acc[NVP];
#pragma unroll
      for (int v = 0; v < NVP; ++v) acc[v] = 0.f;
      for (int k = lane; k < npx; k += 32) {
        const int ry = (int)(((float)k + 0.5f) * inv_bw);
        const int lx_ = x0 + (k - ry * bw), ly_ = y0 + ry;
        {
          const float dx = (float)(ox + lx_) - r0.x, dy = (float)(oy + ly_) - r0.y;
          const float p2 = gauss_power(r0, r1, dx, dy);
          if (p2 < r1.y) continue;
          const int pix = ly_ * CGH_TILE + lx_;
          const float G = pow2_clamped(p2);
          const float aG = r1.z * G;
          const float a = fminf(kAlphaCap, aG);
          float S = 0.f;
#pragma unroll
          for (int c = 0; c < C; ++c) {
            const float2 g = sdu[c][pix];
            acc[c] = fmaf(a, g.x, acc[c]);
            acc[C + c] = fmaf(a, g.y, acc[C + c]);
            S = fmaf(Ac[c], g.x, fmaf(Bc[c], g.y, S));
          }
          if (aG < kAlphaCap) {
            acc[2 * C] = fmaf(S, G, acc[2 * C]);
            if (p2 > kP2Floor) {
              const float u = S * aG;
              const float udx = u * dx, udy = u * dy;
              acc[2 * C + 1] += udx;
              acc[2 * C + 2] += udy;
              acc[2 * C + 3] = fmaf(udx, dx, acc[2 * C + 3]);
              acc[2 * C + 4] = fmaf(udx, dy, acc[2 * C + 4]);
              acc[2 * C + 5] = fmaf(udy, dy, acc[2 * C + 5]);
            }
          }
        }
      }
      int vidx = 0;
      ReduceScatter<NVP, 16>::run(acc, lane, vidx);
      if ((lane & (32 / NVP - 1)) == 0 && vidx < NV && acc[0] != 0.f)
        atomicAdd(&raw[(size_t)sgid[j] * CGH_RAW_STRIDE + vidx], acc[0]);
    }
  }
}

#ifndef CGH_ITEMS_ONLY
template <int C>
__global__ void __launch_bounds__(256) k_raster_bwd(RasterConsts rc, const float4* __restrict__ rec,
                                                    const int4* __restrict__ rect,
                                                    const int* __restrict__ tile_start,
                                                    const int* __restrict__ pairs,
                                                    const float2* __restrict__ dU,
                                                    float* __restrict__ raw) {
  __shared__ float4 srec[256 * CGH_REC_F4];
  __shared__ int sgid[256];
  __shared__ float2 sdu[C][CGH_TILE * CGH_TILE];
  raster_bwd_tile<C>(rc, rec, rect, tile_start, pairs, dU, raw, blockIdx.x, blockIdx.y, srec,
                     sgid, sdu);
}
#endif  // CGH_ITEMS_ONLY

// Backward over a 32 x 32 region (2 x 2 tiles) per CTA of 256 threads: the region's dL/dU is
// staged in shared memory; the CTA walks the lists of its four 16 x 16 tiles and keeps a
// Gaussian only from its home tile -- the first of its tiles inside the region,
// (max(r.x, 2 STX), max(r.y, 2 STY)) -- so every Gaussian meets the region once; each warp then
// sweeps one kept Gaussian's box inside the region (up to 1024 pixels, flattened), with the
// moments, reduction and atomics of raster_bwd_tile.  Compared with one CTA per tile, a
// Gaussian that straddles tile borders is reduced once per region instead of once per tile.
// The four lists are walked as one stream of candidates (list q after lists 0..q-1), 256 per
// batch; within a batch the warps take the kept Gaussians one at a time from a shared counter,
// so a warp that drew small boxes takes more of them instead of waiting at the next barrier.
// Shared memory: srec[256 * CGH_REC_F4], sgid[256], sdu[C][1024], then 16 ints: kept count,
// next kept index, and per tile q of the region its list start [2 + q], candidate count
// [6 + q] and exhaustive flag [10 + q].
constexpr int kSuper = 2 * CGH_TILE;
constexpr int kRegionCtl = 16;
// 1 / w for box widths w = 1..32 (warp-uniform: one broadcast load instead of a division)
static __constant__ float kInvWidth[kSuper + 1] = {
    0.f,          1.f,          1.f / 2.f,    1.f / 3.f,    1.f / 4.f,    1.f / 5.f,
    1.f / 6.f,    1.f / 7.f,    1.f / 8.f,    1.f / 9.f,    1.f / 10.f,   1.f / 11.f,
    1.f / 12.f,   1.f / 13.f,   1.f / 14.f,   1.f / 15.f,   1.f / 16.f,   1.f / 17.f,
    1.f / 18.f,   1.f / 19.f,   1.f / 20.f,   1.f / 21.f,   1.f / 22.f,   1.f / 23.f,
    1.f / 24.f,   1.f / 25.f,   1.f / 26.f,   1.f / 27.f,   1.f / 28.f,   1.f / 29.f,
    1.f / 30.f,   1.f / 31.f,   1.f / 32.f};
template <int C>
__device__ __forceinline__ void raster_bwd_region(const RasterConsts& rc,
                                                  const float4* __restrict__ rec,
                                                  const int4* __restrict__ rect,
                                                  const int* __restrict__ tile_start,
                                                  const int* __restrict__ pairs,
                                                  const float2* __restrict__ dU,
                                                  float* __restrict__ raw, int STX, int STY,
                                                  float4* srec, int* sgid,
                                                  float2 (*sdu)[kSuper * kSuper], int* sctl) {
  constexpr int NV = 2 * C + 6;
  constexpr int NVP = NV <= 8 ? 8 : 16;  // padded to a power of two for the reduce-scatter
  const int lane = threadIdx.x & 31;
  const int ox = STX * kSuper, oy = STY * kSuper;
  if (threadIdx.x < 4) {
    const int q = threadIdx.x;
    const int sx = 2 * STX + (q & 1), sy = 2 * STY + (q >> 1);
    int st = 0, cnt = 0, ex = 0;
    if (sx < rc.tiles_x && sy < rc.tiles_y) {
      const int tile = sy * rc.tiles_x + sx;
      st = CGH_WS_LOAD(&tile_start[tile]);
      const int end = CGH_WS_LOAD(&tile_start[tile + 1]);
      ex = (long long)end > rc.cap;
      cnt = ex ? rc.N : end - st;
    }
    sctl[2 + q] = st;
    sctl[6 + q] = cnt;
    sctl[10 + q] = ex;
  }
  {
    const size_t plane = (size_t)rc.H * rc.W;
    for (int i = threadIdx.x; i < kSuper * kSuper; i += blockDim.x) {
      const int px = ox + (i & (kSuper - 1)), py = oy + i / kSuper;
      const bool inside = px < rc.W && py < rc.H;
      const size_t o = (size_t)py * rc.W + px;
#pragma unroll
      for (int c = 0; c < C; ++c)
        sdu[c][i] = inside ? CGH_WS_LOAD(&dU[c * plane + o]) : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();  // tile lists and dU are staged
  const int e1 = sctl[6], e2 = e1 + sctl[7], e3 = e2 + sctl[8], total = e3 + sctl[9];
  const float fox = (float)ox, foy = (float)oy;
  for (int base = 0; base < total; base += 256) {
    __syncthreads();  // the previous batch has been swept
    if (threadIdx.x == 0) { sctl[0] = 0; sctl[1] = 0; }
    __syncthreads();
    const int i = base + threadIdx.x;
    int gid = 0;
    bool keep = false;
    if (i < total) {
      const int q = (i >= e1) + (i >= e2) + (i >= e3);
      const int li = i - (q == 0 ? 0 : q == 1 ? e1 : q == 2 ? e2 : e3);
      const int sx = 2 * STX + (q & 1), sy = 2 * STY + (q >> 1);
      gid = sctl[10 + q] ? li : CGH_WS_LOAD(&pairs[sctl[2 + q] + li]);
      const int4 r = CGH_WS_LOAD(&rect[gid]);
      keep = r.x <= sx && sx <= r.z && r.y <= sy && sy <= r.w &&
             sx == max(r.x, 2 * STX) && sy == max(r.y, 2 * STY);
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    int wbase = 0;
    if (lane == 0 && bal) wbase = atomicAdd(&sctl[0], __popc(bal));
    wbase = __shfl_sync(0xffffffffu, wbase, 0);
    if (keep) {
      const int slot = wbase + __popc(bal & ((1u << lane) - 1u));
      const float4* g = rec + (size_t)gid * CGH_REC_F4;
#pragma unroll
      for (int k = 0; k < CGH_REC_F4; ++k) srec[slot * CGH_REC_F4 + k] = CGH_WS_LOAD(&g[k]);
      sgid[slot] = gid;
    }
    __syncthreads();
    const int nb = sctl[0];
    for (;;) {
      int j = 0;
      if (lane == 0) j = atomicAdd(&sctl[1], 1);
      j = __shfl_sync(0xffffffffu, j, 0);
      if (j >= nb) break;  // warp-uniform
      const float4 bb = srec[j * CGH_REC_F4 + 2];
      // pixel box of the Gaussian inside this region (region coordinates)
      const int x0 = (int)ceilf(fmaxf(bb.x, fox)) - ox;
      const int x1 = (int)floorf(fminf(bb.y, fox + (float)(kSuper - 1))) - ox;
      const int y0 = (int)ceilf(fmaxf(bb.z, foy)) - oy;
      const int y1 = (int)floorf(fminf(bb.w, foy + (float)(kSuper - 1))) - oy;
      if (x0 > x1 || y0 > y1) continue;  // warp-uniform
      const float4 r0 = srec[j * CGH_REC_F4 + 0];
      const float4 r1 = srec[j * CGH_REC_F4 + 1];
      const float4 r3 = srec[j * CGH_REC_F4 + 3];
      const float4 r4 = srec[j * CGH_REC_F4 + 4];
      const float Ac[4] = {r3.x, r3.z, r4.x, r4.z};
      const float Bc[4] = {r3.y, r3.w, r4.y, r4.w};
      // flattened box pixels: floor(k / bw) from one FP32 product with the correctly rounded
      // 1 / bw (bw <= 32: the box lies inside the region), exact here because k < 1024 and
      // the fractional part of (k + 1/2) / bw stays at least 1/64 away from an integer
      const int bw = x1 - x0 + 1, npx = bw * (y1 - y0 + 1);
      const float inv_bw = kInvWidth[bw];
      float acc[NVP];
#pragma unroll
      for (int v = 0; v < NVP; ++v) acc[v] = 0.f;
      for (int k = lane; k < npx; k += 32) {
        const int ry = (int)(((float)k + 0.5f) * inv_bw);
        const int lx_ = x0 + (k - ry * bw), ly_ = y0 + ry;
        const float dx = (float)(ox + lx_) - r0.x, dy = (float)(oy + ly_) - r0.y;
        const float p2 = gauss_power(r0, r1, dx, dy);
        if (p2 < r1.y) continue;
        const int pix = ly_ * kSuper + lx_;
        const float G = pow2_clamped(p2);
        const float aG = r1.z * G;
        const float a = fminf(kAlphaCap, aG);
        float S = 0.f;
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const float2 gv = sdu[c][pix];
          acc[c] = fmaf(a, gv.x, acc[c]);
          acc[C + c] = fmaf(a, gv.y, acc[C + c]);
          S = fmaf(Ac[c], gv.x, fmaf(Bc[c], gv.y, S));
        }
        if (aG < kAlphaCap) {
          acc[2 * C] = fmaf(S, G, acc[2 * C]);
          if (p2 > kP2Floor) {
            const float u = S * aG;
            const float udx = u * dx, udy = u * dy;
            acc[2 * C + 1] += udx;
            acc[2 * C + 2] += udy;
            acc[2 * C + 3] = fmaf(udx, dx, acc[2 * C + 3]);
            acc[2 * C + 4] = fmaf(udx, dy, acc[2 * C + 4]);
            acc[2 * C + 5] = fmaf(udy, dy, acc[2 * C + 5]);
          }
        }
      }
      int vidx = 0;
      if constexpr (NV == 12) {
        bool owner;
        reduce_scatter_12(acc, lane, vidx, owner);
        if (owner && acc[0] != 0.f) atomicAdd(&raw[(size_t)sgid[j] * CGH_RAW_STRIDE + vidx], acc[0]);
      } else {
        ReduceScatter<NVP, 16>::run(acc, lane, vidx);
        if ((lane & (32 / NVP - 1)) == 0 && vidx < NV && acc[0] != 0.f)
          atomicAdd(&raw[(size_t)sgid[j] * CGH_RAW_STRIDE + vidx], acc[0]);
      }
    }
  }
}

#ifndef CGH_ITEMS_ONLY
template <int C>
__global__ void __launch_bounds__(256) k_raster_bwd_region(RasterConsts rc,
                                                           const float4* __restrict__ rec,
                                                           const int4* __restrict__ rect,
                                                           const int* __restrict__ tile_start,
                                                           const int* __restrict__ pairs,
                                                           const float2* __restrict__ dU,
                                                           float* __restrict__ raw) {
  extern __shared__ __align__(16) unsigned char smem_rb[];
  float4* srec = reinterpret_cast<float4*>(smem_rb);
  int* sgid = reinterpret_cast<int*>(srec + 256 * CGH_REC_F4);
  float2(*sdu)[kSuper * kSuper] = reinterpret_cast<float2(*)[kSuper * kSuper]>(sgid + 256);
  int* sctl = reinterpret_cast<int*>(&sdu[C][0]);
  raster_bwd_region<C>(rc, rec, rect, tile_start, pairs, dU, raw, blockIdx.x, blockIdx.y, srec,
                       sgid, sdu, sctl);
}
#endif  // CGH_ITEMS_ONLY

// shared memory of k_raster_bwd_region<C>
__host__ __device__ constexpr size_t raster_bwd_region_smem(int C) {
  return sizeof(float4) * 256 * CGH_REC_F4 + sizeof(int) * 256 +
         sizeof(float2) * (size_t)C * kSuper * kSuper + sizeof(int) * kRegionCtl;
}

template <int C>
__device__ __forceinline__ void grad_finalize_one(const RasterConsts& rc, const cgh_params& p,
                                                  const float* __restrict__ raw,
                                                  const cgh_grads& g,
                                                  const float* __restrict__ grad_scale, int n) {
  const RawParams<C> q = load_params<C>(p, n);
  // every gradient is linear in the moments: the upstream scale is applied to them
  const float sc = grad_scale ? __ldg(grad_scale) : 1.f;
  float r[2 * C + 6];
#pragma unroll
  for (int k = 0; k < 2 * C + 6; ++k) r[k] = sc * CGH_WS_LOAD(&raw[(size_t)n * CGH_RAW_STRIDE + k]);
  if (!all_finite(q)) {
    g.xy_raw[2 * n] = 0.f; g.xy_raw[2 * n + 1] = 0.f; g.s_raw[2 * n] = 0.f;
    g.s_raw[2 * n + 1] = 0.f; g.theta[n] = 0.f; g.alpha_raw[n] = 0.f;
    for (int c = 0; c < C; ++c) { g.amp[n * C + c] = 0.f; g.phase[n * C + c] = 0.f; }
    return;
  }
  Act a = activate(q, rc.W, rc.H);
  // items 1, 2: amplitude and phase
#pragma unroll
  for (int c = 0; c < C; ++c) {
    float sp, cp;
    sincosf(q.ph[c], &sp, &cp);
    const float P = r[c], Q = r[C + c];
    g.amp[n * C + c] = cp * P + sp * Q;
    g.phase[n * C + c] = q.amp[c] * (cp * Q - sp * P);
  }
  // item 3: opacity through the sigmoid
  g.alpha_raw[n] = r[2 * C] * a.alpha * (1.f - a.alpha);
  // item 4: mean, dL/dx = inv . sum(u d), then tanh: W/2 (1 - tanh^2)
  const float Sx = r[2 * C + 1], Sy = r[2 * C + 2];
  const float dmx = a.i00 * Sx + a.i01 * Sy;
  const float dmy = a.i01 * Sx + a.i11 * Sy;
  g.xy_raw[2 * n + 0] = dmx * 0.5f * (float)rc.W * (1.f - a.tx * a.tx);
  g.xy_raw[2 * n + 1] = dmy * 0.5f * (float)rc.H * (1.f - a.ty * a.ty);
  // item 5: inverse covariance, dL/dinv = -1/2 sum u (dx^2, 2 dx dy, dy^2)
  const float d00 = -0.5f * r[2 * C + 3], d01 = -r[2 * C + 4], d11 = -0.5f * r[2 * C + 5];
  // inverse -> covariance: inv = (S11, -S01, S00) / D, D = S00 S11 - S01^2
  float dS00, dS01, dS11;
  const float A_ = a.S00, B_ = a.S01, C_ = a.S11;
  if (a.det > 1e-10f) {
    const float iD2 = 1.f / (a.det * a.det);
    dS00 = (-C_ * C_ * d00 + B_ * C_ * d01 - B_ * B_ * d11) * iD2;
    dS01 = (2.f * B_ * C_ * d00 - (A_ * C_ + B_ * B_) * d01 + 2.f * A_ * B_ * d11) * iD2;
    dS11 = (-B_ * B_ * d00 + A_ * B_ * d01 - A_ * A_ * d11) * iD2;
  } else {
    dS00 = d11 / 1e-10f;
    dS01 = -d01 / 1e-10f;
    dS11 = d00 / 1e-10f;
  }
  // items 6, 7: scales (then exp) and rotation
  const float cc = a.c * a.c, ss = a.s * a.s, cs = a.c * a.s;
  const float sx2 = a.sx * a.sx, sy2 = a.sy * a.sy;
  const float dsx = 2.f * a.sx * (cc * dS00 + cs * dS01 + ss * dS11);
  const float dsy = 2.f * a.sy * (ss * dS00 - cs * dS01 + cc * dS11);
  g.s_raw[2 * n + 0] = dsx * a.esx;
  g.s_raw[2 * n + 1] = dsy * a.esy;
  g.theta[n] = 2.f * (sy2 - sx2) * cs * dS00 + (sx2 - sy2) * (cc - ss) * dS01 +
               2.f * (sx2 - sy2) * cs * dS11;
}

#ifndef CGH_ITEMS_ONLY
template <int C>
__global__ void k_grad_finalize(RasterConsts rc, cgh_params p, const float* __restrict__ raw,
                                cgh_grads g, const float* __restrict__ grad_scale) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < rc.N) grad_finalize_one<C>(rc, p, raw, g, grad_scale, n);
}
#endif  // CGH_ITEMS_ONLY

}  // namespace cgh
