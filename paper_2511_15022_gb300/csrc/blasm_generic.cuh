// blasm_generic.cuh -- device code of the generic (runtime-length) BLASM passes described in
// blasm.cu: per-item functions and the kernels that run one item per CTA.  Included by
// blasm.cu (the planned launches) and persist.cu (the persistent batched step).
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "cgh_internal.h"
#include "fft.cuh"
#include "blasm_common.cuh"

// Loads of the fields and half grids the passes exchange through global memory: plain loads
// in the planned kernels; a kernel that writes and reads them in one launch (the persistent
// step) defines CGH_FIELD_LOAD as an L2 load before including this file.
#ifndef CGH_FIELD_LOAD
#define CGH_FIELD_LOAD(p) (*(p))
#endif

namespace cgh {

// Item functions of the generic passes: one (row block, batch) or (column block, channel)
// per CTA, shared memory `sm` as the launchers size it.  The kernels below run one item per
// CTA; the persistent batched step (persist.cu) calls the same functions.
template <int MAXB>
__device__ __forceinline__ void rows_pad_fwd_item(const BlasmDev& bl, const FFTDesc& fx, int RB,
                                                  int CB, int bs, int batch, int y0,
                                                  const float2* __restrict__ in,
                                                  float2* __restrict__ half, float2* sm) {
  const int rows = min(RB, bl.H - y0);
  const int Nx = bl.Nx, W = bl.W, H = bl.H;
  const float2* src = in + (size_t)batch * H * W;
  for (int idx = threadIdx.x; idx < rows * Nx; idx += blockDim.x) {
    const int b = idx / Nx, k = idx - b * Nx;
    const int x = k - bl.ox;
    float2 v = make_float2(0.f, 0.f);
    if (x >= 0 && x < W) v = CGH_FIELD_LOAD(&src[(size_t)(y0 + b) * W + x]);
    sm[b * bs + sidx(k)] = v;
  }
  __syncthreads();
  block_fft<false, MAXB>(sm, bs, rows, fx);
  float2* dst = half + (size_t)batch * H * Nx;
  for (int idx = threadIdx.x; idx < rows * Nx; idx += blockDim.x) {
    const int kk = idx % CB, rest = idx / CB;
    const int b = rest % rows, kb = rest / rows;
    dst[((size_t)kb * H + y0 + b) * CB + kk] = sm[b * bs + sidx(kb * CB + kk)];
  }
}

#ifndef CGH_ITEMS_ONLY
template <int MAXB>
__global__ void __launch_bounds__(512, 1) k_rows_pad_fwd(const __grid_constant__ BlasmDev bl,
                                                       const FFTDesc fx, int RB, int CB, int bs,
                                                       const float2* __restrict__ in,
                                                       float2* __restrict__ half) {
  extern __shared__ float2 sm[];
  rows_pad_fwd_item<MAXB>(bl, fx, RB, CB, bs, blockIdx.y, blockIdx.x * RB, in, half, sm);
}
#endif  // CGH_ITEMS_ONLY

template <int MAXB>
__device__ __forceinline__ void cols_fwd_planes_item(const BlasmDev& bl, const FFTDesc& fy,
                                                     int CB, int bs, int c, int kb,
                                                     const float2* __restrict__ Y,
                                                     float2* __restrict__ V, float2* sm) {
  float2* S = sm;
  float2* Wk = sm + CB * bs;
  const int H = bl.H, Ny = bl.Ny, Nx = bl.Nx, C = bl.C, oy = bl.oy;
  const float2* src = Y + (size_t)c * H * Nx + (size_t)kb * H * CB;
  for (int idx = threadIdx.x; idx < CB * Ny; idx += blockDim.x) {
    const int b = idx % CB, i = idx / CB;
    const int y = i - oy;
    S[b * bs + sidx(i)] = (y >= 0 && y < H) ? CGH_FIELD_LOAD(&src[(size_t)y * CB + b]) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  block_fft<false, MAXB>(S, bs, CB, fy);
  for (int l = 0; l < bl.L; ++l) {
    const int cl = c * bl.Ltot + bl.plane[l];
    for (int idx = threadIdx.x; idx < CB * Ny; idx += blockDim.x) {
      const int b = idx / Ny, i = idx - b * Ny;
      const int sx = signed_index(kb * CB + b, Nx), sy = signed_index(i, Ny);
      const int a = b * bs + sidx(i);
      Wk[a] = cmul(S[a], transfer(bl, cl, sx, sy, bl.inv_ntot));
    }
    __syncthreads();
    block_fft<true, MAXB>(Wk, bs, CB, fy);
    float2* dst = V + (size_t)(l * C + c) * H * Nx + (size_t)kb * H * CB;
    for (int idx = threadIdx.x; idx < CB * H; idx += blockDim.x) {
      const int b = idx % CB, y = idx / CB;
      dst[(size_t)y * CB + b] = Wk[b * bs + sidx(oy + y)];
    }
    __syncthreads();
  }
}

#ifndef CGH_ITEMS_ONLY
template <int MAXB>
__global__ void __launch_bounds__(512, 1) k_cols_fwd_planes(const __grid_constant__ BlasmDev bl,
                                                          const FFTDesc fy, int CB, int bs,
                                                          const float2* __restrict__ Y,
                                                          float2* __restrict__ V) {
  extern __shared__ float2 sm[];
  cols_fwd_planes_item<MAXB>(bl, fy, CB, bs, blockIdx.y, blockIdx.x, Y, V, sm);
}
#endif  // CGH_ITEMS_ONLY

template <int MAXB>
__device__ __forceinline__ void rows_inv_crop_item(const BlasmDev& bl, const FFTDesc& fx, int RB,
                                                   int CB, int bs, int batch, int y0,
                                                   const float2* __restrict__ half,
                                                   float2* __restrict__ out, int accum,
                                                   float2* sm) {
  const int rows = min(RB, bl.H - y0);
  const int Nx = bl.Nx, W = bl.W, H = bl.H;
  const float2* src = half + (size_t)batch * H * Nx;
  for (int idx = threadIdx.x; idx < rows * Nx; idx += blockDim.x) {
    const int kk = idx % CB, rest = idx / CB;
    const int b = rest % rows, kb = rest / rows;
    sm[b * bs + sidx(kb * CB + kk)] = CGH_FIELD_LOAD(&src[((size_t)kb * H + y0 + b) * CB + kk]);
  }
  __syncthreads();
  block_fft<true, MAXB>(sm, bs, rows, fx);
  float2* dst = out + (size_t)batch * H * W;
  for (int idx = threadIdx.x; idx < rows * W; idx += blockDim.x) {
    const int b = idx / W, x = idx - b * W;
    const float2 v = sm[b * bs + sidx(bl.ox + x)];
    float2* o = &dst[(size_t)(y0 + b) * W + x];
    *o = accum ? cadd(CGH_FIELD_LOAD(o), v) : v;
  }
}

#ifndef CGH_ITEMS_ONLY
template <int MAXB>
__global__ void __launch_bounds__(512, 1) k_rows_inv_crop(const __grid_constant__ BlasmDev bl,
                                                        const FFTDesc fx, int RB, int CB, int bs,
                                                        const float2* __restrict__ half,
                                                        float2* __restrict__ out, int accum) {
  extern __shared__ float2 sm[];
  rows_inv_crop_item<MAXB>(bl, fx, RB, CB, bs, blockIdx.y, blockIdx.x * RB, half, out, accum, sm);
}
#endif  // CGH_ITEMS_ONLY

// partial_index: where this item's loss partial goes; red: 32 floats of shared memory
template <int MAXB>
__device__ __forceinline__ void rows_loss_item(const BlasmDev& bl, const FFTDesc& fx, int RB,
                                               int CB, int bs, int batch, int y0,
                                               float2* __restrict__ V,
                                               const float* __restrict__ target,
                                               float* __restrict__ partials, int partial_index,
                                               int want_grad, float2* sm, float* red) {
  const int plane = bl.plane[batch / bl.C];  // the hologram plane: target, mask
  const int rows = min(RB, bl.H - y0);
  const int Nx = bl.Nx, W = bl.W, H = bl.H;
  float2* half = V + (size_t)batch * H * Nx;
  for (int idx = threadIdx.x; idx < rows * Nx; idx += blockDim.x) {
    const int kk = idx % CB, rest = idx / CB;
    const int b = rest % rows, kb = rest / rows;
    sm[b * bs + sidx(kb * CB + kk)] = CGH_FIELD_LOAD(&half[((size_t)kb * H + y0 + b) * CB + kk]);
  }
  __syncthreads();
  block_fft<true, MAXB>(sm, bs, rows, fx);
  const float gscale = 4.0f / ((float)bl.Ltot * (float)bl.C * (float)H * (float)W);
  const float* tg = target + ((size_t)plane * bl.C + batch % bl.C) * H * W;
  float acc = 0.f;
  for (int idx = threadIdx.x; idx < rows * Nx; idx += blockDim.x) {
    const int b = idx / Nx, k = idx - b * Nx;
    const int x = k - bl.ox;
    const int a = b * bs + sidx(k);
    float2 g = make_float2(0.f, 0.f);
    if (x >= 0 && x < W) {
      const float2 u = sm[a];
      const float I = fmaf(u.x, u.x, u.y * u.y);
      const float t = tg[(size_t)(y0 + b) * W + x];
      const float d = I - t;
      const float wd = loss_weight(bl, plane, y0 + b, x, t) * d;
      acc = fmaf(wd, d, acc);
      g = cscale(u, gscale * wd);
    }
    sm[a] = g;
  }
  const float tot = block_sum(acc, red);
  if (threadIdx.x == 0) partials[partial_index] = tot;
  if (!want_grad) return;
  __syncthreads();
  block_fft<false, MAXB>(sm, bs, rows, fx);
  for (int idx = threadIdx.x; idx < rows * Nx; idx += blockDim.x) {
    const int kk = idx % CB, rest = idx / CB;
    const int b = rest % rows, kb = rest / rows;
    half[((size_t)kb * H + y0 + b) * CB + kk] = sm[b * bs + sidx(kb * CB + kk)];
  }
}

#ifndef CGH_ITEMS_ONLY
template <int MAXB>
__global__ void __launch_bounds__(512, 1) k_rows_loss(const __grid_constant__ BlasmDev bl,
                                                    const FFTDesc fx, int RB, int CB, int bs,
                                                    float2* __restrict__ V,
                                                    const float* __restrict__ target,
                                                    float* __restrict__ partials, int want_grad) {
  extern __shared__ float2 sm[];
  __shared__ float red[32];
  rows_loss_item<MAXB>(bl, fx, RB, CB, bs, blockIdx.y, blockIdx.x * RB, V, target, partials,
                       blockIdx.y * gridDim.x + blockIdx.x, want_grad, sm, red);
}
#endif  // CGH_ITEMS_ONLY

template <int MAXB>
__device__ __forceinline__ void cols_bwd_planes_item(const BlasmDev& bl, const FFTDesc& fy,
                                                     int CB, int bs, int c, int kb,
                                                     const float2* __restrict__ G,
                                                     float2* __restrict__ D, float2* sm) {
  float2* S = sm;
  float2* Wk = sm + CB * bs;
  const int H = bl.H, Ny = bl.Ny, Nx = bl.Nx, C = bl.C, oy = bl.oy;
  for (int l = 0; l < bl.L; ++l) {
    const float2* src = G + (size_t)(l * C + c) * H * Nx + (size_t)kb * H * CB;
    for (int idx = threadIdx.x; idx < CB * Ny; idx += blockDim.x) {
      const int b = idx % CB, i = idx / CB;
      const int y = i - oy;
      Wk[b * bs + sidx(i)] = (y >= 0 && y < H) ? CGH_FIELD_LOAD(&src[(size_t)y * CB + b]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    block_fft<false, MAXB>(Wk, bs, CB, fy);
    const int cl = c * bl.Ltot + bl.plane[l];
    for (int idx = threadIdx.x; idx < CB * Ny; idx += blockDim.x) {
      const int b = idx / Ny, i = idx - b * Ny;
      const int sx = signed_index(kb * CB + b, Nx), sy = signed_index(i, Ny);
      const int a = b * bs + sidx(i);
      const float2 t = cmulc(Wk[a], transfer(bl, cl, sx, sy, bl.inv_ntot));
      S[a] = (l == 0) ? t : cadd(S[a], t);
    }
    __syncthreads();
  }
  block_fft<true, MAXB>(S, bs, CB, fy);
  float2* dst = D + (size_t)c * H * Nx + (size_t)kb * H * CB;
  for (int idx = threadIdx.x; idx < CB * H; idx += blockDim.x) {
    const int b = idx % CB, y = idx / CB;
    dst[(size_t)y * CB + b] = S[b * bs + sidx(oy + y)];
  }
}

#ifndef CGH_ITEMS_ONLY
template <int MAXB>
__global__ void __launch_bounds__(512, 1) k_cols_bwd_planes(const __grid_constant__ BlasmDev bl,
                                                          const FFTDesc fy, int CB, int bs,
                                                          const float2* __restrict__ G,
                                                          float2* __restrict__ D) {
  extern __shared__ float2 sm[];
  cols_bwd_planes_item<MAXB>(bl, fy, CB, bs, blockIdx.y, blockIdx.x, G, D, sm);
}
#endif  // CGH_ITEMS_ONLY

// Unfused intensity loss for the standalone API: partials per block, optional gradient.
#ifndef CGH_ITEMS_ONLY
__global__ void k_loss_pointwise(const __grid_constant__ BlasmDev bl, long long total,
                                 float gscale, const float2* __restrict__ Ud,
                                 const float* __restrict__ target, float* __restrict__ partials,
                                 float2* __restrict__ dUd) {
  __shared__ float red[32];
  float acc = 0.f;
  const long long HW = (long long)bl.H * bl.W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 u = Ud[i];
    const float t = target[i];
    const float d = fmaf(u.x, u.x, u.y * u.y) - t;
    const long long lc = i / HW, r = i - lc * HW;  // i = ((l C + c) H + y) W + x
    const float wd = loss_weight(bl, (int)(lc / bl.C), (int)(r / bl.W), (int)(r % bl.W), t) * d;
    acc = fmaf(wd, d, acc);
    if (dUd) dUd[i] = cscale(u, gscale * wd);
  }
  const float tot = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}
#endif  // CGH_ITEMS_ONLY

// Loss and gradient seed of the planes whose propagation is the identity (distance 0, no
// aperture, every bin inside the band: H = 1 in Algorithm 3, so U(d_l) = U(0)), taken on
// U(0) itself, as one work item of the persistent batched step (the planned step takes it in
// the forward raster's epilogue instead).  One CTA per image row y and channel c; per pixel,
// for each such plane l, d = |U|^2 - T_l: the loss partial gains w_l d^2 and the seed
// sum_l gscale w_l d U (the seed the loss row pass forms, Sec. 3.2) replaces U when
// want_grad (each element read and written by one thread).  Each thread loads its kIdentU
// elements of a row before using any (a 1920-pixel row is one round), so enough loads are
// in flight to cover the memory latency.
constexpr int kIdentU = 8;
__device__ __forceinline__ void ident_loss_item(const BlasmDev& bl, unsigned mask, float gscale,
                                                float2* __restrict__ U,
                                                const float* __restrict__ target,
                                                float* __restrict__ partials, int partial_index,
                                                int want_grad, int y, int c, float* red) {
  const int W = bl.W;
  const size_t HW = (size_t)bl.H * W, row = (size_t)c * HW + (size_t)y * W;
  float2* u_row = U + row;
  float acc = 0.f;
  for (int x0 = 0; x0 < W; x0 += kIdentU * 256) {
    float2 u[kIdentU];
    float gs[kIdentU];
#pragma unroll
    for (int k = 0; k < kIdentU; ++k) {
      const int x = x0 + k * 256 + threadIdx.x;
      u[k] = x < W ? CGH_FIELD_LOAD(&u_row[x]) : make_float2(0.f, 0.f);
      gs[k] = 0.f;
    }
    for (int l = 0; l < bl.Ltot; ++l) {
      if (!((mask >> l) & 1u)) continue;
      const float* t_row = target + (size_t)l * bl.C * HW + row;
      float t[kIdentU];
#pragma unroll
      for (int k = 0; k < kIdentU; ++k) {
        const int x = x0 + k * 256 + threadIdx.x;
        t[k] = x < W ? __ldg(&t_row[x]) : 0.f;
      }
#pragma unroll
      for (int k = 0; k < kIdentU; ++k) {
        const int x = x0 + k * 256 + threadIdx.x;
        if (x >= W) continue;
        const float d = fmaf(u[k].x, u[k].x, u[k].y * u[k].y) - t[k];
        const float wd = loss_weight(bl, l, y, x, t[k]) * d;
        acc = fmaf(wd, d, acc);
        gs[k] += wd;
      }
    }
    if (want_grad) {
#pragma unroll
      for (int k = 0; k < kIdentU; ++k) {
        const int x = x0 + k * 256 + threadIdx.x;
        if (x < W) u_row[x] = cscale(u[k], gscale * gs[k]);
      }
    }
  }
  const float tot = block_sum(acc, red);
  if (threadIdx.x == 0) partials[partial_index] = tot;
}

// Intensity of a complex field (Sec. 3.2: I = |U|^2), element-wise over `total` values.
#ifndef CGH_ITEMS_ONLY
__global__ void k_intensity(long long total, const float2* __restrict__ U, float* __restrict__ I) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 u = __ldg(&U[i]);
    I[i] = fmaf(u.x, u.x, u.y * u.y);
  }
}
#endif  // CGH_ITEMS_ONLY

// Its adjoint: with dL/dI given, dL/dRe + j dL/dIm = 2 dL/dI (Re U + j Im U).
#ifndef CGH_ITEMS_ONLY
__global__ void k_intensity_bwd(long long total, const float2* __restrict__ U,
                                const float* __restrict__ dI, float2* __restrict__ dU) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 u = __ldg(&U[i]);
    const float g = 2.0f * __ldg(&dI[i]);
    dU[i] = make_float2(g * u.x, g * u.y);
  }
}
#endif  // CGH_ITEMS_ONLY

// loss = sum(partials) / (L C H W), summed in FP64 in a fixed order.
#ifndef CGH_ITEMS_ONLY
__global__ void k_loss_finalize(const float* __restrict__ partials, int count, double inv_norm,
                                float* __restrict__ out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += (double)partials[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[0] = (float)(t * inv_norm);
  }
}
#endif  // CGH_ITEMS_ONLY

}  // namespace cgh
