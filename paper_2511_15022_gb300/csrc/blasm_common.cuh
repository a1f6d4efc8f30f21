// blasm_common.cuh -- device helpers shared by the generic and specialised BLASM passes.
#pragma once

#include <cuda_runtime.h>

#include "cgh_internal.h"
#include "fft.cuh"

namespace cgh {

__device__ __forceinline__ int signed_index(int k, int n) { return k < (n + 1) / 2 ? k : k - n; }

// H_{c,l}(s_x, s_y) * scale, Algorithm 3.  Phase k_z d / 2 pi is evaluated as
// frac(d / lambda) - (d/lambda) q / (1 + sqrt(1 - q)) with q = lambda^2 (f_x^2 + f_y^2)
// (the same value as (d / lambda) sqrt(1 - q); the large integer number of turns is removed
// on the host in FP64).  Evanescent bins inside the band get k_z = 0 (H = 1).
// Column-invariant part of H_{c,l}: everything that depends on s_x only.
struct TFCol {
  float qx2, ax2;  // qx sx^2, ax sx^2
  float ax_half;   // sx + 1/2 (aperture)
  bool in_band;    // |s_x| <= kx_max
};

__device__ __forceinline__ TFCol tf_col(const TFConst& t, int sx) {
  const float fx2 = (float)(sx * sx);
  return {t.qx * fx2, t.ax * fx2, (float)sx + 0.5f, abs(sx) <= t.kx_max};
}

// H_{c,l}(s_x, s_y) * scale from the column part (same formula as transfer() below).
__device__ __forceinline__ float2 transfer_col(const BlasmDev& bl, const TFConst& t,
                                               const TFCol& col, int sy, float scale) {
  if (!col.in_band || abs(sy) > t.ky_max) return make_float2(0.f, 0.f);
  if (bl.aperture2 > 0.f) {
    const float ay = (float)sy + 0.5f;
    if (col.ax_half * col.ax_half + ay * ay >= bl.aperture2) return make_float2(0.f, 0.f);
  }
  const float fy2 = (float)(sy * sy);
  const float q = fmaf(t.qy, fy2, col.qx2);
  float turns = 0.f;
  if (q < 1.f) {
    const float num = fmaf(t.ay, fy2, col.ax2);
    float g;
    if (q < 0.05f) {
      g = fmaf(q, 0.01611328125f, 0.0205078125f);
      g = fmaf(q, g, 0.02734375f);
      g = fmaf(q, g, 0.0390625f);
      g = fmaf(q, g, 0.0625f);
      g = fmaf(q, g, 0.125f);
      g = fmaf(q, g, 0.5f);
    } else {
      g = 1.f / (1.f + sqrtf(1.f - q));
    }
    turns = fmaf(-num, g, t.turns0);
    turns -= rintf(turns);
  }
  float s, c;
  __sincosf(6.28318530717958647692f * turns, &s, &c);
  return make_float2(c * scale, s * scale);
}

// Branch-free H_{c,l} * scale for plans where every bin has q < 0.04 (bl.series_ok, checked
// on the host): the series for 1 - sqrt(1 - q) applies everywhere, no bin is evanescent,
// and the band and aperture masks become a select on the scale.  The series for g stops at
// q^4: the omitted terms are below 21/1024 q^5 < 2.1e-9 relative at q < 0.04, i.e. under
// 1e-5 turns even for num = (d / lambda) q of 1e4 turns, where the FP32 product num * g is
// itself only good to ~5e-4 turns.
__device__ __forceinline__ float2 transfer_series(const BlasmDev& bl, const TFConst& t,
                                                  const TFCol& col, int sy, float scale) {
  const float fy2 = (float)(sy * sy);
  const float ay = (float)sy + 0.5f;
  const bool keep = col.in_band && abs(sy) <= t.ky_max &&
                    !(bl.aperture2 > 0.f && fmaf(col.ax_half, col.ax_half, ay * ay) >= bl.aperture2);
  const float q = fmaf(t.qy, fy2, col.qx2);
  const float num = fmaf(t.ay, fy2, col.ax2);
  float g = fmaf(q, 0.02734375f, 0.0390625f);  // series through q^4 (see below)
  g = fmaf(q, g, 0.0625f);
  g = fmaf(q, g, 0.125f);
  g = fmaf(q, g, 0.5f);
  float turns = fmaf(-num, g, t.turns0);
  turns -= rintf(turns);
  float s, c;
  __sincosf(6.28318530717958647692f * turns, &s, &c);
  const float sc = keep ? scale : 0.f;
  return make_float2(c * sc, s * sc);
}

// The same H_{c,l} (scale 1) where the caller knows the bin lies inside the band and there
// is no aperture: phase polynomial and one sine/cosine, nothing else.
__device__ __forceinline__ float2 transfer_inband(const TFConst& t, const TFCol& col, int sy) {
  const float fy2 = (float)(sy * sy);
  const float q = fmaf(t.qy, fy2, col.qx2);
  const float num = fmaf(t.ay, fy2, col.ax2);
  float g = fmaf(q, 0.02734375f, 0.0390625f);  // series through q^4 (see below)
  g = fmaf(q, g, 0.0625f);
  g = fmaf(q, g, 0.125f);
  g = fmaf(q, g, 0.5f);
  float turns = fmaf(-num, g, t.turns0);
  turns -= rintf(turns);
  float s, c;
  __sincosf(6.28318530717958647692f * turns, &s, &c);
  return make_float2(c, s);
}

__device__ __forceinline__ float2 transfer(const BlasmDev& bl, int cl, int sx, int sy,
                                           float scale) {
  const TFConst& t = bl.tf[cl];
  if (abs(sx) > t.kx_max || abs(sy) > t.ky_max) return make_float2(0.f, 0.f);
  if (bl.aperture2 > 0.f) {
    const float ax = (float)sx + 0.5f, ay = (float)sy + 0.5f;
    if (ax * ax + ay * ay >= bl.aperture2) return make_float2(0.f, 0.f);
  }
  const float fx2 = (float)(sx * sx), fy2 = (float)(sy * sy);
  const float q = fmaf(t.qx, fx2, t.qy * fy2);
  float turns = 0.f;
  if (q < 1.f) {
    // (d/lambda) (1 - sqrt(1 - q)) = num * g(q), num = (d/lambda) q.  For q < 0.05 g is the
    // binomial series of (1 - sqrt(1 - q)) / q, truncated after q^6 (remainder < 3e-10
    // relative); otherwise the closed form 1 / (1 + sqrt(1 - q)).
    const float num = fmaf(t.ax, fx2, t.ay * fy2);
    float g;
    if (q < 0.05f) {
      g = fmaf(q, 0.01611328125f, 0.0205078125f);  // 33/2048, 21/1024
      g = fmaf(q, g, 0.02734375f);                  // 7/256
      g = fmaf(q, g, 0.0390625f);                   // 5/128
      g = fmaf(q, g, 0.0625f);                      // 1/16
      g = fmaf(q, g, 0.125f);                       // 1/8
      g = fmaf(q, g, 0.5f);                         // 1/2
    } else {
      g = 1.f / (1.f + sqrtf(1.f - q));
    }
    turns = fmaf(-num, g, t.turns0);
    turns -= rintf(turns);
  }
  // |turns| <= 1/2 after the exact reduction above: the hardware sine/cosine on
  // [-pi, pi] is accurate to ~4e-7 absolute, far inside the field tolerance
  float s, c;
  __sincosf(6.28318530717958647692f * turns, &s, &c);
  return make_float2(c * scale, s * scale);
}


__device__ __forceinline__ float block_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

// Loss finalisation by the last CTA of a pass of `ncta` CTAs: each CTA has written its
// partial (thread 0) before calling; the CTA that draws the last ticket sums all `count`
// partials (the pass's own and any written by earlier kernels after them) in FP64 in index
// order (the result does not depend on which CTA is last), writes sum * inv_norm to out[0]
// and resets the ticket for the next launch.
__device__ __forceinline__ void finalize_if_last(const float* partials, int ncta, int count,
                                                 double inv_norm, float* out, int* ticket) {
  __shared__ int s_last;
  __shared__ double s_red[32];
  if (threadIdx.x == 0) {
    __threadfence();  // this CTA's partial is visible before its ticket is
    s_last = atomicAdd(ticket, 1) == ncta - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += (double)__ldcg(&partials[i]);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) s_red[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
    out[0] = (float)(t * inv_norm);
    *ticket = 0;
  }
}

}  // namespace cgh
