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
    const float den = 1.f + sqrtf(1.f - q);
    const float num = fmaf(t.ax, fx2, t.ay * fy2);
    turns = t.turns0 - num / den;
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

}  // namespace cgh
