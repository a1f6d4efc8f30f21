// encoder.cu -- the learned initialiser's kernels: 3x3 convolutions with BF16 weights and
// activations and FP32 accumulation (forward, data gradient, weight/bias gradient), the
// FP32 -> BF16 cast, and the decode from the last layer's channels to Gaussian parameters.
//
// The paper has no learned part (it lists feed-forward prediction as future work, Sec. 6);
// the encoder follows the workload description: four stride-2 convolutions from a target
// intensity to 16 Gaussians per output cell.  The network is ~0.9 GMAC per 512x512 image, so
// these are direct convolutions on the FP32 pipes with the weight tile of a block of output
// (or input) channels staged in shared memory; every CTA of an output-channel block reuses it
// for 128 pixels.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "cgh_internal.h"

namespace {

constexpr int kPix = 128;  // pixels per CTA
constexpr int kCOT = 8;    // output channels per thread (forward)
constexpr int kCIT = 4;    // input channels per thread (data gradient)

__device__ __forceinline__ float ld(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// y[b][co][oy][ox] = bias[co] + sum_{ci,ky,kx} w[co][ci][ky][kx] x[b][ci][oy*s+ky-1][ox*s+kx-1]
template <bool OUT_F32>
__global__ void __launch_bounds__(kPix) k_conv_fwd(int CI, int Hi, int Wi, int CO, int Ho, int Wo,
                                                  int stride, int relu,
                                                  const __nv_bfloat16* __restrict__ x,
                                                  const __nv_bfloat16* __restrict__ w,
                                                  const float* __restrict__ bias, void* yv) {
  extern __shared__ float ws[];  // [CI * 9][kCOT]
  const int b = blockIdx.z, co0 = blockIdx.y * kCOT;
  for (int i = threadIdx.x; i < CI * 9 * kCOT; i += blockDim.x) {
    const int t = i % kCOT, ck = i / kCOT;  // ck = ci * 9 + k
    ws[i] = (co0 + t < CO) ? ld(&w[(size_t)(co0 + t) * CI * 9 + ck]) : 0.f;
  }
  __syncthreads();
  const int p = blockIdx.x * kPix + threadIdx.x;
  if (p >= Ho * Wo) return;
  const int oy = p / Wo, ox = p % Wo;
  float acc[kCOT];
#pragma unroll
  for (int t = 0; t < kCOT; ++t) acc[t] = (co0 + t < CO) ? bias[co0 + t] : 0.f;
  const __nv_bfloat16* xb = x + (size_t)b * CI * Hi * Wi;
  for (int ci = 0; ci < CI; ++ci) {
    float xv[9];
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int iy = oy * stride + ky - 1, ix = ox * stride + kx - 1;
        xv[ky * 3 + kx] = (iy >= 0 && iy < Hi && ix >= 0 && ix < Wi)
                              ? ld(&xb[((size_t)ci * Hi + iy) * Wi + ix]) : 0.f;
      }
    const float* wc = ws + ci * 9 * kCOT;
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
      for (int t = 0; t < kCOT; ++t) acc[t] = fmaf(wc[k * kCOT + t], xv[k], acc[t]);
  }
#pragma unroll
  for (int t = 0; t < kCOT; ++t) {
    if (co0 + t >= CO) break;
    float v = acc[t];
    if (relu) v = fmaxf(v, 0.f);
    const size_t o = (((size_t)b * CO + co0 + t) * Ho + oy) * Wo + ox;
    if (OUT_F32) static_cast<float*>(yv)[o] = v;
    else static_cast<__nv_bfloat16*>(yv)[o] = __float2bfloat16(v);
  }
}

// upstream gradient through the ReLU: dy * [y > 0] (y = the layer's forward output)
__device__ __forceinline__ float grad_through(const float* dy, const void* y, int y_f32,
                                              int relu, size_t o) {
  float g = dy[o];
  if (relu) {
    const float yv = y_f32 ? static_cast<const float*>(y)[o]
                           : __bfloat162float(static_cast<const __nv_bfloat16*>(y)[o]);
    if (!(yv > 0.f)) g = 0.f;
  }
  return g;
}

// dx[b][ci][iy][ix] = sum_{co, (ky,kx): iy = oy*s+ky-1, ix = ox*s+kx-1} w[co][ci][ky][kx] g[b][co][oy][ox]
__global__ void __launch_bounds__(kPix) k_conv_bwd_data(int CI, int Hi, int Wi, int CO, int Ho, int Wo,
                                                       int stride, int relu,
                                                       const __nv_bfloat16* __restrict__ w,
                                                       const void* y, int y_f32,
                                                       const float* __restrict__ dy,
                                                       float* __restrict__ dx) {
  extern __shared__ float ws[];  // [CO * 9][kCIT]
  const int b = blockIdx.z, ci0 = blockIdx.y * kCIT;
  for (int i = threadIdx.x; i < CO * 9 * kCIT; i += blockDim.x) {
    const int t = i % kCIT, ck = i / kCIT;  // ck = co * 9 + k
    const int co = ck / 9, k = ck % 9;
    ws[i] = (ci0 + t < CI) ? ld(&w[((size_t)co * CI + ci0 + t) * 9 + k]) : 0.f;
  }
  __syncthreads();
  const int p = blockIdx.x * kPix + threadIdx.x;
  if (p >= Hi * Wi) return;
  const int iy = p / Wi, ix = p % Wi;
  float acc[kCIT];
#pragma unroll
  for (int t = 0; t < kCIT; ++t) acc[t] = 0.f;
  for (int ky = 0; ky < 3; ++ky) {
    const int ty = iy + 1 - ky;
    if (ty < 0 || ty % stride) continue;
    const int oy = ty / stride;
    if (oy >= Ho) continue;
    for (int kx = 0; kx < 3; ++kx) {
      const int tx = ix + 1 - kx;
      if (tx < 0 || tx % stride) continue;
      const int ox = tx / stride;
      if (ox >= Wo) continue;
      const int k = ky * 3 + kx;
      for (int co = 0; co < CO; ++co) {
        const size_t o = (((size_t)b * CO + co) * Ho + oy) * Wo + ox;
        const float g = grad_through(dy, y, y_f32, relu, o);
        const float* wc = ws + (co * 9 + k) * kCIT;
#pragma unroll
        for (int t = 0; t < kCIT; ++t) acc[t] = fmaf(wc[t], g, acc[t]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < kCIT; ++t)
    if (ci0 + t < CI) dx[(((size_t)b * CI + ci0 + t) * Hi + iy) * Wi + ix] = acc[t];
}

// dw[co][ci][k] += sum over (b, oy, ox) in this CTA's slice of g x;  db[co] += sum g.
// One CTA per (slice, co, block of 4 input channels); warp shuffles then one atomic per value.
constexpr int kWCI = 4;
__global__ void __launch_bounds__(256) k_conv_bwd_weight(int B, int CI, int Hi, int Wi, int CO, int Ho,
                                                         int Wo, int stride, int relu,
                                                         const __nv_bfloat16* __restrict__ x,
                                                         const void* y, int y_f32,
                                                         const float* __restrict__ dy,
                                                         float* __restrict__ dw,
                                                         float* __restrict__ db, int slices) {
  const int co = blockIdx.y, ci0 = blockIdx.z * kWCI, slice = blockIdx.x;
  const long long P = (long long)B * Ho * Wo;
  const long long per = (P + slices - 1) / slices;
  const long long p0 = slice * per, p1 = min(P, p0 + per);
  float acc[kWCI][9];
  float gsum = 0.f;
#pragma unroll
  for (int c = 0; c < kWCI; ++c)
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[c][k] = 0.f;
  for (long long p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
    const int b = (int)(p / (Ho * Wo));
    const int r = (int)(p % (Ho * Wo));
    const int oy = r / Wo, ox = r % Wo;
    const size_t o = (((size_t)b * CO + co) * Ho + oy) * Wo + ox;
    const float g = grad_through(dy, y, y_f32, relu, o);
    if (g == 0.f) continue;
    gsum += g;
#pragma unroll
    for (int c = 0; c < kWCI; ++c) {
      if (ci0 + c >= CI) break;
      const __nv_bfloat16* xc = x + ((size_t)b * CI + ci0 + c) * Hi * Wi;
#pragma unroll
      for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const int iy = oy * stride + ky - 1, ix = ox * stride + kx - 1;
          if (iy >= 0 && iy < Hi && ix >= 0 && ix < Wi)
            acc[c][ky * 3 + kx] = fmaf(g, ld(&xc[(size_t)iy * Wi + ix]), acc[c][ky * 3 + kx]);
        }
    }
  }
  __shared__ float red[8][kWCI * 9 + 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < kWCI; ++c)
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float v = acc[c][k];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0) red[wid][c * 9 + k] = v;
    }
  for (int off = 16; off > 0; off >>= 1) gsum += __shfl_xor_sync(0xffffffffu, gsum, off);
  if (lane == 0) red[wid][kWCI * 9] = gsum;
  __syncthreads();
  if (threadIdx.x < kWCI * 9 + 1) {
    float v = 0.f;
    for (int w8 = 0; w8 < (int)(blockDim.x >> 5); ++w8) v += red[w8][threadIdx.x];
    if (threadIdx.x < kWCI * 9) {
      const int c = threadIdx.x / 9, k = threadIdx.x % 9;
      if (ci0 + c < CI && v != 0.f) atomicAdd(&dw[((size_t)co * CI + ci0 + c) * 9 + k], v);
    } else if (blockIdx.z == 0 && v != 0.f) {
      atomicAdd(&db[co], v);
    }
  }
}

__global__ void k_cast_bf16(long long n, const float* __restrict__ src,
                            __nv_bfloat16* __restrict__ dst) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16(src[i]);
}

// Decode: channel g*P + p of cell (cy, cx) -> parameter p of Gaussian n = (cy*CX + cx)*S + g.
// param = base + scale * out, with base = the slot's anchor for the two positions and fixed
// values otherwise (see cgh.h).  P = 6 + 2C: dx, dy, sx, sy, theta, amp[C], phase[C], alpha.
struct DecodeConsts {
  int CY, CX, S, C, H, W, side;
  float pos_scale, scale_scale, s_base, amp_base, amp_scale, alpha_base;
};

__device__ __forceinline__ float anchor_raw(float center, int extent) {
  // pre-activation of a mean at `center` pixels: atanh(2 center / extent - 1)
  const float u = fminf(fmaxf(2.f * center / (float)extent - 1.f, -0.999999f), 0.999999f);
  return atanhf(u);
}

__global__ void k_decode(DecodeConsts d, long long total, const float* __restrict__ out,
                         float* xy, float* s, float* th, float* amp, float* ph, float* al) {
  const int P = 6 + 2 * d.C;
  const int cells = d.CY * d.CX;
  const int N = cells * d.S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / ((long long)N * P));
    const int rem = (int)(i % ((long long)N * P));
    const int n = rem / P, p = rem % P;
    const int cell = n / d.S, g = n % d.S;
    const int cy = cell / d.CX, cx = cell % d.CX;
    const float o = out[(((size_t)b * d.S * P + g * P + p) * d.CY + cy) * d.CX + cx];
    const size_t gn = (size_t)b * N + n;
    const int side = d.side;  // slots form a side x side grid inside a cell
    const float cw = (float)d.W / d.CX, chh = (float)d.H / d.CY;
    if (p == 0) {
      const float c = (cx + ((g % side) + 0.5f) / side) * cw;
      xy[gn * 2 + 0] = anchor_raw(c, d.W) + d.pos_scale * o;
    } else if (p == 1) {
      const float c = (cy + ((g / side) + 0.5f) / side) * chh;
      xy[gn * 2 + 1] = anchor_raw(c, d.H) + d.pos_scale * o;
    } else if (p < 4) {
      s[gn * 2 + (p - 2)] = d.s_base + d.scale_scale * o;
    } else if (p == 4) {
      th[gn] = o;
    } else if (p < 5 + d.C) {
      amp[gn * d.C + (p - 5)] = d.amp_base + d.amp_scale * o;
    } else if (p < 5 + 2 * d.C) {
      ph[gn * d.C + (p - 5 - d.C)] = o;
    } else {
      al[gn] = d.alpha_base + o;
    }
  }
}

// d out = scale * d param (the adjoint of the affine decode)
__global__ void k_decode_bwd(DecodeConsts d, long long total, float* __restrict__ dout,
                             const float* gxy, const float* gs, const float* gth, const float* gamp,
                             const float* gph, const float* gal) {
  const int P = 6 + 2 * d.C;
  const int N = d.CY * d.CX * d.S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / ((long long)N * P));
    const int rem = (int)(i % ((long long)N * P));
    const int n = rem / P, p = rem % P;
    const int cell = n / d.S, g = n % d.S;
    const int cy = cell / d.CX, cx = cell % d.CX;
    const size_t gn = (size_t)b * N + n;
    float v;
    if (p < 2) v = d.pos_scale * gxy[gn * 2 + p];
    else if (p < 4) v = d.scale_scale * gs[gn * 2 + (p - 2)];
    else if (p == 4) v = gth[gn];
    else if (p < 5 + d.C) v = d.amp_scale * gamp[gn * d.C + (p - 5)];
    else if (p < 5 + 2 * d.C) v = gph[gn * d.C + (p - 5 - d.C)];
    else v = gal[gn];
    dout[(((size_t)b * d.S * P + g * P + p) * d.CY + cy) * d.CX + cx] = v;
  }
}

// grad (+)= 2 w (pred - target); *loss += w sum (pred - target)^2 (block sums, one atomic each)
__global__ void k_mse_grad(long long n, const float* __restrict__ pred,
                           const float* __restrict__ target, float w, int accumulate,
                           float* __restrict__ grad, float* __restrict__ loss) {
  float acc = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float d = pred[i] - target[i];
    grad[i] = (accumulate ? grad[i] : 0.f) + 2.f * w * d;
    acc = fmaf(d, d, acc);
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  __shared__ float red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0 && loss) {
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    atomicAdd(loss, w * t);
  }
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g > 152 * 16 ? 152 * 16 : (g < 1 ? 1 : g));
}

cgh_status cuda_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CGH_OK : cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
}

DecodeConsts decode_consts(int CY, int CX, int S, int C, int H, int W) {
  DecodeConsts d;
  d.CY = CY; d.CX = CX; d.S = S; d.C = C; d.H = H; d.W = W;
  d.side = 1;
  while (d.side * d.side < S) ++d.side;
  d.pos_scale = 0.02f;
  d.scale_scale = 0.5f;
  d.s_base = 0.4054651f;  // log(1.5)
  d.amp_base = 0.5f;
  d.amp_scale = 0.5f;
  d.alpha_base = -0.5f;
  return d;
}

}  // namespace

extern "C" cgh_status cgh_conv3x3_fwd(int32_t B, int32_t CI, int32_t Hi, int32_t Wi, int32_t CO,
                                      int32_t stride, const void* x, const void* w,
                                      const float* bias, int32_t relu, void* y, int32_t y_f32,
                                      void* stream) {
  if (B < 1 || CI < 1 || Hi < 1 || Wi < 1 || CO < 1 || stride < 1 || !x || !w || !bias || !y)
    return cgh_record_error(CGH_ERR_ARG, "cgh_conv3x3_fwd: bad argument");
  const int Ho = (Hi - 1) / stride + 1, Wo = (Wi - 1) / stride + 1;
  const size_t smem = sizeof(float) * (size_t)CI * 9 * kCOT;
  if (smem > 48 * 1024) return cgh_record_error(CGH_ERR_UNSUPPORTED_SIZE, "cgh_conv3x3_fwd: CI too large");
  dim3 grid((Ho * Wo + kPix - 1) / kPix, (CO + kCOT - 1) / kCOT, B);
  cudaStream_t s = (cudaStream_t)stream;
  prof_begin(KID_ENCODER, s);
  if (y_f32)
    k_conv_fwd<true><<<grid, kPix, smem, s>>>(CI, Hi, Wi, CO, Ho, Wo, stride, relu,
                                              (const __nv_bfloat16*)x, (const __nv_bfloat16*)w, bias, y);
  else
    k_conv_fwd<false><<<grid, kPix, smem, s>>>(CI, Hi, Wi, CO, Ho, Wo, stride, relu,
                                               (const __nv_bfloat16*)x, (const __nv_bfloat16*)w, bias, y);
  prof_end(KID_ENCODER, s);
  return cuda_status();
}

extern "C" cgh_status cgh_conv3x3_bwd(int32_t B, int32_t CI, int32_t Hi, int32_t Wi, int32_t CO,
                                      int32_t stride, const void* x, const void* w, int32_t relu,
                                      const void* y, int32_t y_f32, const float* dy, float* dx,
                                      float* dw, float* db, void* stream) {
  if (B < 1 || CI < 1 || Hi < 1 || Wi < 1 || CO < 1 || stride < 1 || !x || !w || !dy || !dw || !db ||
      (relu && !y))
    return cgh_record_error(CGH_ERR_ARG, "cgh_conv3x3_bwd: bad argument");
  const int Ho = (Hi - 1) / stride + 1, Wo = (Wi - 1) / stride + 1;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(dw, 0, sizeof(float) * (size_t)CO * CI * 9, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(db, 0, sizeof(float) * (size_t)CO, s);
  if (e != cudaSuccess) return cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
  prof_begin(KID_ENCODER, s);
  if (dx) {
    const size_t smem = sizeof(float) * (size_t)CO * 9 * kCIT;
    if (smem > 48 * 1024) return cgh_record_error(CGH_ERR_UNSUPPORTED_SIZE, "cgh_conv3x3_bwd: CO too large");
    dim3 grid((Hi * Wi + kPix - 1) / kPix, (CI + kCIT - 1) / kCIT, B);
    k_conv_bwd_data<<<grid, kPix, smem, s>>>(CI, Hi, Wi, CO, Ho, Wo, stride, relu,
                                             (const __nv_bfloat16*)w, y, y_f32, dy, dx);
  }
  const long long P = (long long)B * Ho * Wo;
  int slices = (int)((P + 4095) / 4096);
  if (slices > 256) slices = 256;
  dim3 gw(slices, CO, (CI + kWCI - 1) / kWCI);
  k_conv_bwd_weight<<<gw, 256, 0, s>>>(B, CI, Hi, Wi, CO, Ho, Wo, stride, relu,
                                       (const __nv_bfloat16*)x, y, y_f32, dy, dw, db, slices);
  prof_end(KID_ENCODER, s);
  return cuda_status();
}

extern "C" cgh_status cgh_cast_bf16(int64_t n, const float* src, void* dst, void* stream) {
  if (n < 0 || (n > 0 && (!src || !dst))) return cgh_record_error(CGH_ERR_ARG, "cgh_cast_bf16: bad argument");
  if (n == 0) return CGH_OK;
  cudaStream_t s = (cudaStream_t)stream;
  prof_begin(KID_ENCODER, s);
  k_cast_bf16<<<grid_for(n), 256, 0, s>>>(n, src, (__nv_bfloat16*)dst);
  prof_end(KID_ENCODER, s);
  return cuda_status();
}

extern "C" cgh_status cgh_encoder_decode(int32_t B, int32_t CY, int32_t CX, int32_t S, int32_t C,
                                         int32_t H, int32_t W, const float* out,
                                         const cgh_grads* params_out, void* stream) {
  if (B < 1 || CY < 1 || CX < 1 || S < 1 || C < 1 || C > CGH_MAX_C || !out || !params_out)
    return cgh_record_error(CGH_ERR_ARG, "cgh_encoder_decode: bad argument");
  const DecodeConsts d = decode_consts(CY, CX, S, C, H, W);
  const long long total = (long long)B * CY * CX * S * (6 + 2 * C);
  cudaStream_t s = (cudaStream_t)stream;
  prof_begin(KID_ENCODER, s);
  k_decode<<<grid_for(total), 256, 0, s>>>(d, total, out, params_out->xy_raw, params_out->s_raw,
                                           params_out->theta, params_out->amp, params_out->phase,
                                           params_out->alpha_raw);
  prof_end(KID_ENCODER, s);
  return cuda_status();
}

extern "C" cgh_status cgh_encoder_decode_bwd(int32_t B, int32_t CY, int32_t CX, int32_t S, int32_t C,
                                             int32_t H, int32_t W, const cgh_grads* param_grads,
                                             float* dout, void* stream) {
  if (B < 1 || CY < 1 || CX < 1 || S < 1 || C < 1 || C > CGH_MAX_C || !dout || !param_grads)
    return cgh_record_error(CGH_ERR_ARG, "cgh_encoder_decode_bwd: bad argument");
  const DecodeConsts d = decode_consts(CY, CX, S, C, H, W);
  const long long total = (long long)B * CY * CX * S * (6 + 2 * C);
  cudaStream_t s = (cudaStream_t)stream;
  prof_begin(KID_ENCODER, s);
  k_decode_bwd<<<grid_for(total), 256, 0, s>>>(d, total, dout, param_grads->xy_raw,
                                               param_grads->s_raw, param_grads->theta,
                                               param_grads->amp, param_grads->phase,
                                               param_grads->alpha_raw);
  prof_end(KID_ENCODER, s);
  return cuda_status();
}

extern "C" cgh_status cgh_mse_grad(int64_t n, const float* pred, const float* target, float weight,
                                   int32_t accumulate, float* grad, float* loss_accum,
                                   void* stream) {
  if (n < 0 || (n > 0 && (!pred || !target || !grad)))
    return cgh_record_error(CGH_ERR_ARG, "cgh_mse_grad: bad argument");
  if (n == 0) return CGH_OK;
  cudaStream_t s = (cudaStream_t)stream;
  prof_begin(KID_ENCODER, s);
  k_mse_grad<<<grid_for(n), 256, 0, s>>>(n, pred, target, weight, accumulate, grad, loss_accum);
  prof_end(KID_ENCODER, s);
  return cuda_status();
}
