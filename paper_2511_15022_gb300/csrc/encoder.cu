// encoder.cu -- the learned initialiser's entry points: 3x3 convolutions with BF16 weights
// and activations and FP32 accumulation (forward, data gradient, weight/bias gradient: the
// tensor-core kernels of conv_tc.cu), the FP32 -> BF16 cast, and the decode from the last
// layer's channels to Gaussian parameters and its adjoint.
//
// The paper has no learned part (it lists feed-forward prediction as future work, Sec. 6);
// the encoder follows the workload description: four stride-2 convolutions from a target
// intensity to 16 Gaussians per output cell.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "cgh_internal.h"

namespace {

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
  if (B < 1 || CI < 1 || Hi < 1 || Wi < 1 || CO < 1 || !x || !w || !bias || !y)
    return cgh_record_error(CGH_ERR_ARG, "cgh_conv3x3_fwd: bad argument");
  if (stride != 1 && stride != 2)
    return cgh_record_error(CGH_ERR_UNSUPPORTED_SIZE, "cgh_conv3x3_fwd: stride must be 1 or 2");
  const cudaError_t e = conv3x3_fwd_tc(B, CI, Hi, Wi, CO, stride, x, w, bias, relu, y, y_f32,
                                       (cudaStream_t)stream);
  return e == cudaSuccess ? CGH_OK : cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" cgh_status cgh_conv3x3_bwd(int32_t B, int32_t CI, int32_t Hi, int32_t Wi, int32_t CO,
                                      int32_t stride, const void* x, const void* w, int32_t relu,
                                      const void* y, int32_t y_f32, const float* dy, float* dx,
                                      float* dw, float* db, void* stream) {
  if (B < 1 || CI < 1 || Hi < 1 || Wi < 1 || CO < 1 || !x || !w || !dy || !dw || !db ||
      (relu && !y))
    return cgh_record_error(CGH_ERR_ARG, "cgh_conv3x3_bwd: bad argument");
  if (stride != 1 && stride != 2)
    return cgh_record_error(CGH_ERR_UNSUPPORTED_SIZE, "cgh_conv3x3_bwd: stride must be 1 or 2");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(dw, 0, sizeof(float) * (size_t)CO * CI * 9, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(db, 0, sizeof(float) * (size_t)CO, s);
  if (e == cudaSuccess && dx)
    e = conv3x3_dgrad_tc(B, CI, Hi, Wi, CO, stride, w, relu, y, y_f32, dy, dx, s);
  if (e == cudaSuccess)
    e = conv3x3_wgrad_tc(B, CI, Hi, Wi, CO, stride, x, relu, y, y_f32, dy, dw, db, s);
  return e == cudaSuccess ? CGH_OK : cgh_record_error(CGH_ERR_CUDA, cudaGetErrorString(e));
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
