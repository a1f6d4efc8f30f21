// poh.cu -- phase-only hologram (POH) conversion of Sec. 3.3.
//
//   * smooth POH by double-phase amplitude coding (the method the paper cites):
//     phi_DPAC = arg H +- acos(|H| / max|H|) on the two colours of the (i + j) checkerboard,
//     H_smooth = exp(j phi_DPAC); the formula as printed (|H| where i + j is even, arg H
//     where odd) is mode 0;
//   * random POH: a learnable phase field phi [C][H][W], H_rand = exp(j phi), propagated
//     beside the Gaussians' field H, with the joint objective
//       L_extract = sum_l [ R_l(I_l) + R_l(I_rand,l) + lambda_comp mean (I_l - I_rand,l)^2
//                           + lambda_field mean (|Re(U_l - U_rand,l)| + |Im(U_l - U_rand,l)|) ]
//     where R_l = mean over the plane of (I - T)^2 (1 + M + T^2) is plane l's part of
//     L_recon (binary depth masks M of the plan, or M = 0) and every mean runs over the
//     C H W values of one plane.
// cgh_poh_step runs the joint forward + backward pass with the library's raster and BLASM
// kernels; the elementwise pieces (the phase field, L_extract and its two gradients, the
// phase gradient) are the kernels here.
#include <cuda_runtime.h>

#include "cgh_internal.h"

namespace {

__device__ __forceinline__ float sgnf(float v) { return (float)((v > 0.f) - (v < 0.f)); }

// per-channel max |U| (non-negative floats order like their bit patterns)
__global__ void k_chan_absmax(long long per_channel, const float2* __restrict__ U,
                              unsigned int* __restrict__ amax_bits) {
  const int c = blockIdx.y;
  const float2* src = U + (size_t)c * per_channel;
  float m = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per_channel;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 u = src[i];
    m = fmaxf(m, sqrtf(fmaf(u.x, u.x, u.y * u.y)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(&amax_bits[c], __float_as_uint(m));
}

// mode 1 (double-phase amplitude coding): phi +- acos(|U| / max|U|) on the two checkerboard
// colours; mode 0 (as printed): |U| on even i + j, arg U on odd.
__global__ void k_poh_dpac(long long total, int C, int H, int W, int mode,
                           const unsigned int* __restrict__ amax_bits,
                           const float2* __restrict__ U, float2* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % W), y = (int)((i / W) % H), c = (int)(i / ((long long)H * W));
    const float2 u = U[i];
    const float A = sqrtf(fmaf(u.x, u.x, u.y * u.y)), ph = atan2f(u.y, u.x);
    const bool even = ((x + y) & 1) == 0;
    float pd;
    if (mode == 0) {
      pd = even ? A : ph;
    } else {
      const float amax = __uint_as_float(amax_bits[c]);
      const float a = acosf(fminf(amax > 0.f ? A / amax : 0.f, 1.f));
      pd = even ? ph + a : ph - a;
    }
    float s, co;
    sincosf(pd, &s, &co);
    out[i] = make_float2(co, s);
  }
}

__global__ void k_poh_field(long long total, const float* __restrict__ phi,
                            float2* __restrict__ Hr) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    float s, c;
    sincosf(phi[i], &s, &c);
    Hr[i] = make_float2(c, s);
  }
}

// dL/dphi = -sin(phi) dRe + cos(phi) dIm for H_rand = exp(j phi)
__global__ void k_poh_phase_grad(long long total, const float* __restrict__ phi,
                                 const float2* __restrict__ dH, float* __restrict__ dphi) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    float s, c;
    sincosf(phi[i], &s, &c);
    const float2 g = dH[i];
    dphi[i] = fmaf(-s, g.x, c * g.y);
  }
}

// Per element of the L planes: loss partials of L_extract (times n = C H W) and the two
// gradients, written in place over Ud and Ur.
__global__ void k_extract_loss(const __grid_constant__ BlasmDev bl, long long total, float inv_n,
                               float lambda_comp, float lambda_field, float2* __restrict__ Ud,
                               float2* __restrict__ Ur, const float* __restrict__ target,
                               float* __restrict__ partials) {
  __shared__ float red[32];
  float acc = 0.f;
  const long long HW = (long long)bl.H * bl.W;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 u = Ud[i], r = Ur[i];
    const float t = target[i];
    const long long lc = i / HW, pix = i - lc * HW;
    const int l = (int)(lc / bl.C), y = (int)(pix / bl.W), x = (int)(pix % bl.W);
    const float m = bl.recon_mask ? (bl.recon_mask[((size_t)l * bl.H + y) * bl.W + x] ? 1.f : 0.f) : 0.f;
    const float w = 1.f + m + t * t;
    const float I = fmaf(u.x, u.x, u.y * u.y), Ir = fmaf(r.x, r.x, r.y * r.y);
    const float e = I - t, er = Ir - t, dI = I - Ir;
    const float dx = u.x - r.x, dy = u.y - r.y;
    acc += w * (e * e + er * er) + lambda_comp * dI * dI + lambda_field * (fabsf(dx) + fabsf(dy));
    // dL/dI and dL/dI_rand (times n), then through I = |U|^2
    const float gI = 2.f * (w * e + lambda_comp * dI) * inv_n;
    const float gR = 2.f * (w * er - lambda_comp * dI) * inv_n;
    const float fx = lambda_field * sgnf(dx) * inv_n, fy = lambda_field * sgnf(dy) * inv_n;
    Ud[i] = make_float2(fmaf(2.f * gI, u.x, fx), fmaf(2.f * gI, u.y, fy));
    Ur[i] = make_float2(fmaf(2.f * gR, r.x, -fx), fmaf(2.f * gR, r.y, -fy));
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tsum = 0.f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tsum += red[k];
    partials[blockIdx.x] = tsum;
  }
}

int grid_of(long long n) {
  long long g = (n + 255) / 256;
  return (int)(g > 152 * 8 ? 152 * 8 : (g < 1 ? 1 : g));
}

cgh_status cuda_status(cudaError_t e, const char* where) {
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? CGH_OK : cgh_record_error(CGH_ERR_CUDA, where);
}

constexpr int kExtractBlocks = 152 * 4;

}  // namespace

extern "C" cgh_status cgh_poh_scratch_bytes(const cgh_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return cgh_record_error(CGH_ERR_ARG, "cgh_poh_scratch_bytes: NULL argument");
  const size_t hw = (size_t)plan->H * plan->W;
  *bytes = sizeof(float2) * hw * ((size_t)2 * plan->L * plan->C + plan->C);
  return CGH_OK;
}

extern "C" cgh_status cgh_poh_dpac(const cgh_plan* plan, const void* U0, void* H_out,
                                   int32_t mode, void* stream) {
  if (!plan || !U0 || !H_out) return cgh_record_error(CGH_ERR_ARG, "cgh_poh_dpac: NULL argument");
  if (mode != 0 && mode != 1) return cgh_record_error(CGH_ERR_ARG, "cgh_poh_dpac: mode must be 0 or 1");
  if (!plan->ws) return cgh_record_error(CGH_ERR_WORKSPACE, "cgh_poh_dpac: no workspace attached");
  const long long per = (long long)plan->H * plan->W, total = per * plan->C;
  cudaStream_t s = (cudaStream_t)stream;
  // per-channel maxima in the plan's loss-partials area (C words)
  unsigned int* amax = (unsigned int*)(plan->ws + plan->off_loss);
  cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(unsigned int) * plan->C, s);
  if (e != cudaSuccess) return cuda_status(e, "cgh_poh_dpac");
  prof_begin(KID_POH, s);
  if (mode == 1) {
    long long g = (per + 255) / 256;
    if (g > 152 * 4) g = 152 * 4;
    k_chan_absmax<<<dim3((unsigned)g, plan->C), 256, 0, s>>>(per, (const float2*)U0, amax);
  }
  k_poh_dpac<<<grid_of(total), 256, 0, s>>>(total, plan->C, plan->H, plan->W, mode, amax,
                                             (const float2*)U0, (float2*)H_out);
  prof_end(KID_POH, s);
  return cuda_status(cudaSuccess, "cgh_poh_dpac");
}

extern "C" cgh_status cgh_poh_field(const cgh_plan* plan, const float* phi, void* H_out,
                                    void* stream) {
  if (!plan || !phi || !H_out) return cgh_record_error(CGH_ERR_ARG, "cgh_poh_field: NULL argument");
  const long long total = (long long)plan->C * plan->H * plan->W;
  cudaStream_t s = (cudaStream_t)stream;
  prof_begin(KID_POH, s);
  k_poh_field<<<grid_of(total), 256, 0, s>>>(total, phi, (float2*)H_out);
  prof_end(KID_POH, s);
  return cuda_status(cudaSuccess, "cgh_poh_field");
}

extern "C" cgh_status cgh_poh_step(cgh_plan* plan, const cgh_params* params, const float* phi,
                                   const float* target, float lambda_comp, float lambda_field,
                                   float* loss_out, const cgh_grads* grads, float* dphi,
                                   void* scratch, size_t scratch_bytes, void* stream) {
  if (!plan || !params || !phi || !target || !loss_out || !grads || !dphi || !scratch)
    return cgh_record_error(CGH_ERR_ARG, "cgh_poh_step: NULL argument");
  if (!plan->ws) return cgh_record_error(CGH_ERR_WORKSPACE, "cgh_poh_step: no workspace attached");
  if (params->N < 0 || params->N > plan->max_gaussians)
    return cgh_record_error(CGH_ERR_CAPACITY, "cgh_poh_step: N outside [0, max_gaussians]");
  if (params->N > 0 && (!params->xy_raw || !params->s_raw || !params->theta || !params->amp ||
                        !params->phase || !params->alpha_raw || !grads->xy_raw || !grads->s_raw ||
                        !grads->theta || !grads->amp || !grads->phase || !grads->alpha_raw))
    return cgh_record_error(CGH_ERR_ARG, "cgh_poh_step: NULL parameter or gradient array");
  size_t need = 0;
  cgh_poh_scratch_bytes(plan, &need);
  if (scratch_bytes < need)
    return cgh_record_error(CGH_ERR_WORKSPACE, "cgh_poh_step: scratch smaller than cgh_poh_scratch_bytes");
  cudaStream_t s = (cudaStream_t)stream;
  const int L = plan->L, C = plan->C;
  const size_t hw = (size_t)plan->H * plan->W;
  float2* UdA = (float2*)scratch;                 // [L][C][H][W]: U(d_l), then dL/dU(d_l)
  float2* UdB = UdA + (size_t)L * C * hw;         // U_rand(d_l), then its gradient
  float2* Hr = UdB + (size_t)L * C * hw;          // exp(j phi), then dL/dH_rand
  float2* U0 = (float2*)(plan->ws + plan->off_U0);
  float2* Y = (float2*)(plan->ws + plan->off_Y);
  float2* V = (float2*)(plan->ws + plan->off_V);
  float* partials = (float*)(plan->ws + plan->off_loss);
  const long long nf = (long long)C * hw, nl = (long long)L * C * hw;
  cudaError_t e;
  const char* where = "cgh_poh_step";
#define POH_TRY(expr) \
  do { e = (expr); if (e != cudaSuccess) return cuda_status(e, where); } while (0)
  // the Gaussians' field at every plane
  POH_TRY(launch_raster_fwd(plan, params, U0, s));
  POH_TRY(launch_rows_pad_fwd(plan, U0, Y, C, s));
  POH_TRY(launch_cols_fwd_planes(plan, Y, V, s));
  POH_TRY(launch_rows_inv_crop(plan, V, UdA, L * C, s));
  // the random POH at every plane
  prof_begin(KID_POH, s);
  k_poh_field<<<grid_of(nf), 256, 0, s>>>(nf, phi, Hr);
  prof_end(KID_POH, s);
  POH_TRY(launch_rows_pad_fwd(plan, Hr, Y, C, s));
  POH_TRY(launch_cols_fwd_planes(plan, Y, V, s));
  POH_TRY(launch_rows_inv_crop(plan, V, UdB, L * C, s));
  // L_extract and both gradients
  prof_begin(KID_POH, s);
  k_extract_loss<<<kExtractBlocks, 256, 0, s>>>(plan->bl, nl, (float)(1.0 / (double)nf),
                                                lambda_comp, lambda_field, UdA, UdB, target,
                                                partials);
  prof_end(KID_POH, s);
  POH_TRY(launch_loss_finalize_scaled(partials, kExtractBlocks, 1.0 / (double)nf, loss_out, s));
  // adjoint propagation of the Gaussians' gradient, raster backward (binning reused)
  POH_TRY(launch_rows_pad_fwd(plan, UdA, V, L * C, s));
  POH_TRY(launch_cols_bwd_planes(plan, V, Y, s));
  POH_TRY(launch_rows_inv_crop(plan, Y, U0, C, s));
  POH_TRY(launch_raster_bwd(plan, params, U0, grads, s, false));
  // adjoint propagation of the random POH's gradient, then through exp(j phi)
  POH_TRY(launch_rows_pad_fwd(plan, UdB, V, L * C, s));
  POH_TRY(launch_cols_bwd_planes(plan, V, Y, s));
  POH_TRY(launch_rows_inv_crop(plan, Y, Hr, C, s));
  prof_begin(KID_POH, s);
  k_poh_phase_grad<<<grid_of(nf), 256, 0, s>>>(nf, phi, Hr, dphi);
  prof_end(KID_POH, s);
#undef POH_TRY
  return cuda_status(cudaSuccess, where);
}
