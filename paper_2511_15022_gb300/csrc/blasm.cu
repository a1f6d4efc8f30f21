// blasm.cu -- band-limited angular spectrum propagation as fused row/column FFT passes.
//
// The 2D transform of the zero-padded Ny x Nx grid (Ny = pad*H, Nx = pad*W) is split into
// row and column passes that never materialise the padded grid:
//   rows_pad_fwd    pad each image row into the Nx-long row (zeros outside the centred
//                   window) and FFT it; only the H rows that hold data are transformed.
//                   Output: the "half grid" H x Nx.
//   cols_fwd_planes per column block: pad the column to Ny, FFT, keep the spectrum in
//                   shared memory and for every plane l multiply by H_{c,l} (Algorithm 3:
//                   band limit, k_z, exp(j k_z d), optional aperture) / (Ny Nx), inverse
//                   FFT and keep the H cropped rows.  Output: L half grids.
//   rows_loss       per plane and row: inverse row FFT, crop, I = |U|^2, loss partials
//                   (I - I^)^2, seed dL/dU = 4 (I - I^) U / (L C H W), re-pad and forward
//                   row FFT -- written back in place.
//   cols_bwd_planes per column block: for every plane FFT the column, multiply by
//                   conj(H_{c,l}) / (Ny Nx) and accumulate, inverse FFT once, crop.
//   rows_inv_crop   inverse row FFT and crop back to H x W.
// Half grids are stored column-blocked: element (row r, column k) of a half grid lives at
// ((k / CB) * H + r) * CB + k % CB, so a column pass reads one contiguous slab and a row
// pass of RB rows reads/writes runs of RB * CB complex values.
#include <cuda_runtime.h>
#include <math.h>

#include "cgh_internal.h"
#include "fft.cuh"
#include "blasm_common.cuh"
#include "blasm_spec.h"

namespace cgh {

template <int MAXB>
__global__ void __launch_bounds__(512, 1) k_rows_pad_fwd(const __grid_constant__ BlasmDev bl,
                                                       const FFTDesc fx, int RB, int CB, int bs,
                                                       const float2* __restrict__ in,
                                                       float2* __restrict__ half) {
  extern __shared__ float2 sm[];
  const int batch = blockIdx.y;
  const int y0 = blockIdx.x * RB;
  const int rows = min(RB, bl.H - y0);
  const int Nx = bl.Nx, W = bl.W, H = bl.H;
  const float2* src = in + (size_t)batch * H * W;
  for (int idx = threadIdx.x; idx < rows * Nx; idx += blockDim.x) {
    const int b = idx / Nx, k = idx - b * Nx;
    const int x = k - bl.ox;
    float2 v = make_float2(0.f, 0.f);
    if (x >= 0 && x < W) v = src[(size_t)(y0 + b) * W + x];
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

template <int MAXB>
__global__ void __launch_bounds__(512, 1) k_cols_fwd_planes(const __grid_constant__ BlasmDev bl,
                                                          const FFTDesc fy, int CB, int bs,
                                                          const float2* __restrict__ Y,
                                                          float2* __restrict__ V) {
  extern __shared__ float2 sm[];
  float2* S = sm;
  float2* Wk = sm + CB * bs;
  const int c = blockIdx.y, kb = blockIdx.x;
  const int H = bl.H, Ny = bl.Ny, Nx = bl.Nx, C = bl.C, oy = bl.oy;
  const float2* src = Y + (size_t)c * H * Nx + (size_t)kb * H * CB;
  for (int idx = threadIdx.x; idx < CB * Ny; idx += blockDim.x) {
    const int b = idx % CB, i = idx / CB;
    const int y = i - oy;
    S[b * bs + sidx(i)] = (y >= 0 && y < H) ? src[(size_t)y * CB + b] : make_float2(0.f, 0.f);
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

template <int MAXB>
__global__ void __launch_bounds__(512, 1) k_rows_inv_crop(const __grid_constant__ BlasmDev bl,
                                                        const FFTDesc fx, int RB, int CB, int bs,
                                                        const float2* __restrict__ half,
                                                        float2* __restrict__ out, int accum) {
  extern __shared__ float2 sm[];
  const int batch = blockIdx.y;
  const int y0 = blockIdx.x * RB;
  const int rows = min(RB, bl.H - y0);
  const int Nx = bl.Nx, W = bl.W, H = bl.H;
  const float2* src = half + (size_t)batch * H * Nx;
  for (int idx = threadIdx.x; idx < rows * Nx; idx += blockDim.x) {
    const int kk = idx % CB, rest = idx / CB;
    const int b = rest % rows, kb = rest / rows;
    sm[b * bs + sidx(kb * CB + kk)] = src[((size_t)kb * H + y0 + b) * CB + kk];
  }
  __syncthreads();
  block_fft<true, MAXB>(sm, bs, rows, fx);
  float2* dst = out + (size_t)batch * H * W;
  for (int idx = threadIdx.x; idx < rows * W; idx += blockDim.x) {
    const int b = idx / W, x = idx - b * W;
    const float2 v = sm[b * bs + sidx(bl.ox + x)];
    float2* o = &dst[(size_t)(y0 + b) * W + x];
    *o = accum ? cadd(*o, v) : v;
  }
}

template <int MAXB>
__global__ void __launch_bounds__(512, 1) k_rows_loss(const __grid_constant__ BlasmDev bl,
                                                    const FFTDesc fx, int RB, int CB, int bs,
                                                    float2* __restrict__ V,
                                                    const float* __restrict__ target,
                                                    float* __restrict__ partials, int want_grad) {
  extern __shared__ float2 sm[];
  __shared__ float red[32];
  const int batch = blockIdx.y;  // l * C + c (kernel planes)
  const int plane = bl.plane[batch / bl.C];  // the hologram plane: target, mask
  const int y0 = blockIdx.x * RB;
  const int rows = min(RB, bl.H - y0);
  const int Nx = bl.Nx, W = bl.W, H = bl.H;
  float2* half = V + (size_t)batch * H * Nx;
  for (int idx = threadIdx.x; idx < rows * Nx; idx += blockDim.x) {
    const int kk = idx % CB, rest = idx / CB;
    const int b = rest % rows, kb = rest / rows;
    sm[b * bs + sidx(kb * CB + kk)] = half[((size_t)kb * H + y0 + b) * CB + kk];
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
  if (threadIdx.x == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = tot;
  if (!want_grad) return;
  __syncthreads();
  block_fft<false, MAXB>(sm, bs, rows, fx);
  for (int idx = threadIdx.x; idx < rows * Nx; idx += blockDim.x) {
    const int kk = idx % CB, rest = idx / CB;
    const int b = rest % rows, kb = rest / rows;
    half[((size_t)kb * H + y0 + b) * CB + kk] = sm[b * bs + sidx(kb * CB + kk)];
  }
}

template <int MAXB>
__global__ void __launch_bounds__(512, 1) k_cols_bwd_planes(const __grid_constant__ BlasmDev bl,
                                                          const FFTDesc fy, int CB, int bs,
                                                          const float2* __restrict__ G,
                                                          float2* __restrict__ D) {
  extern __shared__ float2 sm[];
  float2* S = sm;
  float2* Wk = sm + CB * bs;
  const int c = blockIdx.y, kb = blockIdx.x;
  const int H = bl.H, Ny = bl.Ny, Nx = bl.Nx, C = bl.C, oy = bl.oy;
  for (int l = 0; l < bl.L; ++l) {
    const float2* src = G + (size_t)(l * C + c) * H * Nx + (size_t)kb * H * CB;
    for (int idx = threadIdx.x; idx < CB * Ny; idx += blockDim.x) {
      const int b = idx % CB, i = idx / CB;
      const int y = i - oy;
      Wk[b * bs + sidx(i)] = (y >= 0 && y < H) ? src[(size_t)y * CB + b] : make_float2(0.f, 0.f);
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

// Unfused intensity loss for the standalone API: partials per block, optional gradient.
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

// Loss and gradient seed of the planes whose propagation is the identity (distance 0, no
// aperture, every bin inside the band: H = 1 in Algorithm 3, so U(d_l) = U(0)), taken on
// U(0) itself.  One CTA per image row y (blockIdx.x) and channel c (blockIdx.y); per pixel,
// for each such plane l, d = |U|^2 - T_l: the loss partial gains w_l d^2 and the seed
// sum_l gscale w_l d U (the seed the loss row pass forms, Sec. 3.2) replaces U when
// want_grad (each element read and written by one thread).  Each thread loads its kIdentU
// elements of a row before using any (a 1920-pixel row is one round), so enough loads are
// in flight to cover the memory latency.
constexpr int kIdentU = 8;
__global__ void __launch_bounds__(256) k_ident_loss(const __grid_constant__ BlasmDev bl,
                                                    unsigned mask, float gscale,
                                                    float2* __restrict__ U,
                                                    const float* __restrict__ target,
                                                    float* __restrict__ partials, int want_grad) {
  __shared__ float red[32];
  const int y = blockIdx.x, c = blockIdx.y, W = bl.W;
  const size_t HW = (size_t)bl.H * W, row = (size_t)c * HW + (size_t)y * W;
  float2* u_row = U + row;
  float acc = 0.f;
  for (int x0 = 0; x0 < W; x0 += kIdentU * 256) {
    float2 u[kIdentU];
    float gs[kIdentU];
#pragma unroll
    for (int k = 0; k < kIdentU; ++k) {
      const int x = x0 + k * 256 + threadIdx.x;
      u[k] = x < W ? u_row[x] : make_float2(0.f, 0.f);
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
  if (threadIdx.x == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = tot;
}

// Intensity of a complex field (Sec. 3.2: I = |U|^2), element-wise over `total` values.
__global__ void k_intensity(long long total, const float2* __restrict__ U, float* __restrict__ I) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 u = __ldg(&U[i]);
    I[i] = fmaf(u.x, u.x, u.y * u.y);
  }
}

// Its adjoint: with dL/dI given, dL/dRe + j dL/dIm = 2 dL/dI (Re U + j Im U).
__global__ void k_intensity_bwd(long long total, const float2* __restrict__ U,
                                const float* __restrict__ dI, float2* __restrict__ dU) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 u = __ldg(&U[i]);
    const float g = 2.0f * __ldg(&dI[i]);
    dU[i] = make_float2(g * u.x, g * u.y);
  }
}

// loss = sum(partials) / (L C H W), summed in FP64 in a fixed order.
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

}  // namespace cgh

using namespace cgh;

namespace {

// shared-memory stride of one transform of length n: n + n/16 swizzle slots, rounded so
// that consecutive batch slots start 1 (mod 16) complex values apart.
int smem_stride(int n) {
  int s = n + n / 16 + 1;
  while (s % 16 != 1) ++s;
  return s;
}

int max_butterflies(const FFTDesc& d, int nb) {
  int mb = 0;
  for (int p = 0; p < d.npass; ++p) mb = mb > (d.n / d.radix[p]) * nb ? mb : (d.n / d.radix[p]) * nb;
  return mb;
}


}  // namespace

// Threads per CTA and butterflies per thread (MAXB) for nb transforms of d: the smallest
// thread count >= the tuned one that needs at most 2 butterflies per thread per pass.
LaunchShape fft_shape(const cgh_plan* p, const FFTDesc& d, int nb, int buffers) {
  const size_t smem = sizeof(float2) * (size_t)smem_stride(d.n) * nb * buffers + 256;
  if (smem > kMaxSmemBytes) return {0, 0, false};
  const int mb = max_butterflies(d, nb);
  for (int t = p->fft_threads; t <= kMaxFFTThreads; t += 32) {
    const int need = (mb + t - 1) / t;
    if (need <= 1) return {t, 1, true};
    if (need <= 2 && t * 2 >= mb) {
      // prefer one butterfly per thread when a legal thread count allows it
      if (mb <= kMaxFFTThreads) return {((mb + 31) / 32) * 32, 1, true};
      return {t, 2, true};
    }
  }
  return {kMaxFFTThreads, 0, false};
}

namespace {

template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define CGH_DISPATCH_MAXB(kid, maxb, KERNEL, grid, block, smem, stream, ...)                     \
  do {                                                                                      \
    cudaError_t _e = cudaSuccess;                                                           \
    prof_begin(kid, stream);                                                                \
    switch (maxb) {                                                                         \
      case 1: _e = set_smem(KERNEL<1>, smem);                                               \
        if (_e == cudaSuccess) KERNEL<1><<<grid, block, smem, stream>>>(__VA_ARGS__); break; \
      case 2: _e = set_smem(KERNEL<2>, smem);                                               \
        if (_e == cudaSuccess) KERNEL<2><<<grid, block, smem, stream>>>(__VA_ARGS__); break; \
      default: _e = cudaErrorInvalidConfiguration; break;                                   \
    }                                                                                       \
    prof_end(kid, stream);                                                                  \
    if (_e != cudaSuccess) return _e;                                                       \
  } while (0)

}  // namespace

int rows_loss_blocks(const cgh_plan* p, const BlasmDev* planes) {
  const int L = planes ? planes->L : p->L;
  return ((p->H + p->row_block - 1) / p->row_block) * L * p->C;
}

int ident_loss_blocks(const cgh_plan* p) { return p->H * p->C; }  // one per row and channel

int pointwise_loss_blocks(const cgh_plan* p) {
  (void)p;
  return 592;  // 4 blocks of 256 threads per SM on a 148-152 SM part
}

bool spec_rows(int kind, int N, int RB, int CB, const cgh_plan* p, const SpecRowArgs* a,
               cudaStream_t s, cudaError_t* err, bool dry) {
  return spec_rows_a(kind, N, RB, CB, p, a, s, err, dry) ||
         spec_rows_b(kind, N, RB, CB, p, a, s, err, dry) ||
         spec_rows_c(kind, N, RB, CB, p, a, s, err, dry) ||
         spec_rows_d(kind, N, RB, CB, p, a, s, err, dry) ||
         spec_rows_e(kind, N, RB, CB, p, a, s, err, dry) ||
         spec_rows_f(kind, N, RB, CB, p, a, s, err, dry) ||
         spec_rows_g(kind, N, RB, CB, p, a, s, err, dry);
}

bool spec_cols(int kind, int N, int CB, const cgh_plan* p, const BlasmDev* bl, const float2* in,
               float2* out, cudaStream_t s, cudaError_t* err, bool dry) {
  return spec_cols_a(kind, N, CB, p, bl, in, out, s, err, dry) ||
         spec_cols_b(kind, N, CB, p, bl, in, out, s, err, dry) ||
         spec_cols_c(kind, N, CB, p, bl, in, out, s, err, dry) ||
         spec_cols_d(kind, N, CB, p, bl, in, out, s, err, dry) ||
         spec_cols_e(kind, N, CB, p, bl, in, out, s, err, dry) ||
         spec_cols_f(kind, N, CB, p, bl, in, out, s, err, dry) ||
         spec_cols_g(kind, N, CB, p, bl, in, out, s, err, dry);
}

static bool try_spec_rows(int kind, cgh_plan* p, const SpecRowArgs& a, cudaStream_t s,
                          cudaError_t* err) {
  if (!p->use_spec) return false;
  return spec_rows(kind, p->fx.n, p->row_block, p->col_block, p, &a, s, err, false);
}

static bool try_spec_cols(int kind, cgh_plan* p, const BlasmDev* bl, const float2* in,
                          float2* out, cudaStream_t s, cudaError_t* err) {
  // the specialised column kernels evaluate H with the series form only
  if (!p->use_spec || !p->bl.series_ok) return false;
  return spec_cols(kind, p->fy.n, p->col_block, p, bl, in, out, s, err, false);
}

cudaError_t launch_rows_pad_fwd(cgh_plan* p, const float2* in, float2* half, int batches,
                                cudaStream_t s) {
  {
    cudaError_t e;
    SpecRowArgs a{&p->bl, in, half, nullptr, nullptr, batches, 0, nullptr, nullptr, 0.0, 0, 0};
    if (try_spec_rows(SPEC_ROWS_PAD_FWD, p, a, s, &e)) return e;
  }
  const int RB = p->row_block, CB = p->col_block, bs = smem_stride(p->fx.n);
  LaunchShape sh = fft_shape(p, p->fx, RB, 1);
  if (!sh.ok) return cudaErrorInvalidConfiguration;
  dim3 grid((p->H + RB - 1) / RB, batches);
  const size_t smem = sizeof(float2) * (size_t)bs * RB;
  CGH_DISPATCH_MAXB(KID_ROWS_PAD_FWD, sh.maxb, k_rows_pad_fwd, grid, sh.threads, smem, s, p->bl, p->fx, RB, CB,
                    bs, in, half);
  return cudaGetLastError();
}

cudaError_t launch_cols_fwd_planes(cgh_plan* p, const float2* Y, float2* V, cudaStream_t s,
                                   const BlasmDev* planes) {
  const BlasmDev& bl = planes ? *planes : p->bl;
  if (bl.L == 0) return cudaSuccess;
  {
    cudaError_t e;
    if (try_spec_cols(SPEC_COLS_FWD_PLANES, p, &bl, Y, V, s, &e)) return e;
  }
  const int CB = p->col_block, bs = smem_stride(p->fy.n);
  LaunchShape sh = fft_shape(p, p->fy, CB, 2);
  if (!sh.ok) return cudaErrorInvalidConfiguration;
  dim3 grid(p->bl.Nx / CB, p->C);
  const size_t smem = sizeof(float2) * (size_t)bs * CB * 2;
  CGH_DISPATCH_MAXB(KID_COLS_FWD_PLANES, sh.maxb, k_cols_fwd_planes, grid, sh.threads, smem, s, bl, p->fy, CB, bs,
                    Y, V);
  return cudaGetLastError();
}

cudaError_t launch_rows_inv_crop(cgh_plan* p, const float2* half, float2* out, int batches,
                                 cudaStream_t s, bool accumulate) {
  {
    cudaError_t e;
    SpecRowArgs a{&p->bl, half, out, nullptr, nullptr, batches, 0, nullptr, nullptr, 0.0, 0,
                  accumulate ? 1 : 0};
    if (try_spec_rows(SPEC_ROWS_INV_CROP, p, a, s, &e)) return e;
  }
  const int RB = p->row_block, CB = p->col_block, bs = smem_stride(p->fx.n);
  LaunchShape sh = fft_shape(p, p->fx, RB, 1);
  if (!sh.ok) return cudaErrorInvalidConfiguration;
  dim3 grid((p->H + RB - 1) / RB, batches);
  const size_t smem = sizeof(float2) * (size_t)bs * RB;
  CGH_DISPATCH_MAXB(KID_ROWS_INV_CROP, sh.maxb, k_rows_inv_crop, grid, sh.threads, smem, s, p->bl, p->fx, RB, CB,
                    bs, half, out, accumulate ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_rows_loss(cgh_plan* p, float2* V, const float* target, float* partials,
                             cudaStream_t s, bool want_grad, float* loss_out,
                             const BlasmDev* planes, int extra) {
  const BlasmDev& bl = planes ? *planes : p->bl;
  const double inv = 1.0 / ((double)p->L * p->C * p->H * p->W);
  if (bl.L == 0) return launch_loss_finalize(p, partials, extra, loss_out, s);
  {
    cudaError_t e;
    SpecRowArgs a{&bl, nullptr, V, target, partials, bl.L * p->C, want_grad ? 1 : 0, loss_out,
                  (int*)(p->ws + p->off_status) + ST_LOSS_TICKET, inv, extra, 0};
    if (try_spec_rows(SPEC_ROWS_LOSS, p, a, s, &e)) return e;
  }
  const int RB = p->row_block, CB = p->col_block, bs = smem_stride(p->fx.n);
  LaunchShape sh = fft_shape(p, p->fx, RB, 1);
  if (!sh.ok) return cudaErrorInvalidConfiguration;
  dim3 grid((p->H + RB - 1) / RB, bl.L * p->C);
  const size_t smem = sizeof(float2) * (size_t)bs * RB;
  CGH_DISPATCH_MAXB(KID_ROWS_LOSS, sh.maxb, k_rows_loss, grid, sh.threads, smem, s, bl, p->fx, RB, CB, bs,
                    V, target, partials, want_grad ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_loss_finalize(p, partials, rows_loss_blocks(p, &bl) + extra, loss_out, s);
}

cudaError_t launch_ident_loss(cgh_plan* p, float2* U, const float* target, float* partials,
                              bool want_grad, cudaStream_t s) {
  const float gscale = 4.0f / ((float)p->L * (float)p->C * (float)p->H * (float)p->W);
  prof_begin(KID_IDENT_LOSS, s);
  k_ident_loss<<<dim3(p->H, p->C), 256, 0, s>>>(p->bl, p->ident_mask, gscale, U, target,
                                                partials, want_grad ? 1 : 0);
  prof_end(KID_IDENT_LOSS, s);
  return cudaGetLastError();
}

cudaError_t launch_cols_bwd_planes(cgh_plan* p, const float2* G, float2* D, cudaStream_t s,
                                   const BlasmDev* planes) {
  const BlasmDev& bl = planes ? *planes : p->bl;
  if (bl.L == 0) return cudaSuccess;
  {
    cudaError_t e;
    if (try_spec_cols(SPEC_COLS_BWD_PLANES, p, &bl, G, D, s, &e)) return e;
  }
  const int CB = p->col_block, bs = smem_stride(p->fy.n);
  LaunchShape sh = fft_shape(p, p->fy, CB, 2);
  if (!sh.ok) return cudaErrorInvalidConfiguration;
  dim3 grid(p->bl.Nx / CB, p->C);
  const size_t smem = sizeof(float2) * (size_t)bs * CB * 2;
  CGH_DISPATCH_MAXB(KID_COLS_BWD_PLANES, sh.maxb, k_cols_bwd_planes, grid, sh.threads, smem, s, bl, p->fy, CB, bs,
                    G, D);
  return cudaGetLastError();
}

cudaError_t launch_loss_pointwise(cgh_plan* p, const float2* Ud, const float* target,
                                  float* partials, float2* dUd, cudaStream_t s) {
  const long long total = (long long)p->L * p->C * p->H * p->W;
  const float gscale = 4.0f / (float)total;
  prof_begin(KID_LOSS_POINTWISE, s);
  k_loss_pointwise<<<pointwise_loss_blocks(p), 256, 0, s>>>(p->bl, total, gscale, Ud, target,
                                                           partials, dUd);
  prof_end(KID_LOSS_POINTWISE, s);
  return cudaGetLastError();
}

static unsigned elementwise_blocks(long long total) {
  long long b = (total + 255) / 256;
  return (unsigned)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

cudaError_t launch_intensity(long long total, const float2* U, float* I, cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  prof_begin(KID_LOSS_POINTWISE, s);
  k_intensity<<<elementwise_blocks(total), 256, 0, s>>>(total, U, I);
  prof_end(KID_LOSS_POINTWISE, s);
  return cudaGetLastError();
}

cudaError_t launch_intensity_bwd(long long total, const float2* U, const float* dI, float2* dU,
                                 cudaStream_t s) {
  if (total <= 0) return cudaSuccess;
  prof_begin(KID_LOSS_POINTWISE, s);
  k_intensity_bwd<<<elementwise_blocks(total), 256, 0, s>>>(total, U, dI, dU);
  prof_end(KID_LOSS_POINTWISE, s);
  return cudaGetLastError();
}

cudaError_t launch_loss_finalize_scaled(const float* partials, int count, double inv, float* out,
                                        cudaStream_t s) {
  prof_begin(KID_LOSS_FINALIZE, s);
  k_loss_finalize<<<1, 1024, 0, s>>>(partials, count, inv, out);
  prof_end(KID_LOSS_FINALIZE, s);
  return cudaGetLastError();
}

cudaError_t launch_loss_finalize(cgh_plan* p, const float* partials, int count, float* out,
                                 cudaStream_t s) {
  const double inv = 1.0 / ((double)p->L * p->C * p->H * p->W);
  prof_begin(KID_LOSS_FINALIZE, s);
  k_loss_finalize<<<1, 1024, 0, s>>>(partials, count, inv, out);
  prof_end(KID_LOSS_FINALIZE, s);
  return cudaGetLastError();
}
