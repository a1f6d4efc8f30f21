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

#include "blasm_generic.cuh"
#include "blasm_spec.h"


using namespace cgh;

namespace {

// shared-memory stride of one transform of length n: n + n/16 swizzle slots, rounded so
// that consecutive batch slots start 1 (mod 16) complex values apart.
int smem_stride(int n) {
  int s = n + n / 16 + 1;
  while (s % 16 != 1) ++s;
  return s;
}

}  // namespace

int fft_smem_stride(int n) { return smem_stride(n); }

namespace {

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

int ident_loss_blocks(const cgh_plan* p) { return p->tiles_x * p->tiles_y; }  // one per tile

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
