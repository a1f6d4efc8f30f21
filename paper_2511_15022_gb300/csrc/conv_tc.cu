// conv_tc.cu -- tensor-core 3x3 convolutions of the learned initialiser (sm_103a).
//
// The encoder's convolutions are dense contractions, so they run on the tensor cores as
// implicit GEMMs: warp-level mma.sync m16n8k16 with BF16 operands and FP32 accumulation,
// operands staged in shared memory and loaded into fragments with ldmatrix.
//
//   k_conv_tc<MODE_FWD>   y = act(bias + W * x): one CTA per 8 x 16 tile of output pixels and
//                         64 output channels; the input patch of each 16-channel chunk is
//                         staged channel-innermost ([position][channel]), so the 16 pixels x
//                         16 channels A fragment of one filter tap is one ldmatrix.x4 of 16
//                         rows (the im2col gather happens in the row addresses); weights are
//                         staged [tap][out channel][channel] (the B fragments).
//   k_conv_tc<MODE_DGRAD> dx = W^T * g with g = dy [y > 0]: for a stride-s convolution this is
//                         the stride-1 convolution of g zero-upsampled by s with the transposed,
//                         flipped weights W'[ci][co][2-ky][2-kx]; the same kernel stages that
//                         virtual input.  g is FP32, so it is split into two BF16 parts, hi =
//                         bf16(g) and lo = bf16(g - hi) (|g - hi - lo| <= 2^-18 |g|), and both
//                         are multiplied: the product keeps FP32 accuracy.
//   k_conv_wgrad_tc       dW[co][ci][tap] = sum over pixels of g x_shifted, db[co] = sum g:
//                         M = 64 output channels, N = 16 input channels x 9 taps, K = pixels
//                         (16 per step, one output row of a tile); each CTA walks a range of
//                         pixel tiles, accumulating in registers, and adds its partial sums
//                         with one atomic per value.  g is split as above.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cgh_internal.h"

namespace cgh {
namespace tc {

constexpr int TH = 8, TW = 16;  // output pixel tile: one warp per row of 16 pixels
constexpr int NT = 64;          // output channels per CTA (8 n8 blocks)
constexpr int KC = 16;          // channels per staged chunk (one k16 step per tap)
constexpr int PS = 24;          // bf16 per staged position / weight row: 48-byte rows, 16-byte
                                // aligned for ldmatrix, consecutive rows on different banks
constexpr int kThreads = 256;
constexpr int kSU = 8;          // staged elements per thread per round (their loads in flight)
constexpr int GS = TH * TW + 8; // bf16 per staged row of the weight-gradient tiles (272 bytes)

enum { MODE_FWD = 0, MODE_DGRAD = 1 };

struct ConvArgs {
  int B;
  int Kc, Nc;        // contraction channels (per tap) and output channels of this convolution
  int Hin, Win;      // the convolution's input grid (DGRAD: the zero-upsampled g, s * Ho x s * Wo)
  int Hout, Wout;    // output grid
  int sc;            // convolution stride (FWD: s; DGRAD: 1)
  int up;            // DGRAD: upsampling factor s of g
  int Hg, Wg;        // DGRAD: grid of g (Ho x Wo)
  int relu, y_f32, out_f32;
  const __nv_bfloat16* x;  // FWD input [B][Kc][Hin][Win]
  const float* dy;         // DGRAD upstream gradient [B][Kc][Hg][Wg]
  const void* y;           // DGRAD: forward output of the layer (ReLU mask), same layout as dy
  const __nv_bfloat16* w;  // forward weights [CO][CI][3][3]
  const float* bias;       // FWD
  void* out;               // [B][Nc][Hout][Wout], bf16 or f32
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t (&r)[2], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(addr));
}

// D = A B + D, A 16 x 16 (row), B 16 x 8 (col), BF16 inputs, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// g = dy [y > 0] (no mask without ReLU)
__device__ __forceinline__ float grad_in(const float* dy, const void* y, int y_f32, int relu,
                                         size_t o) {
  float g = __ldg(&dy[o]);
  if (relu) {
    const float yv = y_f32 ? __ldg(&static_cast<const float*>(y)[o])
                           : __bfloat162float(static_cast<const __nv_bfloat16*>(y)[o]);
    if (!(yv > 0.f)) g = 0.f;
  }
  return g;
}

__device__ __forceinline__ void split_bf16(float g, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(g);
  lo = __float2bfloat16_rn(g - __bfloat162float(hi));
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_conv_tc(ConvArgs a) {
  constexpr int NPART = MODE == MODE_DGRAD ? 2 : 1;  // hi / lo parts of the input
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int sc = a.sc;
  const int PH = (TH - 1) * sc + 3, PW = (TW - 1) * sc + 3;
  __nv_bfloat16* wt = reinterpret_cast<__nv_bfloat16*>(smem_raw);  // [9][NT][PS]
  __nv_bfloat16* patch = wt + 9 * NT * PS;                           // [NPART][PH * PW][PS]
  const int npos = PH * PW;
  const int ntx = (a.Wout + TW - 1) / TW;
  const int ox0 = (blockIdx.x % ntx) * TW, oy0 = (blockIdx.x / ntx) * TH;
  const int nblk = (a.Nc + NT - 1) / NT;
  const int b = blockIdx.y / nblk, n0 = (blockIdx.y % nblk) * NT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int iy0 = oy0 * sc - 1, ix0 = ox0 * sc - 1;  // input position of patch (0, 0)
  // 16-byte weight rows: w + (n Kc + c0) 9 is 16-byte aligned for every n when Kc % 8 == 0
  const bool vec_w = (a.Kc % 8 == 0) && ((reinterpret_cast<uintptr_t>(a.w) & 15u) == 0);

  float acc[NT / 8][4];
#pragma unroll
  for (int j = 0; j < NT / 8; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;

  for (int c0 = 0; c0 < a.Kc; c0 += KC) {
    __syncthreads();  // the previous chunk's fragments have been loaded
    // weights of this chunk: wt[tap][n][c] = W(n0 + n, c0 + c, tap).  Forward weights of a
    // full chunk are 144 consecutive BF16 per output channel: staged with 16-byte loads
    // (when aligned), each scattered to its 8 (tap, channel) slots.
    if (MODE == MODE_FWD && vec_w && c0 + KC <= a.Kc) {
      for (int e = threadIdx.x; e < NT * 18; e += kThreads) {
        const int n = e / 18, q = e % 18, nn = n0 + n;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (nn < a.Nc) v = __ldg(reinterpret_cast<const uint4*>(a.w + ((size_t)nn * a.Kc + c0) * 9) + q);
        const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int r = q * 8 + k;  // r = c * 9 + tap within the chunk
          wt[((r % 9) * NT + n) * PS + r / 9] = h[k];
        }
      }
    } else
    for (int e0 = threadIdx.x; e0 < 9 * NT * KC; e0 += kSU * kThreads) {
      __nv_bfloat16 v[kSU];
      int dst[kSU];
#pragma unroll
      for (int u = 0; u < kSU; ++u) {
        const int e = e0 + u * kThreads;
        int n, c, tap;
        if (MODE == MODE_FWD) {  // e = (n * KC + c) * 9 + tap: w[n][c0 + c][tap] contiguous
          tap = e % 9; c = (e / 9) % KC; n = e / (9 * KC);
        } else {                 // e = (c * NT + n) * 9 + tap: w[c0 + c][n][8 - tap] contiguous
          tap = e % 9; n = (e / 9) % NT; c = e / (9 * NT);
        }
        const int nn = n0 + n, cc = c0 + c;
        v[u] = __float2bfloat16_rn(0.f);
        dst[u] = -1;
        if (e < 9 * NT * KC) {
          dst[u] = (tap * NT + n) * PS + c;
          if (nn < a.Nc && cc < a.Kc)
            v[u] = MODE == MODE_FWD ? a.w[((size_t)nn * a.Kc + cc) * 9 + tap]
                                    : a.w[((size_t)cc * a.Nc + nn) * 9 + (8 - tap)];
        }
      }
#pragma unroll
      for (int u = 0; u < kSU; ++u)
        if (dst[u] >= 0) wt[dst[u]] = v[u];
    }
    // the input patch of this chunk, channel-innermost (the chunk's real channels only; in a
    // partial last chunk the slots beyond Kc are zeroed here, earlier chunks filled them)
    const int kcr = min(KC, a.Kc - c0);
    if (kcr < KC)
      for (int e = threadIdx.x; e < npos * NPART; e += kThreads)
        for (int c = kcr; c < KC; ++c) patch[e * PS + c] = __float2bfloat16_rn(0.f);
    for (int e0 = threadIdx.x; e0 < kcr * npos; e0 += kSU * kThreads) {
      float g[kSU];
      __nv_bfloat16 xv[kSU];
#pragma unroll
      for (int u = 0; u < kSU; ++u) {
        const int e = e0 + u * kThreads;
        const int pos = e % npos, cc = c0 + e / npos;
        const int Y = iy0 + pos / PW, X = ix0 + pos % PW;
        g[u] = 0.f;
        xv[u] = __float2bfloat16_rn(0.f);
        if (e < kcr * npos) {
          if (MODE == MODE_FWD) {
            if (Y >= 0 && Y < a.Hin && X >= 0 && X < a.Win)
              xv[u] = a.x[(((size_t)b * a.Kc + cc) * a.Hin + Y) * a.Win + X];
          } else if (Y >= 0 && X >= 0 && Y % a.up == 0 && X % a.up == 0) {
            const int gy = Y / a.up, gx = X / a.up;
            if (gy < a.Hg && gx < a.Wg)
              g[u] = grad_in(a.dy, a.y, a.y_f32, a.relu,
                             (((size_t)b * a.Kc + cc) * a.Hg + gy) * a.Wg + gx);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kSU; ++u) {
        const int e = e0 + u * kThreads;
        if (e >= kcr * npos) continue;
        const int pos = e % npos, c = e / npos;
        if (MODE == MODE_FWD) {
          patch[pos * PS + c] = xv[u];
        } else {
          __nv_bfloat16 hi, lo;
          split_bf16(g[u], hi, lo);
          patch[pos * PS + c] = hi;
          patch[(npos + pos) * PS + c] = lo;
        }
      }
    }
    __syncthreads();
    // warp `warp` computes output row oy0 + warp: A rows are its 16 pixels
    const int arow = lane & 15, akh = lane >> 4;
    const int bn = (lane & 7) + ((lane >> 4) << 3), bkh = (lane >> 3) & 1;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int ky = tap / 3, kx = tap % 3;
      const int pos = (warp * sc + ky) * PW + arow * sc + kx;
      uint32_t af[NPART][4];
#pragma unroll
      for (int part = 0; part < NPART; ++part)
        ldsm_x4(af[part], smem_u32(&patch[(part * npos + pos) * PS + akh * 8]));
#pragma unroll
      for (int j = 0; j < NT / 16; ++j) {  // two n8 blocks per ldmatrix.x4
        uint32_t bf[4];
        ldsm_x4(bf, smem_u32(&wt[(tap * NT + 16 * j + bn) * PS + bkh * 8]));
#pragma unroll
        for (int part = 0; part < NPART; ++part) {
          mma_bf16(acc[2 * j], af[part], bf[0], bf[1]);
          mma_bf16(acc[2 * j + 1], af[part], bf[2], bf[3]);
        }
      }
    }
  }
  // epilogue: acc[j] = (pixel g, channels 8j + 2t, +1) and (pixel g + 8, ...)
  const int oy = oy0 + warp, gq = lane >> 2, tq = lane & 3;
  if (oy >= a.Hout) return;
#pragma unroll
  for (int j = 0; j < NT / 8; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int n = n0 + 8 * j + 2 * tq + (q & 1);
      const int ox = ox0 + gq + ((q >> 1) << 3);
      if (n >= a.Nc || ox >= a.Wout) continue;
      float v = acc[j][q];
      if (MODE == MODE_FWD) {
        v += __ldg(&a.bias[n]);
        if (a.relu) v = fmaxf(v, 0.f);
      }
      const size_t o = (((size_t)b * a.Nc + n) * a.Hout + oy) * a.Wout + ox;
      if (a.out_f32) static_cast<float*>(a.out)[o] = v;
      else static_cast<__nv_bfloat16*>(a.out)[o] = __float2bfloat16_rn(v);
    }
}

// Data gradient of a stride-2 convolution, one output parity class per CTA (blockIdx.z =
// 2 py + px).  dx[2m + py][2n + px] gets W[co][ci][ky][kx] g[co][m + dy][n + dx] only from the
// taps with ky = 1 (py = 0; dy = 0) or ky in {0, 2} (py = 1; dy = 1, 0), and likewise in x:
// 1, 2, 2 or 4 taps, i.e. exactly the multiply-adds of the forward convolution, no zeros.
// A CTA covers an 8 x 16 tile (m0, n0) of the g grid; the g patch (9 x 17 positions x 16
// channels, hi and lo parts) and the class's weights are staged per 16-channel chunk.
__global__ void __launch_bounds__(kThreads) k_conv_dgrad2_tc(ConvArgs a) {
  constexpr int GH = TH + 1, GW = TW + 1;  // g positions of a tile plus the +1 taps
  __shared__ __align__(16) __nv_bfloat16 wt[4 * NT * PS];        // [tap of the class][n][c]
  __shared__ __align__(16) __nv_bfloat16 patch[2 * GH * GW * PS];  // [hi, lo][pos][c]
  const int py = blockIdx.z >> 1, px = blockIdx.z & 1;
  const int nty = py ? 2 : 1, ntx_ = px ? 2 : 1, ntap = nty * ntx_;
  const int ntx = (a.Wg + TW - 1) / TW;
  const int gx0 = (blockIdx.x % ntx) * TW, gy0 = (blockIdx.x / ntx) * TH;
  const int nblk = (a.Nc + NT - 1) / NT;
  const int b = blockIdx.y / nblk, n0 = (blockIdx.y % nblk) * NT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float acc[NT / 8][4];
#pragma unroll
  for (int j = 0; j < NT / 8; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
  for (int c0 = 0; c0 < a.Kc; c0 += KC) {
    __syncthreads();  // the previous chunk's fragments have been loaded
    // class weights: wt[t][n][c] = W[c0 + c][n0 + n][ky_t][kx_t] (only the class's taps)
    for (int e0 = threadIdx.x; e0 < ntap * NT * KC; e0 += kSU * kThreads) {
      __nv_bfloat16 v[kSU];
      int dst[kSU];
#pragma unroll
      for (int u = 0; u < kSU; ++u) {
        const int e = e0 + u * kThreads;
        const int t = e % ntap, n = (e / ntap) % NT, c = e / (ntap * NT);
        const int ky = py ? 2 * (t / ntx_) : 1, kx = px ? 2 * (t % ntx_) : 1;
        const int nn = n0 + n, cc = c0 + c;
        v[u] = __float2bfloat16_rn(0.f);
        dst[u] = -1;
        if (e < ntap * NT * KC) {
          dst[u] = (t * NT + n) * PS + c;
          if (nn < a.Nc && cc < a.Kc) v[u] = a.w[((size_t)cc * a.Nc + nn) * 9 + ky * 3 + kx];
        }
      }
#pragma unroll
      for (int u = 0; u < kSU; ++u)
        if (dst[u] >= 0) wt[dst[u]] = v[u];
    }
    for (int e0 = threadIdx.x; e0 < KC * GH * GW; e0 += kSU * kThreads) {
      float g[kSU];
#pragma unroll
      for (int u = 0; u < kSU; ++u) {
        const int e = e0 + u * kThreads;
        const int pos = e % (GH * GW), cc = c0 + e / (GH * GW);
        const int gy = gy0 + pos / GW, gx = gx0 + pos % GW;
        g[u] = 0.f;
        if (e < KC * GH * GW && cc < a.Kc && gy < a.Hg && gx < a.Wg)
          g[u] = grad_in(a.dy, a.y, a.y_f32, a.relu,
                         (((size_t)b * a.Kc + cc) * a.Hg + gy) * a.Wg + gx);
      }
#pragma unroll
      for (int u = 0; u < kSU; ++u) {
        const int e = e0 + u * kThreads;
        if (e >= KC * GH * GW) continue;
        const int pos = e % (GH * GW), c = e / (GH * GW);
        __nv_bfloat16 hi, lo;
        split_bf16(g[u], hi, lo);
        patch[pos * PS + c] = hi;
        patch[(GH * GW + pos) * PS + c] = lo;
      }
    }
    __syncthreads();
    const int arow = lane & 15, akh = lane >> 4;
    const int bn = (lane & 7) + ((lane >> 4) << 3), bkh = (lane >> 3) & 1;
    for (int t = 0; t < ntap; ++t) {
      const int ky = py ? 2 * (t / ntx_) : 1, kx = px ? 2 * (t % ntx_) : 1;
      const int dyo = (py + 1 - ky) >> 1, dxo = (px + 1 - kx) >> 1;  // 0 or 1
      const int pos = (warp + dyo) * GW + arow + dxo;
      uint32_t af[2][4];
#pragma unroll
      for (int part = 0; part < 2; ++part)
        ldsm_x4(af[part], smem_u32(&patch[(part * GH * GW + pos) * PS + akh * 8]));
#pragma unroll
      for (int j = 0; j < NT / 16; ++j) {
        uint32_t bf[4];
        ldsm_x4(bf, smem_u32(&wt[(t * NT + 16 * j + bn) * PS + bkh * 8]));
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          mma_bf16(acc[2 * j], af[part], bf[0], bf[1]);
          mma_bf16(acc[2 * j + 1], af[part], bf[2], bf[3]);
        }
      }
    }
  }
  const int gq = lane >> 2, tq = lane & 3;
  const int iy = 2 * (gy0 + warp) + py;
  if (iy >= a.Hout) return;
#pragma unroll
  for (int j = 0; j < NT / 8; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int n = n0 + 8 * j + 2 * tq + (q & 1);
      const int ix = 2 * (gx0 + gq + ((q >> 1) << 3)) + px;
      if (n >= a.Nc || ix >= a.Wout) continue;
      static_cast<float*>(a.out)[(((size_t)b * a.Nc + n) * a.Hout + iy) * a.Wout + ix] = acc[j][q];
    }
}

struct WgradArgs {
  int B, CI, Hi, Wi, CO, Ho, Wo, stride, relu, y_f32;
  int per_cta;  // pixel tiles per CTA
  const __nv_bfloat16* x;
  const void* y;
  const float* dy;
  float* dw;
  float* db;
};

// dW partial sums of one CTA: co block blockIdx.y (64 channels), ci chunk blockIdx.z (16
// channels x 9 taps), pixel tiles [blockIdx.x * per_cta, +per_cta).  Warp w: m16 block w & 3
// (16 output channels), n8 blocks 9 (w >> 2) .. + 9 of the 18 (tap, ci) blocks.
__global__ void __launch_bounds__(kThreads, 2) k_conv_wgrad_tc(WgradArgs a) {
  constexpr int kSU = 4;  // two resident CTAs: fewer staged loads in flight per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* gs = reinterpret_cast<__nv_bfloat16*>(smem_raw);  // [2][NT][GS] g hi / lo
  __nv_bfloat16* xs = gs + 2 * NT * GS;                              // [9 * KC][GS] shifted x
  const int co0 = blockIdx.y * NT, ci0 = blockIdx.z * KC;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mb = warp & 3, nb0 = 9 * (warp >> 2);
  const int ntx = (a.Wo + TW - 1) / TW, nty = (a.Ho + TH - 1) / TH;
  const long long tiles = (long long)a.B * ntx * nty;
  const long long t0 = (long long)blockIdx.x * a.per_cta;
  const long long t1 = t0 + a.per_cta < tiles ? t0 + a.per_cta : tiles;
  float acc[9][4];
#pragma unroll
  for (int j = 0; j < 9; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
  __shared__ float sdb[NT];  // this CTA's bias-gradient partial sums (ci chunk 0 only)
  if (threadIdx.x < NT) sdb[threadIdx.x] = 0.f;
  // rows of padding channels (co >= CO, ci >= CI) stay zero: cleared once, never restaged
  const int cor = min(NT, a.CO - co0), cir = min(KC, a.CI - ci0);
  for (int e = threadIdx.x; e < (NT - cor) * TH * TW; e += kThreads) {
    const int co = cor + e / (TH * TW), p = e % (TH * TW);
    gs[co * GS + p] = __float2bfloat16_rn(0.f);
    gs[(NT + co) * GS + p] = __float2bfloat16_rn(0.f);
  }
  for (int e = threadIdx.x; e < 9 * (KC - cir) * TH * TW; e += kThreads) {
    const int p = e % (TH * TW), r = e / (TH * TW), tap = r / (KC - cir), ci = cir + r % (KC - cir);
    xs[(tap * KC + ci) * GS + p] = __float2bfloat16_rn(0.f);
  }
  for (long long t = t0; t < t1; ++t) {
    const int b = (int)(t / ((long long)ntx * nty));
    const int r = (int)(t % ((long long)ntx * nty));
    const int oy0 = (r / ntx) * TH, ox0 = (r % ntx) * TW;
    __syncthreads();  // the previous tile's fragments have been loaded
    // g of 64 channels x 128 pixels; a warp's elements of one round share one channel, so
    // the bias gradient is a warp sum per round (of the FP32 g, not of its split parts)
    for (int e0 = threadIdx.x; e0 < cor * TH * TW; e0 += kSU * kThreads) {
      float g[kSU];
#pragma unroll
      for (int u = 0; u < kSU; ++u) {
        const int e = e0 + u * kThreads;
        const int p = e % (TH * TW), co = e / (TH * TW);
        const int oy = oy0 + p / TW, ox = ox0 + p % TW;
        g[u] = 0.f;
        if (e < cor * TH * TW && oy < a.Ho && ox < a.Wo)
          g[u] = grad_in(a.dy, a.y, a.y_f32, a.relu,
                         (((size_t)b * a.CO + co0 + co) * a.Ho + oy) * a.Wo + ox);
      }
#pragma unroll
      for (int u = 0; u < kSU; ++u) {
        const int e = e0 + u * kThreads;
        if (e >= cor * TH * TW) continue;  // warp-uniform (the bound is a multiple of 32)
        const int p = e % (TH * TW), co = e / (TH * TW);
        __nv_bfloat16 hi, lo;
        split_bf16(g[u], hi, lo);
        gs[co * GS + p] = hi;
        gs[(NT + co) * GS + p] = lo;
        if (blockIdx.z == 0) {
          float v = g[u];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) atomicAdd(&sdb[co], v);
        }
      }
    }
    for (int e0 = threadIdx.x; e0 < 9 * cir * TH * TW; e0 += kSU * kThreads) {
      __nv_bfloat16 v[kSU];
      int dst[kSU];
#pragma unroll
      for (int u = 0; u < kSU; ++u) {
        const int e = e0 + u * kThreads;
        const int p = e % (TH * TW), r = e / (TH * TW);  // r = tap * cir + real channel
        const int tap = cir == KC ? r / KC : r / cir;  // full chunks: constant divisor
        const int cl = r - tap * cir, ci = ci0 + cl;
        const int oy = oy0 + p / TW, ox = ox0 + p % TW;
        const int iy = oy * a.stride + tap / 3 - 1, ix = ox * a.stride + tap % 3 - 1;
        v[u] = __float2bfloat16_rn(0.f);
        dst[u] = e < 9 * cir * TH * TW ? (tap * KC + cl) * GS + p : -1;
        if (dst[u] >= 0 && oy < a.Ho && ox < a.Wo && iy >= 0 && iy < a.Hi && ix >= 0 &&
            ix < a.Wi)
          v[u] = a.x[(((size_t)b * a.CI + ci) * a.Hi + iy) * a.Wi + ix];
      }
#pragma unroll
      for (int u = 0; u < kSU; ++u)
        if (dst[u] >= 0) xs[dst[u]] = v[u];
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < TH * TW / 16; ++ks) {
      uint32_t af[2][4];
      const int arow = 16 * mb + (lane & 15), ak = 16 * ks + 8 * (lane >> 4);
#pragma unroll
      for (int part = 0; part < 2; ++part)
        ldsm_x4(af[part], smem_u32(&gs[(part * NT + arow) * GS + ak]));
      const int bk = 16 * ks + 8 * ((lane >> 3) & 1);
#pragma unroll
      for (int j = 0; j < 4; ++j) {  // n8 blocks nb0 + 2j, + 1
        uint32_t bf[4];
        const int n = 8 * (nb0 + 2 * j) + (lane & 7) + ((lane >> 4) << 3);
        ldsm_x4(bf, smem_u32(&xs[n * GS + bk]));
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          mma_bf16(acc[2 * j], af[part], bf[0], bf[1]);
          mma_bf16(acc[2 * j + 1], af[part], bf[2], bf[3]);
        }
      }
      {  // the ninth n8 block
        uint32_t bf[2];
        const int n = 8 * (nb0 + 8) + (lane & 7);
        ldsm_x2(bf, smem_u32(&xs[n * GS + bk]));
#pragma unroll
        for (int part = 0; part < 2; ++part) mma_bf16(acc[8], af[part], bf[0], bf[1]);
      }
    }
  }
  // partial sums to global: acc[j] = (co 16 mb + g (+8), n = 8 (nb0 + j) + 2t, +1)
  const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int j = 0; j < 9; ++j)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int co = co0 + 16 * mb + gq + ((q >> 1) << 3);
      const int n = 8 * (nb0 + j) + 2 * tq + (q & 1);
      const int tap = n / KC, ci = ci0 + n % KC;
      if (co < a.CO && ci < a.CI && acc[j][q] != 0.f)
        atomicAdd(&a.dw[((size_t)co * a.CI + ci) * 9 + tap], acc[j][q]);
    }
  __syncthreads();
  if (blockIdx.z == 0 && threadIdx.x < NT && co0 + threadIdx.x < a.CO && sdb[threadIdx.x] != 0.f)
    atomicAdd(&a.db[co0 + threadIdx.x], sdb[threadIdx.x]);
}

}  // namespace tc
}  // namespace cgh

using namespace cgh;

namespace {

size_t conv_smem_bytes(int mode, int sc) {
  const int PH = (tc::TH - 1) * sc + 3, PW = (tc::TW - 1) * sc + 3;
  return sizeof(__nv_bfloat16) * ((size_t)9 * tc::NT * tc::PS +
                                  (size_t)(mode == tc::MODE_DGRAD ? 2 : 1) * PH * PW * tc::PS);
}

template <int MODE>
cudaError_t launch_conv_tc(const tc::ConvArgs& a, cudaStream_t s) {
  const size_t smem = conv_smem_bytes(MODE, a.sc);
  cudaError_t e = cudaFuncSetAttribute(tc::k_conv_tc<MODE>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int tiles = ((a.Hout + tc::TH - 1) / tc::TH) * ((a.Wout + tc::TW - 1) / tc::TW);
  dim3 grid(tiles, a.B * ((a.Nc + tc::NT - 1) / tc::NT));
  prof_begin(KID_ENCODER, s);
  tc::k_conv_tc<MODE><<<grid, tc::kThreads, smem, s>>>(a);
  prof_end(KID_ENCODER, s);
  return cudaGetLastError();
}

}  // namespace

// Tensor-core forward convolution (strides 1 and 2); see encoder.cu for the entry point.
cudaError_t conv3x3_fwd_tc(int B, int CI, int Hi, int Wi, int CO, int stride,
                           const void* x, const void* w, const float* bias, int relu, void* y,
                           int y_f32, cudaStream_t s) {
  tc::ConvArgs a = {};
  a.B = B; a.Kc = CI; a.Nc = CO; a.Hin = Hi; a.Win = Wi;
  a.Hout = (Hi - 1) / stride + 1; a.Wout = (Wi - 1) / stride + 1;
  a.sc = stride; a.up = 1; a.relu = relu; a.out_f32 = y_f32;
  a.x = (const __nv_bfloat16*)x; a.w = (const __nv_bfloat16*)w; a.bias = bias; a.out = y;
  return launch_conv_tc<tc::MODE_FWD>(a, s);
}

// Tensor-core data gradient dx (f32) of a stride-`stride` convolution (strides 1 and 2).
cudaError_t conv3x3_dgrad_tc(int B, int CI, int Hi, int Wi, int CO, int stride, const void* w,
                             int relu, const void* y, int y_f32, const float* dy, float* dx,
                             cudaStream_t s) {
  tc::ConvArgs a = {};
  a.B = B; a.Kc = CO; a.Nc = CI;
  a.Hg = (Hi - 1) / stride + 1; a.Wg = (Wi - 1) / stride + 1;
  a.Hin = a.Hg * stride; a.Win = a.Wg * stride;
  a.Hout = Hi; a.Wout = Wi; a.sc = 1; a.up = stride;
  a.relu = relu; a.y_f32 = y_f32; a.out_f32 = 1;
  a.dy = dy; a.y = y; a.w = (const __nv_bfloat16*)w; a.out = dx;
  if (stride == 1) return launch_conv_tc<tc::MODE_DGRAD>(a, s);
  // stride 2: one launch over the four output parity classes
  const int tiles = ((a.Hg + tc::TH - 1) / tc::TH) * ((a.Wg + tc::TW - 1) / tc::TW);
  dim3 grid(tiles, B * ((a.Nc + tc::NT - 1) / tc::NT), 4);
  prof_begin(KID_ENCODER, s);
  tc::k_conv_dgrad2_tc<<<grid, tc::kThreads, 0, s>>>(a);
  prof_end(KID_ENCODER, s);
  return cudaGetLastError();
}

// Tensor-core weight and bias gradients (accumulated into dw, db with atomics).
cudaError_t conv3x3_wgrad_tc(int B, int CI, int Hi, int Wi, int CO, int stride, const void* x,
                             int relu, const void* y, int y_f32, const float* dy, float* dw,
                             float* db, cudaStream_t s) {
  tc::WgradArgs a = {};
  a.B = B; a.CI = CI; a.Hi = Hi; a.Wi = Wi; a.CO = CO;
  a.Ho = (Hi - 1) / stride + 1; a.Wo = (Wi - 1) / stride + 1;
  a.stride = stride; a.relu = relu; a.y_f32 = y_f32;
  a.x = (const __nv_bfloat16*)x; a.y = y; a.dy = dy; a.dw = dw; a.db = db;
  const long long tiles = (long long)B * ((a.Ho + tc::TH - 1) / tc::TH) *
                          ((a.Wo + tc::TW - 1) / tc::TW);
  const int cob = (CO + tc::NT - 1) / tc::NT, cib = (CI + tc::KC - 1) / tc::KC;
  // about two CTAs per SM over all (co block, ci chunk) pairs, at least 4 tiles each
  long long ctas = (2LL * 152 + cob * cib - 1) / (cob * cib);
  long long per = (tiles + ctas - 1) / ctas;
  if (per < 4) per = 4;
  ctas = (tiles + per - 1) / per;
  a.per_cta = (int)per;
  const size_t smem = sizeof(__nv_bfloat16) * ((size_t)2 * tc::NT + 9 * tc::KC) * tc::GS;
  cudaError_t e = cudaFuncSetAttribute(tc::k_conv_wgrad_tc,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  prof_begin(KID_ENCODER, s);
  tc::k_conv_wgrad_tc<<<dim3((unsigned)ctas, cob, cib), tc::kThreads, smem, s>>>(a);
  prof_end(KID_ENCODER, s);
  return cudaGetLastError();
}
