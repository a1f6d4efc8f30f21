// blasm_reg.cuh -- BLASM row / column passes on the specialised register FFT engine.
//
// Same passes and data layouts as the generic kernels of blasm.cu (see there), with
// every transform length a template constant:
//   kr_rows_pad_fwd    global rows (zero-skipped pad) -> FFT -> blocked half grid
//   kr_cols_fwd_planes column slab -> FFT -> spectrum in registers -> for each plane
//                      x H_{c,l}/(Ny Nx) -> inverse FFT -> cropped rows
//   kr_rows_loss       inverse row FFT -> crop, |U|^2, loss partials, dL/dU seed in
//                      registers -> forward row FFT -> in place; the pass's last CTA sums
//                      the partials into the loss
//   kr_cols_bwd_planes for each plane: FFT -> x conj(H_{c,l}), accumulated in
//                      thread-private shared-memory slots -> one inverse FFT -> cropped rows
//   kr_rows_inv_crop   blocked half grid -> inverse FFT -> cropped image rows
// Where two exchange buffers fit the resident CTAs, each transform alternates between them
// (two barriers per transform instead of four).
#pragma once

#include "blasm_common.cuh"
#include "blasm_spec.h"
#include "fftreg.cuh"

// resident CTAs per SM the register allocation is sized for
#ifndef CGH_REG_MINB
#define CGH_REG_MINB(T) ((T) <= 256 ? 3 : (T) <= 512 ? 2 : 1)
#endif

namespace cgh {

template <int N, int R0, int R1, int R2, int NB, int T, class E = float2>
struct RegPlan {
  using F = reg::Seq<N, R0, R1, R2, NB, T, false, E>;
  using I = reg::Seq<N, R0, R1, R2, NB, T, true, E>;
  static constexpr int BUF = reg::BufSize<N, NB, R0, R1, R2>::elems;
  static constexpr size_t SMEM = sizeof(E) * (size_t)BUF;
  // exchange buffer + one thread-private slot per register of a last pass (column kernels)
  static constexpr size_t SLOTS = sizeof(E) * (size_t)F::GC::MB * F::C * T;
  static constexpr size_t SMEM_SLOTS = SMEM + SLOTS;
  // ... with a second, dense exchange buffer (two barriers per transform instead of four)
  static constexpr int BUF2 = N * NB;
  static constexpr size_t SMEM_SLOTS_DB = SMEM + sizeof(E) * (size_t)BUF2 + SLOTS;
  // double-buffer when `resident` CTAs still fit in the SM's 228 KB (1 KB reserved per CTA)
  static constexpr bool db_fits(int resident) {
    return (size_t)resident * (SMEM_SLOTS_DB + 1024) <= (size_t)228 * 1024;
  }
  // row kernels: exchange buffers (+ `extra` bytes of staging) without slots; only for
  // CTAs of several rows (single-row CTAs measured slower with the smaller L1 it leaves)
  static constexpr bool db_rows_fits(int resident, size_t extra) {
    return NB >= 2 && (size_t)resident * (SMEM + sizeof(E) * (size_t)BUF2 + extra + 1024) <=
                          (size_t)228 * 1024;
  }
};

// largest target stage of kr_rows_loss (NB rows of W = N / 2 floats)
template <int N, int NB>
constexpr size_t rows_stage_bytes() { return sizeof(float) * (size_t)NB * (N / 2); }

// The zeros of the padding (and of the cropped-away seed) as -0.0: a transform input known
// at compile time to be -0.0 lets the compiler drop the additions it enters (x + (-0.0) and
// (-0.0) - x are exact for every x, while x + (+0.0) is not: it maps -0.0 to +0.0); the
// results differ at most in the sign of exact zeros.
__device__ __forceinline__ float2 nz2() { return make_float2(-0.f, -0.f); }
__device__ __forceinline__ float4 nz4() { return make_float4(-0.f, -0.f, -0.f, -0.f); }

// Offset of element (row y, position a) of a column-blocked half grid (CB columns per
// block): ((a / CB) H + y) CB + a % CB.  For the positions a = j + r M of one pass, with M a
// multiple of CB, this is blk_base(j, y) + r M H: the butterfly's part is computed once and
// each element adds one product (unsigned, so the division and remainder need no sign fix-up).
template <int CB>
__device__ __forceinline__ unsigned blk_base(int j, int y, int H) {
  return ((unsigned)j / CB * (unsigned)H + (unsigned)y) * CB + (unsigned)j % CB;
}

// Image coordinate of position j + r M (0 <= j < M = N / R) of a pass over a padded length
// N, and whether it lies inside the image window [off, off + len).  CA (centred window of half
// the length: off = N / 4, len = N / 2, i.e. pad factor 2 with an even image size): the
// coordinate is j plus a compile-time constant, and registers whose positions lie wholly
// inside or wholly outside the window need no test at all (for R % 4 == 0 that is every
// register); what their values feed is then folded or dropped at compile time.
template <int N, int R, bool CA>
__device__ __forceinline__ bool in_window(int j, int r, int off, int len, int& x) {
  constexpr int M = N / R;
  if constexpr (CA) {
    x = j + (r * M - N / 4);
    if (r * M + M <= N / 4 || r * M >= 3 * N / 4) return false;  // wholly outside
    if (r * M >= N / 4 && r * M + M <= 3 * N / 4) return true;   // wholly inside
    return (unsigned)x < (unsigned)(N / 2);
  } else {
    x = j - off + r * M;
    return (unsigned)x < (unsigned)len;
  }
}

// Registers of a pass of radix R over the padded length N whose positions lie outside the
// image window for every butterfly (aligned window only; 0 otherwise): the zero padding the
// first pass of a forward transform leaves out (DFTZ).
template <int N, int R, bool CA>
constexpr unsigned outside_mask() {
  unsigned m = 0u;
  if (CA) {
    constexpr int M = N / R;
    for (int r = 0; r < R; ++r)
      if (r * M + M <= N / 4 || r * M >= 3 * N / 4) m |= 1u << r;
  }
  return m;
}

template <int N, int R0, int R1, int R2, int NB, int CB, int T, bool CA>
__global__ void __launch_bounds__(T, CGH_REG_MINB(T)) kr_rows_pad_fwd(const __grid_constant__ BlasmDev bl,
                                                     const float2* __restrict__ tw,
                                                     const float2* __restrict__ in,
                                                     float2* __restrict__ half) {
  using P = RegPlan<N, R0, R1, R2, NB, T>;
  using F = typename P::F;
  static_assert((N / F::C) % CB == 0, "column blocks must tile the output stride");
  constexpr bool DB = P::db_rows_fits(CGH_REG_MINB(T), 0);
  extern __shared__ float2 buf[];
  const int batch = blockIdx.y, y0 = blockIdx.x * NB;
  const int H = bl.H, W = bl.W, ox = bl.ox;
  const float2* src = in + (size_t)batch * H * W;
  float2 v[F::GA::MB][F::A];
  constexpr unsigned ZM = outside_mask<N, F::A, CA>();  // zero padding of the first pass
  reg::first_from_jr<N, F::A, NB, T, false, ZM>(v, [&](int b, int j, int r) {
    const int y = y0 + b;
    int x;
    const bool in_img = in_window<N, F::A, CA>(j, r, ox, W, x);
    return (in_img && y < H) ? __ldg(&src[(size_t)y * W + x]) : nz2();
  });
  float2 out[F::GC::MB][F::C];
  if constexpr (DB) F::rest2(v, out, buf, buf + P::BUF, tw);
  else F::template rest<false>(v, out, buf, tw);  // first transform: no earlier reader
  float2* dst = half + (size_t)batch * H * N;
  const unsigned MH = (unsigned)(N / F::C) * (unsigned)H;
  reg::for_each_jr<N, F::C, NB, T>(out, [&](int b, int j, int r, float2& val) {
    const int y = y0 + b;
    if (y < H) dst[blk_base<CB>(j, y, H) + (unsigned)r * MH] = val;
  });
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst))),
               "l"(gmem_src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// largest addend stage of kr_rows_inv_crop (NB rows of W = N / 2 complex values)
template <int N, int NB>
constexpr size_t rows_addend_bytes() { return sizeof(float2) * (size_t)NB * (N / 2); }

// accum = 0: out = the cropped rows.  accum = 1: out += them, the CTA's NB rows of `out`
// staged in shared memory (after the exchange buffers) by asynchronous 16-byte copies issued
// before the transform, so their latency hides behind it (needs W even and a 16-byte
// aligned `out`); accum = 2: out += them with plain loads in the epilogue.
template <int N, int R0, int R1, int R2, int NB, int CB, int T, bool ACC, bool CA>
__global__ void __launch_bounds__(T, CGH_REG_MINB(T)) kr_rows_inv_crop(const __grid_constant__ BlasmDev bl,
                                                      const float2* __restrict__ tw,
                                                      const float2* __restrict__ half,
                                                      float2* __restrict__ out, int accum) {
  using P = RegPlan<N, R0, R1, R2, NB, T>;
  using I = typename P::I;
  static_assert((N / I::A) % CB == 0, "column blocks must tile the input stride");
  constexpr bool DB = P::db_rows_fits(CGH_REG_MINB(T), ACC ? rows_addend_bytes<N, NB>() : 0);
  if (!ACC) accum = 0;
  extern __shared__ float2 buf[];
  const int batch = blockIdx.y, y0 = blockIdx.x * NB;
  const int H = bl.H, W = bl.W, ox = bl.ox;
  const float2* src = half + (size_t)batch * H * N;
  float2* dst = out + (size_t)batch * H * W;
  float2* asm_ = buf + P::BUF + (DB ? P::BUF2 : 0);  // addend stage (accum = 1)
  if (accum == 1) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (y0 + b >= H) break;
      const float2* row = dst + (size_t)(y0 + b) * W;
      for (int x = 2 * threadIdx.x; x < W; x += 2 * T) cp_async16(&asm_[b * W + x], &row[x]);
    }
    cp_async_commit();
  }
  float2 v[I::GA::MB][I::A];
  const unsigned MH = (unsigned)(N / I::A) * (unsigned)H;
  reg::first_from_jr<N, I::A, NB, T, true>(v, [&](int b, int j, int r) {
    const int y = y0 + b;
    return y < H ? __ldg(&src[blk_base<CB>(j, y, H) + (unsigned)r * MH]) : make_float2(0.f, 0.f);
  });
  float2 u[I::GC::MB][I::C];
  if constexpr (DB) I::rest2(v, u, buf, buf + P::BUF, tw);
  else I::template rest<false>(v, u, buf, tw);  // first transform: no earlier reader
  if (accum == 1) {
    cp_async_wait_all();
    __syncthreads();
  }
  reg::for_each_jr<N, I::C, NB, T>(u, [&](int b, int j, int r, float2& val) {
    const int y = y0 + b;
    int x;
    if (in_window<N, I::C, CA>(j, r, ox, W, x) && y < H) {
      float2* o = &dst[(size_t)y * W + x];
      if (accum == 1) val = cadd(asm_[b * W + x], val);
      else if (accum == 2) val = cadd(*o, val);  // each element read and written by one thread
      *o = val;
    }
  });
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// tstage = 1: the CTA's NB target rows are copied into shared memory (after the exchange
// buffer) with asynchronous 16-byte copies issued before the inverse transform, so their
// latency hides behind it (needs a 16-byte aligned target and W % 4 == 0).
// GRAD = false: loss only (the forward-only pass), compiled without the forward transform
// so that none of its register pressure reaches the loss-only kernel.  GENERAL = false: the
// intensity MSE (weight 1) with the target staged (tstage = 1), the common case, compiled
// without the runtime choices, which keeps the gradient kernel inside its 64 registers.
template <int N, int R0, int R1, int R2, int NB, int CB, int T, bool GRAD, bool GENERAL, bool CA>
__global__ void __launch_bounds__(T, CGH_REG_MINB(T)) kr_rows_loss(const __grid_constant__ BlasmDev bl,
                                                  const float2* __restrict__ tw,
                                                  float2* __restrict__ V,
                                                  const float* __restrict__ target,
                                                  float* __restrict__ partials,
                                                  int tstage, float* __restrict__ loss_out,
                                                  int* __restrict__ ticket, double inv_norm,
                                                  int extra) {
  using P = RegPlan<N, R0, R1, R2, NB, T>;
  using F = typename P::F;
  using I = typename P::I;
  static_assert(I::C == F::A, "inverse must end where the forward starts");
  static_assert(T % 32 == 0, "the loss reduction shuffles over whole warps");
  static_assert((N / I::A) % CB == 0 && (N / F::C) % CB == 0,
                "column blocks must tile the input and output strides");
  constexpr bool DB = P::db_rows_fits(CGH_REG_MINB(T), rows_stage_bytes<N, NB>());
  extern __shared__ float2 buf[];
  __shared__ float red[32];
  const int batch = blockIdx.y, y0 = blockIdx.x * NB;  // batch = l * C + c (kernel planes)
  const int H = bl.H, W = bl.W, ox = bl.ox;
  const int plane = bl.plane[batch / bl.C];  // the hologram plane: target, mask
  float2* half = V + (size_t)batch * H * N;
  const float* tg = target + ((size_t)plane * bl.C + batch % bl.C) * H * W;
  float2* by = buf + P::BUF;  // second exchange buffer (DB)
  float* tsm = reinterpret_cast<float*>(buf + P::BUF + (DB ? P::BUF2 : 0));
  if (!GENERAL) tstage = 1;
  if (tstage) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (y0 + b >= H) break;
      const float* row = tg + (size_t)(y0 + b) * W;
      for (int x = 4 * threadIdx.x; x < W; x += 4 * T) cp_async16(&tsm[b * W + x], &row[x]);
    }
    cp_async_commit();
  }
  float2 v[I::GA::MB][I::A];
  const unsigned MHI = (unsigned)(N / I::A) * (unsigned)H;
  reg::first_from_jr<N, I::A, NB, T, true>(v, [&](int b, int j, int r) {
    const int y = y0 + b;
    return y < H ? __ldg(&half[blk_base<CB>(j, y, H) + (unsigned)r * MHI]) : make_float2(0.f, 0.f);
  });
  float2 u[I::GC::MB][I::C];
  if constexpr (DB) I::rest2(v, u, buf, by, tw);
  else I::template rest<false>(v, u, buf, tw);  // first transform: no earlier reader
  if (tstage) {
    cp_async_wait_all();
    __syncthreads();
  }
  const float gscale = 4.0f / ((float)bl.Ltot * (float)bl.C * (float)H * (float)W);
  float acc = 0.f;
  reg::for_each_jr<N, I::C, NB, T>(u, [&](int b, int j, int r, float2& val) {
    const int y = y0 + b;
    int x;
    if (in_window<N, I::C, CA>(j, r, ox, W, x) && y < H) {
      const float I_ = fmaf(val.x, val.x, val.y * val.y);
      const float t_ = tstage ? tsm[b * W + x] : __ldg(&tg[(size_t)y * W + x]);
      const float d = I_ - t_;
      const float wd = GENERAL ? loss_weight(bl, plane, y, x, t_) * d : d;
      acc = fmaf(wd, d, acc);
      val = cscale(val, gscale * wd);
    } else {
      val = nz2();
    }
  });
  const float tot = block_sum(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = tot;
  if constexpr (GRAD) {
    // the seed is zero outside the crop: the forward transform's first pass leaves it out
    reg::first_in_regs<N, F::A, NB, T, false, outside_mask<N, I::C, CA>()>(u);
    float2 w[F::GC::MB][F::C];
    // block_sum's barriers follow the inverse transform's last reads of buf
    if constexpr (DB) F::rest2(u, w, buf, by, tw);
    else F::template rest<false>(u, w, buf, tw);
    // row and base re-derived from the block index (fewer values live across the transform)
    float2* hv = V + (size_t)blockIdx.y * bl.H * N;
    const unsigned MHF = (unsigned)(N / F::C) * (unsigned)bl.H;
    reg::for_each_jr<N, F::C, NB, T>(w, [&](int b, int j, int r, float2& val) {
      const int y = blockIdx.x * NB + b;
      if (y < bl.H) hv[blk_base<CB>(j, y, bl.H) + (unsigned)r * MHF] = val;
    });
  }
  // at the end, where no transform state is live
  if (loss_out)
    finalize_if_last(partials, gridDim.x * gridDim.y, gridDim.x * gridDim.y + extra, inv_norm,
                     loss_out, ticket);
}

// Column kernels work on float4 elements: columns 2 s and 2 s + 1 of the CTA's column block
// transformed in lockstep (NB float4 slots, CB = 2 NB columns per CTA).  The 1 / (Ny Nx)
// of the inverse transform is applied once per element outside (to the parked spectrum in
// the forward kernel, to the plane sum in the backward one), so H is taken with scale 1;
// `inband` (both columns inside the band, every row inside it, no aperture: uniform across
// a CTA of one column pair) drops the mask.
template <bool CONJ>
__device__ __forceinline__ float4 transfer_pair(const BlasmDev& bl, const TFConst& t,
                                                const TFCol& c0, const TFCol& c1, int sy,
                                                float4 v, bool inband) {
  float2 h0, h1;
  if (inband) {
    h0 = transfer_inband(t, c0, sy);
    h1 = transfer_inband(t, c1, sy);
  } else {
    h0 = transfer_series(bl, t, c0, sy, 1.0f);
    h1 = transfer_series(bl, t, c1, sy, 1.0f);
  }
  return CONJ ? pack(cmulc(lo(v), h0), cmulc(hi(v), h1)) : pack(cmul(lo(v), h0), cmul(hi(v), h1));
}

// every row of the transform inside the band and no aperture (then only the column's own
// band membership remains to check)
template <int N>
__device__ __forceinline__ bool rows_inband(const BlasmDev& bl, const TFConst& t) {
  return bl.aperture2 <= 0.f && t.ky_max >= N / 2;
}

// INBAND: every bin of every channel and plane lies inside the band and there is no
// aperture (checked on the host), so the masked evaluation of H is not even compiled.
template <int N, int R0, int R1, int R2, int NB, int T, int MINB, bool INBAND, bool CA>
__global__ void __launch_bounds__(T, MINB) kr_cols_fwd_planes(const __grid_constant__ BlasmDev bl,
                                                        const float2* __restrict__ tw,
                                                        const float2* __restrict__ Y,
                                                        float2* __restrict__ V) {
  using P = RegPlan<N, R0, R1, R2, NB, T, float4>;
  using F = typename P::F;
  using I = typename P::I;
  static_assert(F::C == I::A, "inverse must start where the forward ends");
  constexpr int CB = 2 * NB;
  constexpr bool DB = P::db_fits(MINB);
  extern __shared__ float4 buf4[];
  float4* by = buf4 + P::BUF;  // second exchange buffer (DB)
  const int c = blockIdx.y, kb = blockIdx.x;
  const int H = bl.H, Nx = bl.Nx, C = bl.C, oy = bl.oy;
  const float4* src = reinterpret_cast<const float4*>(Y + (size_t)c * H * Nx + (size_t)kb * H * CB);
  float4 v[F::GA::MB][F::A];
  constexpr unsigned ZM = outside_mask<N, F::A, CA>();  // zero padding of the first pass
  reg::first_from_jr<N, F::A, NB, T, false, ZM>(v, [&](int b, int j, int r) {
    int y;
    return in_window<N, F::A, CA>(j, r, oy, H, y) ? __ldg(&src[y * NB + b])
                                                   : nz4();
  });
  // the spectrum is parked in thread-private shared-memory slots (one 16-byte load per
  // element per plane) so that the inverse passes get the registers
  float4* spec = buf4 + P::BUF + (DB ? P::BUF2 : 0);
  {
    float4 S[F::GC::MB][F::C];
    if constexpr (DB) F::rest2(v, S, buf4, by, tw); else F::rest(v, S, buf4, tw);
#pragma unroll
    for (int i = 0; i < F::GC::MB; ++i)
#pragma unroll
      for (int r = 0; r < F::C; ++r)
        spec[(i * F::C + r) * T + threadIdx.x] = cscale(S[i][r], bl.inv_ntot);
  }
  for (int l = 0; l < bl.L; ++l) {
    const TFConst& tc = bl.tf[c * bl.Ltot + bl.plane[l]];
    float4 Z[I::GA::MB][I::A];
#pragma unroll
    for (int i = 0; i < I::GA::MB; ++i) {
      const int q = threadIdx.x + i * T;
      if (reg::valid<N, I::A, NB, T>(q)) {
        const int b = q % NB, j = q / NB;
        const TFCol c0 = tf_col(tc, signed_index(kb * CB + 2 * b, Nx));
        const TFCol c1 = tf_col(tc, signed_index(kb * CB + 2 * b + 1, Nx));
        const bool inband = INBAND || (rows_inband<N>(bl, tc) && c0.in_band && c1.in_band);
#pragma unroll
        for (int r = 0; r < I::A; ++r)
          Z[i][r] = transfer_pair<false>(bl, tc, c0, c1, signed_index(j + r * I::GA::M, N),
                                         spec[(i * I::A + r) * T + threadIdx.x], inband);
      }
    }
    reg::first_in_regs<N, I::A, NB, T, true>(Z);
    float4 u[I::GC::MB][I::C];
    if constexpr (DB) I::rest2(Z, u, buf4, by, tw); else I::rest(Z, u, buf4, tw);
    float4* dst = reinterpret_cast<float4*>(V + (size_t)(l * C + c) * H * Nx + (size_t)kb * H * CB);
    reg::for_each_jr<N, I::C, NB, T>(u, [&](int b, int j, int r, float4& val) {
      int y;
      if (in_window<N, I::C, CA>(j, r, oy, H, y)) dst[y * NB + b] = val;
    });
  }
}

template <int N, int R0, int R1, int R2, int NB, int T, int MINB, bool INBAND, bool CA>
__global__ void __launch_bounds__(T, MINB) kr_cols_bwd_planes(const __grid_constant__ BlasmDev bl,
                                                        const float2* __restrict__ tw,
                                                        const float2* __restrict__ G,
                                                        float2* __restrict__ D) {
  using P = RegPlan<N, R0, R1, R2, NB, T, float4>;
  using F = typename P::F;
  using I = typename P::I;
  static_assert(F::C == I::A, "inverse must start where the forward ends");
  constexpr int CB = 2 * NB;
  constexpr bool DB = P::db_fits(MINB);
  extern __shared__ float4 buf4[];
  float4* by = buf4 + P::BUF;  // second exchange buffer (DB)
  const int c = blockIdx.y, kb = blockIdx.x;
  const int H = bl.H, Nx = bl.Nx, C = bl.C, oy = bl.oy;
  // the running sum over planes lives in thread-private shared-memory slots
  float4* accs = buf4 + P::BUF + (DB ? P::BUF2 : 0);
  for (int l = 0; l < bl.L; ++l) {
    const TFConst& tc = bl.tf[c * bl.Ltot + bl.plane[l]];
    const float4* src =
        reinterpret_cast<const float4*>(G + (size_t)(l * C + c) * H * Nx + (size_t)kb * H * CB);
    if (l + 1 < bl.L) {
      // the next plane's slab (contiguous) into L2 while this one is transformed
      const char* nxt = reinterpret_cast<const char*>(G + (size_t)((l + 1) * C + c) * H * Nx +
                                                      (size_t)kb * H * CB);
      for (int i = threadIdx.x; i * 128 < H * CB * 8; i += T) prefetch_l2(nxt + i * 128);
    }
    float4 v[F::GA::MB][F::A];
    constexpr unsigned ZM = outside_mask<N, F::A, CA>();  // zero padding of the first pass
    reg::first_from_jr<N, F::A, NB, T, false, ZM>(v, [&](int b, int j, int r) {
      int y;
      return in_window<N, F::A, CA>(j, r, oy, H, y) ? __ldg(&src[y * NB + b])
                                                     : nz4();
    });
    float4 S[F::GC::MB][F::C];
    if constexpr (DB) F::rest2(v, S, buf4, by, tw); else F::rest(v, S, buf4, tw);
#pragma unroll
    for (int i = 0; i < F::GC::MB; ++i) {
      const int q = threadIdx.x + i * T;
      if (reg::valid<N, F::C, NB, T>(q)) {
        const int b = q % NB, j = q / NB;
        const TFCol c0 = tf_col(tc, signed_index(kb * CB + 2 * b, Nx));
        const TFCol c1 = tf_col(tc, signed_index(kb * CB + 2 * b + 1, Nx));
        const bool inband = INBAND || (rows_inband<N>(bl, tc) && c0.in_band && c1.in_band);
#pragma unroll
        for (int r = 0; r < F::C; ++r) {
          const float4 t = transfer_pair<true>(bl, tc, c0, c1, signed_index(j + r * F::GC::M, N),
                                               S[i][r], inband);
          float4& a = accs[(i * F::C + r) * T + threadIdx.x];
          a = (l == 0) ? t : cadd(a, t);
        }
      }
    }
  }
  float4 acc[I::GA::MB][I::A];
#pragma unroll
  for (int i = 0; i < I::GA::MB; ++i)
#pragma unroll
    for (int r = 0; r < I::A; ++r) acc[i][r] = cscale(accs[(i * I::A + r) * T + threadIdx.x], bl.inv_ntot);
  reg::first_in_regs<N, I::A, NB, T, true>(acc);
  float4 u[I::GC::MB][I::C];
  if constexpr (DB) I::rest2(acc, u, buf4, by, tw); else I::rest(acc, u, buf4, tw);
  float4* dst = reinterpret_cast<float4*>(D + (size_t)c * H * Nx + (size_t)kb * H * CB);
  reg::for_each_jr<N, I::C, NB, T>(u, [&](int b, int j, int r, float4& val) {
    int y;
    if (in_window<N, I::C, CA>(j, r, oy, H, y)) dst[y * NB + b] = val;
  });
}

// ---------------------------------------------------------------- host launchers
template <class K>
inline cudaError_t reg_set_smem(K kernel, size_t bytes, int resident) {
  cudaError_t e =
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  // ask for just the shared memory `resident` CTAs need (plus the 1 KB the system reserves
  // per CTA): the split is otherwise chosen per launch and can cap residency at one CTA,
  // while the maximum carve-out leaves L1 too small for the spill traffic
  const size_t per_sm = 228u * 1024u;
  size_t pct = (100u * (size_t)resident * (bytes + 1024u) + per_sm - 1) / per_sm;
  if (pct > 100u) pct = 100u;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)pct);
}

template <int N, int R0, int R1, int R2, int NB, int CB, int T, bool CA>
cudaError_t reg_rows_launch_ca(int kind, const cgh_plan* p, const SpecRowArgs* a,
                               const BlasmDev& bl, cudaStream_t s) {
  using P = RegPlan<N, R0, R1, R2, NB, T>;
  constexpr size_t smem_db =
      P::SMEM + (P::db_rows_fits(CGH_REG_MINB(T), 0) ? sizeof(float2) * (size_t)P::BUF2 : 0);
  // accumulating rows_inv_crop: exchange buffers as that kernel sizes them, plus the stage
  constexpr bool db_acc = P::db_rows_fits(CGH_REG_MINB(T), rows_addend_bytes<N, NB>());
  constexpr size_t smem_acc = P::SMEM + (db_acc ? sizeof(float2) * (size_t)P::BUF2 : 0);
  dim3 grid((p->H + NB - 1) / NB, a->batches);
  const float2* tw = p->fx.tw;
  cudaError_t e = cudaSuccess;
  switch (kind) {
    case SPEC_ROWS_PAD_FWD: {
      auto k = kr_rows_pad_fwd<N, R0, R1, R2, NB, CB, T, CA>;
      e = reg_set_smem(k, smem_db, CGH_REG_MINB(T));
      if (e != cudaSuccess) return e;
      prof_begin(KID_ROWS_PAD_FWD, s);
      k<<<grid, T, smem_db, s>>>(bl, tw, a->in, a->out);
      prof_end(KID_ROWS_PAD_FWD, s);
      break;
    }
    case SPEC_ROWS_INV_CROP: {
      auto k = a->accumulate ? kr_rows_inv_crop<N, R0, R1, R2, NB, CB, T, true, CA>
                             : kr_rows_inv_crop<N, R0, R1, R2, NB, CB, T, false, CA>;
      const bool stage = a->accumulate && p->W % 2 == 0 &&
                         (reinterpret_cast<uintptr_t>(a->out) & 15u) == 0;
      const int accum = a->accumulate ? (stage ? 1 : 2) : 0;
      const size_t smem = a->accumulate ? smem_acc + (stage ? sizeof(float2) * (size_t)NB * p->W : 0)
                                        : smem_db;
      e = reg_set_smem(k, smem, CGH_REG_MINB(T));
      if (e != cudaSuccess) return e;
      prof_begin(KID_ROWS_INV_CROP, s);
      k<<<grid, T, smem, s>>>(bl, tw, a->in, a->out, accum);
      prof_end(KID_ROWS_INV_CROP, s);
      break;
    }
    default: {
      const int tstage = (p->W % 4 == 0 && (reinterpret_cast<uintptr_t>(a->target) & 15u) == 0);
      const bool general = !tstage || bl.loss_kind != 0;
      auto k = a->want_grad ? (general ? kr_rows_loss<N, R0, R1, R2, NB, CB, T, true, true, CA>
                                       : kr_rows_loss<N, R0, R1, R2, NB, CB, T, true, false, CA>)
                            : (general ? kr_rows_loss<N, R0, R1, R2, NB, CB, T, false, true, CA>
                                       : kr_rows_loss<N, R0, R1, R2, NB, CB, T, false, false, CA>);
      constexpr bool db = P::db_rows_fits(CGH_REG_MINB(T), rows_stage_bytes<N, NB>());
      const size_t smem = P::SMEM + (db ? sizeof(float2) * (size_t)P::BUF2 : 0) +
                          (tstage ? sizeof(float) * (size_t)NB * p->W : 0);
      e = reg_set_smem(k, smem, CGH_REG_MINB(T));
      if (e != cudaSuccess) return e;
      prof_begin(KID_ROWS_LOSS, s);
      k<<<grid, T, smem, s>>>(bl, tw, a->out, a->target, a->partials, tstage,
                              a->loss_out, a->ticket, a->inv_norm, a->extra);
      prof_end(KID_ROWS_LOSS, s);
      break;
    }
  }
  return cudaGetLastError();
}

// The row kernels come in two forms: with the image window aligned to the passes' geometry
// (W = N / 2, ox = N / 4: pad factor 2, compile-time crop tests) and the general one.
template <int N, int R0, int R1, int R2, int NB, int CB, int T>
cudaError_t reg_rows_launch(int kind, const cgh_plan* p, const SpecRowArgs* a, cudaStream_t s) {
  const BlasmDev& bl = a->bl ? *a->bl : p->bl;
  if (2 * bl.W == N && 4 * bl.ox == N)
    return reg_rows_launch_ca<N, R0, R1, R2, NB, CB, T, true>(kind, p, a, bl, s);
  return reg_rows_launch_ca<N, R0, R1, R2, NB, CB, T, false>(kind, p, a, bl, s);
}

// (R0, R1, R2): radix order of the forward-model kernel; (Q0, Q1, Q2): that of the adjoint one
// (each kernel runs its own complete transforms, so the two orders are independent).
template <int N, int R0, int R1, int R2, int Q0, int Q1, int Q2, int NB, int T, int MINBF,
          int MINBB, bool CA>
cudaError_t reg_cols_launch_ca(int kind, const cgh_plan* p, const BlasmDev& bl, const float2* in,
                               float2* out, cudaStream_t s) {
  using P = RegPlan<N, R0, R1, R2, NB, T, float4>;
  using PB = RegPlan<N, Q0, Q1, Q2, NB, T, float4>;
  static_assert(P::F::C == P::I::A, "slot layout shared by the forward end and inverse start");
  static_assert(PB::F::C == PB::I::A, "slot layout shared by the forward end and inverse start");
  constexpr int MINB = MINBF;  // in-band forward kernel
  constexpr size_t smem = P::db_fits(MINB) ? P::SMEM_SLOTS_DB : P::SMEM_SLOTS;
  constexpr size_t smem_m = P::db_fits(MINBB) ? P::SMEM_SLOTS_DB : P::SMEM_SLOTS;
  constexpr size_t smem_b = PB::db_fits(MINBB) ? PB::SMEM_SLOTS_DB : PB::SMEM_SLOTS;
  dim3 grid(bl.Nx / (2 * NB), p->C);
  const float2* tw = p->fy.tw;
  cudaError_t e = cudaSuccess;
  bool all_in = bl.aperture2 <= 0.f;
  for (int c = 0; c < bl.C; ++c)
    for (int l = 0; l < bl.L; ++l) {
      const TFConst& t = bl.tf[c * bl.Ltot + bl.plane[l]];
      all_in = all_in && t.kx_max >= bl.Nx / 2 && t.ky_max >= N / 2;
    }
  if (kind == SPEC_COLS_FWD_PLANES) {
    // MINBF applies to the in-band form (the masked one keeps the general residency)
    auto k = all_in ? kr_cols_fwd_planes<N, R0, R1, R2, NB, T, MINB, true, CA>
                    : kr_cols_fwd_planes<N, R0, R1, R2, NB, T, MINBB, false, CA>;
    const size_t sm = all_in ? smem : smem_m;
    e = reg_set_smem(k, sm, all_in ? MINB : MINBB);
    if (e != cudaSuccess) return e;
    prof_begin(KID_COLS_FWD_PLANES, s);
    k<<<grid, T, sm, s>>>(bl, tw, in, out);
    prof_end(KID_COLS_FWD_PLANES, s);
  } else {
    auto k = all_in ? kr_cols_bwd_planes<N, Q0, Q1, Q2, NB, T, MINBB, true, CA>
                    : kr_cols_bwd_planes<N, Q0, Q1, Q2, NB, T, MINBB, false, CA>;
    e = reg_set_smem(k, smem_b, MINBB);
    if (e != cudaSuccess) return e;
    prof_begin(KID_COLS_BWD_PLANES, s);
    k<<<grid, T, smem_b, s>>>(bl, tw, in, out);
    prof_end(KID_COLS_BWD_PLANES, s);
  }
  return cudaGetLastError();
}

// Column kernels, like the row kernels, come with the image window aligned (H = N / 2,
// oy = N / 4) and in the general form.
// MINBA: resident CTAs per SM of the aligned-window, in-band forward kernel (its dead cropped
// outputs and known zero inputs free registers, so it can fit more CTAs than the others).
template <int N, int R0, int R1, int R2, int Q0, int Q1, int Q2, int NB, int T, int MINB,
          int MINBA>
cudaError_t reg_cols_launch(int kind, const cgh_plan* p, const BlasmDev* blp, const float2* in,
                            float2* out, cudaStream_t s) {
  const BlasmDev& bl = blp ? *blp : p->bl;
  if (2 * bl.H == N && 4 * bl.oy == N)
    return reg_cols_launch_ca<N, R0, R1, R2, Q0, Q1, Q2, NB, T, MINBA, MINB, true>(kind, p, bl,
                                                                                  in, out, s);
  return reg_cols_launch_ca<N, R0, R1, R2, Q0, Q1, Q2, NB, T, MINB, MINB, false>(kind, p, bl, in,
                                                                                out, s);
}

}  // namespace cgh

// One row / column specialisation entry for the spec translation units:
//   N = R0 * R1 * R2, NB transforms per CTA, CB column-block layout (rows), T threads.
#define CGH_ROW_SPEC(N, R0, R1, R2, NB, CB, T)                                              \
  if (N_ == N && RB_ == NB && CB_ == CB) {                                                  \
    if (!dry) *err = cgh::reg_rows_launch<N, R0, R1, R2, NB, CB, T>(kind, p, a, s);         \
    return true;                                                                            \
  }
//   column entries: NB float4 slots per CTA, i.e. CB = 2 NB columns; MINB resident CTAs per
//   SM the registers are sized for.
#define CGH_COL_SPEC(N, R0, R1, R2, NB, T, MINB) CGH_COL_SPEC_A(N, R0, R1, R2, NB, T, MINB, MINB)
//   ... with MINBA resident CTAs for the aligned-window forward kernel
#define CGH_COL_SPEC_A(N, R0, R1, R2, NB, T, MINB, MINBA) \
  CGH_COL_SPEC_FB(N, R0, R1, R2, R0, R1, R2, NB, T, MINB, MINBA)
//   ... with radix order (Q0, Q1, Q2) for the adjoint kernel
#define CGH_COL_SPEC_FB(N, R0, R1, R2, Q0, Q1, Q2, NB, T, MINB, MINBA)                       \
  if (N_ == N && CB_ == 2 * (NB)) {                                                         \
    if (!dry)                                                                               \
      *err = cgh::reg_cols_launch<N, R0, R1, R2, Q0, Q1, Q2, NB, T, MINB, MINBA>(kind, p, bl, \
                                                                               in, out, s);  \
    return true;                                                                            \
  }
