// fftreg.cuh -- compile-time specialised three-pass FFT engine for one CTA (sm_103a).
//
// A CTA transforms NB sequences of length N = R0 * R1 * R2 (batch slots b) with T threads.
// Elements are float2 (one complex number) or float4 (two sequences in lockstep, sharing
// every index computation and twiddle).
// Each pass is a Stockham autosort step (Govindaraju et al., SC'08): butterfly j of radix R
// with stride Ns reads positions j + r N/R, multiplies by exp(-+2 pi i r (j mod Ns)/(Ns R)),
// runs an R-point DFT in registers and writes (j - j mod Ns) R + (j mod Ns) + r Ns.  All
// sizes are template constants, so the index arithmetic folds into shifts and multiplies.
//
// Data movement is arranged so that the sequence rarely touches shared memory:
//   * the first pass reads its inputs through a caller functor (straight from global
//     memory, skipping known zeros of the padding);
//   * the last pass leaves its outputs in registers, at natural positions j + r N/R of the
//     thread that owns butterfly j -- which are exactly the inputs of a following first
//     pass of the same radix.  So a forward transform can feed a pointwise operation and
//     an inverse transform without a shared-memory round trip (spectrum x H, loss seed);
//   * only the two inner exchanges go through shared memory.  The buffer written by a
//     first pass (stride-R stores) is laid out in rows of R padded to an odd length, which
//     makes those stores bank-conflict free; the other buffer is dense.  Batch slots are
//     interleaved innermost ([position][b]).
// Twiddles: exp(-2 pi i k / (Ns R)) from one hardware sine/cosine per butterfly, higher
// powers by complex multiplication; shared-memory addresses of every pass are
// base + r * stride.
#pragma once

#include "fft.cuh"

namespace cgh {
namespace reg {

template <int R>
struct PadRows {  // odd row length for a buffer written with stride R
  static constexpr int P = (R % 2) ? R : R + 1;
};

// Butterfly geometry of one pass.
template <int N, int R, int NB, int T>
struct Geo {
  static constexpr int M = N / R;
  static constexpr int NBF = M * NB;
  static constexpr int MB = (NBF + T - 1) / T;
  static_assert(N % R == 0, "radix must divide N");
};

// layout of the buffer written by a first pass of radix RW (RW = 0: dense)
template <int RW, int NB>
__device__ __forceinline__ int lay(int a, int b) {
  if constexpr (RW == 0) {
    return a * NB + b;
  } else {
    constexpr int P = PadRows<RW>::P;
    return ((a / RW) * P + (a % RW)) * NB + b;
  }
}

template <int N, int NB, int R0, int R1, int R2>
struct BufSize {
  static constexpr int pad(int R) { return (N / R) * ((R % 2) ? R : R + 1); }
  static constexpr int mx(int a, int b) { return a > b ? a : b; }
  static constexpr int elems = mx(mx(pad(R0), pad(R2)), N) * NB;
};

template <int N, int R, int NS, bool INV, class E>
__device__ __forceinline__ void twiddle(E (&v)[R], int j, const float2* __restrict__ tw) {
  if constexpr (NS > 1) {
    // w = exp(-+2 pi i k / (NS R)) from the hardware sine/cosine (the angle lies in
    // [0, 2 pi / R), inside the range where it is accurate to ~4e-7), its powers by complex
    // multiplication; no memory access, so no load latency to hide at this occupancy
    const int k = j % NS;
    float s, c;
    __sincosf((float)k * (float)(6.28318530717958647692 / (NS * R)), &s, &c);
    float2 w = make_float2(c, INV ? s : -s);
    float2 p = w;
#pragma unroll
    for (int r = 1; r < R; ++r) {
      v[r] = cmul(v[r], p);
      if (r + 1 < R) p = cmul(p, w);
    }
  }
}

template <int N, int R, int NB, int T>
__device__ __forceinline__ bool valid(int q) {
  return (Geo<N, R, NB, T>::NBF % T == 0) || q < Geo<N, R, NB, T>::NBF;
}

// First pass (Ns = 1) with inputs from a functor f(b, a) -> float2.
template <int N, int R, int NB, int T, bool INV, class E, class F>
__device__ __forceinline__ void first_from(E (&v)[Geo<N, R, NB, T>::MB][R], F&& f) {
  using G = Geo<N, R, NB, T>;
#pragma unroll
  for (int i = 0; i < G::MB; ++i) {
    const int q = threadIdx.x + i * T;
    if (valid<N, R, NB, T>(q)) {
      const int b = q % NB, j = q / NB;
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = f(b, j + r * G::M);
      DFT<R, INV>::run(v[i]);
    }
  }
}

// Same with the functor called as f(b, j, r) for position j + r N/R, r a constant after
// unrolling: terms of an address that depend only on (b, j) are then computed once per
// butterfly, the r-dependent part folds into a constant or one multiply-add.
// ZM: registers known to be zero in every butterfly (bit r: position j + r N/R is outside the
// data for every j), whose arithmetic the pass leaves out (DFTZ); f is not called for them.
template <int N, int R, int NB, int T, bool INV, unsigned ZM = 0u, class E, class F>
__device__ __forceinline__ void first_from_jr(E (&v)[Geo<N, R, NB, T>::MB][R], F&& f) {
  using G = Geo<N, R, NB, T>;
#pragma unroll
  for (int i = 0; i < G::MB; ++i) {
    const int q = threadIdx.x + i * T;
    if (valid<N, R, NB, T>(q)) {
      const int b = (int)((unsigned)q % NB), j = (int)((unsigned)q / NB);
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (!((ZM >> r) & 1u)) v[i][r] = f(b, j, r);
      DFTZ<R, INV, ZM>::run(v[i]);
    }
  }
}

// First pass (Ns = 1) on values already in registers at positions j + r N/R (ZM: registers
// known to be zero, as for first_from_jr).
template <int N, int R, int NB, int T, bool INV, unsigned ZM = 0u, class E>
__device__ __forceinline__ void first_in_regs(E (&v)[Geo<N, R, NB, T>::MB][R]) {
  using G = Geo<N, R, NB, T>;
#pragma unroll
  for (int i = 0; i < G::MB; ++i) {
    const int q = threadIdx.x + i * T;
    if (valid<N, R, NB, T>(q)) DFTZ<R, INV, ZM>::run(v[i]);
  }
}

// Pass with stride NS reading shared memory laid out by RIN (0 = dense).
template <int N, int R, int NS, int NB, int T, bool INV, int RIN, class E>
__device__ __forceinline__ void pass_from_smem(E (&v)[Geo<N, R, NB, T>::MB][R],
                                               const E* buf,
                                               const float2* __restrict__ tw) {
  using G = Geo<N, R, NB, T>;
#pragma unroll
  for (int i = 0; i < G::MB; ++i) {
    const int q = threadIdx.x + i * T;
    if (valid<N, R, NB, T>(q)) {
      const int b = q % NB, j = q / NB;
      // positions j + r M are linear in r in both layouts (M is a multiple of RIN)
      int base, stride;
      if constexpr (RIN == 0) {
        base = j * NB + b;
        stride = G::M * NB;
      } else {
        static_assert(G::M % RIN == 0, "padded rows must tile the read stride");
        constexpr int P = PadRows<RIN>::P;
        base = ((j / RIN) * P + (j % RIN)) * NB + b;
        stride = (G::M / RIN) * P * NB;
      }
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = buf[base + r * stride];
      twiddle<N, R, NS, INV, E>(v[i], j, tw);
      DFT<R, INV>::run(v[i]);
    }
  }
}

// Store a pass's outputs (stride NS) to shared memory laid out by ROUT (0 = dense).
template <int N, int R, int NS, int NB, int T, int ROUT, class E>
__device__ __forceinline__ void pass_to_smem(const E (&v)[Geo<N, R, NB, T>::MB][R], E* buf) {
  using G = Geo<N, R, NB, T>;
#pragma unroll
  for (int i = 0; i < G::MB; ++i) {
    const int q = threadIdx.x + i * T;
    if (valid<N, R, NB, T>(q)) {
      const int b = q % NB, j = q / NB;
      int base, stride;
      if constexpr (ROUT == 0) {
        const int k = j % NS;
        base = ((j - k) * R + k) * NB + b;
        stride = NS * NB;
      } else {
        // first pass (NS = 1) into rows of R padded to P: position j R + r -> row j, col r
        static_assert(ROUT == R && NS == 1, "padded layout is written by a first pass");
        base = j * PadRows<R>::P * NB + b;
        stride = NB;
      }
#pragma unroll
      for (int r = 0; r < R; ++r) buf[base + r * stride] = v[i][r];
    }
  }
}

// Visit the registers of a last pass (natural positions a = j + r N/R): f(b, a, value&).
template <int N, int R, int NB, int T, class E, class F>
__device__ __forceinline__ void for_each(E (&v)[Geo<N, R, NB, T>::MB][R], F&& f) {
  using G = Geo<N, R, NB, T>;
#pragma unroll
  for (int i = 0; i < G::MB; ++i) {
    const int q = threadIdx.x + i * T;
    if (valid<N, R, NB, T>(q)) {
      const int b = q % NB, j = q / NB;
#pragma unroll
      for (int r = 0; r < R; ++r) f(b, j + r * G::M, v[i][r]);
    }
  }
}

// Same visit with f(b, j, r, value&) for position j + r N/R (see first_from_jr).
template <int N, int R, int NB, int T, class E, class F>
__device__ __forceinline__ void for_each_jr(E (&v)[Geo<N, R, NB, T>::MB][R], F&& f) {
  using G = Geo<N, R, NB, T>;
#pragma unroll
  for (int i = 0; i < G::MB; ++i) {
    const int q = threadIdx.x + i * T;
    if (valid<N, R, NB, T>(q)) {
      const int b = (int)((unsigned)q % NB), j = (int)((unsigned)q / NB);
#pragma unroll
      for (int r = 0; r < R; ++r) f(b, j, r, v[i][r]);
    }
  }
}

// Three-pass transform helpers.  Forward radix order (R0, R1, R2); inverse (R2, R1, R0).
// `in` holds the registers of the first pass, already transformed by first_from /
// first_in_regs; the result is left in `out` (positions j + r N/R_last).  The call starts
// with a barrier, so buf may still be in use by the previous sequence when it is entered.
template <int N, int R0, int R1, int R2, int NB, int T, bool INV, class E = float2>
struct Seq {
  static constexpr int A = INV ? R2 : R0;  // first radix
  static constexpr int B = R1;
  static constexpr int C = INV ? R0 : R2;  // last radix
  using GA = Geo<N, A, NB, T>;
  using GB = Geo<N, B, NB, T>;
  using GC = Geo<N, C, NB, T>;

  // FENCE = false: the caller guarantees that no thread still reads buf (first transform of
  // the kernel, or a barrier since the previous sequence's last pass).
  template <bool FENCE = true>
  __device__ __forceinline__ static void rest(E (&in)[GA::MB][A], E (&out)[GC::MB][C], E* buf,
                                              const float2* __restrict__ tw) {
    if (FENCE) __syncthreads();  // buf may still be read by a previous sequence's last pass
    pass_to_smem<N, A, 1, NB, T, A, E>(in, buf);
    __syncthreads();
    E mid[GB::MB][B];
    pass_from_smem<N, B, A, NB, T, INV, A, E>(mid, buf, tw);
    __syncthreads();
    pass_to_smem<N, B, A, NB, T, 0, E>(mid, buf);
    __syncthreads();
    pass_from_smem<N, C, A * B, NB, T, INV, 0, E>(out, buf, tw);
  }

  // Same with two exchange buffers (bx: first-pass layout, BufSize elements; by: dense, N NB
  // elements) and two barriers instead of four.  A buffer is rewritten only by a thread that
  // has passed a barrier which every reader of its previous contents reached after reading:
  // bx was last read by the previous sequence's middle pass (before that sequence's second
  // barrier), by by its last pass (before this sequence's first barrier).
  __device__ __forceinline__ static void rest2(E (&in)[GA::MB][A], E (&out)[GC::MB][C], E* bx,
                                               E* by, const float2* __restrict__ tw) {
    pass_to_smem<N, A, 1, NB, T, A, E>(in, bx);
    __syncthreads();
    E mid[GB::MB][B];
    pass_from_smem<N, B, A, NB, T, INV, A, E>(mid, bx, tw);
    pass_to_smem<N, B, A, NB, T, 0, E>(mid, by);
    __syncthreads();
    pass_from_smem<N, C, A * B, NB, T, INV, 0, E>(out, by, tw);
  }
};

}  // namespace reg
}  // namespace cgh
