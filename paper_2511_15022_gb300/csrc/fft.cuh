// fft.cuh -- shared-memory mixed-radix FFT for one CTA (sm_103a).
//
// A CTA holds `nb` independent transforms of length n in shared memory, one per batch
// slot b, at swizzled addresses sidx(b, i) = b * bs + i + (i >> 4) (the extra slot every
// 16 complex values breaks the power-of-two strides of the first Stockham pass across
// the 32 banks).  Each pass of radix R runs the Stockham autosort step (Govindaraju et
// al., "High performance discrete Fourier transforms on graphics processors", SC'08):
// butterfly j reads elements j + r n/R, multiplies by exp(-+2 pi i r (j mod Ns) / (Ns R)),
// runs an R-point DFT in registers and writes (j - j mod Ns) R + (j mod Ns) + r Ns.
// Passes run in place: every thread first reads and transforms its butterflies (at most
// MAXB of them), the CTA synchronises, then everybody writes.
//
// The R-point DFTs are unrolled at compile time: radices 2, 3, 4, 5 are written out;
// larger radices are Cooley-Tukey compositions R = A * B whose inner twiddles are
// compile-time constants (evaluated below from the Taylor series of sin and cos on
// [0, pi/4], with exact values at multiples of pi/4 so trivial twiddles cost nothing).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace cgh {

// ---------------------------------------------------------------- compile-time trig
namespace ct {
constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr double sin_series(double x) {
  double x2 = x * x, term = x, sum = x;
  for (int k = 1; k < 14; ++k) {
    term *= -x2 / ((2.0 * k) * (2.0 * k + 1.0));
    sum += term;
  }
  return sum;
}
constexpr double cos_series(double x) {
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int k = 1; k < 14; ++k) {
    term *= -x2 / ((2.0 * k - 1.0) * (2.0 * k));
    sum += term;
  }
  return sum;
}
// cos and sin of 2 pi k / n: quadrant from integers, remainder angle in [0, pi/2)
// folded to [0, pi/4].
constexpr void cs2pi(long k, long n, double& c, double& s) {
  long m = ((k % n) + n) % n;
  long quad = (4 * m) / n;
  long rem = 4 * m - quad * n;  // angle = (quad + rem/n) * pi/2
  double cr = 1.0, sr = 0.0;
  if (rem != 0) {
    if (2 * rem <= n) {
      double x = (kPi / 2.0) * (double)rem / (double)n;
      cr = cos_series(x);
      sr = sin_series(x);
    } else {
      double x = (kPi / 2.0) * (double)(n - rem) / (double)n;
      cr = sin_series(x);
      sr = cos_series(x);
    }
  }
  switch (quad) {
    case 0: c = cr; s = sr; break;
    case 1: c = -sr; s = cr; break;
    case 2: c = -cr; s = -sr; break;
    default: c = sr; s = -cr; break;
  }
}
constexpr double cos2pi(long k, long n) { double c = 0, s = 0; cs2pi(k, n, c, s); return c; }
constexpr double sin2pi(long k, long n) { double c = 0, s = 0; cs2pi(k, n, c, s); return s; }
}  // namespace ct

template <int I, int N, class F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (I < N) {
    f(std::integral_constant<int, I>());
    sfor<I + 1, N>(f);
  }
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// y + s x
__device__ __forceinline__ float2 caxpy(float s, float2 x, float2 y) {
  return make_float2(fmaf(s, x.x, y.x), fmaf(s, x.y, y.y));
}
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 z) {
  return INV ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
}

// multiply by exp(-+2 pi i K / N) with compile-time K, N (sign: - forward, + inverse)
template <int K, int N, bool INV>
__device__ __forceinline__ float2 twmul(float2 x) {
  constexpr long km = ((long)K % N + N) % N;
  if constexpr ((8 * km) % N == 0) {
    constexpr int o8 = (int)((8 * km) / N);
    constexpr int o = INV ? (8 - o8) % 8 : o8;  // forward angle -2 pi o / 8
    constexpr float r = 0.70710678118654752440f;
    if constexpr (o == 0) return x;
    else if constexpr (o == 1) return make_float2((x.x + x.y) * r, (x.y - x.x) * r);
    else if constexpr (o == 2) return make_float2(x.y, -x.x);
    else if constexpr (o == 3) return make_float2((x.y - x.x) * r, -(x.x + x.y) * r);
    else if constexpr (o == 4) return make_float2(-x.x, -x.y);
    else if constexpr (o == 5) return make_float2(-(x.x + x.y) * r, (x.x - x.y) * r);
    else if constexpr (o == 6) return make_float2(-x.y, x.x);
    else return make_float2((x.x - x.y) * r, (x.x + x.y) * r);
  } else {
    constexpr float c = (float)ct::cos2pi(K, N);
    constexpr float s = INV ? (float)ct::sin2pi(K, N) : -(float)ct::sin2pi(K, N);
    return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
  }
}

// float4 = two complex numbers (x, y) and (z, w) transformed in lockstep (two columns that
// share one butterfly's index arithmetic and twiddles).
__device__ __forceinline__ float2 lo(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi(float4 a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ float4 pack(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ float4 cadd(float4 a, float4 b) { return pack(cadd(lo(a), lo(b)), cadd(hi(a), hi(b))); }
__device__ __forceinline__ float4 csub(float4 a, float4 b) { return pack(csub(lo(a), lo(b)), csub(hi(a), hi(b))); }
__device__ __forceinline__ float4 cmul(float4 a, float2 b) { return pack(cmul(lo(a), b), cmul(hi(a), b)); }
__device__ __forceinline__ float4 cscale(float4 a, float s) { return pack(cscale(lo(a), s), cscale(hi(a), s)); }
__device__ __forceinline__ float4 caxpy(float s, float4 x, float4 y) {
  return pack(caxpy(s, lo(x), lo(y)), caxpy(s, hi(x), hi(y)));
}
template <bool INV>
__device__ __forceinline__ float4 mul_mi(float4 z) { return pack(mul_mi<INV>(lo(z)), mul_mi<INV>(hi(z))); }
template <int K, int N, bool INV>
__device__ __forceinline__ float4 twmul(float4 x) {
  return pack(twmul<K, N, INV>(lo(x)), twmul<K, N, INV>(hi(x)));
}

// ---------------------------------------------------------------- R-point DFT codelets
// DFT<R, INV>::run(v) transforms R elements in place; E is float2 (one complex number) or
// float4 (two in lockstep).
template <int R, bool INV>
struct DFT;

template <bool INV>
struct DFT<1, INV> {
  template <class E>
  __device__ __forceinline__ static void run(E (&)[1]) {}
};

template <bool INV>
struct DFT<2, INV> {
  template <class E>
  __device__ __forceinline__ static void run(E (&v)[2]) {
    const E a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <bool INV>
struct DFT<3, INV> {
  template <class E>
  __device__ __forceinline__ static void run(E (&v)[3]) {
    constexpr float h = 0.86602540378443864676f;  // sin(2 pi / 3)
    const E t1 = cadd(v[1], v[2]);
    const E t2 = mul_mi<INV>(cscale(csub(v[1], v[2]), h));
    const E m = caxpy(-0.5f, t1, v[0]);
    v[0] = cadd(v[0], t1);
    v[1] = cadd(m, t2);
    v[2] = csub(m, t2);
  }
};

template <bool INV>
struct DFT<4, INV> {
  template <class E>
  __device__ __forceinline__ static void run(E (&v)[4]) {
    const E t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const E t2 = cadd(v[1], v[3]), t3 = mul_mi<INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <bool INV>
struct DFT<5, INV> {
  template <class E>
  __device__ __forceinline__ static void run(E (&v)[5]) {
    constexpr float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
    constexpr float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
    constexpr float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
    constexpr float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
    const E a = cadd(v[1], v[4]), b = csub(v[1], v[4]);
    const E c = cadd(v[2], v[3]), d = csub(v[2], v[3]);
    const E x0 = v[0];
    const E r1 = caxpy(c2, c, caxpy(c1, a, x0));
    const E r2 = caxpy(c1, c, caxpy(c2, a, x0));
    const E i1 = mul_mi<INV>(caxpy(s2, d, cscale(b, s1)));
    const E i2 = mul_mi<INV>(caxpy(-s1, d, cscale(b, s2)));
    v[0] = cadd(x0, cadd(a, c));
    v[1] = cadd(r1, i1);
    v[4] = csub(r1, i1);
    v[2] = cadd(r2, i2);
    v[3] = csub(r2, i2);
  }
};

template <int R>
struct SplitOf {
  static constexpr int A = (R % 4 == 0 && R > 4) ? 4 : (R % 2 == 0) ? 2 : (R % 3 == 0) ? 3 : 5;
  static constexpr int B = R / A;
};

constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
// x with a x = 1 (mod m), for gcd(a, m) = 1 (m = 1: 0)
constexpr int inv_mod(int a, int m) {
  for (int x = 1; x < m; ++x)
    if ((a * x) % m == 1) return x;
  return 0;
}

// Composite R = A * B.
//   gcd(A, B) = 1: prime-factor (Good-Thomas) form, no twiddles: input n = (B n1 + A n2)
//   mod R, output k = (eA k1 + eB k2) mod R with eA = 1 (mod A), 0 (mod B) and eB = 0
//   (mod A), 1 (mod B); all indices are compile-time constants, so the maps are free.
//   otherwise Cooley-Tukey: input n = B n1 + n2, output k = k1 + A k2, twiddles between.
template <int R, bool INV>
struct DFT {
  static_assert(R % SplitOf<R>::A == 0, "unsupported radix");
  template <class E>
  __device__ __forceinline__ static void run(E (&v)[R]) {
    constexpr int A = SplitOf<R>::A, B = SplitOf<R>::B;
    if constexpr (gcd_c(A, B) == 1) {
      constexpr int eA = B * inv_mod(B % A, A), eB = A * inv_mod(A % B, B);
      E u[B][A];
      sfor<0, B>([&](auto N2) {
        constexpr int n2 = decltype(N2)::value;
        E t[A];
        sfor<0, A>([&](auto N1) {
          constexpr int n1 = decltype(N1)::value;
          t[n1] = v[(B * n1 + A * n2) % R];
        });
        DFT<A, INV>::run(t);
        sfor<0, A>([&](auto K1) { u[n2][decltype(K1)::value] = t[decltype(K1)::value]; });
      });
      sfor<0, A>([&](auto K1) {
        constexpr int k1 = decltype(K1)::value;
        E t[B];
        sfor<0, B>([&](auto N2) { t[decltype(N2)::value] = u[decltype(N2)::value][k1]; });
        DFT<B, INV>::run(t);
        sfor<0, B>([&](auto K2) {
          constexpr int k2 = decltype(K2)::value;
          v[(eA * k1 + eB * k2) % R] = t[k2];
        });
      });
      return;
    }
    E u[B][A];
    sfor<0, B>([&](auto N2) {
      constexpr int n2 = decltype(N2)::value;
      E t[A];
      sfor<0, A>([&](auto N1) { t[decltype(N1)::value] = v[B * decltype(N1)::value + n2]; });
      DFT<A, INV>::run(t);
      sfor<0, A>([&](auto K1) {
        constexpr int k1 = decltype(K1)::value;
        u[n2][k1] = twmul<n2 * k1, R, INV>(t[k1]);
      });
    });
    sfor<0, A>([&](auto K1) {
      constexpr int k1 = decltype(K1)::value;
      E t[B];
      sfor<0, B>([&](auto N2) { t[decltype(N2)::value] = u[decltype(N2)::value][k1]; });
      DFT<B, INV>::run(t);
      sfor<0, B>([&](auto K2) { v[k1 + A * decltype(K2)::value] = t[decltype(K2)::value]; });
    });
  }
};

// ---------------------------------------------------------------- zero-aware codelets
// DFTZ<R, INV, ZM>::run(v) is DFT<R, INV>::run(v) for inputs of which those with bit r of ZM
// set are known to be zero (the zero padding of a first pass): the additions and products such
// an input would enter are left out.  Leaving out x + 0 or y + s 0 changes no result except,
// possibly, the sign of an exact zero; results that are zero only because all their inputs
// are get an explicit zero.  With ZM = 0 it is DFT<R, INV> itself.
template <class E>
__device__ __forceinline__ E czero() {
  E z;
  if constexpr (sizeof(E) == sizeof(float2)) z = E{0.f, 0.f};
  else z = E{0.f, 0.f, 0.f, 0.f};
  return z;
}
__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float4 cneg(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
// a + b, a - b and y + s x with compile-time zero flags of the operands
template <bool ZA, bool ZB, class E>
__device__ __forceinline__ E zadd(const E& a, const E& b) {
  if constexpr (ZA && ZB) return czero<E>();
  else if constexpr (ZA) return b;
  else if constexpr (ZB) return a;
  else return cadd(a, b);
}
template <bool ZA, bool ZB, class E>
__device__ __forceinline__ E zsub(const E& a, const E& b) {
  if constexpr (ZA && ZB) return czero<E>();
  else if constexpr (ZA) return cneg(b);
  else if constexpr (ZB) return a;
  else return csub(a, b);
}
template <bool ZX, bool ZY, class E>
__device__ __forceinline__ E zaxpy(float sc, const E& x, const E& y) {
  if constexpr (ZX && ZY) return czero<E>();
  else if constexpr (ZX) return y;
  else if constexpr (ZY) return cscale(x, sc);
  else return caxpy(sc, x, y);
}

template <int R, bool INV, unsigned ZM>
struct DFTZ;

template <bool INV, unsigned ZM>
struct DFTZ<2, INV, ZM> {
  template <class E>
  __device__ __forceinline__ static void run(E (&v)[2]) {
    constexpr bool z0 = ZM & 1u, z1 = ZM & 2u;
    const E a = v[0], b = v[1];
    v[0] = zadd<z0, z1>(a, b);
    v[1] = zsub<z0, z1>(a, b);
  }
};

template <bool INV, unsigned ZM>
struct DFTZ<3, INV, ZM> {
  template <class E>
  __device__ __forceinline__ static void run(E (&v)[3]) {
    constexpr bool z0 = ZM & 1u, z1 = ZM & 2u, z2 = ZM & 4u;
    constexpr float h = 0.86602540378443864676f;  // sin(2 pi / 3)
    constexpr bool zt = z1 && z2;                // t1 and t2 are zero
    const E t1 = zadd<z1, z2>(v[1], v[2]);
    const E t2 = mul_mi<INV>(cscale(zsub<z1, z2>(v[1], v[2]), h));
    const E m = zaxpy<zt, z0>(-0.5f, t1, v[0]);
    v[0] = zadd<z0, zt>(v[0], t1);
    v[1] = zadd<zt && z0, zt>(m, t2);
    v[2] = zsub<zt && z0, zt>(m, t2);
  }
};

template <bool INV, unsigned ZM>
struct DFTZ<4, INV, ZM> {
  template <class E>
  __device__ __forceinline__ static void run(E (&v)[4]) {
    constexpr bool z0 = ZM & 1u, z1 = ZM & 2u, z2 = ZM & 4u, z3 = ZM & 8u;
    const E t0 = zadd<z0, z2>(v[0], v[2]), t1 = zsub<z0, z2>(v[0], v[2]);
    const E t2 = zadd<z1, z3>(v[1], v[3]), t3 = mul_mi<INV>(zsub<z1, z3>(v[1], v[3]));
    constexpr bool za = z0 && z2, zb = z1 && z3;
    v[0] = zadd<za, zb>(t0, t2);
    v[2] = zsub<za, zb>(t0, t2);
    v[1] = zadd<za, zb>(t1, t3);
    v[3] = zsub<za, zb>(t1, t3);
  }
};

template <bool INV, unsigned ZM>
struct DFTZ<5, INV, ZM> {
  template <class E>
  __device__ __forceinline__ static void run(E (&v)[5]) {
    constexpr bool z0 = ZM & 1u, z1 = ZM & 2u, z2 = ZM & 4u, z3 = ZM & 8u, z4 = ZM & 16u;
    constexpr float c1 = 0.30901699437494742410f;   // cos(2 pi / 5)
    constexpr float c2 = -0.80901699437494742410f;  // cos(4 pi / 5)
    constexpr float s1 = 0.95105651629515357212f;   // sin(2 pi / 5)
    constexpr float s2 = 0.58778525229247312917f;   // sin(4 pi / 5)
    constexpr bool zad = z1 && z4, zcd = z2 && z3;  // a, b zero; c, d zero
    const E a = zadd<z1, z4>(v[1], v[4]), b = zsub<z1, z4>(v[1], v[4]);
    const E c = zadd<z2, z3>(v[2], v[3]), d = zsub<z2, z3>(v[2], v[3]);
    const E x0 = v[0];
    constexpr bool zr = zad && zcd && z0, zi = zad && zcd;
    const E r1 = zaxpy<zcd, zad && z0>(c2, c, zaxpy<zad, z0>(c1, a, x0));
    const E r2 = zaxpy<zcd, zad && z0>(c1, c, zaxpy<zad, z0>(c2, a, x0));
    const E i1 = mul_mi<INV>(zaxpy<zcd, zad>(s2, d, zad ? czero<E>() : cscale(b, s1)));
    const E i2 = mul_mi<INV>(zaxpy<zcd, zad>(-s1, d, zad ? czero<E>() : cscale(b, s2)));
    v[0] = zadd<z0, zi>(x0, zadd<zad, zcd>(a, c));
    v[1] = zadd<zr, zi>(r1, i1);
    v[4] = zsub<zr, zi>(r1, i1);
    v[2] = zadd<zr, zi>(r2, i2);
    v[3] = zsub<zr, zi>(r2, i2);
  }
};

// zero mask of the inner (A-point) DFT for group n2 of a composite R = A B, and of the groups
// whose inputs are all zero (their outputs, inputs of the outer B-point DFTs, are zero too)
template <int R, int A, int B, unsigned ZM>
constexpr unsigned dftz_inner_mask(int n2, bool pfa) {
  unsigned m = 0;
  for (int n1 = 0; n1 < A; ++n1) {
    const int n = pfa ? (B * n1 + A * n2) % R : B * n1 + n2;
    if ((ZM >> n) & 1u) m |= 1u << n1;
  }
  return m;
}
template <int R, int A, int B, unsigned ZM>
constexpr unsigned dftz_outer_mask(bool pfa) {
  unsigned m = 0;
  for (int n2 = 0; n2 < B; ++n2)
    if (dftz_inner_mask<R, A, B, ZM>(n2, pfa) == (1u << A) - 1u) m |= 1u << n2;
  return m;
}

// composite R = A B, the structure of DFT<R, INV> with the masks carried into its parts
template <int R, bool INV, unsigned ZM>
struct DFTZ {
  template <class E>
  __device__ __forceinline__ static void run(E (&v)[R]) {
    if constexpr (ZM == 0u) {
      DFT<R, INV>::run(v);
    } else {
      constexpr int A = SplitOf<R>::A, B = SplitOf<R>::B;
      constexpr bool pfa = gcd_c(A, B) == 1;
      constexpr unsigned ZO = dftz_outer_mask<R, A, B, ZM>(pfa);
      E u[B][A];
      sfor<0, B>([&](auto N2) {
        constexpr int n2 = decltype(N2)::value;
        constexpr unsigned zi = dftz_inner_mask<R, A, B, ZM>(n2, pfa);
        E t[A];
        sfor<0, A>([&](auto N1) {
          constexpr int n1 = decltype(N1)::value;
          t[n1] = pfa ? v[(B * n1 + A * n2) % R] : v[B * n1 + n2];
        });
        DFTZ<A, INV, zi>::run(t);
        sfor<0, A>([&](auto K1) {
          constexpr int k1 = decltype(K1)::value;
          if constexpr (pfa || ((ZO >> n2) & 1u)) u[n2][k1] = t[k1];
          else u[n2][k1] = twmul<n2 * k1, R, INV>(t[k1]);
        });
      });
      constexpr int eA = pfa ? B * inv_mod(B % A, A) : 0, eB = pfa ? A * inv_mod(A % B, B) : 0;
      sfor<0, A>([&](auto K1) {
        constexpr int k1 = decltype(K1)::value;
        E t[B];
        sfor<0, B>([&](auto N2) { t[decltype(N2)::value] = u[decltype(N2)::value][k1]; });
        DFTZ<B, INV, ZO>::run(t);
        sfor<0, B>([&](auto K2) {
          constexpr int k2 = decltype(K2)::value;
          if constexpr (pfa) v[(eA * k1 + eB * k2) % R] = t[k2];
          else v[k1 + A * k2] = t[k2];
        });
      });
    }
  }
};

// ---------------------------------------------------------------- CTA-level transform
__device__ __forceinline__ int sidx(int i) { return i + (i >> 4); }

// One in-place Stockham pass of radix R over nb transforms of length n stored at
// buf + b * bs + sidx(i).  Requires (n / R) * nb <= MAXB * blockDim.x.
template <int R, bool INV, int MAXB>
__device__ __noinline__ void fft_pass(float2* buf, int bs, int n, int nb, int Ns,
                                         const float2* __restrict__ tw) {
  const int m = n / R;
  const int nbf = m * nb;
  const int twstride = n / (Ns * R);
  float2 v[MAXB][R];
#pragma unroll
  for (int it = 0; it < MAXB; ++it) {
    const int t = threadIdx.x + it * blockDim.x;
    if (t < nbf) {
      const int b = t / m, j = t - b * m;
      const int k = j % Ns;
      float2* base = buf + b * bs;
#pragma unroll
      for (int r = 0; r < R; ++r) v[it][r] = base[sidx(j + r * m)];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = __ldg(&tw[r * k * twstride]);
          if (INV) w.y = -w.y;
          v[it][r] = cmul(v[it][r], w);
        }
      }
      DFT<R, INV>::run(v[it]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < MAXB; ++it) {
    const int t = threadIdx.x + it * blockDim.x;
    if (t < nbf) {
      const int b = t / m, j = t - b * m;
      const int k = j % Ns;
      const int o = (j - k) * R + k;
      float2* base = buf + b * bs;
#pragma unroll
      for (int r = 0; r < R; ++r) base[sidx(o + r * Ns)] = v[it][r];
    }
  }
  __syncthreads();
}

// Full transform (unnormalised; INV selects exp(+2 pi i k n / N)).  The caller must
// __syncthreads() after filling buf; the transform ends with a barrier.
template <bool INV, int MAXB>
__device__ __forceinline__ void block_fft(float2* buf, int bs, int nb, const FFTDesc& d) {
  int Ns = 1;
  for (int p = 0; p < d.npass; ++p) {
    const int R = d.radix[p];
    switch (R) {
      case 2: fft_pass<2, INV, MAXB>(buf, bs, d.n, nb, Ns, d.tw); break;
      case 3: fft_pass<3, INV, MAXB>(buf, bs, d.n, nb, Ns, d.tw); break;
      case 4: fft_pass<4, INV, MAXB>(buf, bs, d.n, nb, Ns, d.tw); break;
      case 5: fft_pass<5, INV, MAXB>(buf, bs, d.n, nb, Ns, d.tw); break;
      case 6: fft_pass<6, INV, MAXB>(buf, bs, d.n, nb, Ns, d.tw); break;
      case 8: fft_pass<8, INV, MAXB>(buf, bs, d.n, nb, Ns, d.tw); break;
      case 9: fft_pass<9, INV, MAXB>(buf, bs, d.n, nb, Ns, d.tw); break;
      case 10: fft_pass<10, INV, MAXB>(buf, bs, d.n, nb, Ns, d.tw); break;
      case 12: fft_pass<12, INV, MAXB>(buf, bs, d.n, nb, Ns, d.tw); break;
      case 15: fft_pass<15, INV, MAXB>(buf, bs, d.n, nb, Ns, d.tw); break;
      case 16: fft_pass<16, INV, MAXB>(buf, bs, d.n, nb, Ns, d.tw); break;
      case 20: fft_pass<20, INV, MAXB>(buf, bs, d.n, nb, Ns, d.tw); break;
      case 24: fft_pass<24, INV, MAXB>(buf, bs, d.n, nb, Ns, d.tw); break;
      default: break;  // the host only builds plans from the radices above
    }
    Ns *= R;
  }
}


}  // namespace cgh
