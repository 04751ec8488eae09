// common.cuh - complex arithmetic, twiddle factors and in-register DFTs for
// the FFT passes of the convolution matvec (Section 3, Eq. 3.3.8).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ori {

// ---------------------------------------------------------------------------
// Complex numbers (interleaved re, im; 8 bytes for float, 16 for double)
// ---------------------------------------------------------------------------
template <class T>
struct alignas(2 * sizeof(T)) cpx {
  T x, y;
};

template <class T>
__host__ __device__ __forceinline__ cpx<T> mkc(T a, T b) { return cpx<T>{a, b}; }
template <class T>
__device__ __forceinline__ cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <class T>
__device__ __forceinline__ cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
// FP32 complex sums as one packed two-lane instruction (add/sub.rn.f32x2,
// sm_100 and later): the same rounding per lane as two scalar operations,
// half the issue slots.  The FFT passes are bound by instruction issue, and
// their butterflies are mostly complex additions.
__device__ __forceinline__ unsigned long long pack2(cpx<float> a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ cpx<float> unpack2(unsigned long long v) {
  cpx<float> r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
template <>
__device__ __forceinline__ cpx<float> operator+(cpx<float> a, cpx<float> b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
  return unpack2(r);
}
template <>
__device__ __forceinline__ cpx<float> operator-(cpx<float> a, cpx<float> b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
  return unpack2(r);
}

template <class T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <class T>
__device__ __forceinline__ cpx<T> cscale(cpx<T> a, T s) { return {a.x * s, a.y * s}; }
template <class T>
__device__ __forceinline__ cpx<T> czero() { return {T(0), T(0)}; }

template <class D, class S>
__device__ __forceinline__ cpx<D> ccast(cpx<S> a) { return {D(a.x), D(a.y)}; }

// ---------------------------------------------------------------------------
// Twiddles.  cos/sin of 2 pi j / M are evaluated at compile time from their
// Taylor series on [0, pi/4] after an exact reduction by octant symmetry.
// ---------------------------------------------------------------------------
constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr double taylor_sin(double x) {
  double t = x, s = x;
  for (int i = 1; i < 16; ++i) {
    t *= -x * x / double((2 * i) * (2 * i + 1));
    s += t;
  }
  return s;
}
constexpr double taylor_cos(double x) {
  double t = 1.0, s = 1.0;
  for (int i = 1; i < 16; ++i) {
    t *= -x * x / double((2 * i - 1) * (2 * i));
    s += t;
  }
  return s;
}

// (cos, sin) of 2 pi j / M for M divisible by 8.
struct CosSin {
  double c, s;
};
constexpr CosSin turn_cos_sin(long long j, long long M) {
  long long jm = ((j % M) + M) % M;
  const long long m8 = M / 8;
  const long long oct = jm / m8, rem = jm % m8;
  const double step = 2.0 * kPi / double(M);
  const double phi = double(rem) * step;          // in [0, pi/4)
  const double phr = double(m8 - rem) * step;     // in (0, pi/4]
  const double cp = taylor_cos(phi), sp = taylor_sin(phi);
  const double cr = taylor_cos(phr), sr = taylor_sin(phr);
  switch (oct) {
    case 0: return {cp, sp};
    case 1: return {sr, cr};
    case 2: return {-sp, cp};
    case 3: return {-cr, sr};
    case 4: return {-cp, -sp};
    case 5: return {-sr, -cr};
    case 6: return {sp, -cp};
    default: return {cr, -sr};
  }
}

// cos/sin of 2 pi j / 64 for the in-register DFTs (radix up to 64).
struct Tw64 {
  double c[64];
  double s[64];
  float cf[64];
  float sf[64];
};
constexpr Tw64 make_tw64() {
  Tw64 t{};
  for (int j = 0; j < 64; ++j) {
    CosSin v = turn_cos_sin(j, 64);
    t.c[j] = v.c;
    t.s[j] = v.s;
    t.cf[j] = float(v.c);
    t.sf[j] = float(v.s);
  }
  return t;
}

__constant__ Tw64 c_tw64 = make_tw64();

template <class T>
__device__ __forceinline__ T tw64c(int i);
template <>
__device__ __forceinline__ float tw64c<float>(int i) { return c_tw64.cf[i]; }
template <>
__device__ __forceinline__ double tw64c<double>(int i) { return c_tw64.c[i]; }
template <class T>
__device__ __forceinline__ T tw64s(int i);
template <>
__device__ __forceinline__ float tw64s<float>(int i) { return c_tw64.sf[i]; }
template <>
__device__ __forceinline__ double tw64s<double>(int i) { return c_tw64.s[i]; }

// z * exp(SIGN * 2 pi i idx / 64); idx is a compile-time constant after
// unrolling, so trivial factors cost nothing and the others read the
// constant bank directly.
template <int SIGN, class T>
__device__ __forceinline__ cpx<T> tw64_mul(cpx<T> z, int idx) {
  idx &= 63;
  if (idx == 0) return z;
  if (idx == 32) return {-z.x, -z.y};
  if (idx == 16) return SIGN > 0 ? cpx<T>{-z.y, z.x} : cpx<T>{z.y, -z.x};
  if (idx == 48) return SIGN > 0 ? cpx<T>{z.y, -z.x} : cpx<T>{-z.y, z.x};
  const T c = tw64c<T>(idx);
  const T s = SIGN > 0 ? tw64s<T>(idx) : -tw64s<T>(idx);
  return cmul(z, cpx<T>{c, s});
}

// Read-only cached loads of one complex number.
__device__ __forceinline__ cpx<float> ldgc(const cpx<float>* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ cpx<double> ldgc(const cpx<double>* p) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return {v.x, v.y};
}

// Load and store of one complex value as the FFT stages keep it in shared
// memory and as the twiddle tables hold it: T's own layout here; paired FP32
// specialises the pair (dfloat.cuh).
template <class T> __device__ __forceinline__ cpx<T> ld_stage(const cpx<T>* p) { return *p; }
template <class T> __device__ __forceinline__ void st_stage(cpx<T>* p, cpx<T> v) { *p = v; }

// z * exp(SIGN * 2 pi i m / L) from a table tab[m] = (cos, sin)(2 pi m / L).
template <int SIGN, class T>
__device__ __forceinline__ cpx<T> twL_mul(cpx<T> z, const cpx<T>* __restrict__ tab, int m) {
  // generic load: the table may sit in global memory or in shared memory
  const cpx<T> w = ld_stage(tab + m);
  return cmul(z, cpx<T>{w.x, SIGN > 0 ? w.y : -w.y});
}

constexpr int bitrev(int i, int R) {
  int r = 0;
  for (int b = 1; b < R; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}

// z * (SIGN i): a quarter turn, no arithmetic.
template <int SIGN, class T>
__device__ __forceinline__ cpx<T> mul_i(cpx<T> z) {
  return SIGN > 0 ? cpx<T>{-z.y, z.x} : cpx<T>{z.y, -z.x};
}

// In-register DFT of size R (power of two, R <= 64):
//   a[k] <- sum_j a[j] exp(SIGN 2 pi i j k / R).
// Decimation in frequency, then the bit-reversal permutation (free: all
// indices are compile-time constants).  The stages go two at a time as
// radix-4 butterflies, a final radix-2 stage when log2 R is odd.  A radix-4
// butterfly leaves the array exactly as the two radix-2 stages it replaces
// (spans s and s/2 of a block of M = 2s points, w = exp(SIGN 2 pi i / M)):
// for x0..x3 = a[j], a[j + s/2], a[j + s], a[j + 3s/2] and
// t0 = x0 + x2, t1 = x0 - x2, t2 = x1 + x3, t3 = SIGN i (x1 - x3),
//   a[j] = t0 + t2,           a[j + s/2] = (t0 - t2) w^2j,
//   a[j + s] = (t1 + t3) w^j, a[j + 3s/2] = (t1 - t3) w^3j,
// since w^(s/2) = SIGN i; it needs three twiddle products where the two
// radix-2 stages need four (34 -> 28 nontrivial products at R = 32, measured:
// the FP32 Z pass 3.43 -> 3.36 ms at n = 512).  HALF: a[j] = 0 for j >= R/2
// on input (the zero padding of Section 3), so the first butterflies have
// x2 = x3 = 0.
// Radix-2 form of the same transform (every stage span s = R/2, R/4, ..., 1;
// the outputs multiplied by w^j of their block): the small transforms (R <= 8,
// the radix-8 stages of the paired-FP32 passes), where the radix-4 form
// saves no twiddle product.
template <int R, int SIGN, bool HALF, class T>
__device__ __forceinline__ void dft_radix2(cpx<T> (&a)[R]) {
#pragma unroll
  for (int s = R / 2; s >= 1; s >>= 1) {
#pragma unroll
    for (int b = 0; b < R; b += 2 * s) {
#pragma unroll
      for (int j = 0; j < s; ++j) {
        const int idx = j * (64 / (2 * s));
        const cpx<T> u = a[b + j];
        if (HALF && s == R / 2) {
          a[b + j + s] = tw64_mul<SIGN>(u, idx);
        } else {
          const cpx<T> v = a[b + j + s];
          a[b + j] = u + v;
          a[b + j + s] = tw64_mul<SIGN>(u - v, idx);
        }
      }
    }
  }
  cpx<T> t[R];
#pragma unroll
  for (int i = 0; i < R; ++i) t[i] = a[bitrev(i, R)];
#pragma unroll
  for (int i = 0; i < R; ++i) a[i] = t[i];
}

template <int R, int SIGN, bool HALF, class T>
__device__ __forceinline__ void dft(cpx<T> (&a)[R]) {
  if constexpr (R > 1 && R <= 8) {
    dft_radix2<R, SIGN, HALF>(a);
  } else if constexpr (R > 1) {
    bool first = true;
    int s = R / 2;
#pragma unroll
    for (; s >= 2; s /= 4) {
#pragma unroll
      for (int b = 0; b < R; b += 2 * s) {
#pragma unroll
        for (int j = 0; j < s / 2; ++j) {
          const int idx = j * (64 / (2 * s));   // w^j in 64ths of a turn
          const int h = s / 2;
          cpx<T> t0, t1, t2, t3;
          if (HALF && first) {
            t0 = a[b + j];
            t1 = a[b + j];
            t2 = a[b + j + h];
            t3 = mul_i<SIGN>(a[b + j + h]);
          } else {
            const cpx<T> x0 = a[b + j], x1 = a[b + j + h], x2 = a[b + j + s], x3 = a[b + j + 3 * h];
            t0 = x0 + x2;
            t1 = x0 - x2;
            t2 = x1 + x3;
            t3 = mul_i<SIGN>(x1 - x3);
          }
          a[b + j] = t0 + t2;
          a[b + j + h] = tw64_mul<SIGN>(t0 - t2, 2 * idx);
          a[b + j + s] = tw64_mul<SIGN>(t1 + t3, idx);
          a[b + j + 3 * h] = tw64_mul<SIGN>(t1 - t3, 3 * idx);
        }
      }
      first = false;
    }
    if (s == 1) {   // the last radix-2 stage (span 1: no twiddles)
#pragma unroll
      for (int b = 0; b < R; b += 2) {
        const cpx<T> u = a[b];
        if (HALF && first) {
          a[b + 1] = u;
        } else {
          const cpx<T> v = a[b + 1];
          a[b] = u + v;
          a[b + 1] = u - v;
        }
      }
    }
    cpx<T> t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) t[i] = a[bitrev(i, R)];
#pragma unroll
    for (int i = 0; i < R; ++i) a[i] = t[i];
  }
}

// Split of the padded length L = L1 * L2 into two in-register stages.
constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }
template <int L>
struct Split {
  static constexpr int lg = ilog2(L);
  static constexpr int L1 = 1 << ((lg + 1) / 2);
  static constexpr int L2 = L / L1;
};

}  // namespace ori
