// dfloat.cuh - paired-FP32 ("double-float") arithmetic for the refinement
// residual.  A value is hi + lo with |lo| <= ulp(hi)/2: about 48 significant
// bits.  On a GPU whose FP64 rate is 1/64 of its FP32 rate this gives the
// FP64-class residual of the iterative refinement several times faster than
// native FP64.
//
// Building blocks (error-free transformations, published methods):
//   two_sum     Knuth, TAOCP vol. 2, s + e = a + b exactly (6 flops)
//   fast_two_sum Dekker 1971, same when |a| >= |b| (3 flops)
//   two_prod    p + e = a * b exactly, e by one fused multiply-add
// Addition is the "sloppy" pairwise form (one two_sum on the high parts, the
// low parts added in FP32): its error is bounded by a small multiple of
// 2^-48 (|a| + |b|), which keeps FFT butterflies normwise accurate.
// Products accumulate all four partial products.  Neither renormalises its
// result: the pair hi + lo stays an exact-enough representation (|lo| grows
// by about one unit of 2^-24 |hi| per level of additions), so the FFT stages
// add and multiply unnormalised pairs and renormalise each value once, when
// they store it (settle), instead of after every operation: an addition
// costs 8 FP32 operations instead of 11, a product 16 instead of 19.
#pragma once

#include "common.cuh"

namespace ori {

struct alignas(8) dfl {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return {s, e + (a.lo + b.lo)};
}
__device__ __forceinline__ dfl operator-(dfl a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = a.hi * b.hi;
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return {p, e};
}

// Renormalise: |lo| <= ulp(hi) / 2 again.  The fast form is exact when
// |hi| >= |lo|; where cancellation left |hi| < |lo| the value is tiny next to
// the operands that produced it, so the normwise error bound still holds.
__device__ __forceinline__ dfl settle(dfl a) {
  dfl r;
  fast_two_sum(a.hi, a.lo, r.hi, r.lo);
  return r;
}

// a*b - c*d with one renormalisation (the real part of a complex product).
__device__ __forceinline__ dfl df_dot2(dfl a, dfl b, dfl c, dfl d, float sign) {
  const float p1 = a.hi * b.hi;
  const float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  const float p2 = sign * (c.hi * d.hi);
  const float e2 = __fmaf_rn(sign * c.hi, d.hi, -p2);
  float s, e;
  two_sum(p1, p2, s, e);
  e += e1 + e2;
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  e = __fmaf_rn(sign * c.hi, d.lo, e);
  e = __fmaf_rn(sign * c.lo, d.hi, e);
  return {s, e};
}

// Complex product in double-float.
__device__ __forceinline__ cpx<dfl> cmul(cpx<dfl> a, cpx<dfl> b) {
  return {df_dot2(a.x, b.x, a.y, b.y, -1.0f), df_dot2(a.x, b.y, a.y, b.x, 1.0f)};
}

// Complex sums and the renormalisation in packed two-lane FP32 instructions
// (f32x2, sm_100 and later): the real and imaginary parts go through the
// same error-free transformation side by side, each lane rounded as the
// scalar operation would be, in half the issue slots.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(unsigned long long v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ unsigned long long fadd2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long fsub2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

// a + b (SUB = false) or a - b (SUB = true): two_sum of the high parts
// (Knuth; with c = -b for the difference: e = (a - (s - bb)) - (b + bb)), the
// low parts added, no renormalisation.
template <bool SUB>
__device__ __forceinline__ cpx<dfl> df_cadd(cpx<dfl> a, cpx<dfl> b) {
  const unsigned long long ah = pk2(a.x.hi, a.y.hi), bh = pk2(b.x.hi, b.y.hi);
  const unsigned long long s = SUB ? fsub2(ah, bh) : fadd2(ah, bh);
  const unsigned long long bb = fsub2(s, ah);
  const unsigned long long e = SUB ? fsub2(fsub2(ah, fsub2(s, bb)), fadd2(bh, bb))
                                   : fadd2(fsub2(ah, fsub2(s, bb)), fsub2(bh, bb));
  const unsigned long long al = pk2(a.x.lo, a.y.lo), bl = pk2(b.x.lo, b.y.lo);
  const unsigned long long lo = fadd2(e, SUB ? fsub2(al, bl) : fadd2(al, bl));
  cpx<dfl> r;
  upk2(s, r.x.hi, r.y.hi);
  upk2(lo, r.x.lo, r.y.lo);
  return r;
}
// Between FFT stages (shared-memory tiles) and in the twiddle tables a
// paired-FP32 complex value is stored as (re.hi, im.hi, re.lo, im.lo): one
// 16-byte access then yields the two lane pairs the packed instructions take.
template <>
__device__ __forceinline__ cpx<dfl> ld_stage<dfl>(const cpx<dfl>* p) {
  const float4 f = *reinterpret_cast<const float4*>(p);
  return {{f.x, f.z}, {f.y, f.w}};
}
template <>
__device__ __forceinline__ void st_stage<dfl>(cpx<dfl>* p, cpx<dfl> v) {
  *reinterpret_cast<float4*>(p) = make_float4(v.x.hi, v.y.hi, v.x.lo, v.y.lo);
}

template <>
__device__ __forceinline__ cpx<dfl> operator+(cpx<dfl> a, cpx<dfl> b) { return df_cadd<false>(a, b); }
template <>
__device__ __forceinline__ cpx<dfl> operator-(cpx<dfl> a, cpx<dfl> b) { return df_cadd<true>(a, b); }

// A value as it is stored between FFT stages: renormalised for paired FP32
// (fast_two_sum on both lanes), unchanged for the other arithmetics.
template <class T> __device__ __forceinline__ cpx<T> settle(cpx<T> v) { return v; }
template <> __device__ __forceinline__ cpx<dfl> settle<dfl>(cpx<dfl> v) {
  const unsigned long long h = pk2(v.x.hi, v.y.hi), l = pk2(v.x.lo, v.y.lo);
  const unsigned long long s = fadd2(h, l);
  const unsigned long long e = fsub2(l, fsub2(s, h));
  cpx<dfl> r;
  upk2(s, r.x.hi, r.y.hi);
  upk2(e, r.x.lo, r.y.lo);
  return r;
}

// Split a double into hi + lo (hi = nearest float, lo = nearest float of the rest).
__device__ __forceinline__ dfl df_from_double(double v) {
  const float hi = __double2float_rn(v);
  const float lo = __double2float_rn(v - double(hi));
  return {hi, lo};
}
__device__ __forceinline__ double df_to_double(dfl v) { return double(v.hi) + double(v.lo); }

__host__ __forceinline__ dfl df_from_double_host(double v) {
  const float hi = float(v);
  const float lo = float(v - double(hi));
  return {hi, lo};
}

// Conversions between complex128 and the pass arithmetic T.
template <class T> __device__ __forceinline__ cpx<T> c_from_c64(cpx<double> v) {
  return {T(v.x), T(v.y)};
}
template <> __device__ __forceinline__ cpx<dfl> c_from_c64<dfl>(cpx<double> v) {
  return {df_from_double(v.x), df_from_double(v.y)};
}
template <class T> __device__ __forceinline__ cpx<double> c_to_c64(cpx<T> v) {
  return {double(v.x), double(v.y)};
}
template <> __device__ __forceinline__ cpx<double> c_to_c64<dfl>(cpx<dfl> v) {
  return {df_to_double(v.x), df_to_double(v.y)};
}

// Twiddles of the in-register DFTs in double-float: hi and lo of the FP64
// compile-time values.
struct Tw64df {
  float ch[64], cl[64], sh[64], sl[64];
};
constexpr Tw64df make_tw64df() {
  Tw64df t{};
  for (int j = 0; j < 64; ++j) {
    CosSin v = turn_cos_sin(j, 64);
    t.ch[j] = float(v.c);
    t.cl[j] = float(v.c - double(float(v.c)));
    t.sh[j] = float(v.s);
    t.sl[j] = float(v.s - double(float(v.s)));
  }
  return t;
}
__constant__ Tw64df c_tw64df = make_tw64df();

template <>
__device__ __forceinline__ dfl tw64c<dfl>(int i) { return {c_tw64df.ch[i], c_tw64df.cl[i]}; }
template <>
__device__ __forceinline__ dfl tw64s<dfl>(int i) { return {c_tw64df.sh[i], c_tw64df.sl[i]}; }

__device__ __forceinline__ cpx<dfl> ldgc(const cpx<dfl>* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return {{v.x, v.y}, {v.z, v.w}};
}

template <>
__device__ __forceinline__ cpx<dfl> czero<dfl>() { return {{0.f, 0.f}, {0.f, 0.f}}; }

}  // namespace ori
