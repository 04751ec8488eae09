// dfft.cuh - shared-memory-resident FFTs for the paired-FP32 (double-float)
// passes.  Paired-FP32 arithmetic costs about ten FP32 instructions per
// operation, so these passes are bound by instruction issue, not memory;
// fully unrolled register transforms of 32 points made the code too large
// for the instruction cache.  Here a tile of C columns x L points sits in
// shared memory and is transformed in place by a loop over radix-8 stages
// (one radix-2 or radix-4 stage closes when log2 L is not a multiple of 3):
//
//   forward: decimation in frequency, natural order in, digit-reversed out
//   inverse: decimation in time, digit-reversed in, natural order out
//
// so a forward transform, a pointwise product (indexed through the digit
// reversal) and an inverse need no reordering pass.  The X inverse pass,
// whose input comes in natural order from global memory, runs the DIF
// stages with the inverse sign instead and gathers its outputs.
#pragma once

#include "dfloat.cuh"

namespace ori {

// Stages of a length-L transform: NST8 radix-8 stages, then one radix-RL
// stage (RL = 1, 2 or 4).
template <int L>
struct DRad {
  static constexpr int lg = ilog2(L);
  static constexpr int NST8 = lg / 3;
  static constexpr int RL = 1 << (lg - 3 * NST8);
};

// Frequency held at position p after the forward (DIF) stages: the mixed-
// radix digits of p reversed (the first stage's digit is the least
// significant digit of the frequency).
template <int L>
__device__ __forceinline__ int digit_rev(int p) {
  using DR = DRad<L>;
  int k = 0, w = 1;
  // digits of p, least significant first, belong to the stages last-to-first
  int q = p;
  int dig[DR::NST8 + 1];
  int nd = 0;
  if (DR::RL > 1) { dig[nd++] = q % DR::RL; q /= DR::RL; }
#pragma unroll
  for (int i = 0; i < DR::NST8; ++i) { dig[nd++] = q & 7; q >>= 3; }
  // the first stage (radix 8) digit is the last one extracted
#pragma unroll
  for (int i = DR::NST8 + (DR::RL > 1 ? 1 : 0) - 1; i >= 0; --i) {
    const int R = (DR::RL > 1 && i == 0) ? DR::RL : 8;
    k += dig[i] * w;
    w *= R;
  }
  return k;
}

// Position that holds frequency k after the forward stages (inverse of digit_rev).
template <int L>
__device__ __forceinline__ int inv_digit_rev(int k) {
  using DR = DRad<L>;
  // k = d_1 + 8 d_2 + ... (first stage's digit least significant), last digit radix RL
  int q = k;
  int p = 0;
  int dig[DR::NST8];
#pragma unroll
  for (int i = 0; i < DR::NST8; ++i) { dig[i] = q & 7; q >>= 3; }
  p = (DR::RL > 1) ? q : 0;   // the radix-RL digit (most significant in k) is least significant in p
  int w = DR::RL;
#pragma unroll
  for (int i = DR::NST8 - 1; i >= 0; --i) { p += dig[i] * w; w *= 8; }
  return p;
}

// Shared-memory index of point j of column c: rows of C columns, the column
// index swizzled by the row so that both row-wise and column-wise warp
// accesses avoid bank conflicts.
template <int C>
__device__ __forceinline__ int sidx(int j, int c) { return j * C + (c ^ (j & (C - 1))); }

// One in-place decimation-in-frequency stage of radix R on all C columns:
// blocks of M points, span s = M / R; outputs multiplied by w_M^(j t').
template <int R, int SIGN, int L, int C, class T>
__device__ __forceinline__ void dif_stage(cpx<T>* X, int M, const cpx<T>* tw, int tid, int nt) {
  const int s = M / R;
  const int step = L / M;
  for (int g = tid; g < C * (L / R); g += nt) {
    const int c = g % C, bi = g / C;
    const int blk = bi / s, j = bi - blk * s;
    const int base = blk * M + j;
    cpx<T> v[R];
#pragma unroll
    for (int t = 0; t < R; ++t) v[t] = ld_stage(X + sidx<C>(base + t * s, c));
    dft<R, SIGN, false>(v);
#pragma unroll
    for (int t = 1; t < R; ++t) v[t] = twL_mul<SIGN>(v[t], tw, (j * t * step) & (L - 1));
#pragma unroll
    for (int t = 0; t < R; ++t) st_stage(X + sidx<C>(base + t * s, c), settle(v[t]));
  }
}

// One in-place decimation-in-time stage: inputs multiplied by w_M^(j t), then
// the radix-R butterfly.
template <int R, int SIGN, int L, int C, class T>
__device__ __forceinline__ void dit_stage(cpx<T>* X, int M, const cpx<T>* tw, int tid, int nt) {
  const int s = M / R;
  const int step = L / M;
  for (int g = tid; g < C * (L / R); g += nt) {
    const int c = g % C, bi = g / C;
    const int blk = bi / s, j = bi - blk * s;
    const int base = blk * M + j;
    cpx<T> v[R];
#pragma unroll
    for (int t = 0; t < R; ++t) v[t] = ld_stage(X + sidx<C>(base + t * s, c));
#pragma unroll
    for (int t = 1; t < R; ++t) v[t] = twL_mul<SIGN>(v[t], tw, (j * t * step) & (L - 1));
    dft<R, SIGN, false>(v);
#pragma unroll
    for (int t = 0; t < R; ++t) st_stage(X + sidx<C>(base + t * s, c), settle(v[t]));
  }
}

// DIF stages after the first one (which the callers fuse with their loads):
// block sizes L/8, L/64, ...  SIGN -1: forward transform; +1: inverse.
template <int L, int C, int SIGN = -1, class T>
__device__ __forceinline__ void dif_rest(cpx<T>* X, const cpx<T>* tw, int tid, int nt) {
  using DR = DRad<L>;
  int M = L / 8;
#pragma unroll 1
  for (int st = 1; st < DR::NST8; ++st) {
    dif_stage<8, SIGN, L, C>(X, M, tw, tid, nt);
    __syncthreads();
    M /= 8;
  }
  if constexpr (DR::RL > 1) {
    dif_stage<DR::RL, SIGN, L, C>(X, M, tw, tid, nt);
    __syncthreads();
  }
}

// Inverse DIT stages except the last (block size L), which the callers fuse
// with their stores: block sizes RL (if any), then 8 RL, 64 RL, ... up to L/8.
template <int L, int C, class T>
__device__ __forceinline__ void dit_head(cpx<T>* X, const cpx<T>* tw, int tid, int nt) {
  using DR = DRad<L>;
  int M = 1;
  if constexpr (DR::RL > 1) {
    M = DR::RL;
    dit_stage<DR::RL, +1, L, C>(X, M, tw, tid, nt);
    __syncthreads();
  }
#pragma unroll 1
  for (int st = 1; st < DR::NST8; ++st) {
    M *= 8;
    dit_stage<8, +1, L, C>(X, M, tw, tid, nt);
    __syncthreads();
  }
}

}  // namespace ori
