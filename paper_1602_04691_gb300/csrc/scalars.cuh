// scalars.cuh - device-resident COCG scalars and deterministic grid reductions.
//
// COCG (van der Vorst & Melissen; the solver of Section 1 and Section 3) needs
// two global reductions per iteration: mu = p^T B p, and rho' = r^T r with
// ||r||^2 for the stop test ||r|| / ||RHS|| (Section 4).  The kernels that
// produce the vectors also produce per-block partial sums; the last block to
// finish (an atomic arrival counter, no waiting) adds the partials in a fixed
// order and updates the scalars below on the device, so the host never sits
// in the iteration loop and the result does not depend on block timing.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace ori {

enum { FIN_NONE = 0,    // no reduction
       FIN_ALPHA = 1,   // mu = sum p^T q; alpha = rho / mu
       FIN_SUM = 2,     // sum -> sc->sum (generic)
       FIN_UPDATE = 3,  // rho' and ||r||^2 -> beta, stop test
       FIN_INIT = 4 };  // rho and ||r||^2 of the initial residual

enum { DONE_RUNNING = 0, DONE_CONVERGED = 1, DONE_BREAKDOWN = 2,
       DONE_NONFINITE = 3, DONE_MAXIT = 4 };

constexpr int kHistMax = 512;

struct alignas(16) Scalars {
  double2 rho;       // r^T r (unconjugated) of the current residual
  double2 mu;        // p^T q
  double2 alpha;     // rho / mu
  double2 beta;      // rho' / rho
  double2 sum;       // result of FIN_SUM
  double rnorm2;     // ||r||^2 (conjugated) of the current residual
  double rnorm2_0;   // ||r_0||^2
  double target2;    // stop when rnorm2 <= target2
  double tol;        // relative tolerance for FIN_INIT
  int done;          // DONE_*
  int iter;          // iterations finished
  int maxit;
  unsigned count;    // arrival counter of the last-block protocol
  double hist[kHistMax];  // ||r||^2 after each iteration (first kHistMax)
};

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double den = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}

__device__ __forceinline__ bool isfinite2(double2 v) { return isfinite(v.x) && isfinite(v.y); }

// Every block calls this after writing its partial(s).  Returns true in the
// block that arrived last.
__device__ __forceinline__ bool last_block_arrives(Scalars* sc, int& s_last) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned prev = atomicAdd(&sc->count, 1u);
    s_last = (prev == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Sum partials[stride*i + which] over i in [0, nparts) in a fixed order.
// Called by all threads of the last block; result valid in thread 0.
__device__ __forceinline__ double2 reduce_partials(const double2* partials, int nparts, int stride,
                                                   int which, double2* red) {
  double2 acc = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    const double2 v = __ldcg(partials + (long long)stride * i + which);
    acc.x += v.x;
    acc.y += v.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[w] = acc;
  __syncthreads();
  double2 s = make_double2(0.0, 0.0);
  if (threadIdx.x == 0)
    for (int i = 0; i < nw; ++i) { s.x += red[i].x; s.y += red[i].y; }
  __syncthreads();
  return s;
}

// Scalar update by the last block.  Partials hold one double2 per block
// (FIN_ALPHA, FIN_SUM) or two (FIN_UPDATE, FIN_INIT: r^T r, then (||r||^2, 0)).
__device__ __forceinline__ void finalize(Scalars* sc, const double2* partials, int nparts, int fin,
                                         double2* red) {
  if (fin == FIN_ALPHA || fin == FIN_SUM) {
    const double2 s = reduce_partials(partials, nparts, 1, 0, red);
    if (threadIdx.x == 0) {
      if (fin == FIN_SUM) {
        sc->sum = s;
      } else {
        sc->mu = s;
        if (!isfinite2(s)) {
          sc->done = DONE_NONFINITE;
        } else if (s.x == 0.0 && s.y == 0.0) {
          sc->done = DONE_BREAKDOWN;
        } else {
          sc->alpha = cdiv(sc->rho, s);
          if (!isfinite2(sc->alpha)) sc->done = DONE_BREAKDOWN;
        }
      }
      sc->count = 0;
    }
    return;
  }
  const double2 rr = reduce_partials(partials, nparts, 2, 0, red);
  const double2 nn = reduce_partials(partials, nparts, 2, 1, red);
  if (threadIdx.x == 0) {
    const double rn2 = nn.x;
    if (fin == FIN_INIT) {
      sc->rho = rr;
      sc->rnorm2 = rn2;
      sc->rnorm2_0 = rn2;
      sc->target2 = sc->tol * sc->tol * rn2;
      sc->iter = 0;
      sc->beta = make_double2(0.0, 0.0);
      // a residual that already meets the target needs no iteration; a nonzero
      // residual with r^T r = 0 cannot start COCG (rho is the divisor of beta)
      sc->done = (!isfinite(rn2) || !isfinite2(rr)) ? DONE_NONFINITE
               : ((rn2 == 0.0 || rn2 <= sc->target2) ? DONE_CONVERGED
               : ((rr.x == 0.0 && rr.y == 0.0) ? DONE_BREAKDOWN : DONE_RUNNING));
    } else {
      const int it = sc->iter + 1;
      sc->iter = it;
      sc->rnorm2 = rn2;
      if (it <= kHistMax) sc->hist[it - 1] = rn2;
      if (!isfinite(rn2) || !isfinite2(rr)) {
        sc->done = DONE_NONFINITE;
      } else if (rn2 <= sc->target2) {
        sc->done = DONE_CONVERGED;
      } else if (rr.x == 0.0 && rr.y == 0.0) {
        sc->done = DONE_BREAKDOWN;
      } else if (it >= sc->maxit) {
        sc->done = DONE_MAXIT;
      }
      sc->beta = cdiv(rr, sc->rho);
      // beta = rho' / rho: a vanished rho (or a rho' at rounding level over it)
      // is a breakdown, not a NaN to carry into p
      if (sc->done == DONE_RUNNING && !isfinite2(sc->beta)) sc->done = DONE_BREAKDOWN;
      sc->rho = rr;
    }
    sc->count = 0;
  }
}

}  // namespace ori
