// vector_kernels.cuh - elementwise and reduction kernels of the solver:
// medium set-up (S = sqrt(h N)), the spectrum extraction of the plan, the
// right-hand side u0 = exp(ik alpha . x) (Eq. 2.4), the COCG vector update,
// the mixed-precision refinement steps and the adjoint gradient.
#pragma once

#include "common.cuh"
#include "dfloat.cuh"
#include "passes.cuh"
#include "scalars.cuh"

namespace ori {

__device__ __forceinline__ cpx<double> cdivd(cpx<double> a, cpx<double> b) {
  const double den = b.x * b.x + b.y * b.y;
  return {(a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den};
}

// Principal square root s of w = a + ib (Re s >= 0, the branch of the
// symmetrisation S = sqrt(h N)) by the half-angle formulas, with m = |w|:
//   v = (m + |a|) / 2,  t = sqrt(v),  s = (t, b / 2t) if a >= 0, else (|b| / 2t, sign(b) t).
// GB300's FP64 pipe issues a small fraction of the FP32 rate, so the square
// root and the quotient come from one reciprocal square root r = 1/sqrt(v):
// t = v r and b / 2t = b r / 2.  Also returns m, since |s|^2 = m and hence
// 1 / s = conj(s) / m.
__device__ __forceinline__ cpx<double> csqrt_principal(cpx<double> w, double& m) {
  m = hypot(w.x, w.y);
  if (m == 0.0) return {0.0, 0.0};
  const double v = 0.5 * (m + fabs(w.x));
  const double r = rsqrt(v);
  const double t = v * r;
  const double q = 0.5 * r * w.y;
  if (w.x >= 0.0) return {t, q};
  return {fabs(q), copysign(t, w.y)};
}

// The medium arrays of a plan from h and N (one pass over the cells):
//   w = h N (scale of the A form), S = sqrt(h N) (scale of the B form), 1/S,
// in FP64, FP32 and paired FP32 (the FP32 value is the pair's high part);
// h and N are also copied into the plan (hcopy, Ncopy) when those are given.
// The A-form arrays, 1/S and the copies are optional (nullptr).  Counts the
// cells with S == 0.
__global__ void k_medium(const cpx<double>* __restrict__ h, const double* __restrict__ N,
                         cpx<double>* hcopy, double* Ncopy,
                         cpx<double>* w64, cpx<double>* S64, cpx<float>* w32, cpx<float>* S32,
                         cpx<double>* Sinv, cpx<dfl>* wdf, cpx<dfl>* Sdf, long long n3,
                         unsigned long long* zero_count) {
  unsigned long long zs = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> hv = h[i];
    const double nv = N[i];
    if (hcopy) hcopy[i] = hv;
    if (Ncopy) Ncopy[i] = nv;
    const cpx<double> w = {hv.x * nv, hv.y * nv};
    double m;
    const cpx<double> s = csqrt_principal(w, m);
    S64[i] = s;
    const cpx<dfl> sd = c_from_c64<dfl>(s);
    Sdf[i] = sd;
    S32[i] = {sd.x.hi, sd.y.hi};
    if (w64) w64[i] = w;
    if (wdf) {
      const cpx<dfl> wd = c_from_c64<dfl>(w);
      wdf[i] = wd;
      if (w32) w32[i] = {wd.x.hi, wd.y.hi};
    } else if (w32) {
      w32[i] = ccast<float>(w);
    }
    const bool zero = m == 0.0;
    if (zero) ++zs;
    if (Sinv) {
      const double im = zero ? 0.0 : 1.0 / m;
      Sinv[i] = {s.x * im, -s.y * im};
    }
  }
  if (zs) atomicAdd(zero_count, zs);
}

// Copies of the solver's small control data (scalar heads, tolerances, skip
// flags, fault and count words) between device memory and mapped pinned host
// memory, made by one CTA instead of a copy engine.  The solver reads and
// writes these on the host between launches; a copy engine busy with a
// caller's large transfer on another stream would hold them back for the
// whole transfer.  rows blocks of `bytes` bytes at the given pitches, in
// 8-byte words when every address, size and pitch allows.
__global__ void k_small_copy(const unsigned char* src, unsigned char* dst, long long bytes, long long spitch,
                             long long dpitch, int rows) {
  const bool words = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) |
                       uintptr_t(bytes) | uintptr_t(spitch) | uintptr_t(dpitch)) & 7u) == 0;
  for (int r = 0; r < rows; ++r) {
    const unsigned char* sr = src + r * spitch;
    unsigned char* dr = dst + r * dpitch;
    if (words) {
      const unsigned long long* s8 = reinterpret_cast<const unsigned long long*>(sr);
      unsigned long long* d8 = reinterpret_cast<unsigned long long*>(dr);
      for (long long i = threadIdx.x; i < bytes / 8; i += blockDim.x) d8[i] = s8[i];
    } else {
      for (long long i = threadIdx.x; i < bytes; i += blockDim.x) dr[i] = sr[i];
    }
  }
}

// dst = src for n16 16-byte words of device memory (an SM copy, for the same
// reason as k_small_copy).
__global__ void k_copy16(const uint4* __restrict__ src, uint4* __restrict__ dst, long long n16) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n16;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

// Spectrum of the kernel cube: keep the (L/2+1)^3 distinct entries of the
// even cube and fold in c_S |Delta| / L^3.
__global__ void k_extract_ghat(const cpx<double>* __restrict__ cube, cpx<double>* g64,
                               cpx<float>* g32, cpx<dfl>* gdf, int ld, int H, double scale) {
  const long long total = (long long)H * H * H;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int m1 = int(i % H), m2 = int((i / H) % H), m3 = int(i / ((long long)H * H));
    const cpx<double> v = cube[((long long)m3 * ld + m2) * ld + m1];
    const cpx<double> s = {v.x * scale, v.y * scale};
    if (g64) g64[i] = s;   // a lean plan keeps no FP64 spectrum
    g32[i] = ccast<float>(s);
    gdf[i] = c_from_c64<dfl>(s);
  }
}

// A saved FP64 spectrum (count entries) into the FP32 and paired-FP32 copies.
__global__ void k_spectrum_convert(const cpx<double>* __restrict__ g64, long long count, cpx<float>* g32,
                                   cpx<dfl>* gdf) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> v = g64[i];
    g32[i] = ccast<float>(v);
    gdf[i] = c_from_c64<dfl>(v);
  }
}

// FP32 spectrum in the order the Z pass reads it: for each my and each block
// of 16 kx columns, the entries mz = 0..L/2 as rows of 16 (one contiguous
// slice per Z tile).  gz[((my * (L/16) + cb) * H + mz) * 16 + c] =
// g32[(mz * H + my) * H + m(cb*16 + c)].
__global__ void k_build_ghatZ(const cpx<float>* __restrict__ g32, cpx<float>* gz, int L, int H) {
  constexpr int G = kZGroup;
  const long long total = (long long)H * (L / G) * H * G;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = int(i % G);
    const long long r = i / G;
    const int mz = int(r % H);
    const long long t = r / H;
    const int cb = int(t % (L / G));
    const int my = int(t / (L / G));
    const int kx = cb * G + c;
    const int mx = kx <= L / 2 ? kx : L - kx;
    gz[i] = g32[((long long)mz * H + my) * H + mx];
  }
}

// Reduction helper for the vector kernels: two double2 partials per block.
__device__ __forceinline__ void block_partial2(double2 a, double2 b, double2* red,
                                               double2* partials) {
  a = warp_sum2(a);
  b = warp_sum2(b);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) { red[w] = a; red[32 + w] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 sa = make_double2(0.0, 0.0), sb = make_double2(0.0, 0.0);
    for (int i = 0; i < nw; ++i) {
      sa.x += red[i].x; sa.y += red[i].y;
      sb.x += red[32 + i].x; sb.y += red[32 + i].y;
    }
    partials[2 * blockIdx.x] = sa;
    partials[2 * blockIdx.x + 1] = sb;
  }
}

// Right-hand side of the symmetrised system: u0 = rhs or exp(ik alpha . x_p)
// (Eq. 2.4, cell centres), b = S u0; sum |b|^2 -> sc->sum.x.  The plane wave
// factors over the axes, exp(ik(a_x x + a_y y + a_z z)) = e_x(ix) e_y(iy)
// e_z(iz), so each block evaluates 3n FP64 phases into shared memory and
// every cell costs two complex products.
// Phase factors of the separable plane wave, once per right-hand side:
// out[rb][axis * n + i] = exp(i k_rb a_rb,axis (o_axis + (i + 1/2) d)).
__global__ void k_phases(const double* __restrict__ kvals, const double* __restrict__ dirs, int n, double d,
                         double ox, double oy, double oz, cpx<double>* out) {
  const int rb = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * n) return;
  const int axis = t / n, i = t - axis * n;
  const double o = axis == 0 ? ox : (axis == 1 ? oy : oz);
  double sn, cs;
  sincos(kvals[rb] * dirs[3 * rb + axis] * (o + (i + 0.5) * d), &sn, &cs);
  out[(long long)rb * 3 * n + t] = {cs, sn};
}

__global__ void k_rhs(const cpx<double>* __restrict__ rhs, const cpx<double>* __restrict__ S,
                      cpx<double>* u0, cpx<double>* b, int n, const cpx<double>* __restrict__ phases,
                      Scalars* sc0, double2* partials0) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<double>* e = reinterpret_cast<cpx<double>*>(smraw);   // [3][n]
  __shared__ double2 red[64];
  __shared__ int s_last;
  const int rb = blockIdx.y;                                  // right-hand side of the batch
  const long long n3 = (long long)n * n * n;
  Scalars* sc = sc0 + rb;
  double2* partials = partials0 + (long long)rb * gridDim.x;
  if (rhs != nullptr) rhs += rb * n3;
  if (u0 != nullptr) u0 += rb * n3;
  b += rb * n3;
  if (rhs == nullptr) {   // the 3n phase factors of this right-hand side (k_phases)
    const cpx<double>* ph = phases + (long long)rb * 3 * n;
    for (int t = threadIdx.x; t < 3 * n; t += blockDim.x) e[t] = ph[t];
    __syncthreads();
  }
  double acc = 0.0;
  // blocks take whole lines (iz, iy): one index division per line, and the
  // line's phase e_y e_z once per thread; threads run along x
  for (int line = blockIdx.x; line < n * n; line += gridDim.x) {
    const int iz = line / n, iy = line - iz * n;
    const cpx<double> pyz = rhs == nullptr ? cmul(e[n + iy], e[2 * n + iz]) : cpx<double>{0.0, 0.0};
    for (int ix = threadIdx.x; ix < n; ix += blockDim.x) {
      const long long i = (long long)line * n + ix;
      const cpx<double> u = rhs != nullptr ? rhs[i] : cmul(e[ix], pyz);
      if (u0 != nullptr) u0[i] = u;
      const cpx<double> bv = cmul(S[i], u);
      b[i] = bv;
      acc += bv.x * bv.x + bv.y * bv.y;
    }
  }
  block_partial(make_double2(acc, 0.0), red, partials);
  if (last_block_arrives(sc, s_last)) finalize(sc, partials, gridDim.x, FIN_SUM, red);
}

// Adjoint right-hand side b = S^-1 conj(e); sum |b|^2 -> sc->sum.x.
__global__ void k_adj_rhs(const cpx<double>* __restrict__ ec, const cpx<double>* __restrict__ S,
                          cpx<double>* b, long long n3, Scalars* sc, double2* partials) {
  __shared__ double2 red[64];
  __shared__ int s_last;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> bv = cdivd(ec[i], S[i]);
    b[i] = bv;
    acc += bv.x * bv.x + bv.y * bv.y;
  }
  block_partial(make_double2(acc, 0.0), red, partials);
  if (last_block_arrives(sc, s_last)) finalize(sc, partials, gridDim.x, FIN_SUM, red);
}

// COCG start: x = 0, rho = r^T r, ||r||^2; sets tol/maxit and the flags.
// Sums in T over 8 elements per thread, then in FP64.
template <class T>
__global__ void k_cocg_init(const cpx<T>* __restrict__ r, cpx<T>* x, long long n3, Scalars* sc0,
                            double2* partials0, const double* __restrict__ tols, int maxit, int zero_x) {
  __shared__ double2 red[64];
  __shared__ int s_last;
  const int rb = blockIdx.y;
  r += rb * n3;
  x += rb * n3;
  Scalars* sc = sc0 + rb;
  double2* partials = partials0 + 2LL * rb * gridDim.x;
  double2 rho = make_double2(0.0, 0.0);
  double nn = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = blockIdx.x * (long long)blockDim.x + threadIdx.x; base < n3;
       base += 8 * stride) {
    cpx<T> rs = czero<T>();
    T ns = T(0);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const long long i = base + u * stride;
      if (i < n3) {
        const cpx<T> rv = r[i];
        if (zero_x) x[i] = czero<T>();   // else x holds an initial guess whose residual is r
        rs = rs + cmul(rv, rv);
        ns += rv.x * rv.x + rv.y * rv.y;
      }
    }
    rho.x += double(rs.x);
    rho.y += double(rs.y);
    nn += double(ns);
  }
  block_partial2(rho, make_double2(nn, 0.0), red, partials);
  if (last_block_arrives(sc, s_last)) {
    if (threadIdx.x == 0) {
      sc->tol = tols[rb];
      sc->maxit = maxit;
    }
    finalize(sc, partials, gridDim.x, FIN_INIT, red);
  }
}

// Compensated (Kahan) FP32 accumulator: keeps the sum of many FP32 terms
// accurate to about FP32 rounding of the total, without FP64 arithmetic.
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// COCG update: x += alpha p, r -= alpha q; rho' = r^T r and ||r||^2 of the new
// residual.  FP64 vectors: sums over 8 elements per thread in FP64.
template <class T>
__global__ void k_cocg_update(cpx<T>* __restrict__ x, const cpx<T>* __restrict__ p,
                              cpx<T>* __restrict__ r, const cpx<T>* __restrict__ q, long long n3,
                              Scalars* sc0, double2* partials0) {
  __shared__ double2 red[64];
  __shared__ int s_last;
  const int rb = blockIdx.y;
  x += rb * n3; p += rb * n3; r += rb * n3; q += rb * n3;
  Scalars* sc = sc0 + rb;
  double2* partials = partials0 + 2LL * rb * gridDim.x;
  if (sc->done != 0) return;
  const double2 ad = sc->alpha;
  const cpx<T> al = {T(ad.x), T(ad.y)};
  double2 rho = make_double2(0.0, 0.0);
  double nn = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = blockIdx.x * (long long)blockDim.x + threadIdx.x; base < n3;
       base += 8 * stride) {
    cpx<T> rs = czero<T>();
    T ns = T(0);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const long long i = base + u * stride;
      if (i < n3) {
        const cpx<T> pv = p[i], qv = q[i];
        cpx<T> xv = x[i], rv = r[i];
        xv = xv + cmul(al, pv);
        rv = rv - cmul(al, qv);
        x[i] = xv;
        r[i] = rv;
        rs = rs + cmul(rv, rv);
        ns += rv.x * rv.x + rv.y * rv.y;
      }
    }
    rho.x += double(rs.x);
    rho.y += double(rs.y);
    nn += double(ns);
  }
  block_partial2(rho, make_double2(nn, 0.0), red, partials);
  if (last_block_arrives(sc, s_last)) finalize(sc, partials, gridDim.x, FIN_UPDATE, red);
}

// FP32 vectors: two complex numbers per 16-byte access, all loads of an
// unrolled group issued before any arithmetic, Kahan-compensated FP32 sums
// widened to FP64 once per thread.
template <>
__global__ void k_cocg_update<float>(cpx<float>* __restrict__ x, const cpx<float>* __restrict__ p,
                                     cpx<float>* __restrict__ r, const cpx<float>* __restrict__ q,
                                     long long n3, Scalars* sc0, double2* partials0) {
  __shared__ double2 red[64];
  __shared__ int s_last;
  const int rb = blockIdx.y;
  x += rb * n3; p += rb * n3; r += rb * n3; q += rb * n3;
  Scalars* sc = sc0 + rb;
  double2* partials = partials0 + 2LL * rb * gridDim.x;
  if (sc->done != 0) return;
  const double2 ad = sc->alpha;
  const float ar = float(ad.x), ai = float(ad.y);
  KahanF kr, ki, kn;
  const long long nv = n3 / 2;                        // float4 = two complex numbers
  float4* x4 = reinterpret_cast<float4*>(x);
  float4* r4 = reinterpret_cast<float4*>(r);
  const float4* p4 = reinterpret_cast<const float4*>(p);
  const float4* q4 = reinterpret_cast<const float4*>(q);
  const long long stride = (long long)gridDim.x * blockDim.x;
  constexpr int U = 4;
  for (long long base = blockIdx.x * (long long)blockDim.x + threadIdx.x; base < nv; base += U * stride) {
    float4 pv[U], qv[U], xv[U], rv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long i = base + u * stride;
      if (i < nv) { pv[u] = __ldcs(p4 + i); qv[u] = __ldcs(q4 + i); xv[u] = x4[i]; rv[u] = r4[i]; }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long i = base + u * stride;
      if (i < nv) {
        float4 X = xv[u], R = rv[u];
        X.x += ar * pv[u].x - ai * pv[u].y;  X.y += ar * pv[u].y + ai * pv[u].x;
        X.z += ar * pv[u].z - ai * pv[u].w;  X.w += ar * pv[u].w + ai * pv[u].z;
        R.x -= ar * qv[u].x - ai * qv[u].y;  R.y -= ar * qv[u].y + ai * qv[u].x;
        R.z -= ar * qv[u].z - ai * qv[u].w;  R.w -= ar * qv[u].w + ai * qv[u].z;
        x4[i] = X;
        r4[i] = R;
        kr.add(R.x * R.x - R.y * R.y + R.z * R.z - R.w * R.w);
        ki.add(2.f * (R.x * R.y + R.z * R.w));
        kn.add(R.x * R.x + R.y * R.y + R.z * R.z + R.w * R.w);
      }
    }
  }
  if ((n3 & 1) && blockIdx.x == 0 && threadIdx.x == 0) {   // odd length: the last element
    const long long i = n3 - 1;
    cpx<float> X = x[i], R = r[i];
    const cpx<float> P = p[i], Q = q[i];
    X.x += ar * P.x - ai * P.y;  X.y += ar * P.y + ai * P.x;
    R.x -= ar * Q.x - ai * Q.y;  R.y -= ar * Q.y + ai * Q.x;
    x[i] = X;
    r[i] = R;
    kr.add(R.x * R.x - R.y * R.y);
    ki.add(2.f * R.x * R.y);
    kn.add(R.x * R.x + R.y * R.y);
  }
  block_partial2(make_double2(double(kr.s) - double(kr.c), double(ki.s) - double(ki.c)),
                 make_double2(double(kn.s) - double(kn.c), 0.0), red, partials);
  if (last_block_arrives(sc, s_last)) finalize(sc, partials, gridDim.x, FIN_UPDATE, red);
}

// Mixed refinement: r32 = r64 / ||r64||.
__global__ void k_normalise_to_f32(const cpx<double>* __restrict__ r64, cpx<float>* r32,
                                   long long n3, const double* __restrict__ invs) {
  const int rb = blockIdx.y;
  const double inv = invs[rb];
  r64 += rb * n3;
  r32 += rb * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> v = r64[i];
    r32[i] = {float(v.x * inv), float(v.y * inv)};
  }
}

// Mixed refinement: w += scale * d32.
__global__ void k_accumulate(cpx<double>* w, const cpx<float>* __restrict__ d32, long long n3,
                             const double* __restrict__ scales) {
  const int rb = blockIdx.y;
  const double scale = scales[rb];
  if (scale == 0.0) return;
  w += rb * n3;
  d32 += rb * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<float> dv = d32[i];
    cpx<double> wv = w[i];
    wv.x += scale * double(dv.x);
    wv.y += scale * double(dv.y);
    w[i] = wv;
  }
}

// u = w / S = w * (1/S) (every S != 0; 1/S is kept by the plan).
__global__ void k_recover(const cpx<double>* __restrict__ w, const cpx<double>* __restrict__ Sinv,
                          const cpx<double>* __restrict__ S, cpx<double>* u, long long n3) {
  w += blockIdx.y * n3;
  u += blockIdx.y * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3;
       i += (long long)gridDim.x * blockDim.x)
    u[i] = Sinv != nullptr ? cmul(w[i], Sinv[i]) : cdivd(w[i], S[i]);   // lean plans keep no 1/S
}

// Adjoint gradient: psi = S z, t = (conj(e) - psi) u,
// grad_h = -2 conj(t / h), grad_N = -2 Re(t / N).
__global__ void k_gradient(const cpx<double>* __restrict__ ec, const cpx<double>* __restrict__ z,
                           const cpx<double>* __restrict__ u, const cpx<double>* __restrict__ S,
                           const cpx<double>* __restrict__ h, const double* __restrict__ N,
                           cpx<double>* gh, double* gN, long long n3) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> psi = cmul(S[i], z[i]);
    const cpx<double> t = cmul(ec[i] - psi, u[i]);
    const cpx<double> th = cdivd(t, h[i]);
    gh[i] = {-2.0 * th.x, 2.0 * th.y};
    gN[i] = -2.0 * t.x / N[i];
  }
}

// Cell charges of Eq. 2.13 summed over a cell: Q_m = coef * h_m N_m u_m with
// coef = -c_S |Delta| (every particle of cell m carries -c_S a^(2-kappa) h u,
// and a^(2-kappa) times their number is N_m |Delta|).
__global__ void k_charges(const cpx<double>* __restrict__ u, const cpx<double>* __restrict__ h,
                          const double* __restrict__ N, double coef, cpx<double>* Q, long long n3) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> hu = cmul(h[i], u[i]);
    const double s = coef * N[i];
    Q[i] = {s * hu.x, s * hu.y};
  }
}

// Field of Eq. 2.10 by direct summation, first stage: block (p, s) adds
// G(x_p, x_m) Q_m over the cells m of slice s (cells m = s, s + S, ...
// strided by threads) and writes one partial per (point, slice).  A cell
// whose point coincides with x_p (r <= 1e-9 d) is left out.
__global__ void k_field_partial(const cpx<double>* __restrict__ Q, const double* __restrict__ pts, int npts,
                                int n, double d, double ox, double oy, double oz, double k,
                                double2* partials) {
  __shared__ double2 red[32];
  const long long n3 = (long long)n * n * n;
  const int S = gridDim.y;
  const long long per = (n3 + S - 1) / S;
  const long long m0 = blockIdx.y * per;
  const long long m1 = m0 + per < n3 ? m0 + per : n3;
  const double inv4pi = 1.0 / (4.0 * kPi);
  for (int pi = blockIdx.x; pi < npts; pi += gridDim.x) {
    const double px = pts[3 * pi], py = pts[3 * pi + 1], pz = pts[3 * pi + 2];
    double ar = 0.0, ai = 0.0;
    for (long long m = m0 + threadIdx.x; m < m1; m += blockDim.x) {
      const unsigned mu = unsigned(m), nu = unsigned(n);   // n^3 <= 2^30: 32-bit division
      const unsigned line = mu / nu;
      const int ix = int(mu - line * nu), iy = int(line % nu), iz = int(line / nu);
      const double dx = px - (ox + (ix + 0.5) * d);
      const double dy = py - (oy + (iy + 0.5) * d);
      const double dz = pz - (oz + (iz + 0.5) * d);
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      if (r > 1e-9 * d) {
        double sn, cs;
        sincos(k * r, &sn, &cs);
        const double g = inv4pi / r;
        const cpx<double> q = Q[m];
        ar += g * (cs * q.x - sn * q.y);
        ai += g * (cs * q.y + sn * q.x);
      }
    }
    const double2 v = warp_sum2(make_double2(ar, ai));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double2 t = make_double2(0.0, 0.0);
      for (int i = 0; i < (int)(blockDim.x + 31) / 32; ++i) { t.x += red[i].x; t.y += red[i].y; }
      partials[(long long)pi * S + blockIdx.y] = t;
    }
  }
}

// Second stage: out_p = sum of the S partials of point p in slice order, plus
// the incident wave exp(i k a . x_p) when add_u0.
__global__ void k_field_finish(const double2* __restrict__ partials, int S, const double* __restrict__ pts,
                               int npts, double k, double ax, double ay, double az, int add_u0,
                               cpx<double>* out) {
  for (int pi = blockIdx.x * blockDim.x + threadIdx.x; pi < npts; pi += gridDim.x * blockDim.x) {
    double2 t = make_double2(0.0, 0.0);
    for (int s = 0; s < S; ++s) {
      const double2 v = partials[(long long)pi * S + s];
      t.x += v.x;
      t.y += v.y;
    }
    if (add_u0) {
      double sn, cs;
      sincos(k * (ax * pts[3 * pi] + ay * pts[3 * pi + 1] + az * pts[3 * pi + 2]), &sn, &cs);
      t.x += cs;
      t.y += sn;
    }
    out[pi] = {t.x, t.y};
  }
}

// Initial guess of the symmetrised system from a guess of u: w = S x0, per system.
__global__ void k_scale_guess(const cpx<double>* __restrict__ x0, const cpx<double>* __restrict__ S,
                              cpx<double>* w, long long n3) {
  x0 += blockIdx.y * n3;
  w += blockIdx.y * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3;
       i += (long long)gridDim.x * blockDim.x)
    w[i] = cmul(S[i], x0[i]);
}

// Widen a complex64 vector to complex128 / narrow complex128 to complex64.
__global__ void k_widen(const cpx<float>* __restrict__ a, cpx<double>* b, long long n3) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = ccast<double>(a[i]);
}

}  // namespace ori
