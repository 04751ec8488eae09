// passes_impl.cuh - kernels of the five FFT passes and their launchers.
// Included by passes_inst.cu, compiled once per arithmetic and part of the passes.
#pragma once

#include "dfloat.cuh"
#include "dfft.cuh"
#include "passes.cuh"
#include "scalars.cuh"

#include <type_traits>

namespace ori {

// Asynchronous 16-byte global -> shared copies (cp.async, L2 only) and their group fences.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Bulk copies (TMA) into shared memory with mbarrier completion.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return unsigned(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// orders this thread's earlier shared-memory accesses before later async-proxy (TMA) writes
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase `parity` of a barrier: false once kMbarWaitNs
// have passed (or kMbarTries unsuccessful tries, should the timer stand still).
constexpr unsigned long long kMbarWaitNs = 2000000000ull;
constexpr int kMbarTries = 1 << 26;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (int i = 0; i < kMbarTries; ++i) {
    if (mbar_test(bar, parity)) return true;
    if (globaltimer_ns() - t0 > kMbarWaitNs) return false;
  }
  return false;
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(smem_addr(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

// z * w (SIGN > 0) or z * conj(w) (SIGN < 0) for a twiddle value w already loaded.
template <int SIGN, class T>
__device__ __forceinline__ cpx<T> tw_mul_val(cpx<T> z, cpx<T> w) {
  return cmul(z, cpx<T>{w.x, SIGN > 0 ? w.y : -w.y});
}

// Two-dimensional twiddle table of a two-stage length-L transform:
// tab2[k1 * L2 + j] = tab[(j * k1) mod L] for k1 < L1, j < L2 (L entries), so
// that a thread with fixed j (or fixed k1) finds its twiddles at constant
// offsets from one base pointer.
template <int L, int L2X = Split<L>::L2, class T>
__device__ __forceinline__ void fill_tw2(cpx<T>* tab2, const cpx<T>* tab, int tid, int nt) {
  constexpr int L2 = L2X;
  for (int i = tid; i < L; i += nt) {
    const int k1 = i / L2, j = i - k1 * L2;
    tab2[i] = tab[(j * k1) & (L - 1)];
  }
}

// Lines per CTA of the FP32 contiguous (X) passes: 256 threads of L2 each.
template <int L>
constexpr int lines_contig_f32() {
  constexpr int want = 256 / Split<L>::L2;
  return want < 1 ? 1 : want;
}

// Lines per tile of the persistent FP32 X passes: 128 threads of L2 each.
template <int L>
constexpr int xpipe_cols() {
  constexpr int c = lines_contig_f32<L>() / 2;
  return c < 1 ? 1 : c;
}

// ---------------------------------------------------------------------------
// Prologue of the X forward pass: the value of the (zero-padded) field that
// enters the transform at cell (line, j) with j < n.
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ int signed_offset(int j, int L) { return j <= L / 2 ? j : j - L; }

template <class T>
__device__ __forceinline__ cpx<T> x_beta(const XArgs& a) {
  if (a.mode != PRO_COCG) return czero<T>();
  const double2 bd = *reinterpret_cast<const double2*>(a.beta);
  return c_from_c64<T>(cpx<double>{bd.x, bd.y});
}

// beta: the COCG coefficient in the pass arithmetic, converted once per thread (x_beta).
template <class T>
__device__ __forceinline__ cpx<T> x_prologue(const XArgs& a, long long line, int j, int L, cpx<T> b) {
  const long long i = line * a.n + j;
  switch (a.mode) {
    case PRO_SCALE: {
      const cpx<T> s = ldgc(reinterpret_cast<const cpx<T>*>(a.scale) + i);
      const cpx<T> v = reinterpret_cast<const cpx<T>*>(a.x)[i];
      return cmul(s, v);
    }
    case PRO_SCALE_D: {
      const cpx<T> s = ldgc(reinterpret_cast<const cpx<T>*>(a.scale) + i);
      const cpx<double> v = reinterpret_cast<const cpx<double>*>(a.x)[i];
      return cmul(s, c_from_c64<T>(v));
    }
    case PRO_COCG_FIRST: {
      const cpx<T> s = ldgc(reinterpret_cast<const cpx<T>*>(a.scale) + i);
      const cpx<T> r = reinterpret_cast<const cpx<T>*>(a.x)[i];
      reinterpret_cast<cpx<T>*>(a.p)[i] = r;
      return cmul(s, r);
    }
    case PRO_COCG: {
      const cpx<T> s = ldgc(reinterpret_cast<const cpx<T>*>(a.scale) + i);
      const cpx<T> r = reinterpret_cast<const cpx<T>*>(a.x)[i];
      cpx<T>* pp = reinterpret_cast<cpx<T>*>(a.p) + i;
      const cpx<T> p = r + cmul(b, *pp);
      *pp = p;
      return cmul(s, p);
    }
    default: {  // PRO_KERNEL: kernel cube entry at signed offsets (FP64)
      const int l3 = a.plane0 + int(line / a.lines_per_plane), l2 = int(line % a.lines_per_plane);
      const int s1 = signed_offset<T>(j, L), s2 = signed_offset<T>(l2, L), s3 = signed_offset<T>(l3, L);
      if (abs(s1) >= a.n || abs(s2) >= a.n || abs(s3) >= a.n) return czero<T>();
      const long long r2 = (long long)s1 * s1 + (long long)s2 * s2 + (long long)s3 * s3;
      if (r2 == 0) return czero<T>();           // p = q is excluded from the sum
      const double r = a.d * sqrt(double(r2));
      double sn, cs;
      sincos(a.k * r, &sn, &cs);
      const double g = 1.0 / (4.0 * kPi * r);   // G = exp(ikr) / (4 pi r)
      return c_from_c64<T>(cpx<double>{cs * g, sn * g});
    }
  }
}

// ---------------------------------------------------------------------------
// X forward pass (contiguous lines): x[line][0..n) -> T1[line][0..L)
// ---------------------------------------------------------------------------
template <class T, int L, int C, bool HALF>
__global__ void __launch_bounds__(Tile<L, C, T>::NT, Tile<L, C, T>::MINB) k_xfwd(XArgs a0) {
  const XArgs a = x_for_rhs(a0, blockIdx.y);
  using TL = Tile<L, C, T>;
  constexpr int L1 = TL::L1, L2 = TL::L2, NT = TL::NT;
  constexpr int PK = TL::PK, PC = TL::PC;
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw);
  if (a.done != nullptr && *a.done != 0) return;
  const cpx<T>* tw = reinterpret_cast<const cpx<T>*>(a.twL);
  const int tid = threadIdx.x;

  int c, j2;
  map_t<LAYOUT_CONTIG, C, L2>(tid, c, j2);
  const long long line = (long long)blockIdx.x * C + c;
  const bool ok = line < a.nlines;
  const cpx<T> beta = x_beta<T>(a);
  cpx<T> r[L1];
#pragma unroll
  for (int j1 = 0; j1 < L1; ++j1) {
    r[j1] = czero<T>();
    if (!HALF || j1 < L1 / 2) {
      const int j = j1 * L2 + j2;
      if (ok && j < a.n_in) r[j1] = x_prologue<T>(a, line, j, L, beta);
    }
  }
  dft<L1, -1, HALF>(r);
#pragma unroll
  for (int k1 = 1; k1 < L1; ++k1) r[k1] = twL_mul<-1>(r[k1], tw, (j2 * k1) & (L - 1));
#pragma unroll
  for (int k1 = 0; k1 < L1; ++k1) sm[c * PC + k1 * PK + j2] = settle(r[k1]);
  __syncthreads();
  cpx<T>* out = reinterpret_cast<cpx<T>*>(a.fft_out);
#pragma unroll
  for (int it = 0; it < L1 / L2; ++it) {
    int c2, k1;
    map_s<LAYOUT_CONTIG, C, L1>(tid + it * NT, c2, k1);
    cpx<T> b[L2];
#pragma unroll
    for (int j = 0; j < L2; ++j) b[j] = sm[c2 * PC + k1 * PK + j];
    dft<L2, -1, false>(b);
    const long long l2 = (long long)blockIdx.x * C + c2;
    if (l2 < a.nlines) {
      cpx<T>* o = out + l2 * a.line_len_out;
#pragma unroll
      for (int k2 = 0; k2 < L2; ++k2) o[k1 + L1 * k2] = settle(b[k2]);
    }
  }
}

// ---------------------------------------------------------------------------
// X forward pass, persistent and pipelined (FP32; prologues PRO_SCALE,
// PRO_COCG_FIRST and PRO_COCG, n even).  A tile is C consecutive lines,
// whose n input points per line form one contiguous block of each streamed
// vector (x or r, p for PRO_COCG, and the scale s); cp.async stages the
// blocks in shared memory, and the next tile's blocks are requested as soon
// as the prologue has read the current ones, so they stream in during the
// two DFT stages.
// ---------------------------------------------------------------------------

template <int L, int C>
struct XFwdPipe {
  using TL = Tile<L, C, float>;
  static constexpr int NT = TL::NT;
  static constexpr int STAGE = 3 * C * (L / 2);     // x or r, p, s: C lines of at most L/2 points each
  static constexpr size_t SMEM_BYTES = size_t(TL::SMEM_ELEMS + STAGE + L) * sizeof(cpx<float>);
};

template <int L, int C>
__device__ __forceinline__ void xfwd_prefetch(const XArgs& a, int tile, cpx<float>* R, cpx<float>* P, cpx<float>* G) {
  constexpr int NT = XFwdPipe<L, C>::NT;
  const long long line0 = (long long)tile * C;
  const long long left = a.nlines - line0;
  const int lines = left < C ? int(left) : C;
  const long long off = line0 * a.n;
  const int chunks = lines * a.n / 2;             // n even: 16 bytes = two complex values
  const cpx<float>* xs = reinterpret_cast<const cpx<float>*>(a.x) + off;
  const cpx<float>* ss = reinterpret_cast<const cpx<float>*>(a.scale) + off;
  for (int k = threadIdx.x; k < chunks; k += NT) {
    cp_async16(R + 2 * k, xs + 2 * k);
    cp_async16(G + 2 * k, ss + 2 * k);
  }
  if (a.mode == PRO_COCG) {
    const cpx<float>* ps = reinterpret_cast<const cpx<float>*>(a.p) + off;
    for (int k = threadIdx.x; k < chunks; k += NT) cp_async16(P + 2 * k, ps + 2 * k);
  }
  cp_async_commit();
}

template <int L, int C>
__global__ void __launch_bounds__(XFwdPipe<L, C>::NT, L > 1024 ? 1 : 2) k_xfwd_pipe(XArgs a0) {
  using T = float;
  const XArgs a = x_for_rhs(a0, blockIdx.y);
  using TL = Tile<L, C, T>;
  using XP = XFwdPipe<L, C>;
  constexpr int L1 = TL::L1, L2 = TL::L2, NT = TL::NT;
  constexpr int PK = TL::PK, PC = TL::PC;
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* E = reinterpret_cast<cpx<T>*>(smraw);
  cpx<T>* R = E + TL::SMEM_ELEMS;
  cpx<T>* P = R + XP::STAGE / 3;
  cpx<T>* G = P + XP::STAGE / 3;
  cpx<T>* TW = G + XP::STAGE / 3;
  if (a.done != nullptr && *a.done != 0) return;
  fill_tw2<L>(TW, reinterpret_cast<const cpx<T>*>(a.twL), threadIdx.x, NT);   // [k1][j] layout
  const int tid = threadIdx.x;
  const int ntiles = int((a.nlines + C - 1) / C);
  const cpx<T> beta = x_beta<T>(a);
  int c, j2;
  map_t<LAYOUT_CONTIG, C, L2>(tid, c, j2);
  cpx<T>* out = reinterpret_cast<cpx<T>*>(a.fft_out);
  int tile = blockIdx.x;
  if (tile < ntiles) xfwd_prefetch<L, C>(a, tile, R, P, G);
  for (; tile < ntiles; tile += gridDim.x) {
    cp_async_wait_all();
    __syncthreads();
    const long long line = (long long)tile * C + c;
    const bool ok = line < a.nlines;
    cpx<T> r[L1];
#pragma unroll
    for (int j1 = 0; j1 < L1; ++j1) {
      r[j1] = czero<T>();
      const int j = j1 * L2 + j2;
      if (j1 < L1 / 2 && ok && j < a.n) {
        const long long i = line * a.n + j;
        const cpx<T> s = G[c * a.n + j];
        cpx<T> v = R[c * a.n + j];
        if (a.mode == PRO_COCG) {
          v = v + cmul(beta, P[c * a.n + j]);
          reinterpret_cast<cpx<T>*>(a.p)[i] = v;
        } else if (a.mode == PRO_COCG_FIRST) {
          reinterpret_cast<cpx<T>*>(a.p)[i] = v;
        }
        r[j1] = cmul(s, v);
      }
    }
    __syncthreads();   // staged inputs consumed: request the next tile
    if (tile + (int)gridDim.x < ntiles) xfwd_prefetch<L, C>(a, tile + gridDim.x, R, P, G);
    dft<L1, -1, true>(r);
    const cpx<T>* t2 = TW + j2;
#pragma unroll
    for (int k1 = 1; k1 < L1; ++k1) r[k1] = tw_mul_val<-1>(r[k1], t2[k1 * L2]);
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) E[c * PC + k1 * PK + j2] = r[k1];
    __syncthreads();
#pragma unroll
    for (int it = 0; it < L1 / L2; ++it) {
      int c2, k1;
      map_s<LAYOUT_CONTIG, C, L1>(tid + it * NT, c2, k1);
      cpx<T> b[L2];
#pragma unroll
      for (int j = 0; j < L2; ++j) b[j] = E[c2 * PC + k1 * PK + j];
      dft<L2, -1, false>(b);
      const long long l2 = (long long)tile * C + c2;
      if (l2 < a.nlines) {
        cpx<T>* o = out + l2 * a.line_len_out;
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) o[k1 + L1 * k2] = b[k2];
      }
    }
  }
  cp_async_wait_all();
}

// Operator epilogue at cell i (conv value v): see EPI_* in passes.cuh.
// accT collects p^T q in the pass arithmetic, acc the FP64 sums.
template <class T>
__device__ __forceinline__ void x_epilogue(const XArgs& a, long long i, cpx<T> v, cpx<T>& accT, double2& acc) {
    switch (a.mode) {
      case EPI_PLUS: {
        const cpx<T> xi = reinterpret_cast<const cpx<T>*>(a.xin)[i];
        reinterpret_cast<cpx<T>*>(a.out)[i] = settle(xi + v);
      } break;
      case EPI_PLUS_S: {
        const cpx<T> xi = reinterpret_cast<const cpx<T>*>(a.xin)[i];
        const cpx<T> s = ldgc(reinterpret_cast<const cpx<T>*>(a.scale) + i);
        reinterpret_cast<cpx<T>*>(a.out)[i] = settle(xi + cmul(s, v));
      } break;
      case EPI_PLUS_D: {
        const cpx<double> xi = reinterpret_cast<const cpx<double>*>(a.xin)[i];
        const cpx<double> vd = c_to_c64(v);
        reinterpret_cast<cpx<double>*>(a.out)[i] = xi + vd;
      } break;
      case EPI_PLUS_S_D: {
        const cpx<double> xi = reinterpret_cast<const cpx<double>*>(a.xin)[i];
        const cpx<T> s = ldgc(reinterpret_cast<const cpx<T>*>(a.scale) + i);
        reinterpret_cast<cpx<double>*>(a.out)[i] = xi + c_to_c64(cmul(s, v));
      } break;
      case EPI_COCG: {
        const cpx<T> p = reinterpret_cast<const cpx<T>*>(a.xin)[i];
        const cpx<T> s = ldgc(reinterpret_cast<const cpx<T>*>(a.scale) + i);
        const cpx<T> q = settle(p + cmul(s, v));
        reinterpret_cast<cpx<T>*>(a.out)[i] = q;
        accT = accT + cmul(p, q);                 // p^T q, no conjugate
      } break;
      case EPI_RESID: {   // complex128 vectors whatever T is
        const cpx<double> w = reinterpret_cast<const cpx<double>*>(a.xin)[i];
        const cpx<double> b = reinterpret_cast<const cpx<double>*>(a.bvec)[i];
        const cpx<double> s = ldgc(reinterpret_cast<const cpx<double>*>(a.scale) + i);
        const cpx<double> rr = b - (w + cmul(s, c_to_c64(v)));
        reinterpret_cast<cpx<double>*>(a.out)[i] = rr;
        acc.x += rr.x * rr.x + rr.y * rr.y;
      } break;
      case EPI_RUPDATE: {  // r -= c (d + s v): residual update with this precision's operator
        const cpx<double> dv = c_to_c64(reinterpret_cast<const cpx<T>*>(a.xin)[i]);
        const cpx<T> s = ldgc(reinterpret_cast<const cpx<T>*>(a.scale) + i);
        const cpx<double> bd = c_to_c64(cmul(s, v));
        cpx<double>* rp = reinterpret_cast<cpx<double>*>(const_cast<void*>(a.bvec)) + i;
        cpx<double> rr = *rp;
        rr.x -= a.coef * (dv.x + bd.x);
        rr.y -= a.coef * (dv.y + bd.y);
        *rp = rr;
        acc.x += rr.x * rr.x + rr.y * rr.y;
      } break;
      default: {  // EPI_RECOVER: u = w / s where s != 0, else b - v (complex128)
        const cpx<double> w = reinterpret_cast<const cpx<double>*>(a.xin)[i];
        const cpx<double> s = ldgc(reinterpret_cast<const cpx<double>*>(a.scale) + i);
        const cpx<double> vd = c_to_c64(v);
        cpx<double> u;
        if (s.x != 0.0 || s.y != 0.0) {
          const double den = s.x * s.x + s.y * s.y;
          u = {(w.x * s.x + w.y * s.y) / den, (w.y * s.x - w.x * s.y) / den};
        } else {
          const cpx<double> b = reinterpret_cast<const cpx<double>*>(a.bvec)[i];
          u = b - vd;
        }
        reinterpret_cast<cpx<double>*>(a.out)[i] = u;
      } break;
    }
}

// ---------------------------------------------------------------------------
// X inverse pass + operator epilogue: T1[line][0..L) -> y[line][0..n)
// ---------------------------------------------------------------------------
template <class T, int L, int C>
__global__ void __launch_bounds__(Tile<L, C, T>::NT, Tile<L, C, T>::MINB) k_xinv(XArgs a0, Scalars* sc0, int fin) {
  const XArgs a = x_for_rhs(a0, blockIdx.y);
  Scalars* sc = sc0 == nullptr ? nullptr : sc0 + blockIdx.y;
  using TL = Tile<L, C, T>;
  constexpr int L1 = TL::L1, L2 = TL::L2, NT = TL::NT;
  constexpr int PKI = TL::PKI, PCI = TL::PCI;
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw);
  __shared__ double2 red[32];
  __shared__ int s_last;
  if (a.done != nullptr && *a.done != 0) return;
  const cpx<T>* tw = reinterpret_cast<const cpx<T>*>(a.twL);
  const cpx<T>* in = reinterpret_cast<const cpx<T>*>(a.in);
  const int tid = threadIdx.x;

  // stage A: DFT over k2 of X[k1 + L1 k2], twiddle, exchange
#pragma unroll
  for (int it = 0; it < L1 / L2; ++it) {
    int c2, k1;
    map_s<LAYOUT_CONTIG, C, L1>(tid + it * NT, c2, k1);
    const long long l2 = (long long)blockIdx.x * C + c2;
    cpx<T> b[L2];
#pragma unroll
    for (int k2 = 0; k2 < L2; ++k2)
      b[k2] = l2 < a.nlines ? in[l2 * a.line_len_in + k1 + L1 * k2] : czero<T>();
    dft<L2, +1, false>(b);
#pragma unroll
    for (int ja = 1; ja < L2; ++ja) b[ja] = twL_mul<+1>(b[ja], tw, (ja * k1) & (L - 1));
#pragma unroll
    for (int ja = 0; ja < L2; ++ja) sm[c2 * PCI + ja * PKI + k1] = settle(b[ja]);
  }
  __syncthreads();
  // stage B: DFT over k1 -> x[ja + L2 jb]
  int c, ja;
  map_t<LAYOUT_CONTIG, C, L2>(tid, c, ja);
  const long long line = (long long)blockIdx.x * C + c;
  cpx<T> r[L1];
#pragma unroll
  for (int k1 = 0; k1 < L1; ++k1) r[k1] = sm[c * PCI + ja * PKI + k1];
  dft<L1, +1, false>(r);

  double2 acc = make_double2(0.0, 0.0);
  cpx<T> accT = czero<T>();
  if (line < a.nlines) {
#pragma unroll
    for (int jb = 0; jb < L1 / 2; ++jb) {
      const int x = ja + L2 * jb;
      if (x < a.n) x_epilogue<T>(a, line * a.n + x, r[jb], accT, acc);
    }
    if constexpr (sizeof(T) != 4) {
      const cpx<double> accD = c_to_c64(accT);
      acc.x += accD.x;
      acc.y += accD.y;
    }
  }
  if (fin == FIN_NONE) return;
  bool done_partial = false;
  if constexpr (sizeof(T) == 4) {
    if (a.mode == EPI_COCG) {
      // FP32 sums (p^T q): reduce across the warp in FP32, widen once per warp
      float ax = accT.x, ay = accT.y;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
      }
      block_partial_lane0(make_double2(double(ax), double(ay)), red, a.partials + (long long)blockIdx.y * gridDim.x);
      done_partial = true;
    }
  }
  double2* parts = a.partials + (long long)blockIdx.y * gridDim.x;
  if (!done_partial) block_partial(acc, red, parts);
  if (last_block_arrives(sc, s_last)) finalize(sc, parts, gridDim.x, fin, red);
}

// ---------------------------------------------------------------------------
// X inverse pass, persistent and pipelined (FP32).  A CTA loops over tiles
// of C consecutive lines; a tile's L points per line (one contiguous block
// of C L complex values) are staged in shared memory by one bulk copy (or
// cp.async when an address is not 16-byte aligned), the exchange between the
// two DFT stages reuses that buffer in place, and as soon as the second stage
// has read the exchange the next tile starts streaming in, overlapping the
// inverse DFT and the epilogue.
// ---------------------------------------------------------------------------
template <int L, int C>
struct XInvPipe {
  using TL = Tile<L, C, float>;
  static constexpr int NT = TL::NT;
  static constexpr int BUF = (C * L > TL::SMEM_ELEMS) ? C * L : TL::SMEM_ELEMS;
  static constexpr int EPI = 2 * C * (L / 2);       // epilogue inputs: xin and s, C lines of <= L/2
  static constexpr size_t SMEM_BYTES = size_t(BUF + EPI) * sizeof(cpx<float>);
};

// The epilogue's complex64 inputs of a tile (xin and the scale s, n points
// per line) when every epilogue reads exactly those: the FP32 operator forms.
inline __host__ __device__ bool xinv_stage_epi(int mode) {
  return mode == EPI_COCG || mode == EPI_PLUS_S;
}

template <int L, int C>
__device__ __forceinline__ void xinv_prefetch_epi(const XArgs& a, int tile, cpx<float>* X, cpx<float>* G) {
  constexpr int NT = XInvPipe<L, C>::NT;
  if (xinv_stage_epi(a.mode)) {
    const long long line0 = (long long)tile * C;
    const long long left = a.nlines - line0;
    const int lines = left < C ? int(left) : C;
    const long long off = line0 * a.n;
    const int chunks = lines * a.n / 2;
    const cpx<float>* xs = reinterpret_cast<const cpx<float>*>(a.xin) + off;
    const cpx<float>* ss = reinterpret_cast<const cpx<float>*>(a.scale) + off;
    for (int k = threadIdx.x; k < chunks; k += NT) {
      cp_async16(X + 2 * k, xs + 2 * k);
      cp_async16(G + 2 * k, ss + 2 * k);
    }
  }
  cp_async_commit();   // always one group, so that the group count stays fixed
}
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }


template <int L, int C>
__device__ __forceinline__ void xinv_prefetch(const XArgs& a, int tile, cpx<float>* B) {
  constexpr int NT = XInvPipe<L, C>::NT;
  const long long line0 = (long long)tile * C;
  const long long left = a.nlines - line0;
  const int lines = left < C ? int(left) : C;
  const cpx<float>* src = reinterpret_cast<const cpx<float>*>(a.in) + line0 * L;
  const int chunks = lines * (L / 2);          // 16 bytes = two complex values
  for (int k = threadIdx.x; k < chunks; k += NT) cp_async16(B + 2 * k, src + 2 * k);
  cp_async_commit();
}

template <int L, int C>
__global__ void __launch_bounds__(XInvPipe<L, C>::NT, L > 1024 ? 1 : 3) k_xinv_pipe(XArgs a0, Scalars* sc0, int fin) {
  using T = float;
  using XP = XInvPipe<L, C>;
  const XArgs a = x_for_rhs(a0, blockIdx.y);
  Scalars* sc = sc0 == nullptr ? nullptr : sc0 + blockIdx.y;
  using TL = Tile<L, C, T>;
  constexpr int L1 = TL::L1, L2 = TL::L2, NT = TL::NT, NI = L1 / L2;
  constexpr int PKI = TL::PKI, PCI = TL::PCI;
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* B = reinterpret_cast<cpx<T>*>(smraw);
  cpx<T>* XI = B + XP::BUF;
  cpx<T>* GI = XI + XP::EPI / 2;
  __shared__ double2 red[32];
  __shared__ int s_last;
  __shared__ __align__(8) unsigned long long bars[2];   // bulk copies: [0] the T1 tile, [1] the epilogue inputs
  if (a.done != nullptr && *a.done != 0) return;
  const cpx<T>* tw = reinterpret_cast<const cpx<T>*>(a.twL);
  const int tid = threadIdx.x;
  const int ntiles = int((a.nlines + C - 1) / C);
  const bool staged = xinv_stage_epi(a.mode) && (a.n % 2 == 0);
  // Bulk copies (TMA, one thread issues them): a tile's C lines of T1 are one
  // contiguous block and its epilogue inputs two more (n even keeps every
  // offset and size a multiple of 16 bytes; the shared-memory regions start
  // on 16-byte boundaries when their element counts are even).
  constexpr bool kBulkFits = XP::BUF % 2 == 0 && (XP::EPI / 2) % 2 == 0;
  const bool bulk = kBulkFits && staged &&
                    ((reinterpret_cast<uintptr_t>(a.in) | reinterpret_cast<uintptr_t>(a.xin) |
                      reinterpret_cast<uintptr_t>(a.scale)) & 15u) == 0;
  unsigned ph_t = 0, ph_e = 0;      // barrier phases awaited next
  bool pend_t = false, pend_e = false, failed = false;
  if (bulk) {
    if (tid == 0) {
      mbar_init(&bars[0], 1);
      mbar_init(&bars[1], 1);
      fence_mbar_init();
    }
    __syncthreads();
  }
  auto lines_of = [&](int t) {
    const long long left = a.nlines - (long long)t * C;
    return left < C ? int(left) : C;
  };
  auto bulk_tile = [&](int t) {
    if (tid == 0) {
      const unsigned bytes = unsigned(lines_of(t)) * unsigned(L) * unsigned(sizeof(cpx<T>));
      fence_proxy_async();
      mbar_expect_tx(&bars[0], bytes);
      bulk_load(B, reinterpret_cast<const cpx<T>*>(a.in) + (long long)t * C * L, bytes, &bars[0]);
    }
    pend_t = true;
  };
  auto bulk_epi = [&](int t) {
    if (tid == 0) {
      const unsigned bytes = unsigned(lines_of(t)) * unsigned(a.n) * unsigned(sizeof(cpx<T>));
      const long long off = (long long)t * C * a.n;
      fence_proxy_async();
      mbar_expect_tx(&bars[1], 2 * bytes);
      bulk_load(XI, reinterpret_cast<const cpx<T>*>(a.xin) + off, bytes, &bars[1]);
      bulk_load(GI, reinterpret_cast<const cpx<T>*>(a.scale) + off, bytes, &bars[1]);
    }
    pend_e = true;
  };
  // Bounded wait for a bulk copy (all threads).  A copy that has not landed
  // after kMbarWaitNs sets *a.err; the CTA then stops working on tiles.
  auto bulk_wait = [&](unsigned long long* bar, unsigned& ph, bool& pend) -> bool {
    const bool ok = mbar_wait(bar, ph);
    if (__syncthreads_or(!ok)) {
      if (tid == 0 && a.err != nullptr) atomicExch(a.err, 1);
      return false;
    }
    ph ^= 1u;
    pend = false;
    return true;
  };
  int c, ja;
  map_t<LAYOUT_CONTIG, C, L2>(tid, c, ja);
  double2 acc = make_double2(0.0, 0.0);
  cpx<T> accT = czero<T>();
  int tile = blockIdx.x;
  // cp.async groups in flight, oldest first: [T1 of this tile] [epilogue inputs of this tile] [T1 of the next]
  if (tile < ntiles) {
    if (bulk) {
      bulk_tile(tile);
      bulk_epi(tile);
    } else {
      xinv_prefetch<L, C>(a, tile, B);
      if (staged) xinv_prefetch_epi<L, C>(a, tile, XI, GI);
      else cp_async_commit();
    }
  }
  for (; tile < ntiles; tile += gridDim.x) {
    if (bulk) {
      if (!bulk_wait(&bars[0], ph_t, pend_t)) { failed = true; break; }
    } else {
      cp_async_wait_1();   // this tile's T1 block has landed
      __syncthreads();
    }
    // stage A: DFT over k2 of X[k1 + L1 k2], twiddle
    cpx<T> b[NI][L2];
#pragma unroll
    for (int it = 0; it < NI; ++it) {
      int c2, k1;
      map_s<LAYOUT_CONTIG, C, L1>(tid + it * NT, c2, k1);
      const bool okl = (long long)tile * C + c2 < a.nlines;
#pragma unroll
      for (int k2 = 0; k2 < L2; ++k2) b[it][k2] = okl ? B[c2 * L + k1 + L1 * k2] : czero<T>();
      dft<L2, +1, false>(b[it]);
#pragma unroll
      for (int j = 1; j < L2; ++j) b[it][j] = twL_mul<+1>(b[it][j], tw, (j * k1) & (L - 1));
    }
    __syncthreads();   // raw tile consumed: the exchange reuses the buffer
#pragma unroll
    for (int it = 0; it < NI; ++it) {
      int c2, k1;
      map_s<LAYOUT_CONTIG, C, L1>(tid + it * NT, c2, k1);
#pragma unroll
      for (int j = 0; j < L2; ++j) B[c2 * PCI + j * PKI + k1] = b[it][j];
    }
    __syncthreads();
    // stage B: DFT over k1 -> x = ja + L2 jb
    cpx<T> r[L1];
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) r[k1] = B[c * PCI + ja * PKI + k1];
    __syncthreads();   // exchange consumed: the buffer takes the next tile
    if (bulk) {
      if (tile + (int)gridDim.x < ntiles) bulk_tile(tile + gridDim.x);
    } else if (tile + (int)gridDim.x < ntiles) {
      xinv_prefetch<L, C>(a, tile + gridDim.x, B);
    } else {
      cp_async_commit();
    }
    dft<L1, +1, false>(r);
    if (bulk) {
      if (!bulk_wait(&bars[1], ph_e, pend_e)) { failed = true; break; }
    } else {
      cp_async_wait_1();   // this tile's epilogue inputs have landed
      __syncthreads();
    }
    const long long line = (long long)tile * C + c;
    if (line < a.nlines) {
      if (staged) {
        cpx<T>* q = reinterpret_cast<cpx<T>*>(a.out);
#pragma unroll
        for (int jb = 0; jb < L1 / 2; ++jb) {
          const int x = ja + L2 * jb;
          if (x < a.n) {
            const cpx<T> pv = XI[c * a.n + x];
            const cpx<T> qv = pv + cmul(GI[c * a.n + x], r[jb]);
            q[line * a.n + x] = qv;
            if (a.mode == EPI_COCG) accT = accT + cmul(pv, qv);   // p^T q, no conjugate
          }
        }
      } else {
#pragma unroll
        for (int jb = 0; jb < L1 / 2; ++jb) {
          const int x = ja + L2 * jb;
          if (x < a.n) x_epilogue<T>(a, line * a.n + x, r[jb], accT, acc);
        }
      }
    }
    __syncthreads();   // epilogue inputs consumed
    if (tile + (int)gridDim.x < ntiles) {
      if (bulk) bulk_epi(tile + gridDim.x);
      else if (staged) xinv_prefetch_epi<L, C>(a, tile + gridDim.x, XI, GI);
      else cp_async_commit();
    }
  }
  if (failed) {   // leave no bulk copy writing into shared memory behind (bounded waits)
    if (pend_t) mbar_wait(&bars[0], ph_t);
    if (pend_e) mbar_wait(&bars[1], ph_e);
  }
  cp_async_wait_all();
  if (fin == FIN_NONE) return;
  double2* parts = a.partials + (long long)blockIdx.y * gridDim.x;
  if (a.mode == EPI_COCG) {
    // FP32 sums (p^T q): reduce across the warp in FP32, widen once per warp
    float ax = accT.x, ay = accT.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    block_partial_lane0(make_double2(double(ax), double(ay)), red, parts);
  } else {
    block_partial(acc, red, parts);
  }
  if (last_block_arrives(sc, s_last)) finalize(sc, parts, gridDim.x, fin, red);
}

// ---------------------------------------------------------------------------
// Strided passes (Y forward, Z convolution, Y inverse, and the plan's full
// forward transforms): a tile of C consecutive columns of L points.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int mirror_index(int k, int L) { return k <= L / 2 ? k : L - k; }

template <class T, int L, int C, int SMODE, bool HALF>
__global__ void __launch_bounds__(Tile<L, C, T>::NT) k_strided(SArgs a0) {
  const SArgs a = s_for_rhs(a0, blockIdx.y);
  using TL = Tile<L, C, T>;
  constexpr int L1 = TL::L1, L2 = TL::L2, NT = TL::NT;
  constexpr int PK = TL::PK, PC = TL::PC, PKI = TL::PKI, PCI = TL::PCI;
  constexpr int NI = L1 / L2;
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* sm = reinterpret_cast<cpx<T>*>(smraw);
  if (a.done != nullptr && *a.done != 0) return;
  const cpx<T>* tw = reinterpret_cast<const cpx<T>*>(a.twL);
  const int tid = threadIdx.x;
  const int outer = blockIdx.x / a.col_blocks;
  const int cb = blockIdx.x - outer * a.col_blocks;
  const cpx<T>* in = reinterpret_cast<const cpx<T>*>(a.in) + outer * a.in_outer + (long long)cb * C;
  cpx<T>* out = reinterpret_cast<cpx<T>*>(a.out) + outer * a.out_outer + (long long)cb * C;
  const int colmax = a.ncols - cb * C;

  cpx<T> b[NI][L2];
  if (SMODE != SMODE_INV) {
    int c, j2;
    map_t<LAYOUT_STRIDED, C, L2>(tid, c, j2);
    cpx<T> r[L1];
#pragma unroll
    for (int j1 = 0; j1 < L1; ++j1) {
      r[j1] = czero<T>();
      if (!HALF || j1 < L1 / 2) {
        const int j = j1 * L2 + j2;
        const int jr = (!HALF && a.mirror_in && j > L / 2) ? L - j : j;
        if (c < colmax && j < a.n_in) r[j1] = in[(long long)jr * a.in_pt + c];
      }
    }
    dft<L1, -1, HALF>(r);
#pragma unroll
    for (int k1 = 1; k1 < L1; ++k1) r[k1] = twL_mul<-1>(r[k1], tw, (j2 * k1) & (L - 1));
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) sm[c * PC + k1 * PK + j2] = settle(r[k1]);
    __syncthreads();
#pragma unroll
    for (int it = 0; it < NI; ++it) {
      int c2, k1;
      map_s<LAYOUT_STRIDED, C, L1>(tid + it * NT, c2, k1);
#pragma unroll
      for (int j = 0; j < L2; ++j) b[it][j] = sm[c2 * PC + k1 * PK + j];
      dft<L2, -1, false>(b[it]);
    }
    if (SMODE == SMODE_FWD) {
#pragma unroll
      for (int it = 0; it < NI; ++it) {
        int c2, k1;
        map_s<LAYOUT_STRIDED, C, L1>(tid + it * NT, c2, k1);
        if (c2 < colmax) {
#pragma unroll
          for (int k2 = 0; k2 < L2; ++k2) {
            const int k = k1 + L1 * k2;
            if (k < a.n_out) out[(long long)k * a.out_pt + c2] = settle(b[it][k2]);
          }
        }
      }
      return;
    }
    // Z convolution: multiply by the spectrum entry of (kx, ky, kz)
    const cpx<T>* gh = reinterpret_cast<const cpx<T>*>(a.ghat);
    const int my = mirror_index(outer, L);
#pragma unroll
    for (int it = 0; it < NI; ++it) {
      int c2, k1;
      map_s<LAYOUT_STRIDED, C, L1>(tid + it * NT, c2, k1);
      const int mx = mirror_index(min(cb * C + c2, L - 1), L);
#pragma unroll
      for (int k2 = 0; k2 < L2; ++k2) {
        const int mz = mirror_index(k1 + L1 * k2, L);
        const cpx<T> g = ldgc(gh + ((long long)mz * a.H + my) * a.H + mx);
        b[it][k2] = cmul(b[it][k2], g);
      }
    }
    __syncthreads();   // every read of the forward exchange is done
  } else {
#pragma unroll
    for (int it = 0; it < NI; ++it) {
      int c2, k1;
      map_s<LAYOUT_STRIDED, C, L1>(tid + it * NT, c2, k1);
#pragma unroll
      for (int k2 = 0; k2 < L2; ++k2)
        b[it][k2] = c2 < colmax ? in[(long long)(k1 + L1 * k2) * a.in_pt + c2] : czero<T>();
    }
  }
  // inverse stage A: DFT over k2, twiddle, exchange
#pragma unroll
  for (int it = 0; it < NI; ++it) {
    int c2, k1;
    map_s<LAYOUT_STRIDED, C, L1>(tid + it * NT, c2, k1);
    dft<L2, +1, false>(b[it]);
#pragma unroll
    for (int ja = 1; ja < L2; ++ja) b[it][ja] = twL_mul<+1>(b[it][ja], tw, (ja * k1) & (L - 1));
#pragma unroll
    for (int ja = 0; ja < L2; ++ja) sm[c2 * PCI + ja * PKI + k1] = settle(b[it][ja]);
  }
  __syncthreads();
  // inverse stage B
  int c, ja;
  map_t<LAYOUT_STRIDED, C, L2>(tid, c, ja);
  cpx<T> r[L1];
#pragma unroll
  for (int k1 = 0; k1 < L1; ++k1) r[k1] = sm[c * PCI + ja * PKI + k1];
  dft<L1, +1, false>(r);
  if (c < colmax) {
#pragma unroll
    for (int jb = 0; jb < L1; ++jb) {
      const int j = ja + L2 * jb;
      if (j < a.n_out) out[(long long)j * a.out_pt + c] = settle(r[jb]);
    }
  }
}

// ---------------------------------------------------------------------------
// X and Y passes for the paired-FP32 residual, shared-memory resident (see
// dfft.cuh): a tile of C lines (X) or C columns (Y) of L points per CTA.
// ---------------------------------------------------------------------------
template <int L, int C, class T>
struct LSmem {
  static constexpr int NT = C >= 4 ? 256 : 64 * C;
  static constexpr int MINB = C >= 4 ? 2 : 4;       // narrow tiles: more independent CTAs per SM
  static constexpr size_t X_ELEMS = size_t(L) * C;
  static constexpr size_t SMEM_BYTES = (X_ELEMS + size_t(L)) * sizeof(cpx<T>);
};

template <class T, int L, int C, int SMODE, bool HALF = true>
__global__ void __launch_bounds__(LSmem<L, C, T>::NT, LSmem<L, C, T>::MINB) k_strided_smem(SArgs a0) {
  const SArgs a = s_for_rhs(a0, blockIdx.y);
  using LS = LSmem<L, C, T>;
  constexpr int NT = LS::NT, S8 = L / 8;
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* X = reinterpret_cast<cpx<T>*>(smraw);
  cpx<T>* TW = X + LS::X_ELEMS;
  if (a.done != nullptr && *a.done != 0) return;
  const cpx<T>* twg = reinterpret_cast<const cpx<T>*>(a.twL);
  const int tid = threadIdx.x;
  for (int i = tid; i < L; i += NT) TW[i] = twg[i];
  const int outer = blockIdx.x / a.col_blocks;
  const int cb = blockIdx.x - outer * a.col_blocks;
  const cpx<T>* in = reinterpret_cast<const cpx<T>*>(a.in) + outer * a.in_outer + (long long)cb * C;
  cpx<T>* out = reinterpret_cast<cpx<T>*>(a.out) + outer * a.out_outer + (long long)cb * C;
  const int colmax = a.ncols - cb * C;
  if (SMODE == SMODE_FWD) {
    __syncthreads();
    for (int g = tid; g < C * S8; g += NT) {
      const int c = g % C, j = g / C;
      cpx<T> v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        v[t] = czero<T>();
        const int jj = j + t * S8;
        const int jr = (!HALF && a.mirror_in && jj > L / 2) ? L - jj : jj;
        if ((!HALF || t < 4) && c < colmax && jj < a.n_in) v[t] = in[(long long)jr * a.in_pt + c];
      }
      dft<8, -1, HALF>(v);
#pragma unroll
      for (int t = 1; t < 8; ++t) v[t] = twL_mul<-1>(v[t], TW, (j * t) & (L - 1));
#pragma unroll
      for (int t = 0; t < 8; ++t) st_stage(X + sidx<C>(j + t * S8, c), settle(v[t]));
    }
    __syncthreads();
    dif_rest<L, C>(X, TW, tid, NT);
    for (int e = tid; e < C * L; e += NT) {
      const int c = e % C, p = e / C;
      const int k = digit_rev<L>(p);
      if (c < colmax && k < a.n_out) out[(long long)k * a.out_pt + c] = ld_stage(X + sidx<C>(p, c));
    }
  } else {
    // the inverse by decimation in frequency with the inverse sign: the first
    // radix-8 stage reads the L input rows in natural order from global
    // memory, the others run in shared memory, and the n_out kept rows are
    // gathered from their digit-reversed positions
    __syncthreads();
    for (int g = tid; g < C * S8; g += NT) {
      const int c = g % C, j = g / C;
      cpx<T> v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int jj = j + t * S8;
        v[t] = (c < colmax && jj < a.n_in) ? in[(long long)jj * a.in_pt + c] : czero<T>();
      }
      dft<8, +1, false>(v);
#pragma unroll
      for (int t = 1; t < 8; ++t) v[t] = twL_mul<+1>(v[t], TW, (j * t) & (L - 1));
#pragma unroll
      for (int t = 0; t < 8; ++t) st_stage(X + sidx<C>(j + t * S8, c), settle(v[t]));
    }
    __syncthreads();
    dif_rest<L, C, +1>(X, TW, tid, NT);
    for (int e = tid; e < C * a.n_out; e += NT) {
      const int c = e % C, z = e / C;
      if (c < colmax) out[(long long)z * a.out_pt + c] = ld_stage(X + sidx<C>(inv_digit_rev<L>(z), c));
    }
  }
}

template <class T, int L, int C, bool HALF = true>
__global__ void __launch_bounds__(LSmem<L, C, T>::NT, LSmem<L, C, T>::MINB) k_xfwd_smem(XArgs a0) {
  const XArgs a = x_for_rhs(a0, blockIdx.y);
  using LS = LSmem<L, C, T>;
  constexpr int NT = LS::NT, S8 = L / 8;
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* X = reinterpret_cast<cpx<T>*>(smraw);
  cpx<T>* TW = X + LS::X_ELEMS;
  if (a.done != nullptr && *a.done != 0) return;
  const cpx<T>* twg = reinterpret_cast<const cpx<T>*>(a.twL);
  const int tid = threadIdx.x;
  for (int i = tid; i < L; i += NT) TW[i] = twg[i];
  __syncthreads();
  const cpx<T> beta = x_beta<T>(a);
  // first stage: consecutive threads take consecutive points of one line
  for (int g = tid; g < C * S8; g += NT) {
    const int j = g % S8, c = g / S8;
    const long long line = (long long)blockIdx.x * C + c;
    cpx<T> v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      v[t] = czero<T>();
      if ((!HALF || t < 4) && line < a.nlines && j + t * S8 < a.n_in) v[t] = x_prologue<T>(a, line, j + t * S8, L, beta);
    }
    dft<8, -1, HALF>(v);
#pragma unroll
    for (int t = 1; t < 8; ++t) v[t] = twL_mul<-1>(v[t], TW, (j * t) & (L - 1));
#pragma unroll
    for (int t = 0; t < 8; ++t) st_stage(X + sidx<C>(j + t * S8, c), settle(v[t]));
  }
  __syncthreads();
  dif_rest<L, C>(X, TW, tid, NT);
  cpx<T>* out = reinterpret_cast<cpx<T>*>(a.fft_out);
  for (int e = tid; e < C * L; e += NT) {
    const int k = e % L, c = e / L;
    const long long line = (long long)blockIdx.x * C + c;
    if (line < a.nlines) out[line * a.line_len_out + k] = ld_stage(X + sidx<C>(inv_digit_rev<L>(k), c));
  }
}

// The inverse X transform runs by decimation in frequency with the inverse
// sign: its first radix-8 stage takes each line's L points in natural order
// straight from global memory (eight independent coalesced loads per thread,
// no scattered shared-memory stores), the remaining stages run in shared
// memory, and the epilogue gathers the n kept points x < n from their
// digit-reversed positions, so its own global reads and writes are coalesced.
template <class T, int L, int C>
__global__ void __launch_bounds__(LSmem<L, C, T>::NT, LSmem<L, C, T>::MINB) k_xinv_smem(XArgs a0, Scalars* sc0, int fin) {
  const XArgs a = x_for_rhs(a0, blockIdx.y);
  Scalars* sc = sc0 == nullptr ? nullptr : sc0 + blockIdx.y;
  using LS = LSmem<L, C, T>;
  constexpr int NT = LS::NT, S8 = L / 8;
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* X = reinterpret_cast<cpx<T>*>(smraw);
  cpx<T>* TW = X + LS::X_ELEMS;
  __shared__ double2 red[32];
  __shared__ int s_last;
  if (a.done != nullptr && *a.done != 0) return;
  const cpx<T>* twg = reinterpret_cast<const cpx<T>*>(a.twL);
  const cpx<T>* in = reinterpret_cast<const cpx<T>*>(a.in);
  const int tid = threadIdx.x;
  for (int i = tid; i < L; i += NT) TW[i] = twg[i];
  __syncthreads();
  for (int g = tid; g < C * S8; g += NT) {
    const int j = g % S8, c = g / S8;
    const long long line = (long long)blockIdx.x * C + c;
    cpx<T> v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = line < a.nlines ? in[line * a.line_len_in + j + t * S8] : czero<T>();
    dft<8, +1, false>(v);
#pragma unroll
    for (int t = 1; t < 8; ++t) v[t] = twL_mul<+1>(v[t], TW, (j * t) & (L - 1));
#pragma unroll
    for (int t = 0; t < 8; ++t) st_stage(X + sidx<C>(j + t * S8, c), settle(v[t]));
  }
  __syncthreads();
  dif_rest<L, C, +1>(X, TW, tid, NT);
  double2 acc = make_double2(0.0, 0.0);
  cpx<T> accT = czero<T>();
  for (int e = tid; e < C * a.n; e += NT) {
    const int x = e % a.n, c = e / a.n;
    const long long line = (long long)blockIdx.x * C + c;
    if (line < a.nlines) x_epilogue<T>(a, line * a.n + x, ld_stage(X + sidx<C>(inv_digit_rev<L>(x), c)), accT, acc);
  }
  const cpx<double> accD = c_to_c64(accT);
  acc.x += accD.x;
  acc.y += accD.y;
  if (fin == FIN_NONE) return;
  double2* parts = a.partials + (long long)blockIdx.y * gridDim.x;
  block_partial(acc, red, parts);
  if (last_block_arrives(sc, s_last)) finalize(sc, parts, gridDim.x, fin, red);
}

// ---------------------------------------------------------------------------
// Launchers (dispatch on the padded length)
// ---------------------------------------------------------------------------
template <class T> constexpr int cols_strided() { return sizeof(T) == 4 ? 8 : 4; }
template <class T, int L> constexpr int lines_contig() {
  constexpr int want = (sizeof(T) == 4 ? 256 : 128) / Split<L>::L2;
  return want < 1 ? 1 : want;
}

template <int L>
cudaError_t launch_xfwd_pipe_L(const XArgs& a, cudaStream_t s, bool setup) {
  constexpr int C = xpipe_cols<L>();
  using XP = XFwdPipe<L, C>;
  auto kfn = k_xfwd_pipe<L, C>;
  static int per_sm = 0;
  if (setup) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(XP::SMEM_BYTES));
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn, XP::NT, XP::SMEM_BYTES);
    per_sm = (e == cudaSuccess && nb > 0) ? nb : 1;
    return e;
  }
  const long long ntiles = (a.nlines + C - 1) / C;
  const int nb = std::max(1, a.nrhs);
  const unsigned gx = unsigned(std::max(1LL, std::min(ntiles, (long long)std::max(1, a.sm_count) * std::max(1, per_sm) / nb)));
  kfn<<<dim3(gx, unsigned(nb)), XP::NT, XP::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

// The pipelined kernel serves the solver's prologues on whole contiguous lines
// of even length; the plan's kernel cube and the mixed-arithmetic prologue
// take the one-tile-per-CTA kernel.
inline bool xfwd_pipe_ok(const XArgs& a, int L) {
  return (a.mode == PRO_SCALE || a.mode == PRO_COCG_FIRST || a.mode == PRO_COCG) && a.n % 2 == 0 &&
         a.n_in == a.n && a.line_len_in == a.n && a.line_len_out == L && 2 * a.n <= L;
}

template <class T, int L, bool HALF>
cudaError_t launch_xfwd_reg_L(const XArgs& a, cudaStream_t s, bool setup) {
  if constexpr (sizeof(T) == 4 && HALF && L >= 64) {
    if (setup) {
      cudaError_t e = launch_xfwd_pipe_L<L>(a, s, true);
      if (e != cudaSuccess) return e;
    } else if (xfwd_pipe_ok(a, L)) {
      return launch_xfwd_pipe_L<L>(a, s, false);
    }
  }
  if constexpr (std::is_same<T, dfl>::value && HALF && L >= 64) {
    constexpr int CS = 2;   // two lines per CTA, four CTAs per SM
    using LS = LSmem<L, CS, T>;
    auto kfs = k_xfwd_smem<T, L, CS>;
    if (setup) return cudaFuncSetAttribute(kfs, cudaFuncAttributeMaxDynamicSharedMemorySize, int(LS::SMEM_BYTES));
    kfs<<<dim3(unsigned((a.nlines + CS - 1) / CS), unsigned(std::max(1, a.nrhs))), LS::NT, LS::SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
  }
  constexpr int C = lines_contig<T, L>();
  using TL = Tile<L, C, T>;
  auto kfn = k_xfwd<T, L, C, HALF>;
  if (setup) return cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(TL::SMEM_BYTES));
  const dim3 grid(unsigned((a.nlines + C - 1) / C), unsigned(std::max(1, a.nrhs)));
  kfn<<<grid, TL::NT, TL::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

template <int L>
cudaError_t launch_xinv_pipe_L(const XArgs& a, Scalars* sc, int fin, cudaStream_t s, bool setup, unsigned* nblocks) {
  constexpr int C = xpipe_cols<L>();
  using XP = XInvPipe<L, C>;
  auto kfn = k_xinv_pipe<L, C>;
  static int per_sm = 0;   // resident CTAs per SM, measured once at set-up
  const long long ntiles = (a.nlines + C - 1) / C;
  if (setup) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(XP::SMEM_BYTES));
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn, XP::NT, XP::SMEM_BYTES);
    per_sm = (e == cudaSuccess && nb > 0) ? nb : 1;
    if (nblocks) *nblocks = unsigned(std::max(1LL, std::min(ntiles, (long long)std::max(1, a.sm_count) * per_sm)));
    return e;
  }
  if (a.line_len_in != L) return cudaErrorInvalidValue;   // tiles are contiguous blocks of whole lines
  const int nb = std::max(1, a.nrhs);
  const unsigned gx = unsigned(std::max(1LL, std::min(ntiles, (long long)std::max(1, a.sm_count) * std::max(1, per_sm) / nb)));
  if (nblocks) *nblocks = gx;
  kfn<<<dim3(gx, unsigned(nb)), XP::NT, XP::SMEM_BYTES, s>>>(a, sc, fin);
  return cudaGetLastError();
}

template <class T, int L>
cudaError_t launch_xinv_reg_L(const XArgs& a, Scalars* sc, int fin, cudaStream_t s, bool setup, unsigned* nblocks) {
  if constexpr (sizeof(T) == 4 && L >= 64) {
    return launch_xinv_pipe_L<L>(a, sc, fin, s, setup, nblocks);
  } else if constexpr (std::is_same<T, dfl>::value && L >= 64) {
    constexpr int CS = 2;   // two lines per CTA, four CTAs per SM
    using LS = LSmem<L, CS, T>;
    auto kfs = k_xinv_smem<T, L, CS>;
    const unsigned grid = unsigned((a.nlines + CS - 1) / CS);
    if (nblocks) *nblocks = grid;
    if (setup) return cudaFuncSetAttribute(kfs, cudaFuncAttributeMaxDynamicSharedMemorySize, int(LS::SMEM_BYTES));
    kfs<<<dim3(grid, unsigned(std::max(1, a.nrhs))), LS::NT, LS::SMEM_BYTES, s>>>(a, sc, fin);
    return cudaGetLastError();
  } else {
    constexpr int C = lines_contig<T, L>();
    using TL = Tile<L, C, T>;
    auto kfn = k_xinv<T, L, C>;
    const unsigned grid = unsigned((a.nlines + C - 1) / C);
    if (nblocks) *nblocks = grid;
    if (setup) return cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(TL::SMEM_BYTES));
    kfn<<<dim3(grid, unsigned(std::max(1, a.nrhs))), TL::NT, TL::SMEM_BYTES, s>>>(a, sc, fin);
    return cudaGetLastError();
  }
}

template <class T, int L>
cudaError_t launch_yfwd_pipe_L(SArgs a, cudaStream_t s, bool setup, int sm_count);
template <int L>
cudaError_t launch_yinv_pipe_L(SArgs a, cudaStream_t s, bool setup, int sm_count);

template <class T, int L, int SMODE, bool HALF>
cudaError_t launch_strided_L(SArgs a, cudaStream_t s, bool setup);
template <class T, int L>
cudaError_t launch_zconv_L(SArgs a, cudaStream_t s, bool setup);

template <class T, int L, int SMODE, bool HALF>
cudaError_t launch_strided_reg_L(SArgs a, cudaStream_t s, bool setup) {
  if constexpr (sizeof(T) == 4 && SMODE == SMODE_FWD && HALF && L >= 64) {
    if (setup) {   // both schedules are set up; the plan picks one per launch
      cudaError_t e = launch_yfwd_pipe_L<T, L>(a, s, true, a.sm_count);
      if (e != cudaSuccess) return e;
    } else if (a.sched == SCHED_PERSISTENT) {
      return launch_yfwd_pipe_L<T, L>(a, s, false, a.sm_count);
    }
  }
  if constexpr (sizeof(T) == 4 && SMODE == SMODE_INV && L >= 64) {
    if (setup) {
      cudaError_t e = launch_yinv_pipe_L<L>(a, s, true, a.sm_count);
      if (e != cudaSuccess) return e;
    } else if (a.sched == SCHED_PERSISTENT && a.ncols == L && a.n_in == L) {
      return launch_yinv_pipe_L<L>(a, s, false, a.sm_count);
    }
  }
  if constexpr (std::is_same<T, dfl>::value && L >= 64 && ((SMODE == SMODE_FWD && HALF) || SMODE == SMODE_INV)) {
    constexpr int CS = 4;
    using LS = LSmem<L, CS, T>;
    auto kfs = k_strided_smem<T, L, CS, SMODE>;
    if (setup) return cudaFuncSetAttribute(kfs, cudaFuncAttributeMaxDynamicSharedMemorySize, int(LS::SMEM_BYTES));
    a.col_blocks = (a.ncols + CS - 1) / CS;
    kfs<<<dim3(unsigned(a.nouter) * unsigned(a.col_blocks), unsigned(std::max(1, a.nrhs))), LS::NT, LS::SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
  }
  constexpr int C = cols_strided<T>();
  using TL = Tile<L, C, T>;
  auto kfn = k_strided<T, L, C, SMODE, HALF>;
  if (setup) return cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(TL::SMEM_BYTES));
  a.col_blocks = (a.ncols + C - 1) / C;
  const dim3 grid(unsigned(a.nouter) * unsigned(a.col_blocks), unsigned(std::max(1, a.nrhs)));
  kfn<<<grid, TL::NT, TL::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Z convolution, persistent and software-pipelined.  Each CTA loops over
// tiles of C columns (C * sizeof(cpx<T>) = 128 B per row).  While a tile is
// transformed, the next tile's n input rows stream into a staging buffer
// with cp.async, so the memory system stays busy through the compute.
// Tiles are visited ky = 0, L/2, 1, L-1, 2, L-2, ... so that rows ky and
// L - ky, which read the same spectrum entries, run at the same time and
// the second read hits L2.
// ---------------------------------------------------------------------------

__device__ __forceinline__ int ky_of_slot(int i, int L) {
  if (i == 0) return 0;
  if (i == 1) return L / 2;
  const int m = (i - 2) / 2 + 1;
  return (i & 1) ? L - m : m;
}

// Persistent passes number the tiles of a batch consecutively: right-hand
// side r owns tiles [r * per_rhs, (r + 1) * per_rhs).  A CTA visits tiles
// t, t + step, ...; this returns the first of them at or after t whose
// right-hand side is still running (ntiles when none is left).
__device__ __forceinline__ int next_live_tile(const SArgs& a, int t, int step, int per_rhs, int ntiles) {
  if (a.done == nullptr) return t;
  while (t < ntiles) {
    const int r = t / per_rhs;
    if (*bflag(a.done, a.done_stride, r) == 0) return t;
    const int first_next = (r + 1) * per_rhs;          // jump past this right-hand side
    t += ((first_next - t + step - 1) / step) * step;
  }
  return t;
}

template <int L, int C, class T, int L1X = Split<L>::L1>
struct ZPipe {
  using TL = Tile<L, C, T, L1X>;
  static constexpr int NT = TL::NT;
  static constexpr bool GZ = sizeof(T) == 4;              // spectrum staged through smem
  // 128-byte rows of the input and of the Z-tile-ordered spectrum: both
  // arrive by bulk copy (TMA) when the host supplied the tensor map
  static constexpr bool TMA = GZ && C == kZGroup;
  static constexpr size_t E_ELEMS = size_t(TL::SMEM_ELEMS);
  static constexpr size_t S_ELEMS = size_t(L / 2 + (GZ ? 1 : 0)) * C;  // input rows / spectrum slice
  static constexpr size_t TW_ELEMS = GZ ? size_t(L) : 0;                // twiddle table copy
  // with TMA: 128 bytes of slack to align the tile to 128 bytes, and the mbarrier
  static constexpr size_t TMA_BYTES = TMA ? 128 + 16 : 0;
  static constexpr size_t SMEM_BYTES = (E_ELEMS + S_ELEMS + TW_ELEMS) * sizeof(cpx<T>) + TMA_BYTES;
};

// Bulk-copy staging of the FP32 Z pass (ZPipe::TMA).  Thread 0 issues the
// copies; every thread waits on the barrier.  The n_in input rows of a tile,
// 128 bytes each, come as ceil(n_in / zbox) boxes of zbox rows through the
// tensor map a.zrows (rows past n_in are zero-filled; zbox is a power of two
// dividing L / 2 or equal to it, so the boxes end within the L / 2 + 1 rows of S).
template <int L, int C>
__device__ __forceinline__ void zpipe_tma_rows(const SArgs& a, int tile, int per_rhs, cpx<float>* S,
                                               unsigned long long* bar) {
  const int col_blocks = L / C;
  const int rhs = tile / per_rhs;
  const int tl = tile - rhs * per_rhs;
  const int ky = ky_of_slot(tl / col_blocks, L);
  const int cb = tl % col_blocks;
  const int nbox = (a.n_in + a.zbox - 1) / a.zbox;
  fence_proxy_async();
  mbar_expect_tx(bar, unsigned(nbox * a.zbox * C * int(sizeof(cpx<float>))));
  for (int q = 0; q < nbox; ++q) tma_load_4d(S + q * a.zbox * C, &a.zrows, cb * C, ky, q * a.zbox, rhs, bar);
}
// The spectrum slice of a tile: with C == kZGroup the L / 2 + 1 rows of C
// entries are one contiguous run of the Z-tile-ordered spectrum.
template <int L, int C>
__device__ __forceinline__ void zpipe_tma_ghat(const SArgs& a, int rhs, int ky, int cb, cpx<float>* S,
                                               unsigned long long* bar) {
  static_assert(C == kZGroup, "one contiguous run per tile");
  const int my = mirror_index(ky, L);
  const int g = a.rhs_per_ghat > 0 ? rhs / a.rhs_per_ghat : 0;
  const cpx<float>* src = reinterpret_cast<const cpx<float>*>(bmove(a.ghatZ, a.bs_ghatZ * g)) +
                          ((long long)my * (L / kZGroup) + cb) * (L / 2 + 1) * kZGroup;
  constexpr unsigned bytes = unsigned(L / 2 + 1) * C * unsigned(sizeof(cpx<float>));
  fence_proxy_async();
  mbar_expect_tx(bar, bytes);
  bulk_load(S, src, bytes, bar);
}

template <class T, int L, int C, int L1X>
__device__ __forceinline__ void zpipe_prefetch(const SArgs& a, int tile, int per_rhs, cpx<T>* S) {
  constexpr int NT = ZPipe<L, C, T, L1X>::NT;
  constexpr int PER_ROW = C * int(sizeof(cpx<T>)) / 16;    // 16-byte chunks per row
  const int col_blocks = L / C;
  const int rhs = tile / per_rhs;
  const int t = tile - rhs * per_rhs;
  const int ky = ky_of_slot(t / col_blocks, L);
  const int cb = t % col_blocks;
  const cpx<T>* src = reinterpret_cast<const cpx<T>*>(bmove(a.in, a.bs_in * rhs)) + (long long)ky * a.in_outer +
                      (long long)cb * C;
  const int chunks = a.n_in * PER_ROW;
  constexpr int EPC = 16 / int(sizeof(cpx<T>));             // elements per chunk
  for (int k = threadIdx.x; k < chunks; k += NT) {
    const int j = k / PER_ROW, cc = (k - j * PER_ROW) * EPC;
    cp_async16(S + j * C + cc, src + (long long)j * a.in_pt + cc);
  }
  cp_async_commit();
}

// Stage the n_in input rows of a Z tile (C columns) into S, NT threads.
template <class T, int L, int C, int NT>
__device__ __forceinline__ void zpipe_prefetch_rows(const SArgs& a, int tile, int per_rhs, cpx<T>* S) {
  constexpr int PER_ROW = C * int(sizeof(cpx<T>)) / 16;
  constexpr int EPC = 16 / int(sizeof(cpx<T>));
  const int col_blocks = L / C;
  const int rhs = tile / per_rhs;
  const int tl = tile - rhs * per_rhs;
  const int ky = ky_of_slot(tl / col_blocks, L);
  const int cb = tl % col_blocks;
  const cpx<T>* src = reinterpret_cast<const cpx<T>*>(bmove(a.in, a.bs_in * rhs)) + (long long)ky * a.in_outer +
                      (long long)cb * C;
  const int chunks = a.n_in * PER_ROW;
  for (int k = threadIdx.x; k < chunks; k += NT) {
    const int j = k / PER_ROW, cc = (k - j * PER_ROW) * EPC;
    cp_async16(S + j * C + cc, src + (long long)j * a.in_pt + cc);
  }
  cp_async_commit();
}

// The spectrum slice of a tile: entries (mz, my(ky), kx) for mz in [0, L/2]
// and kx in the tile, copied to S as [mz][C].  The Z-tile order stores the
// FP32 spectrum in groups of kZGroup columns, [my][kx / kZGroup][mz][kZGroup];
// a tile of C columns (C divides kZGroup) reads C of each group row.
template <class T, int L, int C, int L1X>
__device__ __forceinline__ void zpipe_prefetch_ghat(const SArgs& a, int rhs, int ky, int cb, cpx<T>* S) {
  static_assert(kZGroup % C == 0, "tile width must divide the spectrum group");
  constexpr int NT = ZPipe<L, C, T, L1X>::NT;
  const int my = mirror_index(ky, L);
  const int g = a.rhs_per_ghat > 0 ? rhs / a.rhs_per_ghat : 0;
  const int kx0 = cb * C;
  const int grp = kx0 / kZGroup, off = kx0 - grp * kZGroup;
  const cpx<T>* src = reinterpret_cast<const cpx<T>*>(bmove(a.ghatZ, a.bs_ghatZ * g)) +
                      ((long long)my * (L / kZGroup) + grp) * (L / 2 + 1) * kZGroup + off;
  constexpr int EPC = 16 / int(sizeof(cpx<T>));
  constexpr int PER_ROW = C / EPC;
  constexpr int chunks = (L / 2 + 1) * PER_ROW;
  for (int k = threadIdx.x; k < chunks; k += NT) {
    const int row = k / PER_ROW, cc = (k - row * PER_ROW) * EPC;
    cp_async16(S + row * C + cc, src + row * kZGroup + cc);
  }
  cp_async_commit();
}

template <class T, int L, int C, int L1X = Split<L>::L1>
__global__ void __launch_bounds__(ZPipe<L, C, T, L1X>::NT,
                                  (ZPipe<L, C, T, L1X>::NT <= 256 && sizeof(T) == 4 && L <= 1024 && L1X < 64) ? 2 : 1)
k_zconv_pipe(const __grid_constant__ SArgs a) {
  using TL = Tile<L, C, T, L1X>;
  using ZP = ZPipe<L, C, T, L1X>;
  constexpr bool GZ = ZP::GZ;
  constexpr int L1 = TL::L1, L2 = TL::L2, NT = TL::NT, NI = L1 / L2;
  constexpr int PK = TL::PK, PC = TL::PC, PKI = TL::PKI, PCI = TL::PCI;
  extern __shared__ __align__(128) unsigned char smraw[];
  unsigned char* base = smraw;
  if constexpr (ZP::TMA) base += (128u - (smem_addr(smraw) & 127u)) & 127u;   // E, S: 128-byte aligned
  cpx<T>* E = reinterpret_cast<cpx<T>*>(base);
  cpx<T>* S = E + ZP::E_ELEMS;
  cpx<T>* TWS = S + ZP::S_ELEMS;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(TWS + ZP::TW_ELEMS);
  const cpx<T>* twg = reinterpret_cast<const cpx<T>*>(a.twL);
  if (GZ) fill_tw2<L, L2>(TWS, twg, threadIdx.x, NT);   // [k1][j] layout
  const cpx<T>* tw = GZ ? TWS : twg;
  const int col_blocks = L / C;
  const int per_rhs = L * col_blocks;
  const int ntiles = per_rhs * (a.nrhs > 1 ? a.nrhs : 1);
  const int step = gridDim.x;
  const int tid = threadIdx.x;
  const int c = tid % C, jl = tid / C;
  const bool tma = ZP::TMA && a.zrows_ok != 0;   // uniform over the grid
  unsigned phase = 0;                            // parity of the barrier phase awaited next
  if (tma) {
    if (tid == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
  }
  // Wait for the staged copy (bulk copies: bounded; a copy that has not
  // landed after kMbarWaitNs sets *a.err and the CTA leaves after one more
  // bounded wait for it).  Also the barrier that ends the use of E by the
  // previous step.  Returns false when the CTA must leave.
  auto staged = [&]() -> bool {
    if constexpr (ZP::TMA) {
      if (tma) {
        const bool ok = mbar_wait(bar, phase);
        if (__syncthreads_or(!ok)) {
          if (tid == 0 && a.err != nullptr) atomicExch(a.err, 1);
          if (!ok) mbar_wait(bar, phase);
          return false;
        }
        phase ^= 1u;
        return true;
      }
    }
    cp_async_wait_all();
    __syncthreads();
    return true;
  };
  auto stage_rows = [&](int t) {
    if constexpr (ZP::TMA) {
      if (tma) {
        if (tid == 0) zpipe_tma_rows<L, C>(a, t, per_rhs, reinterpret_cast<cpx<float>*>(S), bar);
        return;
      }
    }
    zpipe_prefetch<T, L, C, L1X>(a, t, per_rhs, S);
  };

  int tile = next_live_tile(a, blockIdx.x, step, per_rhs, ntiles);
  if (tile < ntiles) stage_rows(tile);
  while (tile < ntiles) {
    const int rhs = tile / per_rhs;
    const int tl = tile - rhs * per_rhs;
    const int ky = ky_of_slot(tl / col_blocks, L);
    const int cb = tl % col_blocks;
    const int next = next_live_tile(a, tile + step, step, per_rhs, ntiles);
    if (!staged()) return;   // staged rows visible; previous tile done with E
    // stage 1: DFT over j1 of rows j1*L2 + j2 (zero padded beyond n_in)
    cpx<T> r[L1];
#pragma unroll
    for (int j1 = 0; j1 < L1; ++j1) {
      r[j1] = czero<T>();
      if (j1 < L1 / 2) {
        const int j = j1 * L2 + jl;
        if (j < a.n_in) r[j1] = S[j * C + c];
      }
    }
    __syncthreads();   // staging buffer consumed
    if constexpr (ZP::TMA) {
      if (tma) {
        if (tid == 0) zpipe_tma_ghat<L, C>(a, rhs, ky, cb, reinterpret_cast<cpx<float>*>(S), bar);
      } else {
        zpipe_prefetch_ghat<T, L, C, L1X>(a, rhs, ky, cb, S);
      }
    } else if (GZ) {
      zpipe_prefetch_ghat<T, L, C, L1X>(a, rhs, ky, cb, S);
    } else if (next < ntiles) {
      zpipe_prefetch<T, L, C, L1X>(a, next, per_rhs, S);
    }
    dft<L1, -1, true>(r);
    if (GZ) {
      const cpx<T>* t2 = tw + jl;
#pragma unroll
      for (int k1 = 1; k1 < L1; ++k1) r[k1] = tw_mul_val<-1>(r[k1], t2[k1 * L2]);
    } else {
#pragma unroll
      for (int k1 = 1; k1 < L1; ++k1) r[k1] = twL_mul<-1>(r[k1], tw, (jl * k1) & (L - 1));
    }
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) E[c * PC + k1 * PK + jl] = r[k1];
    if (GZ) {
      if (!staged()) return;   // spectrum slice visible
    } else {
      __syncthreads();
    }
    // stage 2 (DFT over j2), spectrum, inverse stage A (DFT over k2)
    cpx<T> b[NI][L2];
    const int my = mirror_index(ky, L);
    const cpx<T>* gh = GZ ? nullptr
                          : reinterpret_cast<const cpx<T>*>(bmove(a.ghat, a.bs_ghat * (a.rhs_per_ghat > 0 ? rhs / a.rhs_per_ghat : 0)));
#pragma unroll
    for (int it = 0; it < NI; ++it) {
      const int s = tid + it * NT;
      const int c2 = s % C, k1 = s / C;
#pragma unroll
      for (int j = 0; j < L2; ++j) b[it][j] = E[c2 * PC + k1 * PK + j];
      dft<L2, -1, false>(b[it]);
      if (GZ) {
        // kz = k1 + L1 k2 has mirror index kz below L/2 and L - kz from L/2 on
        // (k2 >= L2/2), so the slice [mz][C] is read at constant offsets from
        // two base pointers
        const cpx<T>* lo = S + k1 * C + c2;
        const cpx<T>* hi = S + (L - k1) * C + c2;
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2)
          b[it][k2] = cmul(b[it][k2], k2 < L2 / 2 ? lo[k2 * L1 * C] : hi[-k2 * L1 * C]);
      } else {
        const int mx = mirror_index(cb * C + c2, L);
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) {
          const int mz = mirror_index(k1 + L1 * k2, L);
          b[it][k2] = cmul(b[it][k2], ldgc(gh + ((long long)mz * a.H + my) * a.H + mx));
        }
      }
      dft<L2, +1, false>(b[it]);
      if (GZ) {
        const cpx<T>* t2 = tw + k1 * L2;
#pragma unroll
        for (int ja = 1; ja < L2; ++ja) b[it][ja] = tw_mul_val<+1>(b[it][ja], t2[ja]);
      } else {
#pragma unroll
        for (int ja = 1; ja < L2; ++ja) b[it][ja] = twL_mul<+1>(b[it][ja], tw, (ja * k1) & (L - 1));
      }
    }
    __syncthreads();   // forward exchange and the spectrum slice fully read
    if (GZ && next < ntiles) stage_rows(next);
#pragma unroll
    for (int it = 0; it < NI; ++it) {
      const int s = tid + it * NT;
      const int c2 = s % C, k1 = s / C;
#pragma unroll
      for (int ja = 0; ja < L2; ++ja) E[c2 * PCI + ja * PKI + k1] = b[it][ja];
    }
    __syncthreads();
    // inverse stage B: DFT over k1 -> rows ja + L2 jb (keep z < n_out)
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) r[k1] = E[c * PCI + jl * PKI + k1];
    dft<L1, +1, false>(r);
    cpx<T>* out = reinterpret_cast<cpx<T>*>(bmove(a.out, a.bs_out * rhs)) + (long long)ky * a.out_outer + (long long)cb * C;
#pragma unroll
    for (int jb = 0; jb < L1 / 2; ++jb) {
      const int j = jl + L2 * jb;
      if (j < a.n_out) out[(long long)j * a.out_pt + c] = r[jb];
    }
    tile = next;
  }
  cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// Z convolution for the paired-FP32 residual: persistent CTAs, a tile of C
// columns (C * 16 B = 128 B rows) held in shared memory and transformed in
// place by looped radix-8 stages (dfft.cuh); the next tile's input rows
// stream into a staging buffer with cp.async meanwhile.
// ---------------------------------------------------------------------------
template <int L, int C, class T>
struct ZSmem {
  static constexpr int NT = 512;
  static constexpr int MINB = 1;   // (256 threads, two CTAs per SM measured 9% slower at L = 2048)
  static constexpr size_t X_ELEMS = size_t(L) * C;
  static constexpr size_t S_ELEMS = size_t(L / 2) * C;
  static constexpr size_t SMEM_BYTES = (X_ELEMS + S_ELEMS + size_t(L)) * sizeof(cpx<T>);
};

template <class T, int L, int C>
__global__ void __launch_bounds__(ZSmem<L, C, T>::NT, ZSmem<L, C, T>::MINB) k_zconv_smem(SArgs a) {
  using ZS = ZSmem<L, C, T>;
  constexpr int NT = ZS::NT;
  constexpr int S8 = L / 8;          // span of the first (and last) radix-8 stage
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T>* X = reinterpret_cast<cpx<T>*>(smraw);
  cpx<T>* S = X + ZS::X_ELEMS;
  cpx<T>* TW = S + ZS::S_ELEMS;
  const cpx<T>* twg = reinterpret_cast<const cpx<T>*>(a.twL);
  for (int i = threadIdx.x; i < L; i += NT) TW[i] = twg[i];
  const int col_blocks = L / C;
  const int per_rhs = L * col_blocks;
  const int ntiles = per_rhs * (a.nrhs > 1 ? a.nrhs : 1);
  const int step = gridDim.x;
  const int tid = threadIdx.x;

  int tile = next_live_tile(a, blockIdx.x, step, per_rhs, ntiles);
  if (tile < ntiles) zpipe_prefetch_rows<T, L, C, NT>(a, tile, per_rhs, S);
  while (tile < ntiles) {
    const int rhs = tile / per_rhs;
    const int tl = tile - rhs * per_rhs;
    const int ky = ky_of_slot(tl / col_blocks, L);
    const int cb = tl % col_blocks;
    const int next = next_live_tile(a, tile + step, step, per_rhs, ntiles);
    const cpx<T>* gh = reinterpret_cast<const cpx<T>*>(bmove(a.ghat, a.bs_ghat * (a.rhs_per_ghat > 0 ? rhs / a.rhs_per_ghat : 0)));
    cp_async_wait_all();
    __syncthreads();
    // first forward stage (M = L): inputs beyond L/2 are the zero padding
    for (int g = tid; g < C * S8; g += NT) {
      const int c = g % C, j = g / C;
      cpx<T> v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        v[t] = czero<T>();
        if (t < 4 && j + t * S8 < a.n_in) v[t] = S[(j + t * S8) * C + c];
      }
      dft<8, -1, true>(v);
#pragma unroll
      for (int t = 1; t < 8; ++t) v[t] = twL_mul<-1>(v[t], TW, (j * t) & (L - 1));
#pragma unroll
      for (int t = 0; t < 8; ++t) st_stage(X + sidx<C>(j + t * S8, c), settle(v[t]));
    }
    __syncthreads();
    if (next < ntiles) zpipe_prefetch_rows<T, L, C, NT>(a, next, per_rhs, S);
    dif_rest<L, C>(X, TW, tid, NT);
    // spectrum: position p holds frequency kz = digit_rev(p)
    const int my = mirror_index(ky, L);
    for (int e = tid; e < C * L; e += NT) {
      const int c = e % C, p = e / C;
      const int mz = mirror_index(digit_rev<L>(p), L);
      const int mx = mirror_index(cb * C + c, L);
      const int si = sidx<C>(p, c);
      st_stage(X + si, settle(cmul(ld_stage(X + si), ldgc(gh + ((long long)mz * a.H + my) * a.H + mx))));
    }
    __syncthreads();
    dit_head<L, C>(X, TW, tid, NT);
    // last inverse stage (M = L), keep rows z < n_out
    cpx<T>* out = reinterpret_cast<cpx<T>*>(bmove(a.out, a.bs_out * rhs)) + (long long)ky * a.out_outer + (long long)cb * C;
    for (int g = tid; g < C * S8; g += NT) {
      const int c = g % C, j = g / C;
      cpx<T> v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) v[t] = ld_stage(X + sidx<C>(j + t * S8, c));
#pragma unroll
      for (int t = 1; t < 8; ++t) v[t] = twL_mul<+1>(v[t], TW, (j * t) & (L - 1));
      dft<8, +1, false>(v);
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int z = j + t * S8;
        if (z < a.n_out) out[(long long)z * a.out_pt + c] = settle(v[t]);
      }
    }
    tile = next;
  }
  cp_async_wait_all();
}

template <class T, int L>
cudaError_t launch_zconv_smem_L(SArgs a, cudaStream_t s, bool setup, int sm_count) {
  constexpr int C = (L > 1024 && sizeof(cpx<T>) == 16) ? 4 : 8;   // the tile must fit in 227 KB
  using ZS = ZSmem<L, C, T>;
  auto kfn = k_zconv_smem<T, L, C>;
  static int per_sm = 0;   // resident CTAs per SM, measured once at set-up
  if (setup) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ZS::SMEM_BYTES));
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn, ZS::NT, ZS::SMEM_BYTES);
    per_sm = (e == cudaSuccess && nb > 0) ? nb : 1;
    return e;
  }
  const long long ntiles = (long long)L * (L / C) * std::max(1, a.nrhs);
  const unsigned gx = unsigned(std::max(1LL, std::min(ntiles, (long long)std::max(1, sm_count) * std::max(1, per_sm))));
  kfn<<<gx, ZS::NT, ZS::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Y forward pass, persistent and software-pipelined like the Z pass: each CTA
// loops over tiles (outer index z, C columns); the next tile's n input rows
// stream into shared memory while the current one is transformed, by TMA
// through a tensor map of T1 for 16-column tiles (boxes of up to 256 rows)
// and by cp.async otherwise.
// ---------------------------------------------------------------------------
template <int L, int C, class T, int L1X = Split<L>::L1>
struct YPipe {
  using TL = Tile<L, C, T, L1X>;
  static constexpr int NT = TL::NT;
  // 128-byte rows (16 FP32 columns): the input rows arrive by TMA when the
  // host supplied the tensor map (a.zrows); 128 bytes of slack align the
  // tile to 128 bytes, then the mbarrier
  static constexpr bool TMA = sizeof(T) == 4 && C == kZGroup;
  static constexpr size_t E_ELEMS = size_t(TL::SMEM_ELEMS);
  static constexpr size_t S_ELEMS = size_t(L / 2) * C;
  static constexpr size_t TMA_BYTES = TMA ? 128 + 16 : 0;
  static constexpr size_t SMEM_BYTES = (E_ELEMS + S_ELEMS + size_t(L)) * sizeof(cpx<T>) + TMA_BYTES;
};

// Bulk-copy staging of the rows [0, rows) of a pipelined FP32 Y tile (C ==
// kZGroup columns at x = cb * C of plane `outer`, right-hand side rhs)
// through the tensor map a.zrows (box: C columns x a.zbox rows); rows past
// the map's extent are zero-filled and must fit the staging buffer.  Thread 0
// issues the copies.
template <int C>
__device__ __forceinline__ void ypipe_tma_rows(const SArgs& a, int rhs, int outer, int cb, int rows, cpx<float>* S,
                                               unsigned long long* bar) {
  const int nbox = (rows + a.zbox - 1) / a.zbox;
  fence_proxy_async();
  mbar_expect_tx(bar, unsigned(nbox * a.zbox * C * int(sizeof(cpx<float>))));
  for (int q = 0; q < nbox; ++q) tma_load_4d(S + q * a.zbox * C, &a.zrows, cb * C, q * a.zbox, outer, rhs, bar);
}

template <class T, int L, int C, int L1X>
__device__ __forceinline__ void ypipe_prefetch(const SArgs& a, int tile, int per_rhs, cpx<T>* S) {
  constexpr int NT = YPipe<L, C, T, L1X>::NT;
  constexpr int PER_ROW = C * int(sizeof(cpx<T>)) / 16;
  constexpr int EPC = 16 / int(sizeof(cpx<T>));
  const int rhs = tile / per_rhs;
  const int tl = tile - rhs * per_rhs;
  const int outer = tl / a.col_blocks, cb = tl - outer * a.col_blocks;
  const cpx<T>* src = reinterpret_cast<const cpx<T>*>(bmove(a.in, a.bs_in * rhs)) + outer * a.in_outer + (long long)cb * C;
  const int chunks = a.n_in * PER_ROW;
  for (int k = threadIdx.x; k < chunks; k += NT) {
    const int j = k / PER_ROW, cc = (k - j * PER_ROW) * EPC;
    cp_async16(S + j * C + cc, src + (long long)j * a.in_pt + cc);
  }
  cp_async_commit();
}

template <class T, int L, int C, int L1X = Split<L>::L1>
__global__ void __launch_bounds__(YPipe<L, C, T, L1X>::NT,
                                  (L > 1024 || L1X >= 64 || YPipe<L, C, T, L1X>::NT >= 512)
                                      ? 1 : (YPipe<L, C, T, L1X>::NT >= 256 ? 2 : 512 / YPipe<L, C, T, L1X>::NT))
k_yfwd_pipe(const __grid_constant__ SArgs a) {
  using TL = Tile<L, C, T, L1X>;
  using YP = YPipe<L, C, T, L1X>;
  constexpr int L1 = TL::L1, L2 = TL::L2, NT = TL::NT, NI = L1 / L2;
  constexpr int PK = TL::PK, PC = TL::PC;
  extern __shared__ __align__(128) unsigned char smraw[];
  unsigned char* base = smraw;
  if constexpr (YP::TMA) base += (128u - (smem_addr(smraw) & 127u)) & 127u;   // E, S: 128-byte aligned
  cpx<T>* E = reinterpret_cast<cpx<T>*>(base);
  cpx<T>* S = E + YP::E_ELEMS;
  cpx<T>* TW = S + YP::S_ELEMS;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(TW + L);
  const cpx<T>* twg = reinterpret_cast<const cpx<T>*>(a.twL);
  fill_tw2<L, L2>(TW, twg, threadIdx.x, NT);   // [k1][j] layout
  const int per_rhs = a.nouter * a.col_blocks;
  const int ntiles = per_rhs * (a.nrhs > 1 ? a.nrhs : 1);
  const int step = gridDim.x;
  const int tid = threadIdx.x;
  const int c = tid % C, jl = tid / C;
  const bool tma = YP::TMA && a.zrows_ok != 0;   // uniform over the grid
  unsigned phase = 0;
  if (tma) {
    if (tid == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
  }
  auto stage = [&](int t) {
    if constexpr (YP::TMA) {
      if (tma) {
        if (tid == 0) {
          const int rt = t / per_rhs, tt = t - rt * per_rhs;
          const int o = tt / a.col_blocks;
          ypipe_tma_rows<C>(a, rt, o, tt - o * a.col_blocks, a.n_in, reinterpret_cast<cpx<float>*>(S), bar);
        }
        return;
      }
    }
    ypipe_prefetch<T, L, C, L1X>(a, t, per_rhs, S);
  };
  int tile = next_live_tile(a, blockIdx.x, step, per_rhs, ntiles);
  if (tile < ntiles) stage(tile);
  while (tile < ntiles) {
    const int rhs = tile / per_rhs;
    const int tl = tile - rhs * per_rhs;
    const int outer = tl / a.col_blocks, cb = tl - outer * a.col_blocks;
    const int next = next_live_tile(a, tile + step, step, per_rhs, ntiles);
    if (tma) {
      const bool ok = mbar_wait(bar, phase);
      if (__syncthreads_or(!ok)) {   // rows that have not landed: flag it, wait once more (bounded), leave
        if (tid == 0 && a.err != nullptr) atomicExch(a.err, 1);
        if (!ok) mbar_wait(bar, phase);
        return;
      }
      phase ^= 1u;
    } else {
      cp_async_wait_all();
      __syncthreads();
    }
    cpx<T> r[L1];
#pragma unroll
    for (int j1 = 0; j1 < L1; ++j1) {
      r[j1] = czero<T>();
      if (j1 < L1 / 2) {
        const int j = j1 * L2 + jl;
        if (j < a.n_in) r[j1] = S[j * C + c];
      }
    }
    __syncthreads();
    if (next < ntiles) stage(next);
    dft<L1, -1, true>(r);
    const cpx<T>* t2 = TW + jl;
#pragma unroll
    for (int k1 = 1; k1 < L1; ++k1) r[k1] = tw_mul_val<-1>(r[k1], t2[k1 * L2]);
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) E[c * PC + k1 * PK + jl] = r[k1];
    __syncthreads();
    cpx<T>* out = reinterpret_cast<cpx<T>*>(bmove(a.out, a.bs_out * rhs)) + outer * a.out_outer + (long long)cb * C;
#pragma unroll
    for (int it = 0; it < NI; ++it) {
      const int sidx2 = tid + it * NT;
      const int c2 = sidx2 % C, k1 = sidx2 / C;
      cpx<T> b[L2];
#pragma unroll
      for (int j = 0; j < L2; ++j) b[j] = E[c2 * PC + k1 * PK + j];
      dft<L2, -1, false>(b);
#pragma unroll
      for (int k2 = 0; k2 < L2; ++k2) {
        const int k = k1 + L1 * k2;
        if (k < a.n_out) out[(long long)k * a.out_pt + c2] = b[k2];
      }
    }
    tile = next;
  }
  cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// Y inverse pass, persistent and pipelined (FP32): tiles (outer index z, C
// columns) of every right-hand side numbered together.  A tile's L input
// rows stream into shared memory (TMA through a tensor map of T2 for
// 16-column tiles, cp.async otherwise); the exchange between the two DFT
// stages reuses that buffer in place, and the next tile is requested as soon
// as the second stage has read the exchange.
// ---------------------------------------------------------------------------
template <int L, int C, int L1X = Split<L>::L1>
struct YInvPipe {
  using TL = Tile<L, C, float, L1X>;
  static constexpr int NT = TL::NT;
  static constexpr int BUF = (C * L > TL::SMEM_ELEMS) ? C * L : TL::SMEM_ELEMS;
  // 128-byte rows: TMA staging as in YPipe (slack to align the tile, the mbarrier)
  static constexpr bool TMA = C == kZGroup;
  static constexpr size_t TMA_BYTES = TMA ? 128 + 16 : 0;
  static constexpr size_t SMEM_BYTES = size_t(BUF + L) * sizeof(cpx<float>) + TMA_BYTES;
};

template <int L, int C, int L1X>
__device__ __forceinline__ void yinv_prefetch(const SArgs& a, int tile, int per_rhs, cpx<float>* B) {
  constexpr int NT = YInvPipe<L, C, L1X>::NT;
  constexpr int PER_ROW = C * int(sizeof(cpx<float>)) / 16;
  const int rhs = tile / per_rhs;
  const int tl = tile - rhs * per_rhs;
  const int outer = tl / a.col_blocks, cb = tl - outer * a.col_blocks;
  const cpx<float>* src = reinterpret_cast<const cpx<float>*>(bmove(a.in, a.bs_in * rhs)) + outer * a.in_outer +
                          (long long)cb * C;
  for (int k = threadIdx.x; k < L * PER_ROW; k += NT) {
    const int j = k / PER_ROW, cc = (k - j * PER_ROW) * 2;
    cp_async16(B + j * C + cc, src + (long long)j * a.in_pt + cc);
  }
  cp_async_commit();
}

template <int L, int C, int L1X = Split<L>::L1>
__global__ void __launch_bounds__(YInvPipe<L, C, L1X>::NT,
                                  (L > 1024 || L1X >= 64 || YInvPipe<L, C, L1X>::NT >= 512)
                                      ? 1 : (YInvPipe<L, C, L1X>::NT >= 256 ? 2 : 512 / YInvPipe<L, C, L1X>::NT))
k_yinv_pipe(const __grid_constant__ SArgs a) {
  using T = float;
  using TL = Tile<L, C, T, L1X>;
  using YP = YInvPipe<L, C, L1X>;
  constexpr int L1 = TL::L1, L2 = TL::L2, NT = TL::NT, NI = L1 / L2;
  constexpr int PKI = TL::PKI, PCI = TL::PCI;
  extern __shared__ __align__(128) unsigned char smraw[];
  unsigned char* base = smraw;
  if constexpr (YP::TMA) base += (128u - (smem_addr(smraw) & 127u)) & 127u;   // B: 128-byte aligned
  cpx<T>* B = reinterpret_cast<cpx<T>*>(base);
  cpx<T>* TW = B + YP::BUF;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(TW + L);
  const cpx<T>* twg = reinterpret_cast<const cpx<T>*>(a.twL);
  fill_tw2<L, L2>(TW, twg, threadIdx.x, NT);   // [k1][j] layout
  const int per_rhs = a.nouter * a.col_blocks;
  const int ntiles = per_rhs * (a.nrhs > 1 ? a.nrhs : 1);
  const int step = gridDim.x;
  const int tid = threadIdx.x;
  int c, ja;
  map_t<LAYOUT_STRIDED, C, L2>(tid, c, ja);
  const bool tma = YP::TMA && a.zrows_ok != 0;   // uniform over the grid
  unsigned phase = 0;
  if (tma) {
    if (tid == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
    }
    __syncthreads();
  }
  auto stage = [&](int t) {
    if constexpr (YP::TMA) {
      if (tma) {
        if (tid == 0) {
          const int rt = t / per_rhs, tt = t - rt * per_rhs;
          const int o = tt / a.col_blocks;
          ypipe_tma_rows<C>(a, rt, o, tt - o * a.col_blocks, L, B, bar);
        }
        return;
      }
    }
    yinv_prefetch<L, C, L1X>(a, t, per_rhs, B);
  };
  int tile = next_live_tile(a, blockIdx.x, step, per_rhs, ntiles);
  if (tile < ntiles) stage(tile);
  while (tile < ntiles) {
    const int rhs = tile / per_rhs;
    const int tl = tile - rhs * per_rhs;
    const int outer = tl / a.col_blocks, cb = tl - outer * a.col_blocks;
    const int next = next_live_tile(a, tile + step, step, per_rhs, ntiles);
    if (tma) {
      const bool ok = mbar_wait(bar, phase);
      if (__syncthreads_or(!ok)) {   // rows that have not landed: flag it, wait once more (bounded), leave
        if (tid == 0 && a.err != nullptr) atomicExch(a.err, 1);
        if (!ok) mbar_wait(bar, phase);
        return;
      }
      phase ^= 1u;
    } else {
      cp_async_wait_all();
      __syncthreads();
    }
    // stage A: DFT over k2 of rows k1 + L1 k2, twiddle
    cpx<T> b[NI][L2];
#pragma unroll
    for (int it = 0; it < NI; ++it) {
      int c2, k1;
      map_s<LAYOUT_STRIDED, C, L1>(tid + it * NT, c2, k1);
#pragma unroll
      for (int k2 = 0; k2 < L2; ++k2) b[it][k2] = B[(k1 + L1 * k2) * C + c2];
      dft<L2, +1, false>(b[it]);
      const cpx<T>* t2 = TW + k1 * L2;
#pragma unroll
      for (int j = 1; j < L2; ++j) b[it][j] = tw_mul_val<+1>(b[it][j], t2[j]);
    }
    __syncthreads();   // raw tile consumed: the exchange reuses the buffer
#pragma unroll
    for (int it = 0; it < NI; ++it) {
      int c2, k1;
      map_s<LAYOUT_STRIDED, C, L1>(tid + it * NT, c2, k1);
#pragma unroll
      for (int j = 0; j < L2; ++j) B[c2 * PCI + j * PKI + k1] = b[it][j];
    }
    __syncthreads();
    cpx<T> r[L1];
#pragma unroll
    for (int k1 = 0; k1 < L1; ++k1) r[k1] = B[c * PCI + ja * PKI + k1];
    __syncthreads();   // exchange consumed: the buffer takes the next tile
    if (next < ntiles) stage(next);
    dft<L1, +1, false>(r);
    cpx<T>* out = reinterpret_cast<cpx<T>*>(bmove(a.out, a.bs_out * rhs)) + outer * a.out_outer + (long long)cb * C;
#pragma unroll
    for (int jb = 0; jb < L1; ++jb) {
      const int j = ja + L2 * jb;
      if (j < a.n_out) out[(long long)j * a.out_pt + c] = r[jb];
    }
    tile = next;
  }
  cp_async_wait_all();
}

template <int L, int C, int L1X>
cudaError_t launch_yinv_pipe_V(SArgs a, cudaStream_t s, bool setup, int sm_count) {
  using YP = YInvPipe<L, C, L1X>;
  auto kfn = k_yinv_pipe<L, C, L1X>;
  static int per_sm = 0;
  if (setup) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(YP::SMEM_BYTES));
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn, YP::NT, YP::SMEM_BYTES);
    per_sm = (e == cudaSuccess && nb > 0) ? nb : 1;
    return e;
  }
  if (a.ncols != L || a.n_in != L) return cudaErrorInvalidValue;   // whole columns of L rows
  a.col_blocks = L / C;
  const long long ntiles = (long long)a.nouter * a.col_blocks * std::max(1, a.nrhs);
  const int resident = a.cta_cap > 0 ? std::min(std::max(1, per_sm), a.cta_cap) : std::max(1, per_sm);
  const unsigned gx = unsigned(std::max(1LL, std::min(ntiles, (long long)std::max(1, sm_count) * resident)));
  kfn<<<gx, YP::NT, YP::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

template <class T, int L, int C, int L1X>
cudaError_t launch_yfwd_pipe_V(SArgs a, cudaStream_t s, bool setup, int sm_count) {
  using YP = YPipe<L, C, T, L1X>;
  auto kfn = k_yfwd_pipe<T, L, C, L1X>;
  static int per_sm = 0;
  if (setup) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(YP::SMEM_BYTES));
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn, YP::NT, YP::SMEM_BYTES);
    per_sm = (e == cudaSuccess && nb > 0) ? nb : 1;
    return e;
  }
  a.col_blocks = (a.ncols + C - 1) / C;
  const long long ntiles = (long long)a.nouter * a.col_blocks * std::max(1, a.nrhs);
  const int resident = a.cta_cap > 0 ? std::min(std::max(1, per_sm), a.cta_cap) : std::max(1, per_sm);
  const unsigned gx = unsigned(std::max(1LL, std::min(ntiles, (long long)std::max(1, sm_count) * resident)));
  kfn<<<gx, YP::NT, YP::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

template <class T, int L, int C, int L1X>
cudaError_t launch_zconv_pipe_V(SArgs a, cudaStream_t s, bool setup, int sm_count) {
  using ZP = ZPipe<L, C, T, L1X>;
  auto kfn = k_zconv_pipe<T, L, C, L1X>;
  static int per_sm = 0;   // resident CTAs per SM, measured once at set-up
  if (setup) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ZP::SMEM_BYTES));
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn, ZP::NT, ZP::SMEM_BYTES);
    per_sm = (e == cudaSuccess && nb > 0) ? nb : 1;
    return e;
  }
  const long long ntiles = (long long)L * (L / C) * std::max(1, a.nrhs);
  const int resident = a.cta_cap > 0 ? std::min(std::max(1, per_sm), a.cta_cap) : std::max(1, per_sm);
  const unsigned gx = unsigned(std::max(1LL, std::min(ntiles, (long long)std::max(1, sm_count) * resident)));
  kfn<<<gx, ZP::NT, ZP::SMEM_BYTES, s>>>(a);
  return cudaGetLastError();
}

// Dispatch on the launch variant (has_pipe_variants): the set-up call
// prepares every variant, a launch runs the one a.variant names.
template <class T, int L, int C0, template <class, int, int, int> class Launch>
cudaError_t dispatch_pipe_variant(SArgs a, cudaStream_t s, bool setup, int sm_count) {
  constexpr int L1 = Split<L>::L1;
  if constexpr (sizeof(T) == 4 && has_pipe_variants(L)) {
    if (setup) {
      cudaError_t e = Launch<T, L, 16, L1>::run(a, s, true, sm_count);
      if (e == cudaSuccess) e = Launch<T, L, 8, L1>::run(a, s, true, sm_count);
      if (e == cudaSuccess) e = Launch<T, L, 16, 2 * L1>::run(a, s, true, sm_count);
      return e;
    }
    if (a.variant == 1) return Launch<T, L, 8, L1>::run(a, s, false, sm_count);
    if (a.variant == 2) return Launch<T, L, 16, 2 * L1>::run(a, s, false, sm_count);
    return Launch<T, L, 16, L1>::run(a, s, false, sm_count);
  } else {
    return Launch<T, L, C0, L1>::run(a, s, setup, sm_count);
  }
}

template <class T, int L, int C, int L1X>
struct ZconvPipeLaunch {
  static cudaError_t run(SArgs a, cudaStream_t s, bool setup, int sm) { return launch_zconv_pipe_V<T, L, C, L1X>(a, s, setup, sm); }
};
template <class T, int L, int C, int L1X>
struct YfwdPipeLaunch {
  static cudaError_t run(SArgs a, cudaStream_t s, bool setup, int sm) { return launch_yfwd_pipe_V<T, L, C, L1X>(a, s, setup, sm); }
};
template <class T, int L, int C, int L1X>
struct YinvPipeLaunch {
  static cudaError_t run(SArgs a, cudaStream_t s, bool setup, int sm) { return launch_yinv_pipe_V<L, C, L1X>(a, s, setup, sm); }
};

// Default tile widths: 128-byte rows (Z: 64-byte rows measured slower at
// L <= 1024; Y: 8 columns 1.37 / 1.42 ms against 16 columns 1.30 / 1.24 ms at
// n = 512); at L = 2048 a 16-column tile's exchange buffer exceeds shared
// memory, so 8 columns (256 threads, one CTA per SM, up to 255 registers).
template <class T, int L>
cudaError_t launch_zconv_pipe_L(SArgs a, cudaStream_t s, bool setup, int sm_count) {
  constexpr int C = (L > 1024 && sizeof(T) == 4) ? 8 : 128 / int(sizeof(cpx<T>));
  return dispatch_pipe_variant<T, L, C, ZconvPipeLaunch>(a, s, setup, sm_count);
}
template <class T, int L>
cudaError_t launch_yfwd_pipe_L(SArgs a, cudaStream_t s, bool setup, int sm_count) {
  constexpr int C = L > 1024 ? 8 : 16;
  return dispatch_pipe_variant<T, L, C, YfwdPipeLaunch>(a, s, setup, sm_count);
}
template <int L>
cudaError_t launch_yinv_pipe_L(SArgs a, cudaStream_t s, bool setup, int sm_count) {
  constexpr int C = L > 1024 ? 8 : 16;
  return dispatch_pipe_variant<float, L, C, YinvPipeLaunch>(a, s, setup, sm_count);
}

// Z-pass kernel choice for L >= 64: the shared-memory radix-8 kernel for
// paired FP32; for FP32 the pipelined persistent kernel or, by schedule, the
// one-CTA-per-tile strided kernel; the pipelined kernel for FP64; the plain
// strided kernel for small L.
template <class T, int L>
cudaError_t launch_zconv_reg_L(SArgs a, cudaStream_t s, bool setup) {
  if constexpr (L >= 64 && std::is_same<T, dfl>::value) {
    return launch_zconv_smem_L<T, L>(a, s, setup, a.sm_count);
  } else if constexpr (L >= 64 && sizeof(T) == 4) {
    if (setup) {
      cudaError_t e = launch_zconv_pipe_L<T, L>(a, s, true, a.sm_count);
      if (e != cudaSuccess) return e;
      return launch_strided_L<T, L, SMODE_ZCONV, true>(a, s, true);
    }
    if (a.sched == SCHED_TILES) return launch_strided_L<T, L, SMODE_ZCONV, true>(a, s, false);
    return launch_zconv_pipe_L<T, L>(a, s, false, a.sm_count);
  } else if constexpr (L >= 64) {
    return launch_zconv_pipe_L<T, L>(a, s, setup, a.sm_count);
  } else {
    return launch_strided_L<T, L, SMODE_ZCONV, true>(a, s, setup);
  }
}

// Lengths beyond kMaxRegL: the FP64 and paired-FP32 passes use the
// shared-memory radix-8 kernels (a register tile of L1 = 64 of their points
// per thread does not fit).  The FP32 passes stay pipelined: each 64-point
// stage either has a zero-padded half on input or keeps half its outputs.
constexpr int kMaxRegL = 1024;

template <class T, int L, bool HALF>
cudaError_t launch_xfwd_L(const XArgs& a, cudaStream_t s, bool setup) {
  if constexpr (L > kMaxRegL) {
    // FP32 solver prologues: the pipelined kernel (4-line tiles, one CTA per SM)
    if constexpr (std::is_same<T, float>::value && HALF) {
      if (setup) {
        cudaError_t e = launch_xfwd_pipe_L<L>(a, s, true);
        if (e != cudaSuccess) return e;
      } else if (xfwd_pipe_ok(a, L)) {
        return launch_xfwd_pipe_L<L>(a, s, false);
      }
    }
    constexpr int CS = 4;
    using LS = LSmem<L, CS, T>;
    auto kfs = k_xfwd_smem<T, L, CS, HALF>;
    if (setup) return cudaFuncSetAttribute(kfs, cudaFuncAttributeMaxDynamicSharedMemorySize, int(LS::SMEM_BYTES));
    kfs<<<dim3(unsigned((a.nlines + CS - 1) / CS), unsigned(std::max(1, a.nrhs))), LS::NT, LS::SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
  } else {
    return launch_xfwd_reg_L<T, L, HALF>(a, s, setup);
  }
}

template <class T, int L>
cudaError_t launch_xinv_L(const XArgs& a, Scalars* sc, int fin, cudaStream_t s, bool setup, unsigned* nblocks) {
  if constexpr (L > kMaxRegL && std::is_same<T, float>::value) {
    return launch_xinv_pipe_L<L>(a, sc, fin, s, setup, nblocks);   // as for L <= kMaxRegL
  } else if constexpr (L > kMaxRegL) {
    constexpr int CS = 4;
    using LS = LSmem<L, CS, T>;
    auto kfs = k_xinv_smem<T, L, CS>;
    const unsigned grid = unsigned((a.nlines + CS - 1) / CS);
    if (nblocks) *nblocks = grid;
    if (setup) return cudaFuncSetAttribute(kfs, cudaFuncAttributeMaxDynamicSharedMemorySize, int(LS::SMEM_BYTES));
    kfs<<<dim3(grid, unsigned(std::max(1, a.nrhs))), LS::NT, LS::SMEM_BYTES, s>>>(a, sc, fin);
    return cudaGetLastError();
  } else {
    return launch_xinv_reg_L<T, L>(a, sc, fin, s, setup, nblocks);
  }
}

template <class T, int L, int SMODE, bool HALF>
cudaError_t launch_strided_L(SArgs a, cudaStream_t s, bool setup) {
  if constexpr (L > kMaxRegL) {
    if constexpr (SMODE == SMODE_ZCONV) {
      return launch_zconv_smem_L<T, L>(a, s, setup, a.sm_count);
    } else {
      // FP32 Y passes: the pipelined kernels fit for the reason the Z kernel does
      // (a 64-point stage with a zero half on input, or with half its outputs
      // kept); the TILES schedule keeps the radix-8 kernels below
      if constexpr (std::is_same<T, float>::value && SMODE == SMODE_FWD && HALF) {
        if (setup) {
          cudaError_t e = launch_yfwd_pipe_L<T, L>(a, s, true, a.sm_count);
          if (e != cudaSuccess) return e;
        } else if (a.sched == SCHED_PERSISTENT) {
          return launch_yfwd_pipe_L<T, L>(a, s, false, a.sm_count);
        }
      }
      if constexpr (std::is_same<T, float>::value && SMODE == SMODE_INV) {
        if (setup) {
          cudaError_t e = launch_yinv_pipe_L<L>(a, s, true, a.sm_count);
          if (e != cudaSuccess) return e;
        } else if (a.sched == SCHED_PERSISTENT && a.ncols == L && a.n_in == L) {
          return launch_yinv_pipe_L<L>(a, s, false, a.sm_count);
        }
      }
      constexpr int CS = 4;   // (8 columns measured slower at L = 2048: fewer resident CTAs)
      using LS = LSmem<L, CS, T>;
      auto kfs = k_strided_smem<T, L, CS, SMODE, (SMODE == SMODE_FWD ? HALF : true)>;
      if (setup) return cudaFuncSetAttribute(kfs, cudaFuncAttributeMaxDynamicSharedMemorySize, int(LS::SMEM_BYTES));
      a.col_blocks = (a.ncols + CS - 1) / CS;
      kfs<<<dim3(unsigned(a.nouter) * unsigned(a.col_blocks), unsigned(std::max(1, a.nrhs))), LS::NT, LS::SMEM_BYTES, s>>>(a);
      return cudaGetLastError();
    }
  } else {
    return launch_strided_reg_L<T, L, SMODE, HALF>(a, s, setup);
  }
}

// The Z pass beyond kMaxRegL: for FP32 the pipelined kernel still fits, since
// its first stage holds 32 nonzero inputs of the 64-point DFT (dft<64> with
// the zero-padded half) and its last keeps 32 of 64 outputs; it reads the
// Z-tile-ordered spectrum.  The radix-8 shared-memory kernel is the TILES
// schedule and the kernel of the other arithmetics.
template <class T, int L>
cudaError_t launch_zconv_L(SArgs a, cudaStream_t s, bool setup) {
  if constexpr (L > kMaxRegL) {
    if constexpr (std::is_same<T, float>::value) {
      if (setup) {
        cudaError_t e = launch_zconv_pipe_L<T, L>(a, s, true, a.sm_count);
        if (e != cudaSuccess) return e;
        return launch_zconv_smem_L<T, L>(a, s, true, a.sm_count);
      }
      if (a.ghatZ != nullptr && a.sched != SCHED_TILES) return launch_zconv_pipe_L<T, L>(a, s, false, a.sm_count);
    }
    return launch_zconv_smem_L<T, L>(a, s, setup, a.sm_count);
  } else {
    return launch_zconv_reg_L<T, L>(a, s, setup);
  }
}

#define ORI_FOR_EACH_L(X) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048)

template <class T>
cudaError_t run_xfwd(int L, bool half, const XArgs& a, cudaStream_t s, bool setup) {
  switch (L) {
#define ORI_CASE(LL) \
    case LL: return half ? launch_xfwd_L<T, LL, true>(a, s, setup) : launch_xfwd_L<T, LL, false>(a, s, setup);
    ORI_FOR_EACH_L(ORI_CASE)
#undef ORI_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <class T>
cudaError_t run_xinv(int L, const XArgs& a, Scalars* sc, int fin, cudaStream_t s, bool setup, unsigned* nblocks) {
  switch (L) {
#define ORI_CASE(LL) case LL: return launch_xinv_L<T, LL>(a, sc, fin, s, setup, nblocks);
    ORI_FOR_EACH_L(ORI_CASE)
#undef ORI_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <class T>
cudaError_t run_strided_fwd(int L, bool half, const SArgs& a, cudaStream_t s, bool setup) {
  switch (L) {
#define ORI_CASE(LL) \
    case LL: return half ? launch_strided_L<T, LL, SMODE_FWD, true>(a, s, setup) \
                         : launch_strided_L<T, LL, SMODE_FWD, false>(a, s, setup);
    ORI_FOR_EACH_L(ORI_CASE)
#undef ORI_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <class T>
cudaError_t run_strided_inv(int L, const SArgs& a, cudaStream_t s, bool setup) {
  switch (L) {
#define ORI_CASE(LL) case LL: return launch_strided_L<T, LL, SMODE_INV, false>(a, s, setup);
    ORI_FOR_EACH_L(ORI_CASE)
#undef ORI_CASE
    default: return cudaErrorInvalidValue;
  }
}

template <class T>
cudaError_t run_zconv(int L, const SArgs& a, cudaStream_t s, bool setup) {
  switch (L) {
#define ORI_CASE(LL) case LL: return launch_zconv_L<T, LL>(a, s, setup);
    ORI_FOR_EACH_L(ORI_CASE)
#undef ORI_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ori
