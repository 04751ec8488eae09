// passes.cuh - the FFT passes of the padded 3D convolution (Section 3).
//
// The matvec y = x + K(s x) (K = c_S |Delta| G_off, s = h N or sqrt(h N)) runs
// as five passes over two scratch cubes, each pass an FFT of length L along
// one axis, pruned by the zero padding (Section 3: u is padded with zeros,
// and entries past the n-th are discarded after the inverse transform):
//
//   X fwd : x[z][y][0..n)  --(prologue: scale, COCG update)-->  T1[z][y][0..L)
//   Y fwd : T1[z][0..n)[kx]                                 ->  T2[z][0..L)[kx]
//   Z conv: T2[0..n)[ky][kx] -> FFT -> * Ghat -> IFFT -> keep z < n (in place)
//   Y inv : T2[z][0..L)[kx]                                 ->  T1[z][0..n)[kx]
//   X inv : T1[z][y][0..L) -> keep x < n --(epilogue: y = x + s conv, dots)--> y
//
// T1 is [n][n][L] and T2 is [n][L][L] (C-order, x fastest).  The spectrum is
// stored once for the (L/2+1)^3 distinct entries (the kernel cube is even
// along each axis); column (kx, ky, kz) reads entry (m(kz), m(ky), m(kx)),
// m(k) = min(k, L - k), and already carries c_S |Delta| / L^3.
//
// Every pass computes length-L DFTs on a tile of C lines held by one CTA as
// L = L1 * L2: a length-L1 DFT in registers over j1 (j = j1 L2 + j2), the
// twiddle exp(-2 pi i j2 k1 / L), one exchange through shared memory, and a
// length-L2 DFT over j2 giving X[k1 + L1 k2].  The inverse runs the same two
// stages in the opposite order, so a forward transform followed by an
// inverse (the Z pass) needs no exchange in between.
#pragma once

#include "common.cuh"

#include <cuda.h>   // CUtensorMap (the type only; maps are encoded through the runtime's driver entry point)

#include <algorithm>

namespace ori {

// Layout of the lines a CTA works on.
enum { LAYOUT_STRIDED = 0,     // C consecutive columns, points at a stride
       LAYOUT_CONTIG = 1 };    // C whole lines, points contiguous (X passes)

enum { SMODE_FWD = 0,          // forward transform, store n_out points
       SMODE_INV = 1,          // inverse transform of L points, store n_out
       SMODE_ZCONV = 2 };      // forward, * spectrum, inverse, store n_out

// Prologue of the X forward pass (value fed at cell (line, j), j < n).
enum { PRO_SCALE = 0,          // v = s[i] * x[i]           (x of type T)
       PRO_SCALE_D = 1,        // v = s[i] * x[i]           (x complex128, cast)
       PRO_COCG_FIRST = 2,     // p = r;          v = s[i] * p
       PRO_COCG = 3,           // p = r + beta p; v = s[i] * p
       PRO_KERNEL = 4 };       // v = G(d |signed offset|) (plan; FP64 only)

// Epilogue of the X inverse pass (conv value v at cell i = line*n + x).
enum { EPI_PLUS = 0,           // y = x + v                   (A form)
       EPI_PLUS_S = 1,         // y = x + s v                 (B form)
       EPI_PLUS_D = 2,         // y = x + v, x,y complex128   (A form, FP32 math)
       EPI_PLUS_S_D = 3,       // y = x + s v, x,y complex128 (B form, FP32 math)
       EPI_COCG = 4,           // q = p + s v; partial sum p^T q
       EPI_RESID = 5,          // r = b - (w + s v); partial sum ||r||^2
       EPI_RECOVER = 6,        // u = w / s, or b - v where s == 0
       EPI_RUPDATE = 7 };      // r -= c (d + s v), r complex128; partial ||r||^2

struct XArgs {
  // prologue
  const void* x;        // input vector (T or double), or r for COCG
  void* p;              // COCG search direction (read/write)
  const void* scale;    // complex scale s (T), n^3
  const void* beta;     // device double2 (COCG)
  // kernel-cube generation (PRO_KERNEL)
  double d, k;
  // epilogue
  const void* xin;      // x (EPI_PLUS*), p (EPI_COCG), w (EPI_RESID/RECOVER)
  const void* bvec;     // b (EPI_RESID, EPI_RECOVER); r (EPI_RUPDATE, in place)
  double coef;          // c of EPI_RUPDATE
  void* out;            // y / q / r / u
  double2* partials;    // per-block partial sums
  // geometry
  const void* in;       // FFT input (T1 for the inverse pass)
  void* fft_out;        // FFT output (T1 for the forward pass)
  int n;                // cells per axis
  int nlines;           // number of lines
  int n_in;             // valid input points (forward)
  int line_len_in;      // elements between lines in the input
  int line_len_out;     // elements between lines in the output
  int lines_per_plane;  // PRO_KERNEL: lines in one z plane (= L)
  int plane0;           // PRO_KERNEL: z index of the first plane of the launch
  int mode;             // PRO_* or EPI_*
  const void* twL;      // twiddle table for length L
  const int* done;      // solver flag: the pass returns at once if *done != 0
  // batch of right-hand sides: blockIdx.y selects one; each per-RHS pointer
  // moves by its byte stride (scale, the medium, is shared by all)
  long long bs_x, bs_p, bs_xin, bs_out, bs_bvec, bs_in, bs_fft;
  long long bs_beta;    // bytes between the beta of consecutive RHS
  int done_stride;      // bytes between the flags of consecutive RHS
  const double* coefs;  // EPI_RUPDATE: per-RHS coefficient (overrides coef when set)
  int nrhs;             // right-hand sides in the batch (gridDim.y)
  int sm_count;         // persistent kernels: SMs of the device
  int* err;             // set to 1 by a kernel whose bounded wait on a bulk copy gave up
};

struct SArgs {
  const void* in;
  void* out;
  long long in_outer, out_outer;   // elements between outer indices
  long long in_pt, out_pt;         // elements between points of a line
  int ncols;                       // columns per outer index (stride 1)
  int col_blocks;                  // ceil(ncols / C)
  int n_in, n_out;
  int nouter;
  const void* twL;
  const void* ghat;                // spectrum, H^3 entries (SMODE_ZCONV)
  const void* ghatZ;               // FP32 spectrum in Z-tile order [my][kx/kZGroup][mz][kZGroup]
  int H;                           // L/2 + 1
  const int* done;
  int sm_count;                    // persistent kernels: CTAs to launch
  // batch of right-hand sides (blockIdx.y): byte strides of in/out per RHS,
  // and of the spectra, one spectrum per wave number for rhs_per_ghat RHS
  int nrhs;
  long long bs_in, bs_out, bs_ghat, bs_ghatZ;
  int rhs_per_ghat;
  int done_stride;
  int mirror_in;                   // forward transform of an even sequence stored up to L/2:
                                   // input row j > L/2 is read from row L - j
  // launch schedule of the FP32 Y-forward and Z passes (chosen by the plan's
  // autotuner): SCHED_PERSISTENT = the pipelined persistent kernel
  // with at most cta_cap resident CTAs per SM (0 = as many as fit);
  // SCHED_TILES = one CTA per tile of columns
  int sched;
  int cta_cap;
  int variant;                     // pipelined FP32 kernels: launch variant (has_pipe_variants)
  // FP32 Z and Y passes with 16-column tiles: the input rows of a tile
  // arrive by TMA (cp.async.bulk.tensor) through this map of the input cube,
  // dims (kx, ky, z, right-hand side) and box (16, 1, zbox, 1) for the Z
  // pass, (kx, y, z, right-hand side) and box (16, zbox, 1, 1) for the Y
  // passes; zrows_ok = 0 keeps cp.async
  CUtensorMap zrows;
  int zrows_ok;
  int zbox;
  int* err;                        // set to 1 when a bounded wait on a copy gave up
};

enum { SCHED_PERSISTENT = 0, SCHED_TILES = 1 };

// Columns per group of the Z-tile-ordered FP32 spectrum [my][kx / kZGroup][mz][kZGroup].
constexpr int kZGroup = 16;

// Move a pointer by `bytes` (null stays null).
__device__ __forceinline__ const void* bmove(const void* p, long long bytes) {
  return p == nullptr ? p : static_cast<const void*>(static_cast<const char*>(p) + bytes);
}
__device__ __forceinline__ void* bmove(void* p, long long bytes) {
  return p == nullptr ? p : static_cast<void*>(static_cast<char*>(p) + bytes);
}
__device__ __forceinline__ const int* bflag(const int* f, int stride, int rhs) {
  return f == nullptr ? f : reinterpret_cast<const int*>(reinterpret_cast<const char*>(f) + (long long)stride * rhs);
}

// The view of the arguments seen by right-hand side `rhs` of a batch.
__device__ __forceinline__ XArgs x_for_rhs(XArgs a, int rhs) {
  if (a.coefs != nullptr) a.coef = a.coefs[rhs];
  if (rhs == 0) return a;
  a.x = bmove(a.x, a.bs_x * rhs);
  a.p = bmove(a.p, a.bs_p * rhs);
  a.beta = bmove(a.beta, a.bs_beta * rhs);
  a.xin = bmove(a.xin, a.bs_xin * rhs);
  a.bvec = bmove(a.bvec, a.bs_bvec * rhs);
  a.out = bmove(a.out, a.bs_out * rhs);
  a.in = bmove(a.in, a.bs_fft * rhs);
  a.fft_out = bmove(a.fft_out, a.bs_fft * rhs);
  a.done = bflag(a.done, a.done_stride, rhs);
  return a;
}
__device__ __forceinline__ SArgs s_for_rhs(SArgs a, int rhs) {
  if (rhs == 0) return a;
  a.in = bmove(a.in, a.bs_in * rhs);
  a.out = bmove(a.out, a.bs_out * rhs);
  const int g = a.rhs_per_ghat > 0 ? rhs / a.rhs_per_ghat : 0;
  a.ghat = bmove(a.ghat, a.bs_ghat * g);
  a.ghatZ = bmove(a.ghatZ, a.bs_ghatZ * g);
  a.done = bflag(a.done, a.done_stride, rhs);
  return a;
}

// Launch variants of the pipelined FP32 Y-forward, Z and Y-inverse passes at
// the padded lengths where the autotuner chooses among them:
//   0: the default tile (16 columns) and split L = L1 * L2 of Split<L>;
//   1: 8-column tiles, same split;
//   2: 16-column tiles, first stage of radix 2 * L1 (second of L2 / 2).
constexpr bool has_pipe_variants(int L) { return L >= 256 && L <= 1024; }
constexpr int pipe_variants(int L) { return has_pipe_variants(L) ? 3 : 1; }

template <int L, int C, class T, int L1X = Split<L>::L1>
struct Tile {
  static constexpr int L1 = L1X;
  static constexpr int L2 = L / L1X;
  static constexpr int NT = C * L2;            // threads per CTA
  static constexpr int PK = L2 + 1;            // forward exchange [c][k1][j2]
  static constexpr int PC = (L1 * PK) | 1;
  static constexpr int PKI = L1 + 1;           // inverse exchange [c][ja][k1]
  static constexpr int PCI = (L2 * PKI) | 1;
  static constexpr int SMEM_ELEMS = (C * PC > C * PCI) ? C * PC : C * PCI;
  static constexpr size_t SMEM_BYTES = size_t(SMEM_ELEMS) * sizeof(cpx<T>);
  // The FP32 X passes are latency bound: three resident CTAs per SM (the
  // exchange buffer allows it) keep more loads in flight (measured: the X
  // passes gain 20%, the strided Y passes do not, so only the X passes use it).
  static constexpr int MINB = (sizeof(T) == 4 && NT == 256 && SMEM_BYTES <= 72 * 1024) ? 3 : 1;
};

// ---------------------------------------------------------------------------
// Stage helpers shared by both layouts
// ---------------------------------------------------------------------------

// thread t -> (line c, j2) of the first forward stage / second inverse stage
template <int LAYOUT, int C, int L2>
__device__ __forceinline__ void map_t(int t, int& c, int& j) {
  if (LAYOUT == LAYOUT_STRIDED) { c = t % C; j = t / C; }
  else { j = t % L2; c = t / L2; }
}
// item s -> (line c, k1) of the second forward stage / first inverse stage
template <int LAYOUT, int C, int L1>
__device__ __forceinline__ void map_s(int s, int& c, int& k) {
  if (LAYOUT == LAYOUT_STRIDED) { c = s % C; k = s / C; }
  else { k = s % L1; c = s / L1; }
}

// ---------------------------------------------------------------------------
// Warp + block reduction of a double2 partial into partials[blockIdx.x]
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 warp_sum2(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// All threads of the block must call it.  Uses 32 double2 of scratch smem.
__device__ __forceinline__ void block_partial(double2 v, double2* red, double2* partials) {
  v = warp_sum2(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = make_double2(0.0, 0.0);
    for (int i = 0; i < nw; ++i) { s.x += red[i].x; s.y += red[i].y; }
    partials[blockIdx.x] = s;
  }
}

// Like block_partial, but v is already reduced over the warp (valid in lane 0).
__device__ __forceinline__ void block_partial_lane0(double2 v, double2* red, double2* partials) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = make_double2(0.0, 0.0);
    for (int i = 0; i < nw; ++i) { s.x += red[i].x; s.y += red[i].y; }
    partials[blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------
// Pass launchers.  Each arithmetic T (float, double, dfl) and each part (the
// X passes, the strided forward and inverse passes, the Z pass) is explicitly
// instantiated in a translation unit of its own (passes_inst.cu compiled once
// per pair), so that the library builds in parallel.
// ---------------------------------------------------------------------------
struct Scalars;
template <class T> cudaError_t run_xfwd(int L, bool half, const XArgs& a, cudaStream_t s, bool setup);
template <class T> cudaError_t run_xinv(int L, const XArgs& a, Scalars* sc, int fin, cudaStream_t s, bool setup,
                                        unsigned* nblocks);
template <class T> cudaError_t run_strided_fwd(int L, bool half, const SArgs& a, cudaStream_t s, bool setup);
template <class T> cudaError_t run_strided_inv(int L, const SArgs& a, cudaStream_t s, bool setup);
template <class T> cudaError_t run_zconv(int L, const SArgs& a, cudaStream_t s, bool setup);

// One strided pass (SMODE_FWD, SMODE_INV or SMODE_ZCONV) at padded length L.
template <class T>
inline cudaError_t run_strided(int L, int smode, bool half, const SArgs& a, cudaStream_t s, bool setup) {
  if (smode == SMODE_FWD) return run_strided_fwd<T>(L, half, a, s, setup);
  if (smode == SMODE_INV) return run_strided_inv<T>(L, a, s, setup);
  return run_zconv<T>(L, a, s, setup);
}

}  // namespace ori
