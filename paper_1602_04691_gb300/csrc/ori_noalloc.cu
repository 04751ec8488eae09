// ori_noalloc.cu - ori_matvec_noalloc: the FP64 operator y = A x for small
// grids with every intermediate in one statically allocated device array, so
// the call never allocates device memory.
//
// For callers that cannot allocate: code whose device memory is owned by
// another framework's pool (raw cudaMalloc is forbidden there), latency-
// critical callers that must not risk the device-wide synchronisation that
// cudaMalloc / cudaFree may cause, and code under a rule that forbids dynamic
// allocation after start-up.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/ori.h"
#include "common.cuh"
#include "passes.cuh"
#include "scalars.cuh"

namespace ori {
void set_last_error(const std::string& msg);   // ori_api.cu: the ori_last_error() message
}  // namespace ori

using namespace ori;

namespace {

constexpr int kMaxN = ORI_NOALLOC_MAX_N;   // 16
constexpr int kMaxL = 2 * kMaxN;           // smallest power of two >= 2n for n <= 16
constexpr int kMaxH = kMaxL / 2 + 1;
constexpr size_t kC128 = sizeof(cpx<double>);

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kTwBytes = align256(size_t(kMaxL) * kC128);
constexpr size_t kGhatBytes = align256(size_t(kMaxH) * kMaxH * kMaxH * kC128);
constexpr size_t kScaleBytes = align256(size_t(kMaxN) * kMaxN * kMaxN * kC128);
constexpr size_t kCubeBytes = size_t(kMaxL) * kMaxL * kMaxL * kC128;
constexpr size_t kPassBytes = (size_t(kMaxN) * kMaxN * kMaxL + size_t(kMaxN) * kMaxL * kMaxL) * kC128;
constexpr size_t kWorkBytes = align256(kCubeBytes > kPassBytes ? kCubeBytes : kPassBytes);
constexpr size_t kScratchBytes = kTwBytes + kGhatBytes + kScaleBytes + kWorkBytes;
static_assert(kScratchBytes == ORI_NOALLOC_SCRATCH_BYTES, "header and scratch size disagree");

}  // namespace

// The scratch every call shares.  It keeps the previous call's contents; each
// call writes every element it later reads (twiddles, h N, the kernel cube
// and its spectrum, both FFT work cubes), so nothing needs clearing.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

// Per-device set-up: the device address of the scratch array (the host-side
// name is only a stand-in) and the shared-memory attributes of the kernels.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_dev[kMaxDevices] = {nullptr};

ori_status na_fail(ori_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

__global__ void k_na_twiddles(cpx<double>* tw, int L) {
  const long long M = 1LL << 20;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < L; m += gridDim.x * blockDim.x) {
    const CosSin v = turn_cos_sin((long long)m * (M / L), M);
    tw[m] = {v.c, v.s};
  }
}

__global__ void k_na_scale(const cpx<double>* __restrict__ h, const double* __restrict__ N,
                           cpx<double>* w, long long n3) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3;
       i += (long long)gridDim.x * blockDim.x) {
    const cpx<double> hv = h[i];
    const double nv = N[i];
    w[i] = {hv.x * nv, hv.y * nv};
  }
}

__global__ void k_na_extract(const cpx<double>* __restrict__ cube, cpx<double>* g, int L, int H,
                             double scale) {
  const int total = H * H * H;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int m1 = i % H, m2 = (i / H) % H, m3 = i / (H * H);
    const cpx<double> v = cube[((long long)m3 * L + m2) * L + m1];
    g[i] = {v.x * scale, v.y * scale};
  }
}

// The symbol's address is looked up on every call (a host-side query, no
// allocation): a context created anew on the device (after cudaDeviceReset)
// may place the array elsewhere, and the cached address would then be stale.
// The kernel attributes are set again whenever the address changes.
ori_status setup_device(int dev, void** base) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (dev < 0 || dev >= kMaxDevices) return na_fail(ORI_ERR_UNSUPPORTED, "device index out of range");
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr)
    return na_fail(ORI_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  if (g_scratch_dev[dev] != p) {
    for (int L = 4; L <= kMaxL; L *= 2) {
      XArgs xa{};
      SArgs sa{};
      if ((e = run_xfwd<double>(L, true, xa, nullptr, true)) != cudaSuccess ||
          (e = run_xfwd<double>(L, false, xa, nullptr, true)) != cudaSuccess ||
          (e = run_xinv<double>(L, xa, nullptr, FIN_NONE, nullptr, true, nullptr)) != cudaSuccess ||
          (e = run_strided<double>(L, SMODE_FWD, true, sa, nullptr, true)) != cudaSuccess ||
          (e = run_strided<double>(L, SMODE_FWD, false, sa, nullptr, true)) != cudaSuccess ||
          (e = run_strided<double>(L, SMODE_INV, false, sa, nullptr, true)) != cudaSuccess ||
          (e = run_strided<double>(L, SMODE_ZCONV, true, sa, nullptr, true)) != cudaSuccess)
        return na_fail(ORI_ERR_CUDA, std::string("kernel set-up: ") + cudaGetErrorString(e));
    }
    g_scratch_dev[dev] = p;
  }
  *base = g_scratch_dev[dev];
  return ORI_OK;
}

#define NA_CUDA(call)                                                                     \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return na_fail(ORI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

extern "C" ori_status ori_matvec_noalloc(int64_t n64, double k, const ori_domain* dom, double c_S,
                                         const double* h_dev, const double* N_dev, const double* x_dev,
                                         double* y_dev, void* stream) {
  set_last_error("");
  if (n64 < 2 || n64 > kMaxN)
    return na_fail(ORI_ERR_INVALID_ARG, "ori_matvec_noalloc: n must be in [2, ORI_NOALLOC_MAX_N = 16]");
  if (!std::isfinite(k) || k <= 0) return na_fail(ORI_ERR_INVALID_ARG, "k must be finite and > 0");
  if (!dom || !std::isfinite(dom->side) || dom->side <= 0)
    return na_fail(ORI_ERR_INVALID_ARG, "domain side must be finite and > 0");
  if (c_S == 0.0) c_S = 4.0 * kPi;
  if (!std::isfinite(c_S)) return na_fail(ORI_ERR_INVALID_ARG, "c_S must be finite");
  if (!h_dev || !N_dev || !x_dev || !y_dev) return na_fail(ORI_ERR_INVALID_ARG, "NULL pointer");
  {
    // [x, x + 16 n^3) and [y, y + 16 n^3) must be disjoint: the last pass reads x while other blocks write y
    const uintptr_t xb = reinterpret_cast<uintptr_t>(x_dev), yb = reinterpret_cast<uintptr_t>(y_dev);
    const uintptr_t bytes = uintptr_t(n64) * uintptr_t(n64) * uintptr_t(n64) * sizeof(cpx<double>);
    if (xb < yb + bytes && yb < xb + bytes) return na_fail(ORI_ERR_INVALID_ARG, "x_dev and y_dev must not overlap");
  }

  int dev = 0;
  NA_CUDA(cudaGetDevice(&dev));
  void* base = nullptr;
  ori_status st = setup_device(dev, &base);
  if (st != ORI_OK) return st;

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n = int(n64);
  int L = 4;
  while (L < 2 * n) L *= 2;
  const int H = L / 2 + 1;
  const double d = dom->side / double(n);
  const long long n3 = (long long)n * n * n;
  unsigned char* b = static_cast<unsigned char*>(base);
  cpx<double>* tw = reinterpret_cast<cpx<double>*>(b);
  cpx<double>* ghat = reinterpret_cast<cpx<double>*>(b + kTwBytes);
  cpx<double>* wsc = reinterpret_cast<cpx<double>*>(b + kTwBytes + kGhatBytes);
  cpx<double>* work = reinterpret_cast<cpx<double>*>(b + kTwBytes + kGhatBytes + kScaleBytes);
  cpx<double>* T1 = work;                                  // [n][n][L]
  cpx<double>* T2 = work + (long long)n * n * L;           // [n][L][L]

  k_na_twiddles<<<1, 64, 0, s>>>(tw, L);
  NA_CUDA(cudaGetLastError());
  k_na_scale<<<64, 256, 0, s>>>(reinterpret_cast<const cpx<double>*>(h_dev), N_dev, wsc, n3);
  NA_CUDA(cudaGetLastError());

  // kernel cube c_S |Delta| G(d |j|) (self term 0) -> FP64 3D FFT -> (L/2+1)^3
  {
    XArgs a{};
    a.mode = PRO_KERNEL;
    a.d = d;
    a.k = k;
    a.n = n;
    a.nlines = L * L;
    a.n_in = L;
    a.line_len_in = L;
    a.line_len_out = L;
    a.lines_per_plane = L;
    a.fft_out = work;
    a.twL = tw;
    NA_CUDA(run_xfwd<double>(L, false, a, s, false));
    SArgs y{};
    y.in = work; y.out = work;
    y.in_outer = (long long)L * L; y.out_outer = (long long)L * L;
    y.in_pt = L; y.out_pt = L; y.ncols = L; y.n_in = L; y.n_out = L; y.nouter = L; y.twL = tw;
    NA_CUDA(run_strided<double>(L, SMODE_FWD, false, y, s, false));
    SArgs z{};
    z.in = work; z.out = work;
    z.in_outer = L; z.out_outer = L;
    z.in_pt = (long long)L * L; z.out_pt = (long long)L * L;
    z.ncols = L; z.n_in = L; z.n_out = L; z.nouter = L; z.twL = tw;
    NA_CUDA(run_strided<double>(L, SMODE_FWD, false, z, s, false));
    const double scale = c_S * d * d * d / (double(L) * L * L);
    k_na_extract<<<64, 256, 0, s>>>(work, ghat, L, H, scale);
    NA_CUDA(cudaGetLastError());
  }
  // y = x + conv(w x): X fwd, Y fwd, Z conv, Y inv, X inv (the cube region is reused)
  {
    XArgs pro{};
    pro.mode = PRO_SCALE;
    pro.x = x_dev;
    pro.scale = wsc;
    pro.n = n; pro.nlines = n * n; pro.n_in = n; pro.line_len_in = n; pro.line_len_out = L;
    pro.fft_out = T1; pro.twL = tw;
    NA_CUDA(run_xfwd<double>(L, true, pro, s, false));
    SArgs y{};
    y.in = T1; y.out = T2;
    y.in_outer = (long long)n * L; y.out_outer = (long long)L * L;
    y.in_pt = L; y.out_pt = L; y.ncols = L; y.n_in = n; y.n_out = L; y.nouter = n; y.twL = tw;
    NA_CUDA(run_strided<double>(L, SMODE_FWD, true, y, s, false));
    SArgs z{};
    z.in = T2; z.out = T2;
    z.in_outer = L; z.out_outer = L;
    z.in_pt = (long long)L * L; z.out_pt = (long long)L * L;
    z.ncols = L; z.n_in = n; z.n_out = n; z.nouter = L;
    z.twL = tw; z.ghat = ghat; z.H = H;
    NA_CUDA(run_strided<double>(L, SMODE_ZCONV, true, z, s, false));
    SArgs yi{};
    yi.in = T2; yi.out = T1;
    yi.in_outer = (long long)L * L; yi.out_outer = (long long)n * L;
    yi.in_pt = L; yi.out_pt = L; yi.ncols = L; yi.n_in = L; yi.n_out = n; yi.nouter = n; yi.twL = tw;
    NA_CUDA(run_strided<double>(L, SMODE_INV, false, yi, s, false));
    XArgs epi{};
    epi.mode = EPI_PLUS;
    epi.xin = x_dev;
    epi.out = y_dev;
    epi.n = n; epi.nlines = n * n; epi.line_len_in = L; epi.line_len_out = n;
    epi.in = T1; epi.twL = tw;
    NA_CUDA(run_xinv<double>(L, epi, nullptr, FIN_NONE, s, false, nullptr));
  }
  return ORI_OK;
}
