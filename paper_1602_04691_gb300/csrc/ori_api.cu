// ori_api.cu - the C ABI declared in include/ori.h: plan, matvec, COCG solve
// (FP64, and mixed FP32 / FP64-class refinement), batched solves over several
// incidence directions and wave numbers, and the adjoint gradient.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/ori.h"
#include "common.cuh"
#include "dfloat.cuh"
#include "passes.cuh"
#include "scalars.cuh"
#include "vector_kernels.cuh"

using namespace ori;

// NVTX range for profilers (nsys, ncu --nvtx): pushed on construction, popped
// on scope exit.  Host-side only; costs nothing when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

static ori_status fail(ori_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

namespace ori {
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace ori

#define ORI_CUDA(call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(e_ == cudaErrorMemoryAllocation ? ORI_ERR_OOM : ORI_ERR_CUDA,         \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                  \
  } while (0)

#define ORI_TRY(expr)                 \
  do {                                \
    ori_status s_ = (expr);           \
    if (s_ != ORI_OK) return s_;      \
  } while (0)

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------
struct ori_plan_s {
  int device = 0;
  int n = 0, L = 0, H = 0;
  long long n3 = 0;
  double d = 0, c_S = 0, side = 0, origin[3] = {0, 0, 0};
  std::vector<double> ks;          // wave numbers; one spectrum each
  bool lean = false;               // mixed-solve-only plan (ori_plan_opts.lean)
  std::vector<std::vector<double>> history;   // per system: residual estimates of the last solve
                                              // run with ori_solve_opts.history
  size_t bytes = 0, mem_cap = 0;
  int sm_count = 0;
  unsigned long long zero_S = 0;
  // medium
  cpx<double>* h = nullptr;
  double* N = nullptr;
  cpx<double>* w64 = nullptr;
  cpx<double>* S64 = nullptr;
  cpx<double>* Sinv = nullptr;
  cpx<float>* w32 = nullptr;
  cpx<float>* S32 = nullptr;
  cpx<dfl>* wdf = nullptr;         // h N and sqrt(h N) in paired FP32
  cpx<dfl>* Sdf = nullptr;
  // spectra (one per wave number, contiguous) and twiddles
  cpx<double>* ghat64 = nullptr;
  cpx<float>* ghat32 = nullptr;
  cpx<dfl>* ghatdf = nullptr;
  cpx<float>* ghatZ32 = nullptr;   // FP32 spectrum in Z-tile order
  cpx<double>* tw64 = nullptr;
  cpx<float>* tw32 = nullptr;
  cpx<dfl>* twdf = nullptr;
  unsigned long long* d_count = nullptr;
  int* d_fault = nullptr;          // set by a kernel whose bounded wait on a bulk copy gave up
  int* h_fault = nullptr;          // pinned mirror
  unsigned long long* h_count = nullptr;   // pinned mirror of d_count
  // device addresses of the pinned mirrors (mapped host memory): the control
  // copies between them and device memory run as kernels (k_small_copy)
  void* h_fault_d = nullptr;
  void* h_count_d = nullptr;
  void* h_sc_d = nullptr;
  void* h_small_d = nullptr;
  void* h_skip_d = nullptr;
  // tensor map of the FP32 Z pass's input rows (bulk-copy staging), for T2f
  // and a batch of zmap_R right-hand sides
  CUtensorMap zmap{};
  const void* zmap_ptr = nullptr;
  int zmap_R = 0, zmap_ok = 0, zbox = 0;
  // tensor maps of the FP32 Y passes' input rows: T1f rows (Y forward) and
  // T2f rows (Y inverse), 16 columns by ybox rows a box
  CUtensorMap ymap_f{}, ymap_i{};
  const void* ymap_ptr = nullptr;
  int ymap_R = 0, ymap_ok = 0, ybox_f = 0, ybox_i = 0;
  // batch capacity: pass scratch and solver state for cap right-hand sides
  int cap = 0;
  cpx<float>* T1f = nullptr;
  cpx<float>* T2f = nullptr;
  cpx<double>* T1d = nullptr;      // FP64 and paired-FP32 passes
  cpx<double>* T2d = nullptr;
  Scalars* sc = nullptr;
  Scalars* h_sc = nullptr;         // pinned mirror of the scalar heads
  double2* partials = nullptr;
  size_t part_per_rhs = 0;
  cpx<double>* b64 = nullptr;
  cpx<double>* w = nullptr;
  cpx<double>* r64 = nullptr;
  cpx<double>* u0 = nullptr;
  cpx<double>* p64 = nullptr;
  cpx<double>* q64 = nullptr;
  cpx<float>* x32 = nullptr;
  cpx<float>* r32 = nullptr;
  cpx<float>* p32 = nullptr;
  cpx<float>* q32 = nullptr;
  // per-RHS small arrays: device copies and pinned host staging
  double* d_tols = nullptr;        // inner tolerances
  double* d_scl = nullptr;         // scale factors (normalise / accumulate)
  double* d_coef = nullptr;        // residual-update coefficients
  double* d_kv = nullptr;          // wave number of each RHS (plane waves)
  cpx<double>* d_phase = nullptr;  // 3n plane-wave phase factors per RHS
  double* d_dir = nullptr;         // 3 per RHS (plane waves)
  int* d_skip = nullptr;           // 1 = this RHS takes no part in a pass
  double* h_small = nullptr;       // pinned: 7 * cap doubles
  int* h_skip = nullptr;           // pinned: cap ints
  unsigned xinv_blocks = 0;        // largest X-inverse grid of the three arithmetics
  cudaStream_t ps = nullptr;       // private stream (capturable)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, evj = nullptr;
  // captured COCG blocks (FP32 and FP64 inner solvers)
  cudaGraphExec_t graph_f = nullptr, graph_d = nullptr;
  int graph_f_len = 0, graph_d_len = 0, graph_f_nrhs = 0, graph_d_nrhs = 0;
  bool graph_f_timed = false, graph_d_timed = false;
  int vec_grid = 0;
  // launch schedule (ori_schedule): FP32 Y-forward / Z kernels, CTA cap, vector grid
  int sched_y = SCHED_PERSISTENT, sched_z = SCHED_PERSISTENT, sched_yi = SCHED_PERSISTENT, cta_cap = 0, vec_ctas = 8;
  int var_y = 0, var_z = 0, var_yi = 0;   // launch variants of the persistent FP32 kernels
  // accounting (ori_plan_stats) and optional per-kernel event timing
  ori_plan_stats stats{};
  bool capturing = false;
  int cap_iter = 0;                // iteration being captured (timing attribution)
  unsigned long long cap_launches = 0, graph_f_kernels = 0, graph_d_kernels = 0;
  bool timing = false;
  struct Pend { int kind, e0, e1, iter; };   // iter: iteration index inside a captured block
  cudaEvent_t* tev = nullptr;      // immediate pool
  int tev_n = 0, tev_used = 0;
  Pend* pend = nullptr;
  int npend = 0;
  cudaEvent_t* gev = nullptr;      // pool owned by the captured graphs
  int gev_n = 0, gev_used = 0;
  Pend* gpend_f = nullptr;
  Pend* gpend_d = nullptr;
  int ngpend_f = 0, ngpend_d = 0;
  Pend* gpend_cur = nullptr;
  int* ngpend_cur = nullptr;
};

static constexpr int kEvPool = 4096;
static constexpr int kMaxVecCtasPerSm = 16;   // bound of ori_schedule.vec_ctas_per_sm

// Count one kernel launch (graph nodes are counted at each replay instead).
static inline void launched(ori_plan_s* p) {
  if (p->capturing) ++p->cap_launches;
  else ++p->stats.kernel_launches;
}

// Record a timing event on s; returns its pool index, or -1 (timing off/full).
static int t_rec(ori_plan_s* p, cudaStream_t s) {
  if (!p->timing) return -1;
  if (p->capturing) {
    if (p->gev_used >= p->gev_n) return -1;
    // an external record becomes an event-record node of the graph
    cudaEventRecordWithFlags(p->gev[p->gev_used], s, cudaEventRecordExternal);
    return p->gev_used++;
  }
  if (p->tev_used >= p->tev_n) return -1;
  cudaEventRecord(p->tev[p->tev_used], s);
  return p->tev_used++;
}

static void t_pair(ori_plan_s* p, int kind, int e0, int e1) {
  if (e0 < 0 || e1 < 0) return;
  if (p->capturing) {
    if (p->gpend_cur && *p->ngpend_cur < kEvPool) p->gpend_cur[(*p->ngpend_cur)++] = {kind, e0, e1, p->cap_iter};
  } else if (p->npend < kEvPool) {
    p->pend[p->npend++] = {kind, e0, e1, 0};
  }
}

// Add the elapsed times of recorded pairs (the stream must be synchronised).
static void t_harvest(ori_plan_s* p) {
  for (int i = 0; i < p->npend; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->tev[p->pend[i].e0], p->tev[p->pend[i].e1]) == cudaSuccess) {
      p->stats.pass_ms[p->pend[i].kind] += ms;
      p->stats.pass_count[p->pend[i].kind] += 1;
    }
  }
  cudaGetLastError();
  p->npend = 0;
  p->tev_used = 0;
}

// Only the first `real_iters` iterations of a replayed block ran; the rest
// returned at once (every right-hand side had converged) and are not counted.
static void t_harvest_graph(ori_plan_s* p, const ori_plan_s::Pend* g, int ng, int real_iters) {
  for (int i = 0; i < ng; ++i) {
    if (g[i].iter >= real_iters) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->gev[g[i].e0], p->gev[g[i].e1]) == cudaSuccess) {
      p->stats.pass_ms[g[i].kind] += ms;
      p->stats.pass_count[g[i].kind] += 1;
    }
  }
  cudaGetLastError();
}

static ori_status plan_alloc(ori_plan_s* p, void** ptr, size_t bytes) {
  if (p->mem_cap && p->bytes + bytes > p->mem_cap)
    return fail(ORI_ERR_OOM, "plan memory would exceed opts->mem_cap");
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return fail(ORI_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  p->bytes += bytes;
  return ORI_OK;
}

template <class P>
static ori_status alloc_n(ori_plan_s* p, P** ptr, size_t count) {
  return plan_alloc(p, reinterpret_cast<void**>(ptr), count * sizeof(P));
}

template <class P>
static void free_n(ori_plan_s* p, P*& ptr, size_t count) {
  if (ptr) {
    cudaFree(ptr);
    p->bytes -= count * sizeof(P);
    ptr = nullptr;
  }
}

static void drop_graphs(ori_plan_s* p) {
  if (p->graph_f) cudaGraphExecDestroy(p->graph_f);
  if (p->graph_d) cudaGraphExecDestroy(p->graph_d);
  p->graph_f = p->graph_d = nullptr;
  p->graph_f_len = p->graph_d_len = 0;
}

static size_t t1_elems(const ori_plan_s* p) { return size_t(p->n) * p->n * p->L; }
static size_t t2_elems(const ori_plan_s* p) { return size_t(p->n) * p->L * p->L; }

// Release the batch-sized buffers.
static void free_capacity(ori_plan_s* p) {
  const size_t c = size_t(p->cap), n3 = size_t(p->n3);
  p->T1f = nullptr;   // the FP32 cubes live inside the FP64-class ones
  p->T2f = nullptr;
  free_n(p, p->T1d, c * t1_elems(p));
  free_n(p, p->T2d, c * t2_elems(p));
  free_n(p, p->sc, c);
  free_n(p, p->partials, c * p->part_per_rhs);
  for (cpx<double>** v : {&p->b64, &p->w, &p->r64, &p->u0, &p->p64, &p->q64}) free_n(p, *v, c * n3);
  for (cpx<float>** v : {&p->x32, &p->r32, &p->p32, &p->q32}) free_n(p, *v, c * n3);
  for (double** v : {&p->d_tols, &p->d_scl, &p->d_coef, &p->d_kv}) free_n(p, *v, c);
  free_n(p, p->d_dir, 3 * c);
  free_n(p, p->d_phase, 3 * size_t(p->n) * c);
  free_n(p, p->d_skip, c);
  if (p->h_sc) cudaFreeHost(p->h_sc);
  if (p->h_small) cudaFreeHost(p->h_small);
  if (p->h_skip) cudaFreeHost(p->h_skip);
  p->h_sc = nullptr;
  p->h_small = nullptr;
  p->h_skip = nullptr;
  p->h_sc_d = p->h_small_d = p->h_skip_d = nullptr;
  p->cap = 0;
  drop_graphs(p);
}

// Make room for nrhs right-hand sides (the scratch of every pass and the solver state).
static ori_status ensure_capacity(ori_plan_s* p, int nrhs) {
  if (nrhs <= p->cap) return ORI_OK;
  cudaStreamSynchronize(p->ps);
  free_capacity(p);
  const size_t c = size_t(nrhs), n3 = size_t(p->n3);
  // FP32 passes and FP64-class passes never run at the same time (one
  // stream, one operator application after another), so the FP32 cubes
  // (half the bytes) share the FP64-class allocations
  ORI_TRY(alloc_n(p, &p->T1d, c * t1_elems(p)));
  ORI_TRY(alloc_n(p, &p->T2d, c * t2_elems(p)));
  p->T1f = reinterpret_cast<cpx<float>*>(p->T1d);
  p->T2f = reinterpret_cast<cpx<float>*>(p->T2d);
  ORI_TRY(alloc_n(p, &p->sc, c));
  ORI_CUDA(cudaMemsetAsync(p->sc, 0, c * sizeof(Scalars), p->ps));
  // partials of the X-inverse reductions, or two per block of the widest vector grid
  p->part_per_rhs = std::max<size_t>(size_t(p->xinv_blocks), size_t(2) * std::max(1, p->sm_count) * kMaxVecCtasPerSm) + 16;
  ORI_TRY(alloc_n(p, &p->partials, c * p->part_per_rhs));
  for (cpx<double>** v : {&p->b64, &p->w, &p->r64}) ORI_TRY(alloc_n(p, v, c * n3));
  if (!p->lean)   // FP64 COCG vectors and the incident field kept for S = 0 cells
    for (cpx<double>** v : {&p->u0, &p->p64, &p->q64}) ORI_TRY(alloc_n(p, v, c * n3));
  for (cpx<float>** v : {&p->x32, &p->r32, &p->p32, &p->q32}) ORI_TRY(alloc_n(p, v, c * n3));
  for (double** v : {&p->d_tols, &p->d_scl, &p->d_coef, &p->d_kv}) ORI_TRY(alloc_n(p, v, c));
  ORI_TRY(alloc_n(p, &p->d_dir, 3 * c));
  ORI_TRY(alloc_n(p, &p->d_phase, 3 * size_t(p->n) * c));
  ORI_TRY(alloc_n(p, &p->d_skip, c));
  if (cudaMallocHost(&p->h_sc, c * sizeof(Scalars)) != cudaSuccess ||
      cudaMallocHost(&p->h_small, 7 * c * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&p->h_skip, c * sizeof(int)) != cudaSuccess)
    return fail(ORI_ERR_OOM, "cudaMallocHost failed");
  if (cudaHostGetDevicePointer(&p->h_sc_d, p->h_sc, 0) != cudaSuccess ||
      cudaHostGetDevicePointer(&p->h_small_d, p->h_small, 0) != cudaSuccess ||
      cudaHostGetDevicePointer(&p->h_skip_d, p->h_skip, 0) != cudaSuccess)
    return fail(ORI_ERR_CUDA, "cudaHostGetDevicePointer failed (pinned memory not mapped)");
  std::memset(p->h_sc, 0, c * sizeof(Scalars));
  p->cap = nrhs;
  return ORI_OK;
}

static void plan_free(ori_plan_s* p) {
  if (!p) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  cudaDeviceSynchronize();
  free_capacity(p);
  void* ptrs[] = {p->h, p->N, p->w64, p->S64, p->Sinv, p->w32, p->S32, p->wdf, p->Sdf,
                  p->ghat64, p->ghat32, p->ghatdf, p->ghatZ32, p->tw64, p->tw32, p->twdf, p->d_count,
                  p->d_fault};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->h_fault) cudaFreeHost(p->h_fault);
  if (p->h_count) cudaFreeHost(p->h_count);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  if (p->evj) cudaEventDestroy(p->evj);
  if (p->tev) { for (int i = 0; i < p->tev_n; ++i) cudaEventDestroy(p->tev[i]); delete[] p->tev; }
  if (p->gev) { for (int i = 0; i < 2 * kEvPool; ++i) cudaEventDestroy(p->gev[i]); delete[] p->gev; }
  delete[] p->pend;
  delete[] p->gpend_f;
  delete[] p->gpend_d;
  if (p->ps) cudaStreamDestroy(p->ps);
  cudaSetDevice(prev);
  delete p;
}

// Host twiddle table tab[m] = (cos, sin)(2 pi m / L), from the compile-time
// evaluable series in common.cuh on a fine circle (2^20 points).
template <class T>
static void host_twiddles(int L, cpx<T>* out) {
  const long long M = 1LL << 20;
  for (int m = 0; m < L; ++m) {
    CosSin v = turn_cos_sin((long long)m * (M / L), M);
    out[m] = cpx<T>{T(v.c), T(v.s)};
  }
}

// Stream handoff: the plan's private stream waits for the caller's stream.
static ori_status enter(ori_plan_s* p, cudaStream_t user) {
  ORI_CUDA(cudaEventRecord(p->evj, user));
  ORI_CUDA(cudaStreamWaitEvent(p->ps, p->evj, 0));
  return ORI_OK;
}
static ori_status leave(ori_plan_s* p, cudaStream_t user) {
  ORI_CUDA(cudaEventRecord(p->evj, p->ps));
  ORI_CUDA(cudaStreamWaitEvent(user, p->evj, 0));
  return ORI_OK;
}

// One application of the convolution operator to a batch of nrhs vectors: X
// fwd (prologue), Y fwd, Z conv, Y inv, X inv (epilogue).  `pro` and `epi`
// carry the mode, vectors and the byte strides of their per-RHS vectors;
// rhs_per_k consecutive right-hand sides share one wave number (spectrum).
template <class T> struct ArithOf;
template <> struct ArithOf<float> { static constexpr int kind = 0; };
template <> struct ArithOf<double> { static constexpr int kind = ORI_PASS_FP64; };
template <> struct ArithOf<dfl> { static constexpr int kind = ORI_PASS_DF; };

struct Mask {
  const int* flags = nullptr;   // the pass skips RHS r when flags[r * stride] != 0
  int stride = 0;               // bytes
};

static ori_status check_fault(ori_plan_s* p);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null when the driver does not provide it.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// Whether the FP32 Z pass stages its tiles by bulk copies: the pipelined
// kernel with 16-column tiles (ZPipe::TMA), given a valid tensor map.
static bool z_bulk_staged(const ori_plan_s* p) {
  const int L = p->L;
  if (!p->zmap_ok || L < 64 || L > 1024 || p->sched_z == SCHED_TILES) return false;
  return !(has_pipe_variants(L) && p->var_z == 1);
}

// The tensor map of the FP32 Z pass's input: T2f seen as [rhs][z][ky][kx]
// with dims (kx: L, ky: L, z: n, rhs: R), 8-byte elements, boxes of
// 16 x 1 x zbox x 1 (128-byte rows; zbox = min(L / 2, 256), so that the boxes
// covering z < n end within the tile's L / 2 + 1 staged rows).  Encoded when
// T2f or the batch size changes; without an encoder, an aligned base or a
// length the kernel stages by bulk copies, the kernel keeps cp.async.
static void z_tensor_map(ori_plan_s* p, SArgs& z, int nrhs) {
  const int R = std::max(1, nrhs);
  if (p->zmap_ptr != p->T2f || p->zmap_R != R) {
    p->zmap_ok = 0;
    p->zmap_ptr = p->T2f;
    p->zmap_R = R;
    const int L = p->L;
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (enc != nullptr && L >= 64 && L <= 1024 && (reinterpret_cast<uintptr_t>(p->T2f) & 15u) == 0) {
      const cuuint64_t es = sizeof(cpx<float>);
      const cuuint64_t dims[4] = {cuuint64_t(L), cuuint64_t(L), cuuint64_t(p->n), cuuint64_t(R)};
      const cuuint64_t strides[3] = {cuuint64_t(L) * es, cuuint64_t(L) * L * es, cuuint64_t(t2_elems(p)) * es};
      const int zbox = std::min(L / 2, 256);
      const cuuint32_t box[4] = {cuuint32_t(kZGroup), 1, cuuint32_t(zbox), 1};
      const cuuint32_t estr[4] = {1, 1, 1, 1};
      if (enc(&p->zmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, p->T2f, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
        p->zmap_ok = 1;
        p->zbox = zbox;
      }
    }
  }
  z.zrows = p->zmap;
  z.zrows_ok = p->zmap_ok;
  z.zbox = p->zbox;
  z.err = p->d_fault;
}

// Tensor maps of the rows the pipelined FP32 Y passes stage per tile (16
// FP32 columns = 128 bytes a row): the Y-forward input T1f, dims (kx, y, z,
// right-hand side) and box (16, ybox_f, 1, 1), ybox_f = min(L/2, 256) (a
// power of two dividing L/2: the zero-filled rows past n stay within the L/2
// staged rows); the Y-inverse input T2f, dims (kx, ky, z, right-hand side)
// and box (16, ybox_i, 1, 1), ybox_i = min(L, 256).
static void y_tensor_maps(ori_plan_s* p, SArgs& y, SArgs& yi, int nrhs) {
  const int R = std::max(1, nrhs);
  if (p->ymap_ptr != p->T1f || p->ymap_R != R) {
    p->ymap_ok = 0;
    p->ymap_ptr = p->T1f;
    p->ymap_R = R;
    const int L = p->L, n = p->n;
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (enc != nullptr && L >= 64 && L <= 1024 && ((reinterpret_cast<uintptr_t>(p->T1f) |
                                                    reinterpret_cast<uintptr_t>(p->T2f)) & 15u) == 0) {
      const cuuint64_t es = sizeof(cpx<float>);
      const int bf = std::min(L / 2, 256), bi = std::min(L, 256);
      const cuuint32_t estr[4] = {1, 1, 1, 1};
      const cuuint64_t dims_f[4] = {cuuint64_t(L), cuuint64_t(n), cuuint64_t(n), cuuint64_t(R)};
      const cuuint64_t str_f[3] = {cuuint64_t(L) * es, cuuint64_t(n) * L * es, cuuint64_t(t1_elems(p)) * es};
      const cuuint32_t box_f[4] = {cuuint32_t(kZGroup), cuuint32_t(bf), 1, 1};
      const cuuint64_t dims_i[4] = {cuuint64_t(L), cuuint64_t(L), cuuint64_t(n), cuuint64_t(R)};
      const cuuint64_t str_i[3] = {cuuint64_t(L) * es, cuuint64_t(L) * L * es, cuuint64_t(t2_elems(p)) * es};
      const cuuint32_t box_i[4] = {cuuint32_t(kZGroup), cuuint32_t(bi), 1, 1};
      if (enc(&p->ymap_f, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, p->T1f, dims_f, str_f, box_f, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS &&
          enc(&p->ymap_i, CU_TENSOR_MAP_DATA_TYPE_UINT64, 4, p->T2f, dims_i, str_i, box_i, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
        p->ymap_ok = 1;
        p->ybox_f = bf;
        p->ybox_i = bi;
      }
    }
  }
  y.zrows = p->ymap_f;
  y.zrows_ok = p->ymap_ok;
  y.zbox = p->ybox_f;
  y.err = p->d_fault;
  yi.zrows = p->ymap_i;
  yi.zrows_ok = p->ymap_ok;
  yi.zbox = p->ybox_i;
  yi.err = p->d_fault;
}

template <class T>
static ori_status run_conv(ori_plan_s* p, XArgs pro, XArgs epi, int fin, cudaStream_t s, Mask mask,
                           int nrhs = 1, int rhs_per_k = 1) {
  constexpr int K = ArithOf<T>::kind;
  NvtxRange nvtx(K == 0 ? "ori operator fp32" : (K == ORI_PASS_FP64 ? "ori operator fp64" : "ori operator df"));
  const bool f32 = K == 0;
  cpx<T>* T1 = reinterpret_cast<cpx<T>*>(f32 ? (void*)p->T1f : (void*)p->T1d);
  cpx<T>* T2 = reinterpret_cast<cpx<T>*>(f32 ? (void*)p->T2f : (void*)p->T2d);
  const void* tw = K == 0 ? (const void*)p->tw32 : (K == ORI_PASS_FP64 ? (const void*)p->tw64 : (const void*)p->twdf);
  const void* gh = K == 0 ? (const void*)p->ghat32 : (K == ORI_PASS_FP64 ? (const void*)p->ghat64 : (const void*)p->ghatdf);
  const int n = p->n, L = p->L;
  const long long H3 = (long long)p->H * p->H * p->H;
  const long long bsT1 = (long long)t1_elems(p) * sizeof(cpx<T>);
  const long long bsT2 = (long long)t2_elems(p) * sizeof(cpx<T>);
  int e0 = t_rec(p, s), e1;
  pro.n = n; pro.nlines = n * n; pro.n_in = n; pro.line_len_in = n; pro.line_len_out = L;
  pro.fft_out = T1; pro.twL = tw; pro.done = mask.flags; pro.done_stride = mask.stride;
  pro.nrhs = nrhs; pro.bs_fft = bsT1; pro.bs_beta = sizeof(Scalars); pro.sm_count = p->sm_count;
  ORI_CUDA(run_xfwd<T>(L, true, pro, s, false));
  launched(p);
  e1 = t_rec(p, s); t_pair(p, ORI_PASS_XFWD + K, e0, e1); e0 = e1;

  SArgs y{};
  y.in = T1; y.out = T2;
  y.in_outer = (long long)n * L; y.out_outer = (long long)L * L;
  y.in_pt = L; y.out_pt = L; y.ncols = L; y.n_in = n; y.n_out = L; y.nouter = n;
  y.twL = tw; y.done = mask.flags; y.done_stride = mask.stride; y.sm_count = p->sm_count;
  y.nrhs = nrhs; y.bs_in = bsT1; y.bs_out = bsT2;
  y.sched = p->sched_y; y.cta_cap = p->cta_cap; y.variant = p->var_y;
  SArgs yi{};
  if (f32) y_tensor_maps(p, y, yi, nrhs);
  ORI_CUDA(run_strided<T>(L, SMODE_FWD, true, y, s, false));
  launched(p);
  e1 = t_rec(p, s); t_pair(p, ORI_PASS_YFWD + K, e0, e1); e0 = e1;

  SArgs z{};
  z.in = T2; z.out = T2;
  z.in_outer = L; z.out_outer = L;
  z.in_pt = (long long)L * L; z.out_pt = (long long)L * L;
  z.ncols = L; z.n_in = n; z.n_out = n; z.nouter = L;
  z.twL = tw; z.ghat = gh; z.ghatZ = p->ghatZ32; z.H = p->H;
  z.done = mask.flags; z.done_stride = mask.stride; z.sm_count = p->sm_count;
  z.nrhs = nrhs; z.bs_in = bsT2; z.bs_out = bsT2;
  z.bs_ghat = H3 * (long long)sizeof(cpx<T>);
  z.bs_ghatZ = (long long)p->H * p->H * p->L * (long long)sizeof(cpx<float>);
  z.rhs_per_ghat = rhs_per_k;
  z.sched = p->sched_z; z.cta_cap = p->cta_cap; z.variant = p->var_z;
  if (f32) z_tensor_map(p, z, nrhs);
  ORI_CUDA(run_strided<T>(L, SMODE_ZCONV, true, z, s, false));
  launched(p);
  e1 = t_rec(p, s); t_pair(p, ORI_PASS_ZCONV + K, e0, e1); e0 = e1;

  yi.in = T2; yi.out = T1;
  yi.in_outer = (long long)L * L; yi.out_outer = (long long)n * L;
  yi.in_pt = L; yi.out_pt = L; yi.ncols = L; yi.n_in = L; yi.n_out = n; yi.nouter = n;
  yi.twL = tw; yi.done = mask.flags; yi.done_stride = mask.stride;
  yi.nrhs = nrhs; yi.bs_in = bsT2; yi.bs_out = bsT1;
  yi.sm_count = p->sm_count; yi.sched = p->sched_yi; yi.cta_cap = p->cta_cap; yi.variant = p->var_yi;
  ORI_CUDA(run_strided<T>(L, SMODE_INV, false, yi, s, false));
  launched(p);
  e1 = t_rec(p, s); t_pair(p, ORI_PASS_YINV + K, e0, e1); e0 = e1;

  epi.n = n; epi.nlines = n * n; epi.line_len_in = L; epi.line_len_out = n;
  epi.err = p->d_fault;
  epi.in = T1; epi.twL = tw; epi.done = mask.flags; epi.done_stride = mask.stride;
  epi.partials = p->partials; epi.nrhs = nrhs; epi.bs_fft = bsT1; epi.sm_count = p->sm_count;
  ORI_CUDA(run_xinv<T>(L, epi, p->sc, fin, s, false, nullptr));
  launched(p);
  e1 = t_rec(p, s); t_pair(p, ORI_PASS_XINV + K, e0, e1);
  if (!p->capturing) {
    if (K == 0) p->stats.fp32_matvecs += nrhs;
    if (K == 0 && z_bulk_staged(p)) p->stats.fp32_bulk_matvecs += nrhs;
    else if (K == ORI_PASS_FP64) p->stats.fp64_matvecs += nrhs;
    else p->stats.df_matvecs += nrhs;
  }
  return ORI_OK;
}

// Launch a vector kernel with accounting: ORI_VEC(p, kind, kernel<<<...>>>(...)).
#define ORI_VEC(p, kind, launch_expr)                     \
  do {                                                    \
    int ve0_ = t_rec((p), (p)->ps);                       \
    launch_expr;                                          \
    ORI_CUDA(cudaGetLastError());                         \
    launched(p);                                          \
    int ve1_ = t_rec((p), (p)->ps);                       \
    t_pair((p), (kind), ve0_, ve1_);                      \
  } while (0)

// Blocks per right-hand side of the vector kernels.
static int vgrid(const ori_plan_s* p, int nrhs) { return std::max(16, p->vec_grid / std::max(1, nrhs)); }

// Control copy on the plan's stream by k_small_copy (rows of `bytes` at the
// given pitches); dst and src are device addresses (device memory or the
// mapped address of a pinned mirror).
static ori_status small_copy(ori_plan_s* p, void* dst, const void* src, size_t bytes, int rows = 1,
                             size_t dpitch = 0, size_t spitch = 0) {
  k_small_copy<<<1, 256, 0, p->ps>>>(static_cast<const unsigned char*>(src), static_cast<unsigned char*>(dst),
                                     (long long)bytes, (long long)(spitch ? spitch : bytes),
                                     (long long)(dpitch ? dpitch : bytes), rows);
  ORI_CUDA(cudaGetLastError());
  launched(p);
  return ORI_OK;
}

// Device-to-device copy by k_copy16 (16-byte words) and k_small_copy (the
// tail); buffers not 16-byte aligned (a caller's offset view) take
// cudaMemcpyAsync.
static ori_status dev_copy(ori_plan_s* p, void* dst, const void* src, size_t bytes) {
  if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15u) != 0) {
    ORI_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, p->ps));
    return ORI_OK;
  }
  const size_t n16 = bytes / 16;
  if (n16 > 0) {
    k_copy16<<<p->vec_grid, 256, 0, p->ps>>>(static_cast<const uint4*>(src), static_cast<uint4*>(dst),
                                             (long long)n16);
    ORI_CUDA(cudaGetLastError());
    launched(p);
  }
  if (bytes % 16)
    ORI_TRY(small_copy(p, static_cast<unsigned char*>(dst) + 16 * n16, static_cast<const unsigned char*>(src) + 16 * n16,
                       bytes % 16));
  return ORI_OK;
}

template <class T>
static ori_status setup_kernels(int L, unsigned* xinv_blocks, int n, int sm_count) {
  XArgs a{};
  a.nlines = n * n;
  a.sm_count = sm_count;
  ORI_CUDA(run_xfwd<T>(L, true, a, nullptr, true));
  ORI_CUDA(run_xfwd<T>(L, false, a, nullptr, true));
  ORI_CUDA(run_xinv<T>(L, a, nullptr, FIN_NONE, nullptr, true, xinv_blocks));
  SArgs s{};
  ORI_CUDA(run_strided<T>(L, SMODE_FWD, true, s, nullptr, true));
  ORI_CUDA(run_strided<T>(L, SMODE_FWD, false, s, nullptr, true));
  ORI_CUDA(run_strided<T>(L, SMODE_INV, false, s, nullptr, true));
  ORI_CUDA(run_strided<T>(L, SMODE_ZCONV, true, s, nullptr, true));
  return ORI_OK;
}

static ori_status set_medium(ori_plan_s* p, const double* h_dev, const double* N_dev) {
  const size_t n3 = size_t(p->n3);
  const cpx<double>* h = reinterpret_cast<const cpx<double>*>(h_dev);
  // the plan's copies of h and N (a lean plan keeps none: no adjoint, no field)
  // are written by the same pass; h_dev may alias them (set_medium(p->h, p->N))
  const bool copy = !p->lean && h != p->h;
  if (!p->lean && !copy && N_dev != p->N)
    ORI_TRY(dev_copy(p, p->N, N_dev, n3 * sizeof(double)));
  ORI_CUDA(cudaMemsetAsync(p->d_count, 0, sizeof(unsigned long long), p->ps));
  ORI_VEC(p, ORI_PASS_VECTOR, (k_medium<<<p->vec_grid, 256, 0, p->ps>>>(h, N_dev, copy ? p->h : nullptr,
                                                                        copy && N_dev != p->N ? p->N : nullptr,
                                                                        p->w64, p->S64, p->w32, p->S32,
                                                                        p->Sinv, p->wdf, p->Sdf, p->n3, p->d_count)));
  ORI_TRY(small_copy(p, p->h_count_d, p->d_count, sizeof(unsigned long long)));
  ORI_CUDA(cudaStreamSynchronize(p->ps));
  p->zero_S = *p->h_count;
  if (p->lean && p->zero_S != 0)
    return fail(ORI_ERR_UNSUPPORTED, "a lean plan needs h N != 0 in every cell (no FP64 recovery of S = 0 cells)");
  return ORI_OK;
}

// Spectrum of every wave number.  The kernel cube c(x, y, z) = G(d |offset|)
// (zero at the origin and beyond offsets n - 1) is even along each axis, so
// its DFT is even too and only the octant kx, ky, kz <= L/2 (H = L/2 + 1 per
// axis) is kept.  Planes z = 0..H-1 (the others repeat them) are transformed
// along x and y in batches, keeping kx, ky < H, into an H^3 buffer; the z
// transform then reads row L - z for z > L/2 (the even extension) and keeps
// kz < H in place.  FP64 throughout; the octant is stored in FP64, FP32 and
// paired FP32 with c_S |Delta| / L^3 folded in, plus the Z-tile-ordered FP32
// copy.  Transient memory: the H^3 octant and a batch of L^2 planes.
static ori_status build_spectrum(ori_plan_s* p) {
  NvtxRange nvtx("ori plan spectrum");
  const int L = p->L, n = p->n, H = p->H;
  const long long L3 = (long long)L * L * L;
  const long long H3 = (long long)H * H * H;
  const long long HZ = (long long)H * H * L;
  const long long plane = (long long)L * L;
  const int nz = int(std::max<long long>(1, std::min<long long>(H, (1LL << 26) / plane)));   // <= 1 GiB per batch
  cpx<double>* oct = nullptr;
  cpx<double>* planes = nullptr;
  cudaError_t e = cudaMalloc(&oct, size_t(H3) * sizeof(cpx<double>));
  if (e == cudaSuccess) e = cudaMalloc(&planes, size_t(nz) * size_t(plane) * sizeof(cpx<double>));
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (oct) cudaFree(oct);
    return fail(ORI_ERR_OOM, std::string("cudaMalloc (spectrum build): ") + cudaGetErrorString(e));
  }
  ori_status st = ORI_OK;
  auto check = [&](cudaError_t err, const char* what) {
    if (err != cudaSuccess && st == ORI_OK) st = fail(ORI_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(err));
    return st == ORI_OK;
  };
  for (size_t ik = 0; ik < p->ks.size() && st == ORI_OK; ++ik) {
    for (int z0 = 0; z0 < H && st == ORI_OK; z0 += nz) {
      const int nzb = std::min(nz, H - z0);
      XArgs a{};
      a.mode = PRO_KERNEL;
      a.d = p->d;
      a.k = p->ks[ik];
      a.n = n;
      a.nlines = (long long)nzb * L;
      a.n_in = L;
      a.line_len_in = L;
      a.line_len_out = L;
      a.lines_per_plane = L;
      a.plane0 = z0;
      a.fft_out = planes;
      a.twL = p->tw64;
      a.sm_count = p->sm_count;
      if (!check(run_xfwd<double>(L, false, a, p->ps, false), "plan X pass")) break;
      SArgs y{};
      y.in = planes;
      y.out = oct + (long long)z0 * H * H;
      y.in_outer = plane; y.out_outer = (long long)H * H;
      y.in_pt = L; y.out_pt = H; y.ncols = H; y.n_in = L; y.n_out = H; y.nouter = nzb;
      y.twL = p->tw64;
      y.sm_count = p->sm_count;
      check(run_strided<double>(L, SMODE_FWD, false, y, p->ps, false), "plan Y pass");
    }
    if (st != ORI_OK) break;
    SArgs z{};
    z.in = oct; z.out = oct;
    z.in_outer = H; z.out_outer = H;
    z.in_pt = (long long)H * H; z.out_pt = (long long)H * H;
    z.ncols = H; z.n_in = L; z.n_out = H; z.nouter = H;
    z.mirror_in = 1;
    z.twL = p->tw64;
    z.sm_count = p->sm_count;
    if (!check(run_strided<double>(L, SMODE_FWD, false, z, p->ps, false), "plan Z pass")) break;
    const double scale = p->c_S * p->d * p->d * p->d / double(L3);
    k_extract_ghat<<<p->vec_grid, 256, 0, p->ps>>>(oct, p->ghat64 ? p->ghat64 + ik * H3 : nullptr, p->ghat32 + ik * H3,
                                                   p->ghatdf + ik * H3, H, H, scale);
    if (!check(cudaGetLastError(), "plan extract")) break;
    if (p->ghatZ32) {
      k_build_ghatZ<<<p->vec_grid, 256, 0, p->ps>>>(p->ghat32 + ik * H3, p->ghatZ32 + ik * HZ, L, H);
      if (!check(cudaGetLastError(), "plan Z spectrum")) break;
    }
    check(cudaStreamSynchronize(p->ps), "plan spectrum");
  }
  cudaStreamSynchronize(p->ps);
  cudaFree(planes);
  cudaFree(oct);
  return st;
}

// Saved form of a plan's spectra (ori_plan_save_spectrum): this header, then
// n_k (L/2+1)^3 complex128 entries from byte kSpecPayload on.
struct SpecHeader {
  char tag[8];          // "ORISPEC", NUL-terminated
  int32_t version;      // 1
  int32_t n, L, n_k;
  double c_S, side;
  uint64_t entries;     // n_k (L/2+1)^3
  double ks[64];
};
static constexpr size_t kSpecPayload = 576;
static_assert(sizeof(SpecHeader) <= kSpecPayload, "spectrum header");
static const char kSpecTag[8] = {'O', 'R', 'I', 'S', 'P', 'E', 'C', 0};

static size_t spectrum_bytes(const ori_plan_s* p) {
  return kSpecPayload + p->ks.size() * size_t(p->H) * p->H * p->H * sizeof(cpx<double>);
}

// Fill the plan's spectra from a saved form whose header has been checked.
static ori_status load_spectrum(ori_plan_s* p, const unsigned char* buf) {
  NvtxRange nvtx("ori plan spectrum (saved)");
  const long long H3 = (long long)p->H * p->H * p->H;
  const long long HZ = (long long)p->H * p->H * p->L;
  const cpx<double>* src = reinterpret_cast<const cpx<double>*>(buf + kSpecPayload);
  // a lean plan has no FP64 spectrum: the entries go through a bounded staging buffer
  const long long chunk = p->ghat64 ? H3 : std::min<long long>(H3, 1LL << 26);
  cpx<double>* stage = nullptr;
  if (!p->ghat64) {
    cudaError_t e = cudaMalloc(&stage, size_t(chunk) * sizeof(cpx<double>));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ORI_ERR_OOM, std::string("cudaMalloc (spectrum load): ") + cudaGetErrorString(e));
    }
  }
  ori_status st = ORI_OK;
  for (size_t ik = 0; ik < p->ks.size() && st == ORI_OK; ++ik) {
    for (long long off = 0; off < H3 && st == ORI_OK; off += chunk) {
      const long long cnt = std::min(chunk, H3 - off);
      cpx<double>* dst = p->ghat64 ? p->ghat64 + ik * H3 + off : stage;
      cudaError_t e = cudaMemcpyAsync(dst, src + ik * H3 + off, size_t(cnt) * sizeof(cpx<double>),
                                      cudaMemcpyHostToDevice, p->ps);
      if (e == cudaSuccess) {
        k_spectrum_convert<<<p->vec_grid, 256, 0, p->ps>>>(dst, cnt, p->ghat32 + ik * H3 + off, p->ghatdf + ik * H3 + off);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(p->ps);   // the staging buffer is reused
      if (e != cudaSuccess) st = fail(ORI_ERR_CUDA, std::string("spectrum load: ") + cudaGetErrorString(e));
    }
    if (st == ORI_OK && p->ghatZ32) {
      k_build_ghatZ<<<p->vec_grid, 256, 0, p->ps>>>(p->ghat32 + ik * H3, p->ghatZ32 + ik * HZ, p->L, p->H);
      cudaError_t e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaStreamSynchronize(p->ps);
      if (e != cudaSuccess) st = fail(ORI_ERR_CUDA, std::string("spectrum load: ") + cudaGetErrorString(e));
    }
  }
  if (stage) cudaFree(stage);
  return st;
}

static bool finite3(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

extern "C" {

void ori_default_plan_opts(ori_plan_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->c_S = 4.0 * kPi;
}

void ori_default_solve_opts(ori_solve_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-6;
  o->maxit = 1000;
  o->precision = ORI_MIXED;
  o->inner_tol = 1e-5;
  o->max_outer = 8;
  o->check_every = 8;
  o->alpha[2] = 1.0;
  o->use_graph = 1;
  o->residual = ORI_DF;
  o->resid_update = 1;
}

int ori_abi_version(void) { return ORI_ABI_VERSION; }

const char* ori_last_error(void) { return g_last_error.c_str(); }

const char* ori_status_string(int s) {
  switch (s) {
    case ORI_OK: return "ok";
    case ORI_ERR_INVALID_ARG: return "invalid argument";
    case ORI_ERR_CUDA: return "CUDA error";
    case ORI_ERR_OOM: return "out of device memory";
    case ORI_ERR_NOT_CONVERGED: return "not converged";
    case ORI_ERR_BREAKDOWN: return "COCG breakdown";
    case ORI_ERR_NONFINITE: return "non-finite value";
    case ORI_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

}  // extern "C"

// ori_plan and ori_plan_from_spectrum: spec == NULL builds the spectra.
static ori_status plan_create(int64_t n, double k, const ori_domain* dom, const double* h_dev, const double* N_dev,
                              const ori_plan_opts* opts, void* stream, const void* spec, size_t spec_bytes,
                              ori_plan_t* out) {
  g_last_error.clear();
  if (!out) return fail(ORI_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (n < 2 || n > 1024) return fail(ORI_ERR_INVALID_ARG, "n must be in [2, 1024]");
  if (!dom) return fail(ORI_ERR_INVALID_ARG, "dom is NULL");
  if (!std::isfinite(dom->side) || dom->side <= 0 || !finite3(dom->origin))
    return fail(ORI_ERR_INVALID_ARG, "domain side must be finite and > 0, origin finite");
  if (!h_dev || !N_dev) return fail(ORI_ERR_INVALID_ARG, "h_dev and N_dev must be non-NULL");
  ori_plan_opts o;
  ori_default_plan_opts(&o);
  if (opts) {
    o = *opts;
    if (o.c_S == 0.0) o.c_S = 4.0 * kPi;
  }
  if (!std::isfinite(o.c_S)) return fail(ORI_ERR_INVALID_ARG, "c_S must be finite");
  if (o.min_L != 0 && (o.min_L < 4 || o.min_L > 2048 || (o.min_L & (o.min_L - 1)) != 0))
    return fail(ORI_ERR_INVALID_ARG, "min_L must be 0 or a power of two in [4, 2048]");
  std::vector<double> ks;
  if (spec) {
    SpecHeader hd;
    if (spec_bytes < kSpecPayload) return fail(ORI_ERR_INVALID_ARG, "saved spectrum: buffer shorter than its header");
    std::memcpy(&hd, spec, sizeof(hd));
    if (std::memcmp(hd.tag, kSpecTag, sizeof(kSpecTag)) != 0 || hd.version != 1)
      return fail(ORI_ERR_INVALID_ARG, "saved spectrum: not a saved spectrum of this format");
    int Lw = 4;
    while (Lw < 2 * n) Lw *= 2;
    Lw = std::max(Lw, o.min_L);
    const long long H = Lw / 2 + 1;
    if (hd.n != n || hd.L != Lw)
      return fail(ORI_ERR_INVALID_ARG, "saved spectrum: n or padded length L differs from this plan's");
    if (hd.c_S != o.c_S || hd.side != dom->side)
      return fail(ORI_ERR_INVALID_ARG, "saved spectrum: c_S or the cube side differs from this plan's");
    if (hd.n_k < 1 || hd.n_k > 64 || hd.entries != uint64_t(hd.n_k) * uint64_t(H * H * H) ||
        spec_bytes < kSpecPayload + hd.entries * sizeof(cpx<double>))
      return fail(ORI_ERR_INVALID_ARG, "saved spectrum: truncated or inconsistent");
    ks.assign(hd.ks, hd.ks + hd.n_k);
  } else if (o.n_k > 0) {
    if (!o.ks) return fail(ORI_ERR_INVALID_ARG, "opts->ks is NULL while opts->n_k > 0");
    if (o.n_k > 64) return fail(ORI_ERR_INVALID_ARG, "at most 64 wave numbers per plan");
    ks.assign(o.ks, o.ks + o.n_k);
  } else {
    ks.push_back(k);
  }
  for (double kv : ks)
    if (!std::isfinite(kv) || kv <= 0) return fail(ORI_ERR_INVALID_ARG, "k must be finite and > 0");

  ori_plan_s* p = new (std::nothrow) ori_plan_s();
  if (!p) return fail(ORI_ERR_OOM, "host allocation failed");
  ori_status st = ORI_OK;
  cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
  do {
    if (cudaGetDevice(&p->device) != cudaSuccess) { st = fail(ORI_ERR_CUDA, "cudaGetDevice failed"); break; }
    p->n = int(n);
    p->L = 4;
    while (p->L < 2 * p->n) p->L *= 2;
    p->L = std::max(p->L, o.min_L);
    p->H = p->L / 2 + 1;
    p->n3 = (long long)n * n * n;
    p->ks = ks;
    p->side = dom->side;
    p->d = dom->side / double(n);
    for (int i = 0; i < 3; ++i) p->origin[i] = dom->origin[i];
    p->c_S = o.c_S;
    p->mem_cap = o.mem_cap;
    p->lean = o.lean != 0;
    cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    p->vec_grid = std::max(1, p->sm_count) * p->vec_ctas;
    if (cudaStreamCreateWithFlags(&p->ps, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->evj, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&p->ev0) != cudaSuccess || cudaEventCreate(&p->ev1) != cudaSuccess) {
      st = fail(ORI_ERR_CUDA, "stream/event creation failed");
      break;
    }
    const size_t n3 = size_t(p->n3), nk = ks.size();
    const size_t H3 = size_t(p->H) * p->H * p->H;
    const bool full = !p->lean;   // arrays of the FP64 and A-form operations, the adjoint and the field
    if ((full && ((st = alloc_n(p, &p->h, n3)) || (st = alloc_n(p, &p->N, n3)) || (st = alloc_n(p, &p->w64, n3)) ||
                  (st = alloc_n(p, &p->Sinv, n3)) || (st = alloc_n(p, &p->w32, n3)) || (st = alloc_n(p, &p->wdf, n3)) ||
                  (st = alloc_n(p, &p->ghat64, nk * H3)))) ||
        (st = alloc_n(p, &p->S64, n3)) || (st = alloc_n(p, &p->S32, n3)) || (st = alloc_n(p, &p->Sdf, n3)) ||
        (st = alloc_n(p, &p->ghat32, nk * H3)) ||
        (st = alloc_n(p, &p->ghatdf, nk * H3)) ||
        (st = alloc_n(p, &p->ghatZ32, nk * size_t(p->H) * p->H * p->L)) ||
        (st = alloc_n(p, &p->tw64, size_t(p->L))) || (st = alloc_n(p, &p->tw32, size_t(p->L))) ||
        (st = alloc_n(p, &p->twdf, size_t(p->L))) || (st = alloc_n(p, &p->d_count, 1)) ||
        (st = alloc_n(p, &p->d_fault, 1)))
      break;
    if (cudaMemset(p->d_fault, 0, sizeof(int)) != cudaSuccess || cudaMallocHost(&p->h_fault, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&p->h_count, sizeof(unsigned long long)) != cudaSuccess ||
        cudaHostGetDevicePointer(&p->h_fault_d, p->h_fault, 0) != cudaSuccess ||
        cudaHostGetDevicePointer(&p->h_count_d, p->h_count, 0) != cudaSuccess) {
      st = fail(ORI_ERR_CUDA, "fault flag");
      break;
    }
    *p->h_fault = 0;
    *p->h_count = 0;
    unsigned bx32 = 0, bx64 = 0, bxdf = 0;
    if ((st = setup_kernels<float>(p->L, &bx32, p->n, p->sm_count)) ||
        (st = setup_kernels<double>(p->L, &bx64, p->n, p->sm_count)) ||
        (st = setup_kernels<dfl>(p->L, &bxdf, p->n, p->sm_count)))
      break;
    p->xinv_blocks = std::max({bx32, bx64, bxdf});
    if ((st = enter(p, user))) break;
    {
      cpx<double>* twd = new cpx<double>[p->L];
      cpx<float>* twf = new cpx<float>[p->L];
      cpx<dfl>* twdf = new cpx<dfl>[p->L];
      host_twiddles<double>(p->L, twd);
      host_twiddles<float>(p->L, twf);
      for (int m = 0; m < p->L; ++m) {   // the stage layout of paired FP32: (re.hi, im.hi, re.lo, im.lo)
        const dfl re = df_from_double_host(twd[m].x), im = df_from_double_host(twd[m].y);
        float* f = reinterpret_cast<float*>(twdf + m);
        f[0] = re.hi;
        f[1] = im.hi;
        f[2] = re.lo;
        f[3] = im.lo;
      }
      cudaError_t e1 = cudaMemcpy(p->tw64, twd, sizeof(cpx<double>) * p->L, cudaMemcpyHostToDevice);
      cudaError_t e2 = cudaMemcpy(p->tw32, twf, sizeof(cpx<float>) * p->L, cudaMemcpyHostToDevice);
      cudaError_t e3 = cudaMemcpy(p->twdf, twdf, sizeof(cpx<dfl>) * p->L, cudaMemcpyHostToDevice);
      delete[] twd;
      delete[] twf;
      delete[] twdf;
      if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) { st = fail(ORI_ERR_CUDA, "twiddle upload failed"); break; }
    }
    if ((st = set_medium(p, h_dev, N_dev))) break;
    if ((st = spec ? load_spectrum(p, static_cast<const unsigned char*>(spec)) : build_spectrum(p))) break;
    if ((st = ensure_capacity(p, 1))) break;   // after the spectrum build: lower peak memory
    if ((st = leave(p, user))) break;
  } while (0);
  if (st != ORI_OK) {
    plan_free(p);
    return st;
  }
  *out = p;
  return ORI_OK;
}

extern "C" {

ori_status ori_plan(int64_t n, double k, const ori_domain* dom, const double* h_dev,
                    const double* N_dev, const ori_plan_opts* opts, void* stream, ori_plan_t* out) {
  return plan_create(n, k, dom, h_dev, N_dev, opts, stream, nullptr, 0, out);
}

ori_status ori_plan_from_spectrum(int64_t n, const ori_domain* dom, const double* h_dev, const double* N_dev,
                                  const ori_plan_opts* opts, const void* host_buf, size_t bytes, void* stream,
                                  ori_plan_t* out) {
  if (!host_buf) {
    g_last_error.clear();
    return fail(ORI_ERR_INVALID_ARG, "host_buf is NULL");
  }
  return plan_create(n, 1.0, dom, h_dev, N_dev, opts, stream, host_buf, bytes, out);
}

ori_status ori_plan_spectrum_bytes(ori_plan_t p, size_t* bytes) {
  g_last_error.clear();
  if (!p || !bytes) return fail(ORI_ERR_INVALID_ARG, "NULL argument");
  *bytes = spectrum_bytes(p);
  return ORI_OK;
}

ori_status ori_plan_save_spectrum(ori_plan_t p, void* host_buf, size_t bytes, void* stream) {
  g_last_error.clear();
  if (!p || !host_buf) return fail(ORI_ERR_INVALID_ARG, "NULL argument");
  if (bytes < spectrum_bytes(p)) return fail(ORI_ERR_INVALID_ARG, "host_buf is shorter than ori_plan_spectrum_bytes");
  ORI_TRY(enter(p, reinterpret_cast<cudaStream_t>(stream)));
  SpecHeader hd{};
  std::memcpy(hd.tag, kSpecTag, sizeof(kSpecTag));
  hd.version = 1;
  hd.n = p->n;
  hd.L = p->L;
  hd.n_k = int32_t(p->ks.size());
  hd.c_S = p->c_S;
  hd.side = p->side;
  const size_t H3 = size_t(p->H) * p->H * p->H;
  hd.entries = uint64_t(p->ks.size() * H3);
  for (size_t i = 0; i < p->ks.size(); ++i) hd.ks[i] = p->ks[i];
  unsigned char* out = static_cast<unsigned char*>(host_buf);
  std::memset(out, 0, kSpecPayload);
  std::memcpy(out, &hd, sizeof(hd));
  cpx<double>* dst = reinterpret_cast<cpx<double>*>(out + kSpecPayload);
  const size_t nbytes = p->ks.size() * H3 * sizeof(cpx<double>);
  if (p->ghat64) {
    ORI_CUDA(cudaMemcpyAsync(dst, p->ghat64, nbytes, cudaMemcpyDeviceToHost, p->ps));
    ORI_CUDA(cudaStreamSynchronize(p->ps));
  } else {
    // lean plan: the paired-FP32 spectrum (same 16 bytes per entry), widened in place
    ORI_CUDA(cudaMemcpyAsync(dst, p->ghatdf, nbytes, cudaMemcpyDeviceToHost, p->ps));
    ORI_CUDA(cudaStreamSynchronize(p->ps));
    for (size_t i = 0; i < p->ks.size() * H3; ++i) {
      float f[4];
      std::memcpy(f, dst + i, sizeof(f));   // re.hi, re.lo, im.hi, im.lo
      const cpx<double> v{double(f[0]) + double(f[1]), double(f[2]) + double(f[3])};
      std::memcpy(dst + i, &v, sizeof(v));
    }
  }
  ORI_TRY(leave(p, reinterpret_cast<cudaStream_t>(stream)));
  return ORI_OK;
}

ori_status ori_plan_residual_history(ori_plan_t p, int system, double* out_host, int max, int* count) {
  g_last_error.clear();
  if (!p || !count || max < 0 || (max > 0 && !out_host)) return fail(ORI_ERR_INVALID_ARG, "bad argument");
  if (system < 0 || system >= int(p->history.size()))
    return fail(ORI_ERR_INVALID_ARG, "no residual history for this system (solve with opts.history = 1)");
  const std::vector<double>& h = p->history[size_t(system)];
  *count = int(h.size());
  for (int i = 0; i < std::min(max, int(h.size())); ++i) out_host[i] = h[size_t(i)];
  return ORI_OK;
}

ori_status ori_plan_set_medium(ori_plan_t p, const double* h_dev, const double* N_dev, void* stream) {
  g_last_error.clear();
  if (!p || !h_dev || !N_dev) return fail(ORI_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
  ORI_TRY(enter(p, user));
  ORI_TRY(set_medium(p, h_dev, N_dev));
  return leave(p, user);
}

ori_status ori_plan_set_timing(ori_plan_t p, int on) {
  if (!p) return fail(ORI_ERR_INVALID_ARG, "plan is NULL");
  if (on && !p->tev) {
    p->tev = new (std::nothrow) cudaEvent_t[kEvPool];
    p->gev = new (std::nothrow) cudaEvent_t[2 * kEvPool];
    p->pend = new (std::nothrow) ori_plan_s::Pend[kEvPool];
    if (!p->tev || !p->gev || !p->pend) return fail(ORI_ERR_OOM, "host allocation failed");
    for (int i = 0; i < kEvPool; ++i) ORI_CUDA(cudaEventCreate(&p->tev[i]));
    for (int i = 0; i < 2 * kEvPool; ++i) ORI_CUDA(cudaEventCreate(&p->gev[i]));
    p->tev_n = kEvPool;
  }
  ORI_CUDA(cudaStreamSynchronize(p->ps));
  if (p->timing) t_harvest(p);
  p->timing = on != 0;
  return ORI_OK;
}

ori_status ori_plan_get_stats(ori_plan_t p, ori_plan_stats* out) {
  if (!p || !out) return fail(ORI_ERR_INVALID_ARG, "NULL argument");
  ORI_TRY(small_copy(p, p->h_fault_d, p->d_fault, sizeof(int)));
  ORI_CUDA(cudaStreamSynchronize(p->ps));
  if (p->timing) t_harvest(p);
  *out = p->stats;
  return check_fault(p);
}

ori_status ori_plan_reset_stats(ori_plan_t p) {
  if (!p) return fail(ORI_ERR_INVALID_ARG, "plan is NULL");
  ORI_CUDA(cudaStreamSynchronize(p->ps));
  if (p->timing) t_harvest(p);
  std::memset(&p->stats, 0, sizeof(p->stats));
  return ORI_OK;
}

ori_status ori_plan_destroy(ori_plan_t p) {
  plan_free(p);
  return ORI_OK;
}

ori_status ori_plan_info(ori_plan_t p, int64_t* n, int64_t* L, size_t* bytes) {
  if (!p) return fail(ORI_ERR_INVALID_ARG, "plan is NULL");
  if (n) *n = p->n;
  if (L) *L = p->L;
  if (bytes) *bytes = p->bytes;
  return ORI_OK;
}

ori_status ori_matvec(ori_plan_t p, const double* x_dev, double* y_dev, int form, int precision,
                      void* stream) {
  g_last_error.clear();
  if (!p || !x_dev || !y_dev) return fail(ORI_ERR_INVALID_ARG, "NULL argument");
  if (form != ORI_FORM_A && form != ORI_FORM_B) return fail(ORI_ERR_INVALID_ARG, "form must be ORI_FORM_A or ORI_FORM_B");
  if (precision != ORI_FP64 && precision != ORI_FP32 && precision != ORI_DF)
    return fail(ORI_ERR_INVALID_ARG, "precision must be ORI_FP64, ORI_FP32 or ORI_DF");
  if (x_dev == y_dev) return fail(ORI_ERR_INVALID_ARG, "x_dev and y_dev must not overlap");
  if (p->lean && (form == ORI_FORM_A || precision == ORI_FP64))
    return fail(ORI_ERR_UNSUPPORTED, "a lean plan applies only the B form in FP32 or paired FP32");
  cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
  ORI_TRY(enter(p, user));
  XArgs pro{}, epi{};
  pro.x = x_dev;
  epi.xin = x_dev;
  epi.out = y_dev;
  if (precision == ORI_FP64) {
    pro.mode = PRO_SCALE;
    pro.scale = form == ORI_FORM_A ? (const void*)p->w64 : (const void*)p->S64;
    epi.mode = form == ORI_FORM_A ? EPI_PLUS : EPI_PLUS_S;
    epi.scale = p->S64;
    ORI_TRY(run_conv<double>(p, pro, epi, FIN_NONE, p->ps, Mask{}));
  } else if (precision == ORI_FP32) {
    pro.mode = PRO_SCALE_D;
    pro.scale = form == ORI_FORM_A ? (const void*)p->w32 : (const void*)p->S32;
    epi.mode = form == ORI_FORM_A ? EPI_PLUS_D : EPI_PLUS_S_D;
    epi.scale = p->S32;
    ORI_TRY(run_conv<float>(p, pro, epi, FIN_NONE, p->ps, Mask{}));
  } else {
    pro.mode = PRO_SCALE_D;
    pro.scale = form == ORI_FORM_A ? (const void*)p->wdf : (const void*)p->Sdf;
    epi.mode = form == ORI_FORM_A ? EPI_PLUS_D : EPI_PLUS_S_D;
    epi.scale = p->Sdf;
    ORI_TRY(run_conv<dfl>(p, pro, epi, FIN_NONE, p->ps, Mask{}));
  }
  return leave(p, user);
}

ori_status ori_matvec32(ori_plan_t p, const float* x_dev, float* y_dev, int form, void* stream) {
  g_last_error.clear();
  if (!p || !x_dev || !y_dev) return fail(ORI_ERR_INVALID_ARG, "NULL argument");
  if (form != ORI_FORM_A && form != ORI_FORM_B) return fail(ORI_ERR_INVALID_ARG, "form must be ORI_FORM_A or ORI_FORM_B");
  if (x_dev == y_dev) return fail(ORI_ERR_INVALID_ARG, "x_dev and y_dev must not overlap");
  if (p->lean && form == ORI_FORM_A) return fail(ORI_ERR_UNSUPPORTED, "a lean plan applies only the B form");
  cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
  ORI_TRY(enter(p, user));
  XArgs pro{}, epi{};
  pro.x = x_dev;
  pro.mode = PRO_SCALE;
  pro.scale = form == ORI_FORM_A ? (const void*)p->w32 : (const void*)p->S32;
  epi.xin = x_dev;
  epi.out = y_dev;
  epi.mode = form == ORI_FORM_A ? EPI_PLUS : EPI_PLUS_S;
  epi.scale = p->S32;
  ORI_TRY(run_conv<float>(p, pro, epi, FIN_NONE, p->ps, Mask{}));
  return leave(p, user);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Solver (batched over nrhs right-hand sides; nrhs = 1 is the single solve)
// ---------------------------------------------------------------------------

template <class T>
static ori_status cocg_iteration(ori_plan_s* p, int nrhs, int rhs_per_k, cpx<T>* x, cpx<T>* r, cpx<T>* pp,
                                 cpx<T>* q, const cpx<T>* S, bool first) {
  const long long bsv = p->n3 * (long long)sizeof(cpx<T>);
  XArgs pro{}, epi{};
  pro.mode = first ? PRO_COCG_FIRST : PRO_COCG;
  pro.x = r;
  pro.p = pp;
  pro.scale = S;
  pro.beta = &p->sc->beta;
  pro.bs_x = bsv;
  pro.bs_p = bsv;
  epi.mode = EPI_COCG;
  epi.xin = pp;
  epi.out = q;
  epi.scale = S;
  epi.bs_xin = bsv;
  epi.bs_out = bsv;
  ORI_TRY(run_conv<T>(p, pro, epi, FIN_ALPHA, p->ps, Mask{&p->sc->done, int(sizeof(Scalars))}, nrhs, rhs_per_k));
  const int vg = vgrid(p, nrhs);
  ORI_VEC(p, ORI_PASS_UPDATE + (sizeof(T) == 4 ? 0 : ORI_PASS_FP64),
          (k_cocg_update<T><<<dim3(vg, nrhs), 256, 0, p->ps>>>(x, pp, r, q, p->n3, p->sc, p->partials)));
  return ORI_OK;
}

struct InnerResult {
  int iters = 0;
  int done = 0;
  double relres_recur = 0;
};

// Copy the scalar heads of all right-hand sides to the pinned mirror.
static ori_status read_heads(ori_plan_s* p, int nrhs) {
  ORI_TRY(small_copy(p, p->h_sc_d, p->sc, offsetof(Scalars, hist), nrhs, sizeof(Scalars), sizeof(Scalars)));
  ORI_TRY(small_copy(p, p->h_fault_d, p->d_fault, sizeof(int)));
  ORI_CUDA(cudaStreamSynchronize(p->ps));
  if (p->timing) t_harvest(p);
  return check_fault(p);
}

// After a synchronisation that brought d_fault to h_fault: a kernel that gave
// up waiting for a bulk copy makes the call fail (the flag is cleared).
static ori_status check_fault(ori_plan_s* p) {
  if (*p->h_fault == 0) return ORI_OK;
  *p->h_fault = 0;
  ORI_CUDA(cudaMemsetAsync(p->d_fault, 0, sizeof(int), p->ps));
  ORI_CUDA(cudaStreamSynchronize(p->ps));
  return fail(ORI_ERR_CUDA, "a bulk copy into shared memory did not complete within its time limit");
}

// COCG on B x_r = r_r for every right-hand side r of the batch (r holds the
// right-hand sides on entry, the residuals on exit; x starts at 0).  RHS r
// stops when ||r_r|| <= tols[r] ||r_r(0)|| or after maxit iterations; its
// kernels then return at once, so the batch runs until the last one stops.
template <class T>
static ori_status cocg_inner(ori_plan_s* p, int nrhs, int rhs_per_k, cpx<T>* x, cpx<T>* r, cpx<T>* pp,
                             cpx<T>* q, const cpx<T>* S, const double* tols_host, int maxit, int check_every,
                             bool use_graph, InnerResult* res, bool zero_x = true) {
  NvtxRange nvtx(sizeof(T) == 4 ? "ori cocg fp32" : "ori cocg fp64");
  double* h_tols = p->h_small;
  for (int i = 0; i < nrhs; ++i) h_tols[i] = tols_host[i];
  ORI_TRY(small_copy(p, p->d_tols, p->h_small_d, nrhs * sizeof(double)));   // h_tols is h_small
  const int vg = vgrid(p, nrhs);
  ORI_VEC(p, ORI_PASS_VECTOR + (sizeof(T) == 4 ? 0 : ORI_PASS_FP64),
          (k_cocg_init<T><<<dim3(vg, nrhs), 256, 0, p->ps>>>(r, x, p->n3, p->sc, p->partials, p->d_tols, maxit,
                                                               zero_x ? 1 : 0)));
  ORI_TRY(read_heads(p, nrhs));
  auto any_running = [&]() {
    for (int i = 0; i < nrhs; ++i)
      if (p->h_sc[i].done == DONE_RUNNING) return true;
    return false;
  };
  auto max_iter = [&]() {
    int m = 0;
    for (int i = 0; i < nrhs; ++i) m = std::max(m, p->h_sc[i].iter);
    return m;
  };
  int graph_iters_total = 0;
  if (any_running() && maxit > 0) {
    ORI_TRY(cocg_iteration<T>(p, nrhs, rhs_per_k, x, r, pp, q, S, true));
    const bool f32 = sizeof(T) == 4;
    cudaGraphExec_t& gexec = f32 ? p->graph_f : p->graph_d;
    int& glen = f32 ? p->graph_f_len : p->graph_d_len;
    int& gnr = f32 ? p->graph_f_nrhs : p->graph_d_nrhs;
    bool& gtimed = f32 ? p->graph_f_timed : p->graph_d_timed;
    unsigned long long& gkern = f32 ? p->graph_f_kernels : p->graph_d_kernels;
    ori_plan_s::Pend*& gpend = f32 ? p->gpend_f : p->gpend_d;
    int& ngpend = f32 ? p->ngpend_f : p->ngpend_d;
    if (use_graph && (gexec == nullptr || glen != check_every || gnr != nrhs || gtimed != p->timing)) {
      if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
      if (!gpend) gpend = new ori_plan_s::Pend[kEvPool];
      ngpend = 0;
      p->gpend_cur = gpend;
      p->ngpend_cur = &ngpend;
      p->gev_used = f32 ? 0 : kEvPool;
      p->gev_n = p->gev ? (f32 ? kEvPool : 2 * kEvPool) : 0;
      p->cap_launches = 0;
      cudaGraph_t g = nullptr;
      ORI_CUDA(cudaStreamBeginCapture(p->ps, cudaStreamCaptureModeThreadLocal));
      p->capturing = true;
      ori_status cs = ORI_OK;
      for (int i = 0; i < check_every && cs == ORI_OK; ++i) {
        p->cap_iter = i;
        cs = cocg_iteration<T>(p, nrhs, rhs_per_k, x, r, pp, q, S, false);
      }
      p->capturing = false;
      cudaError_t ee = cudaStreamEndCapture(p->ps, &g);
      if (cs != ORI_OK) { if (g) cudaGraphDestroy(g); return cs; }
      if (ee != cudaSuccess) return fail(ORI_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ee));
      ee = cudaGraphInstantiate(&gexec, g, 0);
      cudaGraphDestroy(g);
      if (ee != cudaSuccess) { gexec = nullptr; return fail(ORI_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ee)); }
      glen = check_every;
      gnr = nrhs;
      gtimed = p->timing;
      gkern = p->cap_launches;
    }
    int launched_iters = 1;
    bool graph_pending = false;
    int iter_before = 0;
    for (;;) {
      ORI_TRY(read_heads(p, nrhs));
      const int it_now = max_iter();
      if (graph_pending) {
        graph_iters_total += it_now - iter_before;
        if (p->timing) t_harvest_graph(p, gpend, ngpend, it_now - iter_before);
      }
      iter_before = it_now;
      graph_pending = false;
      if (!any_running() || launched_iters >= maxit) break;
      if (use_graph) {
        ORI_CUDA(cudaGraphLaunch(gexec, p->ps));
        p->stats.kernel_launches += gkern;
        graph_pending = true;
      } else {
        for (int i = 0; i < check_every; ++i) ORI_TRY(cocg_iteration<T>(p, nrhs, rhs_per_k, x, r, pp, q, S, false));
      }
      launched_iters += check_every;
    }
  }
  ORI_TRY(read_heads(p, nrhs));
  long long real_matvecs = 0;
  for (int i = 0; i < nrhs; ++i) {
    res[i].iters = p->h_sc[i].iter;
    res[i].done = p->h_sc[i].done;
    res[i].relres_recur = p->h_sc[i].rnorm2_0 > 0 ? std::sqrt(p->h_sc[i].rnorm2 / p->h_sc[i].rnorm2_0) : 0.0;
    if (use_graph && res[i].iters > 1) real_matvecs += res[i].iters - 1;   // ran inside replayed graphs
  }
  if (sizeof(T) == 4) {
    p->stats.fp32_matvecs += real_matvecs;
    if (z_bulk_staged(p)) p->stats.fp32_bulk_matvecs += real_matvecs;
  } else {
    p->stats.fp64_matvecs += real_matvecs;
  }
  (void)graph_iters_total;
  return ORI_OK;
}

// r64_r = b64_r - B w_r for the RHS whose skip flag is 0 (complex128 vectors;
// FFT passes in paired FP32 or native FP64).  Fills rn[r] = ||r64_r||.
static ori_status fp64_residual(ori_plan_s* p, int nrhs, int rhs_per_k, bool use_df, double* rn) {
  NvtxRange nvtx("ori refinement residual");
  const long long bsv = p->n3 * (long long)sizeof(cpx<double>);
  XArgs pro{}, epi{};
  pro.mode = use_df ? PRO_SCALE_D : PRO_SCALE;
  pro.x = p->w;
  pro.bs_x = bsv;
  pro.scale = use_df ? (const void*)p->Sdf : (const void*)p->S64;
  epi.mode = EPI_RESID;
  epi.xin = p->w;
  epi.bvec = p->b64;
  epi.out = p->r64;
  epi.scale = p->S64;
  epi.bs_xin = bsv;
  epi.bs_bvec = bsv;
  epi.bs_out = bsv;
  const Mask m{p->d_skip, int(sizeof(int))};
  if (use_df) ORI_TRY(run_conv<dfl>(p, pro, epi, FIN_SUM, p->ps, m, nrhs, rhs_per_k));
  else ORI_TRY(run_conv<double>(p, pro, epi, FIN_SUM, p->ps, m, nrhs, rhs_per_k));
  ORI_TRY(read_heads(p, nrhs));
  for (int i = 0; i < nrhs; ++i)
    if (!p->h_skip[i]) rn[i] = std::sqrt(p->h_sc[i].sum.x);
  return ORI_OK;
}

// Normwise relative error bounds of one operator application, used to decide
// when a refinement residual may be updated with the FP32 operator.  The FP32
// bound is the tolerance the parity tests hold the FP32 operator to (measured
// errors are a few times 1e-7); the paired-FP32 bound is the FP64 test bar.
static constexpr double kFp32OperatorRelErr = 1e-5;
static constexpr double kDfOperatorRelErr = 1e-12;

static ori_status status_of(int done) {
  switch (done) {
    case DONE_CONVERGED: return ORI_OK;
    case DONE_BREAKDOWN: return ORI_ERR_BREAKDOWN;
    case DONE_NONFINITE: return ORI_ERR_NONFINITE;
    default: return ORI_ERR_NOT_CONVERGED;
  }
}

static ori_status push_skip(ori_plan_s* p, int nrhs) {
  ORI_TRY(small_copy(p, p->d_skip, p->h_skip_d, nrhs * sizeof(int)));
  return ORI_OK;
}
static ori_status push_doubles(ori_plan_s* p, double* dst, const double* src, int count) {
  double* stage = p->h_small + 3 * p->cap;   // pinned staging beyond the tolerance slots
  for (int i = 0; i < count; ++i) stage[i] = src[i];
  ORI_TRY(small_copy(p, dst, static_cast<double*>(p->h_small_d) + 3 * p->cap, count * sizeof(double)));
  ORI_CUDA(cudaStreamSynchronize(p->ps));
  return ORI_OK;
}

// Append COCG's recursive residual after each iteration of the last inner run
// to the history of every system taking part: ||r|| / ||RHS||, where the
// inner system was scaled by 1 / scale[r] (FP64 COCG: scale 1).
static ori_status record_history(ori_plan_s* p, int nrhs, const InnerResult* ir, const double* scale,
                                 const double* bnorm, const std::vector<int>& part) {
  std::vector<double> buf(kHistMax);
  for (int i = 0; i < nrhs; ++i) {
    if (!part[i] || bnorm[i] <= 0) continue;
    const int cnt = std::min(ir[i].iters, kHistMax);
    if (cnt <= 0) continue;
    ORI_CUDA(cudaMemcpy(buf.data(), p->sc[i].hist, size_t(cnt) * sizeof(double), cudaMemcpyDeviceToHost));
    for (int t = 0; t < cnt; ++t) p->history[i].push_back(scale[i] * std::sqrt(buf[t]) / bnorm[i]);
  }
  return ORI_OK;
}

// Solve B w_r = b64_r for the batch (b64 and bnorm[r] ready); w -> p->w.
static ori_status solve_B(ori_plan_s* p, int nrhs, int rhs_per_k, const double* bnorm, const ori_solve_opts& o,
                          ori_solve_info* info, bool warm = false) {
  const long long n3 = p->n3;
  const size_t bytes64 = size_t(n3) * sizeof(cpx<double>) * nrhs;
  for (int i = 0; i < nrhs; ++i) {
    info[i] = ori_solve_info{};
  }
  const bool graph = o.use_graph != 0;
  std::vector<InnerResult> ir(nrhs);
  std::vector<double> tin(nrhs);
  // a non-finite right-hand side (NaN/Inf in rhs, h or N) is reported, not solved
  std::vector<char> bad(nrhs);
  for (int i = 0; i < nrhs; ++i) bad[i] = !std::isfinite(bnorm[i]);
  // warm start: w holds S x0; its true residual r0 = b - B w starts the solve
  std::vector<double> rn0(bnorm, bnorm + nrhs);
  if (warm) {
    for (int i = 0; i < nrhs; ++i)   // a zero right-hand side has the solution 0 whatever the guess
      if (bnorm[i] == 0.0) ORI_CUDA(cudaMemsetAsync(p->w + size_t(i) * size_t(n3), 0, size_t(n3) * sizeof(cpx<double>), p->ps));
    for (int i = 0; i < nrhs; ++i) p->h_skip[i] = bnorm[i] > 0 ? 0 : 1;
    ORI_TRY(push_skip(p, nrhs));
    const bool use_df = o.precision != ORI_FP64 && o.residual == ORI_DF;
    ORI_TRY(fp64_residual(p, nrhs, rhs_per_k, use_df, rn0.data()));
    for (int i = 0; i < nrhs; ++i) info[i].fp64_matvecs += bnorm[i] > 0 ? 1 : 0;
  }
  if (o.precision == ORI_FP64) {
    if (!warm) {
      ORI_CUDA(cudaMemsetAsync(p->w, 0, bytes64, p->ps));
      ORI_TRY(dev_copy(p, p->r64, p->b64, bytes64));
    }
    // COCG from w (0, or the warm start) to ||r|| <= tol ||b||.  The recursive
    // residual can drift from the true one b - B w; when the true residual
    // misses tol, COCG restarts from w with the true residual (at most
    // max_outer runs), so ORI_OK always means the true relres <= tol.
    std::vector<double> rn(rn0);
    std::vector<int> active(nrhs), total(nrhs, 0), last_done(nrhs, DONE_CONVERGED), runs(nrhs, 0);
    for (int i = 0; i < nrhs; ++i) active[i] = !bad[i] && bnorm[i] > 0 && rn[i] > o.tol * bnorm[i];
    for (int run = 0; run < o.max_outer; ++run) {
      bool any = false;
      int budget = o.maxit;
      for (int i = 0; i < nrhs; ++i) {
        if (!active[i]) continue;
        any = true;
        budget = std::min(budget, o.maxit - total[i]);
      }
      if (!any || budget <= 0) break;
      // tolerance 1 marks a system that takes no part in this run
      for (int i = 0; i < nrhs; ++i) tin[i] = active[i] ? std::min(1.0, o.tol * bnorm[i] / rn[i]) : 1.0;
      ORI_TRY(cocg_inner<double>(p, nrhs, rhs_per_k, p->w, p->r64, p->p64, p->q64, p->S64, tin.data(), budget,
                                 o.check_every, graph, ir.data(), false));
      if (o.history) {
        const std::vector<double> one(nrhs, 1.0);
        ORI_TRY(record_history(p, nrhs, ir.data(), one.data(), bnorm, active));
      }
      for (int i = 0; i < nrhs; ++i) p->h_skip[i] = active[i] ? 0 : 1;
      ORI_TRY(push_skip(p, nrhs));
      std::vector<double> rn_new(rn);
      ORI_TRY(fp64_residual(p, nrhs, rhs_per_k, false, rn_new.data()));   // r64 = b - B w
      for (int i = 0; i < nrhs; ++i) {
        if (!active[i]) continue;
        total[i] += ir[i].iters;
        last_done[i] = ir[i].done;
        ++runs[i];
        info[i].fp64_matvecs += 1;
        info[i].relres_recur = ir[i].relres_recur;
        const bool progress = rn_new[i] < 0.9 * rn[i];
        rn[i] = rn_new[i];
        if (rn[i] <= o.tol * bnorm[i] || ir[i].done != DONE_CONVERGED || !progress || total[i] >= o.maxit)
          active[i] = 0;
      }
    }
    for (int i = 0; i < nrhs; ++i) {
      info[i].iters = total[i];
      info[i].outer_iters = std::max(1, runs[i]);
      info[i].relres = bnorm[i] > 0 ? rn[i] / bnorm[i] : 0.0;
      info[i].relres_bound = 1e-14;
      if (bad[i] || !std::isfinite(rn[i])) info[i].status = ORI_ERR_NONFINITE;
      else if (bnorm[i] == 0 || info[i].relres <= o.tol) info[i].status = ORI_OK;
      else if (last_done[i] != DONE_CONVERGED) info[i].status = status_of(last_done[i]);
      else info[i].status = ORI_ERR_NOT_CONVERGED;
    }
    return ORI_OK;
  }
  // mixed: FP32 COCG on the normalised residual, FP64-class refinement
  if (!warm) {
    ORI_CUDA(cudaMemsetAsync(p->w, 0, bytes64, p->ps));
    ORI_TRY(dev_copy(p, p->r64, p->b64, bytes64));
  }
  std::vector<double> rn(rn0), err(nrhs, 0.0), recur(nrhs, 0.0);
  if (warm)
    for (int i = 0; i < nrhs; ++i) err[i] = (o.residual == ORI_DF ? kDfOperatorRelErr : 1e-14) * bnorm[i];
  std::vector<int> active(nrhs), last_done(nrhs, DONE_CONVERGED), total(nrhs, 0), outer(nrhs, 0);
  for (int i = 0; i < nrhs; ++i) active[i] = !bad[i] && bnorm[i] > 0 && rn[i] + err[i] > o.tol * bnorm[i];
  for (int step = 0; step < o.max_outer; ++step) {
    bool any = false;
    for (int i = 0; i < nrhs; ++i) any = any || active[i];
    if (!any) break;
    int budget = o.maxit;
    std::vector<double> inv(nrhs, 0.0);
    for (int i = 0; i < nrhs; ++i) {
      if (active[i]) budget = std::min(budget, o.maxit - total[i]);
      inv[i] = active[i] ? 1.0 / rn[i] : 0.0;
      const double want = active[i] ? 0.25 * o.tol * bnorm[i] / rn[i] : 1.0;
      tin[i] = active[i] ? std::min(0.5, std::max(o.inner_tol, want)) : 1.0;
    }
    if (budget <= 0) break;
    ORI_TRY(push_doubles(p, p->d_scl, inv.data(), nrhs));
    const int vg = vgrid(p, nrhs);
    ORI_VEC(p, ORI_PASS_VECTOR, (k_normalise_to_f32<<<dim3(vg, nrhs), 256, 0, p->ps>>>(p->r64, p->r32, n3, p->d_scl)));
    ORI_TRY(cocg_inner<float>(p, nrhs, rhs_per_k, p->x32, p->r32, p->p32, p->q32, p->S32, tin.data(), budget,
                              o.check_every, graph, ir.data()));
    if (o.history) ORI_TRY(record_history(p, nrhs, ir.data(), rn.data(), bnorm, active));
    bool nonfinite_all = true;
    std::vector<double> scl(nrhs, 0.0);
    for (int i = 0; i < nrhs; ++i) {
      if (!active[i]) continue;
      total[i] += ir[i].iters;
      last_done[i] = ir[i].done;
      recur[i] = ir[i].relres_recur;
      ++outer[i];
      if (ir[i].done == DONE_NONFINITE) active[i] = 0;
      else nonfinite_all = false;
      scl[i] = active[i] ? rn[i] : 0.0;
    }
    if (nonfinite_all) break;
    ORI_TRY(push_doubles(p, p->d_scl, scl.data(), nrhs));
    ORI_VEC(p, ORI_PASS_VECTOR, (k_accumulate<<<dim3(vg, nrhs), 256, 0, p->ps>>>(p->w, p->x32, n3, p->d_scl)));
    // residual: updated with the FP32 operator when every active RHS allows it
    bool upd = o.resid_update != 0;
    std::vector<double> upd_err(nrhs, 0.0);
    for (int i = 0; i < nrhs; ++i) {
      if (!active[i]) continue;
      upd_err[i] = kFp32OperatorRelErr * rn[i] * (1.0 + recur[i]);   // |B d| <= 1 + inner residual
      upd = upd && upd_err[i] <= 0.05 * o.tol * bnorm[i];
    }
    for (int i = 0; i < nrhs; ++i) p->h_skip[i] = active[i] ? 0 : 1;
    ORI_TRY(push_skip(p, nrhs));
    std::vector<double> rn_new(rn);
    if (upd) {
      // r -= rn B d with the FP32 operator; error <= kFp32OperatorRelErr rn |B d|
      ORI_TRY(push_doubles(p, p->d_coef, scl.data(), nrhs));
      const long long bs32 = n3 * (long long)sizeof(cpx<float>), bs64 = n3 * (long long)sizeof(cpx<double>);
      XArgs pro{}, epi{};
      pro.mode = PRO_SCALE;
      pro.x = p->x32;
      pro.bs_x = bs32;
      pro.scale = p->S32;
      epi.mode = EPI_RUPDATE;
      epi.xin = p->x32;
      epi.bs_xin = bs32;
      epi.scale = p->S32;
      epi.bvec = p->r64;
      epi.bs_bvec = bs64;
      epi.coefs = p->d_coef;
      ORI_TRY(run_conv<float>(p, pro, epi, FIN_SUM, p->ps, Mask{p->d_skip, int(sizeof(int))}, nrhs, rhs_per_k));
      ORI_TRY(read_heads(p, nrhs));
      for (int i = 0; i < nrhs; ++i) {
        if (!active[i]) continue;
        rn_new[i] = std::sqrt(p->h_sc[i].sum.x);
        err[i] += upd_err[i];
        info[i].resid_updates += 1;
      }
    } else {
      ORI_TRY(fp64_residual(p, nrhs, rhs_per_k, o.residual == ORI_DF, rn_new.data()));
      for (int i = 0; i < nrhs; ++i) {
        if (!active[i]) continue;
        info[i].fp64_matvecs += 1;
        err[i] = (o.residual == ORI_DF ? kDfOperatorRelErr : 1e-14) * bnorm[i];
      }
    }
    for (int i = 0; i < nrhs; ++i) {
      if (!active[i]) continue;
      const bool stalled = rn_new[i] > 0.9 * rn[i];
      rn[i] = rn_new[i];
      if (stalled && ir[i].done != DONE_CONVERGED) active[i] = 0;
      if (rn[i] + err[i] <= o.tol * bnorm[i]) active[i] = 0;
      if (total[i] >= o.maxit) active[i] = 0;
    }
  }
  for (int i = 0; i < nrhs; ++i) {
    info[i].iters = total[i];
    info[i].outer_iters = outer[i];
    info[i].relres = bnorm[i] > 0 ? rn[i] / bnorm[i] : 0.0;
    info[i].relres_bound = bnorm[i] > 0 ? err[i] / bnorm[i] : 0.0;
    info[i].relres_recur = recur[i];
    if (bad[i] || !std::isfinite(rn[i])) info[i].status = ORI_ERR_NONFINITE;
    else if (bnorm[i] == 0 || info[i].relres + info[i].relres_bound <= o.tol) info[i].status = ORI_OK;
    else if (last_done[i] == DONE_NONFINITE) info[i].status = ORI_ERR_NONFINITE;
    else if (last_done[i] == DONE_BREAKDOWN) info[i].status = ORI_ERR_BREAKDOWN;
    else info[i].status = ORI_ERR_NOT_CONVERGED;
  }
  return ORI_OK;
}

static ori_status check_solve_opts(const ori_solve_opts* in, ori_solve_opts* o) {
  ori_default_solve_opts(o);
  if (in) *o = *in;
  if (!std::isfinite(o->tol) || o->tol <= 0) return fail(ORI_ERR_INVALID_ARG, "tol must be finite and > 0");
  if (o->maxit < 0) return fail(ORI_ERR_INVALID_ARG, "maxit must be >= 0");
  if (o->precision != ORI_FP64 && o->precision != ORI_MIXED)
    return fail(ORI_ERR_INVALID_ARG, "precision must be ORI_FP64 or ORI_MIXED");
  if (!std::isfinite(o->inner_tol) || o->inner_tol <= 0 || o->inner_tol >= 1)
    return fail(ORI_ERR_INVALID_ARG, "inner_tol must be in (0, 1)");
  if (o->max_outer < 1) return fail(ORI_ERR_INVALID_ARG, "max_outer must be >= 1");
  if (o->check_every < 1 || o->check_every > 1024) return fail(ORI_ERR_INVALID_ARG, "check_every must be in [1, 1024]");
  if (!finite3(o->alpha)) return fail(ORI_ERR_INVALID_ARG, "alpha must be finite");
  if (o->residual != ORI_DF && o->residual != ORI_FP64)
    return fail(ORI_ERR_INVALID_ARG, "residual must be ORI_DF or ORI_FP64");
  if (o->history != 0 && o->history != 1) return fail(ORI_ERR_INVALID_ARG, "history must be 0 or 1");
  return ORI_OK;
}

// Solve A u_r = rhs_r for r = ik * ndir + id: wave number ks[ik] (ik over the
// plan's wave numbers) and direction id.  rhs_dev == NULL: plane waves.
static ori_status solve_batch(ori_plan_s* p, int nk, int ndir, const double* rhs_dev, const double* dirs_host,
                              double* u_dev, const ori_solve_opts& o, ori_solve_info* infos, cudaStream_t user) {
  NvtxRange nvtx("ori solve");
  const int nrhs = nk * ndir;
  if (p->lean && (o.precision == ORI_FP64 || o.residual == ORI_FP64))
    return fail(ORI_ERR_UNSUPPORTED, "a lean plan solves in mixed precision with the paired-FP32 residual only");
  ORI_TRY(ensure_capacity(p, nrhs));
  if (o.history) p->history.assign(size_t(nrhs), std::vector<double>());
  ORI_TRY(enter(p, user));
  ORI_CUDA(cudaEventRecord(p->ev0, p->ps));
  std::vector<double> kv(nrhs), dv(3 * nrhs);
  for (int ik = 0; ik < nk; ++ik)
    for (int id = 0; id < ndir; ++id) {
      const int r = ik * ndir + id;
      kv[r] = p->ks[ik];
      const double* a = dirs_host + 3 * id;
      const double an = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      for (int c = 0; c < 3; ++c) dv[3 * r + c] = an > 0 ? a[c] / an : (c == 2 ? 1.0 : 0.0);
    }
  ORI_TRY(push_doubles(p, p->d_kv, kv.data(), nrhs));
  ORI_TRY(push_doubles(p, p->d_dir, dv.data(), 3 * nrhs));
  const int vg = vgrid(p, nrhs);
  ORI_VEC(p, ORI_PASS_VECTOR,
          (k_phases<<<dim3(unsigned((3 * p->n + 255) / 256), nrhs), 256, 0, p->ps>>>(
              p->d_kv, p->d_dir, p->n, p->d, p->origin[0], p->origin[1], p->origin[2], p->d_phase)));
  // u0 is kept only where S = 0 cells need it for the recovery
  ORI_VEC(p, ORI_PASS_VECTOR,
          (k_rhs<<<dim3(vg, nrhs), 256, rhs_dev ? 0 : 3 * size_t(p->n) * sizeof(cpx<double>), p->ps>>>(
              reinterpret_cast<const cpx<double>*>(rhs_dev), p->S64, p->zero_S ? p->u0 : nullptr, p->b64, p->n,
              p->d_phase, p->sc, p->partials)));
  ORI_TRY(read_heads(p, nrhs));
  std::vector<double> bnorm(nrhs);
  for (int i = 0; i < nrhs; ++i) bnorm[i] = std::sqrt(p->h_sc[i].sum.x);
  if (o.x0 != nullptr)
    ORI_VEC(p, ORI_PASS_VECTOR, (k_scale_guess<<<dim3(vg, nrhs), 256, 0, p->ps>>>(
                                    reinterpret_cast<const cpx<double>*>(o.x0), p->S64, p->w, p->n3)));
  ORI_TRY(solve_B(p, nrhs, ndir, bnorm.data(), o, infos, o.x0 != nullptr));
  // u = w / S; cells with S = 0 take u = u0 - K (S w) (one more FP64 application)
  if (p->zero_S == 0) {
    ORI_VEC(p, ORI_PASS_VECTOR,
            (k_recover<<<dim3(vg, nrhs), 256, 0, p->ps>>>(p->w, p->Sinv, p->S64, reinterpret_cast<cpx<double>*>(u_dev),
                                                           p->n3)));
  } else {
    const long long bsv = p->n3 * (long long)sizeof(cpx<double>);
    XArgs pro{}, epi{};
    pro.mode = PRO_SCALE;
    pro.x = p->w;
    pro.bs_x = bsv;
    pro.scale = p->S64;
    epi.mode = EPI_RECOVER;
    epi.xin = p->w;
    epi.bvec = p->u0;
    epi.out = u_dev;
    epi.scale = p->S64;
    epi.bs_xin = bsv;
    epi.bs_bvec = bsv;
    epi.bs_out = bsv;
    ORI_TRY(run_conv<double>(p, pro, epi, FIN_NONE, p->ps, Mask{}, nrhs, ndir));
    for (int i = 0; i < nrhs; ++i) infos[i].fp64_matvecs += 1;
  }
  ORI_CUDA(cudaEventRecord(p->ev1, p->ps));
  ORI_CUDA(cudaEventSynchronize(p->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, p->ev0, p->ev1);
  if (p->timing) t_harvest(p);
  for (int i = 0; i < nrhs; ++i) infos[i].ms = ms;
  ORI_TRY(leave(p, user));
  return ORI_OK;
}

extern "C" {

ori_status ori_cocg_solve(ori_plan_t p, const double* rhs_dev, double* u_dev, const ori_solve_opts* opts,
                          ori_solve_info* info_out, void* stream) {
  g_last_error.clear();
  if (!p || !u_dev) return fail(ORI_ERR_INVALID_ARG, "NULL argument");
  ori_solve_opts o;
  ORI_TRY(check_solve_opts(opts, &o));
  ori_solve_info info{};
  ORI_TRY(solve_batch(p, 1, 1, rhs_dev, o.alpha, u_dev, o, &info, reinterpret_cast<cudaStream_t>(stream)));
  if (info_out) *info_out = info;
  if (info.status != ORI_OK)
    return fail(ori_status(info.status), std::string("solve ended with status ") + ori_status_string(info.status));
  return ORI_OK;
}

ori_status ori_cocg_solve_batch(ori_plan_t p, int ndir, const double* alphas_host, const double* rhs_dev,
                                double* u_dev, const ori_solve_opts* opts, ori_solve_info* infos,
                                void* stream) {
  g_last_error.clear();
  if (!p || !u_dev) return fail(ORI_ERR_INVALID_ARG, "NULL argument");
  if (ndir < 1) return fail(ORI_ERR_INVALID_ARG, "ndir must be >= 1");
  if (!rhs_dev && !alphas_host) return fail(ORI_ERR_INVALID_ARG, "alphas_host is NULL and rhs_dev is NULL");
  ori_solve_opts o;
  ORI_TRY(check_solve_opts(opts, &o));
  const int nk = int(p->ks.size());
  const long long nrhs = (long long)nk * ndir;
  if (nrhs > 4096) return fail(ORI_ERR_INVALID_ARG, "at most 4096 right-hand sides per batch");
  std::vector<double> dirs(3 * size_t(ndir));
  for (int id = 0; id < ndir; ++id)
    for (int c = 0; c < 3; ++c) dirs[3 * id + c] = alphas_host ? alphas_host[3 * id + c] : o.alpha[c];
  for (double v : dirs)
    if (!std::isfinite(v)) return fail(ORI_ERR_INVALID_ARG, "directions must be finite");
  std::vector<ori_solve_info> inf(static_cast<size_t>(nrhs));
  ORI_TRY(solve_batch(p, nk, ndir, rhs_dev, dirs.data(), u_dev, o, inf.data(), reinterpret_cast<cudaStream_t>(stream)));
  ori_status worst = ORI_OK;
  for (long long i = 0; i < nrhs; ++i) {
    if (infos) infos[i] = inf[i];
    if (inf[i].status != ORI_OK && worst == ORI_OK) worst = ori_status(inf[i].status);
  }
  if (worst != ORI_OK)
    return fail(worst, std::string("batched solve: some right-hand side ended with status ") + ori_status_string(worst));
  return ORI_OK;
}

ori_status ori_adjoint_solve(ori_plan_t p, const double* u_dev, const double* econj_dev, double* grad_h_dev,
                             double* grad_N_dev, const ori_solve_opts* opts, ori_solve_info* info_out,
                             void* stream) {
  g_last_error.clear();
  if (!p || !u_dev || !econj_dev || !grad_h_dev || !grad_N_dev) return fail(ORI_ERR_INVALID_ARG, "NULL argument");
  if (p->zero_S != 0) return fail(ORI_ERR_UNSUPPORTED, "the adjoint needs h N != 0 in every cell");
  if (p->lean) return fail(ORI_ERR_UNSUPPORTED, "a lean plan has no adjoint (it keeps no copy of h and N)");
  ori_solve_opts o;
  ORI_TRY(check_solve_opts(opts, &o));
  ori_solve_info info{};
  cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
  ORI_TRY(ensure_capacity(p, 1));
  if (o.history) p->history.assign(1, std::vector<double>());
  ORI_TRY(enter(p, user));
  ORI_CUDA(cudaEventRecord(p->ev0, p->ps));
  ORI_VEC(p, ORI_PASS_VECTOR,
          (k_adj_rhs<<<p->vec_grid, 256, 0, p->ps>>>(reinterpret_cast<const cpx<double>*>(econj_dev), p->S64, p->b64,
                                                      p->n3, p->sc, p->partials)));
  ORI_TRY(read_heads(p, 1));
  const double bnorm = std::sqrt(p->h_sc[0].sum.x);
  ORI_TRY(solve_B(p, 1, 1, &bnorm, o, &info));
  ORI_VEC(p, ORI_PASS_VECTOR,
          (k_gradient<<<p->vec_grid, 256, 0, p->ps>>>(reinterpret_cast<const cpx<double>*>(econj_dev), p->w,
                                                       reinterpret_cast<const cpx<double>*>(u_dev), p->S64, p->h,
                                                       p->N, reinterpret_cast<cpx<double>*>(grad_h_dev), grad_N_dev,
                                                       p->n3)));
  ORI_CUDA(cudaEventRecord(p->ev1, p->ps));
  ORI_CUDA(cudaEventSynchronize(p->ev1));
  cudaEventElapsedTime(&info.ms, p->ev0, p->ev1);
  if (p->timing) t_harvest(p);
  ORI_TRY(leave(p, user));
  if (info_out) *info_out = info;
  if (info.status != ORI_OK)
    return fail(ori_status(info.status), std::string("adjoint solve ended with status ") + ori_status_string(info.status));
  return ORI_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Launch schedules and the autotuner
// ---------------------------------------------------------------------------

static_assert(ORI_SCHED_PERSISTENT == SCHED_PERSISTENT && ORI_SCHED_TILES == SCHED_TILES,
              "schedule codes of the ABI and the kernels must agree");

static void apply_schedule(ori_plan_s* p, const ori_schedule& s) {
  p->sched_y = s.yfwd;
  p->sched_z = s.zconv;
  p->sched_yi = s.yinv;
  p->var_y = s.yfwd_variant;
  p->var_z = s.zconv_variant;
  p->var_yi = s.yinv_variant;
  p->cta_cap = s.ctas_per_sm;
  p->vec_ctas = s.vec_ctas_per_sm > 0 ? s.vec_ctas_per_sm : 8;
  p->vec_grid = std::max(1, p->sm_count) * p->vec_ctas;
  drop_graphs(p);   // captured launches carry the old grids
}

static ori_schedule current_schedule(const ori_plan_s* p) {
  ori_schedule s{};
  s.yfwd = p->sched_y;
  s.zconv = p->sched_z;
  s.yinv = p->sched_yi;
  s.yfwd_variant = p->var_y;
  s.zconv_variant = p->var_z;
  s.yinv_variant = p->var_yi;
  s.ctas_per_sm = p->cta_cap;
  s.vec_ctas_per_sm = p->vec_ctas;
  return s;
}

// Device time of `reps` FP32 operator applications y = B x over a batch of
// nrhs systems on the plan's scratch vectors (no masks), per application.
static ori_status time_fp32_operator(ori_plan_s* p, int nrhs, int reps, float* ms) {
  const long long bs32 = p->n3 * (long long)sizeof(cpx<float>);
  const int nk = int(p->ks.size());
  const int per_k = (nrhs + nk - 1) / nk;
  XArgs pro{}, epi{};
  pro.mode = PRO_SCALE;
  pro.x = p->x32;
  pro.bs_x = bs32;
  pro.scale = p->S32;
  epi.mode = EPI_PLUS_S;
  epi.xin = p->x32;
  epi.bs_xin = bs32;
  epi.out = p->q32;
  epi.bs_out = bs32;
  epi.scale = p->S32;
  ORI_TRY(run_conv<float>(p, pro, epi, FIN_NONE, p->ps, Mask{}, nrhs, per_k));   // warm-up
  ORI_CUDA(cudaEventRecord(p->ev0, p->ps));
  for (int i = 0; i < reps; ++i) ORI_TRY(run_conv<float>(p, pro, epi, FIN_NONE, p->ps, Mask{}, nrhs, per_k));
  ORI_CUDA(cudaEventRecord(p->ev1, p->ps));
  ORI_CUDA(cudaEventSynchronize(p->ev1));
  float t = 0.f;
  ORI_CUDA(cudaEventElapsedTime(&t, p->ev0, p->ev1));
  *ms = t / float(reps);
  return ORI_OK;
}

// Device time of one FP32 COCG vector update over the batch (scalars reset
// before each launch so that no system is flagged as finished).
static ori_status time_fp32_update(ori_plan_s* p, int nrhs, int reps, float* ms) {
  const int vg = vgrid(p, nrhs);
  float total = 0.f;
  for (int i = 0; i <= reps; ++i) {
    ORI_CUDA(cudaMemsetAsync(p->sc, 0, size_t(nrhs) * sizeof(Scalars), p->ps));
    ORI_CUDA(cudaEventRecord(p->ev0, p->ps));
    k_cocg_update<float><<<dim3(vg, nrhs), 256, 0, p->ps>>>(p->x32, p->p32, p->r32, p->q32, p->n3, p->sc, p->partials);
    ORI_CUDA(cudaGetLastError());
    ORI_CUDA(cudaEventRecord(p->ev1, p->ps));
    ORI_CUDA(cudaEventSynchronize(p->ev1));
    float t = 0.f;
    ORI_CUDA(cudaEventElapsedTime(&t, p->ev0, p->ev1));
    if (i > 0) total += t;   // the first launch is a warm-up
  }
  *ms = total / float(reps);
  return ORI_OK;
}

static ori_status autotune(ori_plan_s* p, int nrhs, int reps, ori_schedule* best_out, float* best_ms) {
  NvtxRange nvtx("ori autotune");
  ORI_TRY(ensure_capacity(p, nrhs));
  const size_t n3 = size_t(p->n3) * size_t(nrhs);
  for (cpx<float>* v : {p->x32, p->p32, p->r32, p->q32})
    ORI_CUDA(cudaMemsetAsync(v, 0, n3 * sizeof(cpx<float>), p->ps));
  ori_schedule best = current_schedule(p);
  float best_t = 0.f;
  // FFT pass schedules (only the FP32 passes at L >= 64 have alternatives):
  // one field at a time, keeping the best value of each before the next
  ORI_TRY(time_fp32_operator(p, nrhs, reps, &best_t));
  if (p->L >= 64 && p->L <= 1024) {   // longer transforms have one schedule
    const int nv = pipe_variants(p->L);
    // fields: 0-2 kernel choice of Y fwd, Z, Y inv; 3-5 their launch variants
    // (persistent kernels only); 6 the persistent CTA cap
    for (int field = 0; field < 7; ++field) {
      const bool var_field = field >= 3 && field < 6;
      if (var_field) {
        const int sched = field == 3 ? best.yfwd : field == 4 ? best.zconv : best.yinv;
        if (sched != SCHED_PERSISTENT || nv < 2) continue;
      }
      const int nval = field < 3 ? 1 : (var_field ? nv - 1 : 2);
      for (int vi = 0; vi < nval; ++vi) {
        ori_schedule s = best;
        int* f = field == 0 ? &s.yfwd : field == 1 ? &s.zconv : field == 2 ? &s.yinv
               : field == 3 ? &s.yfwd_variant : field == 4 ? &s.zconv_variant : field == 5 ? &s.yinv_variant
               : &s.ctas_per_sm;
        const int value = field < 3 ? SCHED_TILES : (var_field ? (vi + 1 == *f ? 0 : vi + 1) : vi + 1);
        if (value == *f) continue;
        *f = value;
        apply_schedule(p, s);
        float t = 0.f;
        ORI_TRY(time_fp32_operator(p, nrhs, reps, &t));
        if (t < best_t) {
          best_t = t;
          best = s;
        }
        apply_schedule(p, best);
      }
    }
  }
  apply_schedule(p, best);
  // vector-kernel grid
  float best_v = 0.f;
  bool first = true;
  for (int v : {4, 8, 16}) {
    ori_schedule s = best;
    s.vec_ctas_per_sm = v;
    apply_schedule(p, s);
    float t = 0.f;
    ORI_TRY(time_fp32_update(p, nrhs, reps, &t));
    if (first || t < best_v) {
      best_v = t;
      best.vec_ctas_per_sm = v;
      first = false;
    }
  }
  apply_schedule(p, best);
  ORI_CUDA(cudaMemsetAsync(p->sc, 0, size_t(nrhs) * sizeof(Scalars), p->ps));
  ORI_CUDA(cudaStreamSynchronize(p->ps));
  if (best_out) *best_out = best;
  if (best_ms) *best_ms = best_t;
  return ORI_OK;
}

extern "C" {

ori_status ori_plan_get_schedule(ori_plan_t p, ori_schedule* out) {
  if (!p || !out) return fail(ORI_ERR_INVALID_ARG, "NULL argument");
  *out = current_schedule(p);
  return ORI_OK;
}

ori_status ori_plan_set_schedule(ori_plan_t p, const ori_schedule* s) {
  g_last_error.clear();
  if (!p || !s) return fail(ORI_ERR_INVALID_ARG, "NULL argument");
  auto sched_ok = [](int v) { return v == ORI_SCHED_PERSISTENT || v == ORI_SCHED_TILES; };
  if (!sched_ok(s->yfwd) || !sched_ok(s->zconv) || !sched_ok(s->yinv))
    return fail(ORI_ERR_INVALID_ARG, "yfwd, zconv and yinv must be ORI_SCHED_PERSISTENT or ORI_SCHED_TILES");
  if (s->ctas_per_sm < 0 || s->ctas_per_sm > 64) return fail(ORI_ERR_INVALID_ARG, "ctas_per_sm must be in [0, 64]");
  if (s->vec_ctas_per_sm < 0 || s->vec_ctas_per_sm > kMaxVecCtasPerSm)
    return fail(ORI_ERR_INVALID_ARG, "vec_ctas_per_sm must be in [0, 16]");
  const int nv = pipe_variants(p->L);
  auto var_ok = [nv](int v) { return v >= 0 && v < nv; };
  if (!var_ok(s->yfwd_variant) || !var_ok(s->zconv_variant) || !var_ok(s->yinv_variant))
    return fail(ORI_ERR_INVALID_ARG, "launch variants must be in [0, " + std::to_string(nv) +
                                         ") at this padded length");
  ORI_CUDA(cudaStreamSynchronize(p->ps));
  apply_schedule(p, *s);
  return ORI_OK;
}

ori_status ori_plan_autotune(ori_plan_t p, int nrhs, int reps, ori_schedule* best, float* best_ms, void* stream) {
  g_last_error.clear();
  if (!p) return fail(ORI_ERR_INVALID_ARG, "plan is NULL");
  if (nrhs < 1 || nrhs > 4096) return fail(ORI_ERR_INVALID_ARG, "nrhs must be in [1, 4096]");
  if (reps < 1 || reps > 100) return fail(ORI_ERR_INVALID_ARG, "reps must be in [1, 100]");
  cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
  ORI_TRY(enter(p, user));
  ORI_CUDA(cudaStreamSynchronize(p->ps));
  if (p->timing) t_harvest(p);
  const bool timing = p->timing;
  const ori_plan_stats saved = p->stats;
  p->timing = false;
  const ori_status st = autotune(p, nrhs, reps, best, best_ms);
  p->timing = timing;
  p->stats = saved;
  if (st != ORI_OK) return st;
  return leave(p, user);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The field off the grid (Eq. 2.10)
// ---------------------------------------------------------------------------
extern "C" ori_status ori_field(ori_plan_t p, const double* u_dev, int64_t npts, const double* points_dev,
                                const double* alpha_host, double* out_dev, void* stream) {
  g_last_error.clear();
  if (!p || !u_dev) return fail(ORI_ERR_INVALID_ARG, "NULL argument");
  if (p->lean) return fail(ORI_ERR_UNSUPPORTED, "a lean plan has no field evaluation (it keeps no copy of h and N)");
  if (npts < 0 || npts > (int64_t(1) << 30)) return fail(ORI_ERR_INVALID_ARG, "npts must be in [0, 2^30]");
  if (npts == 0) return ORI_OK;
  if (!points_dev || !out_dev) return fail(ORI_ERR_INVALID_ARG, "points_dev and out_dev must be non-NULL");
  double a[3] = {0.0, 0.0, 1.0};
  if (alpha_host) {
    if (!finite3(alpha_host)) return fail(ORI_ERR_INVALID_ARG, "alpha must be finite");
    const double an = std::sqrt(alpha_host[0] * alpha_host[0] + alpha_host[1] * alpha_host[1] +
                                alpha_host[2] * alpha_host[2]);
    if (an > 0)
      for (int c = 0; c < 3; ++c) a[c] = alpha_host[c] / an;
  }
  cudaStream_t user = reinterpret_cast<cudaStream_t>(stream);
  ORI_TRY(ensure_capacity(p, 1));
  ORI_TRY(enter(p, user));
  const double coef = -p->c_S * p->d * p->d * p->d;
  ORI_VEC(p, ORI_PASS_VECTOR,
          (k_charges<<<p->vec_grid, 256, 0, p->ps>>>(reinterpret_cast<const cpx<double>*>(u_dev), p->h, p->N, coef,
                                                      p->p64, p->n3)));
  // slices per point: enough blocks to fill the GPU; partials in the FP64 scratch cube
  const long long cap_entries = (long long)t1_elems(p) * p->cap;
  int S = int(std::max<long long>(1, std::min<long long>(256, (4LL * p->sm_count + npts - 1) / npts)));
  S = int(std::min<long long>(S, std::max<long long>(1, p->n3 / 256)));
  const long long chunk = std::max<long long>(1, std::min<long long>(npts, cap_entries / S));
  double2* partials = reinterpret_cast<double2*>(p->T1d);
  for (long long c0 = 0; c0 < npts; c0 += chunk) {
    const int np = int(std::min<long long>(chunk, npts - c0));
    const double* pts = points_dev + 3 * c0;
    const dim3 grid(unsigned(std::min<long long>(np, 65535)), unsigned(S));
    ORI_VEC(p, ORI_PASS_VECTOR,
            (k_field_partial<<<grid, 256, 0, p->ps>>>(p->p64, pts, np, p->n, p->d, p->origin[0], p->origin[1],
                                                       p->origin[2], p->ks[0], partials)));
    ORI_VEC(p, ORI_PASS_VECTOR,
            (k_field_finish<<<unsigned((np + 255) / 256), 256, 0, p->ps>>>(
                partials, S, pts, np, p->ks[0], a[0], a[1], a[2], alpha_host ? 1 : 0,
                reinterpret_cast<cpx<double>*>(out_dev) + c0)));
  }
  return leave(p, user);
}
