/*
 * ori.h - C ABI of the GB300 solver for the reduced (RED) / original (ORI)
 * linear system of Ramm & Tran, "A fast algorithm for solving scalar wave
 * scattering problem by billions of particles".
 *
 * The system (Eq. 2.19, the sum moved to the left-hand side; Eq. 2.15 is the
 * same system with one particle per cell and N = 1):
 *
 *     u_q + c_S * sum_{p != q} G(x_q, x_p) h_p N_p |Delta_p| u_p = u0_q,
 *     G(x, y) = exp(ik|x-y|) / (4 pi |x-y|)         (Eq. 2.6a, Eq. 3.3.2)
 *     u0(x)   = exp(ik alpha . x)                    (Eq. 2.4)
 *
 * on the n^3 cells of a cube [o, o + side]^3; x_p is the centre of cell p
 * and |Delta_p| = (side/n)^3.  The matrix is never stored (Section 3): the
 * off-diagonal sum is a 3D convolution (Eq. 3.3.6-3.3.7) done with padded
 * FFTs by the convolution theorem (Eq. 3.3.8); the kernel's spectrum is
 * computed once per plan.  The system is solved with COCG (Section 1,
 * Section 3) to the relative residual ||r|| / ||RHS|| (Section 4).
 *
 * Conventions for every entry point:
 *  - Arrays are C-ordered [z][y][x] with x fastest; index p = (iz*n + iy)*n + ix.
 *  - A complex array of m entries is 2*m doubles (or floats for the *32 entry
 *    points), interleaved (re, im): the layout of C99 double complex,
 *    std::complex<double>, numpy complex128 and torch.complex128.
 *  - Pointers named *_dev are CUDA device pointers on the device that was
 *    current when the plan was made; they are owned by the caller, must stay
 *    valid until the call's work on `stream` has finished, and are only read
 *    (const) or written as documented.  Pointers named *_host are host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it; calls return once enqueued unless
 *    documented as synchronising.
 *  - Every call returns an ori_status.  Nothing is thrown across the ABI.
 *    Invalid arguments are rejected before any device work is enqueued.  A
 *    human-readable message for the last failure on the calling thread is
 *    available from ori_last_error().
 *  - A plan is not safe for concurrent use from two streams or two threads.
 */
#ifndef ORI_H_
#define ORI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORI_ABI_VERSION 6

typedef struct ori_plan_s* ori_plan_t;

typedef enum {
  ORI_OK = 0,
  ORI_ERR_INVALID_ARG = 1,   /* bad size, null pointer, non-finite scalar      */
  ORI_ERR_CUDA = 2,          /* a CUDA runtime call failed                      */
  ORI_ERR_OOM = 3,           /* device allocation failed or mem_cap exceeded    */
  ORI_ERR_NOT_CONVERGED = 4, /* maxit reached; best iterate written             */
  ORI_ERR_BREAKDOWN = 5,     /* COCG breakdown (p^T B p or r^T r vanished)      */
  ORI_ERR_NONFINITE = 6,     /* NaN/Inf met in the iteration                    */
  ORI_ERR_UNSUPPORTED = 7    /* valid request this build does not implement     */
} ori_status;

/* Arithmetic of a call. */
enum {
  ORI_FP64 = 0,   /* complex128 data, FP64 FFTs                                      */
  ORI_FP32 = 1,   /* complex64 data, FP32 FFTs (FP64 spectrum rounded once)          */
  ORI_MIXED = 2,  /* solve only: FP32 COCG inside FP64 iterative refinement          */
  ORI_DF = 3      /* paired-FP32 ("double-float", ~48-bit) arithmetic: hi + lo
                     floats with error-free sums and products; complex128 data  */
};

/* Which operator ori_matvec applies. */
enum {
  ORI_FORM_A = 0, /* y = A x = x + c_S K_G (h N |Delta| x)   (Eq. 2.19, left side)   */
  ORI_FORM_B = 1  /* y = B x = x + S c_S K_G (S x), S = diag(sqrt(h N)), principal
                     root.  B = S A S^-1 is complex symmetric; COCG runs on it.     */
};

typedef struct {
  double origin[3]; /* corner of the cube (x, y, z)                                 */
  double side;      /* edge length, > 0; cell size d = side / n                     */
} ori_domain;

typedef struct {
  double c_S;       /* surface constant |S_m| = c_S a^2 (Eq. 2.13); 0 -> 4 pi       */
  size_t mem_cap;   /* 0 = no cap; otherwise ori_plan fails with ORI_ERR_OOM when
                       its device memory would exceed this many bytes              */
  int    n_k;       /* 0: one wave number, ori_plan's k.  1..64: the plan holds one
                       spectrum per entry of ks (each finite and > 0) and ignores
                       k; ori_cocg_solve_batch solves for every one of them, the
                       other calls use ks[0]                                      */
  const double* ks; /* n_k host wave numbers (read during ori_plan only)         */
  int    min_L;     /* 0: padded length L = smallest power of two >= 2n.  Else a
                       power of two in [4, 2048]: L = max(that, min_L).  Any
                       L >= 2n - 1 gives the same operator, because offsets
                       between cells span -(n-1)..n-1 and the cyclic
                       convolution then never wraps onto a kept output; used
                       to exercise long transforms on small grids             */
  int    lean;      /* 0: full plan.  1: a plan for mixed-precision solves only, for
                       the largest grids (n = 1000 needs about 263 GB instead of
                       ~410 GB): it keeps no copy of h and N, no A-form arrays, no
                       1/S, no FP64 spectrum and no FP64 COCG vectors.  On a lean
                       plan ori_matvec supports ORI_FORM_B in ORI_FP32 / ORI_DF,
                       ori_matvec32 ORI_FORM_B, the solves ORI_MIXED with the
                       ORI_DF residual; the A form, FP64 operations, the adjoint
                       and ori_field return ORI_ERR_UNSUPPORTED, and h N must be
                       nonzero in every cell (ORI_ERR_UNSUPPORTED otherwise)  */
  int    reserved[2];
} ori_plan_opts;

typedef struct {
  double tol;          /* target ||r||/||RHS|| of the symmetrised system, def 1e-6  */
  int    maxit;        /* cap on COCG iterations summed over refinements, def 1000  */
  int    precision;    /* ORI_FP64 or ORI_MIXED (default ORI_MIXED)                  */
  double inner_tol;    /* ORI_MIXED: floor of the FP32 inner target, default 1e-5    */
  int    max_outer;    /* cap on refinement steps (ORI_FP64: on COCG runs), def 8    */
  int    check_every;  /* iterations between host reads of the convergence flag (8)  */
  double alpha[3];     /* incidence direction when rhs_dev == NULL; (0,0,0)->(0,0,1) */
  int    use_graph;    /* 1 (default): replay the check_every-iteration block as a
                          captured CUDA graph; 0: plain launches                      */
  int    residual;     /* ORI_MIXED: arithmetic of the FP64-class refinement residual
                          b - B w: ORI_DF (default; inputs and output complex128,
                          FFT passes in paired FP32) or ORI_FP64 (native FP64)      */
  int    resid_update; /* ORI_MIXED: 1 (default) lets later refinement steps update
                          the residual with an FP32 operator application when the
                          error bound allows (see ori_solve_info.resid_updates);
                          0 recomputes b - B w every step                           */
  int    history;      /* 1: record COCG's residual estimate after every iteration
                          (read with ori_plan_residual_history); 0 (default): off  */
  int    reserved[4];
  const double* x0;    /* NULL (default): start from u = 0.  Else an initial guess of u
                          on the device, n^3 complex128 per system (ori_cocg_solve_batch:
                          system r at offset r n^3).  The solve starts from w = S x0
                          with its true residual (one more FP64-class operator
                          application, counted in fp64_matvecs); a zero right-hand
                          side still gives u = 0.  Ignored by ori_adjoint_solve.   */
} ori_solve_opts;

typedef struct {
  int    iters;         /* COCG iterations, all refinement steps together            */
  int    outer_iters;   /* ORI_MIXED: refinement steps.  ORI_FP64: COCG runs (a run
                           restarts from the true residual b - B w when the
                           recursive one met tol but the true one did not)        */
  int    fp64_matvecs;  /* FP64 operator applications (residuals, recovery)          */
  double relres;        /* true residual of the symmetrised system COCG solves,
                           ||S rhs - B w|| / ||S rhs|| with u = w / S, in FP64      */
  double relres_recur;  /* last recursive residual of the inner COCG                 */
  int    status;        /* ori_status of the solve                                   */
  float  ms;            /* device time of the solve (CUDA events)                    */
  int    resid_updates; /* ORI_MIXED: refinement residuals updated as r -= |r| B d
                           with an FP32 operator application (allowed once |r| is
                           small enough that the FP32 error bound times |r| stays
                           under 5% of tol |RHS|)                                     */
  double relres_bound;  /* bound on |relres - true relres| from those updates        */
} ori_solve_info;

/* Fill *o with the defaults named above. */
void ori_default_solve_opts(ori_solve_opts* o);
void ori_default_plan_opts(ori_plan_opts* o);

/*
 * ori_plan - build the operator for one grid, wave number and medium.
 *   n        cells per axis, 2 <= n <= 1024.  The padded FFT length per axis
 *            is L = the smallest power of two >= 2n (the paper pads to 2b-2
 *            by mirroring, Section 3; any L >= 2n-1 gives the same crop), at
 *            most 2048.  L <= 1024 runs the register-tile and persistent
 *            pipelined FFT passes; at L = 2048 the FP32 passes stay pipelined
 *            (the TILES schedules of the Y and Z passes select shared-memory
 *            radix-8 kernels) and the FP64 and paired-FP32 passes run
 *            shared-memory radix-8 kernels.
 *   k        wave number, finite and > 0 (Eq. 2.1).
 *   dom      cube corner and side (Eq. 3.3.5 uses the unit cube at the origin).
 *   h_dev    n^3 complex128 impedance samples h(x_p) (Eq. 2.13), device.
 *   N_dev    n^3 float64 densities N(x_p) >= 0 (Eq. 2.17), device.
 *   opts     may be NULL (defaults).
 * The plan computes, on `stream`, the kernel cube c_S |Delta| G(d |j|) with
 * the self term set to 0 (the sum excludes p = q), its spectrum by an FP64
 * 3D FFT, stores the (L/2+1)^3 distinct entries (the cube is even along each
 * axis) in FP64 and FP32, and copies h, N, h*N and S = sqrt(h N).  Later
 * changes to h_dev / N_dev do not affect the plan (see ori_plan_set_medium).
 * The call synchronises `stream` before returning.  *out receives the plan.
 */
ori_status ori_plan(int64_t n, double k, const ori_domain* dom,
                    const double* h_dev, const double* N_dev,
                    const ori_plan_opts* opts, void* stream, ori_plan_t* out);

/*
 * Saving and reusing a plan's kernel spectra (the plan build's expensive part:
 * the FP64 FFT of the kernel cube per wave number).  The spectra depend on n,
 * the padded length L, c_S, the cell size side / n and the wave numbers, not
 * on h, N or the origin.
 *
 * ori_plan_spectrum_bytes - *bytes = size of the saved form: a 576-byte header
 *   (format tag, n, L, wave numbers, c_S, side) and n_k (L/2+1)^3 complex128
 *   spectrum entries.
 * ori_plan_save_spectrum - write the saved form into host_buf (bytes >= the
 *   size above; pageable or pinned host memory).  A lean plan writes its
 *   paired-FP32 spectrum widened to complex128 (about 48 significant bits).
 *   Synchronises `stream`.
 * ori_plan_from_spectrum - as ori_plan, but the spectra come from a saved form
 *   instead of being computed: n, L (with opts->min_L), c_S (opts->c_S) and
 *   side (dom->side) must equal the saved ones, and the wave numbers are the
 *   saved ones (k, opts->n_k and opts->ks are ignored).  A mismatch, or a
 *   buffer that is too short or not a saved spectrum, returns
 *   ORI_ERR_INVALID_ARG.  Synchronises `stream`.
 */
ori_status ori_plan_spectrum_bytes(ori_plan_t plan, size_t* bytes);
ori_status ori_plan_save_spectrum(ori_plan_t plan, void* host_buf, size_t bytes, void* stream);
ori_status ori_plan_from_spectrum(int64_t n, const ori_domain* dom, const double* h_dev,
                                  const double* N_dev, const ori_plan_opts* opts,
                                  const void* host_buf, size_t bytes, void* stream,
                                  ori_plan_t* out);

/* Replace h and N (same layout as ori_plan) without recomputing the spectrum.
 * Synchronises `stream`. */
ori_status ori_plan_set_medium(ori_plan_t plan, const double* h_dev,
                               const double* N_dev, void* stream);

/* Free the plan and its device memory (synchronises the device first). */
ori_status ori_plan_destroy(ori_plan_t plan);

/* Grid size, padded length, and bytes of device memory the plan holds. */
ori_status ori_plan_info(ori_plan_t plan, int64_t* n, int64_t* L, size_t* bytes);

/*
 * ori_matvec - y = A x or y = B x (form) for n^3 complex128 vectors.
 *   precision ORI_FP64: every pass in FP64.
 *   precision ORI_FP32: x is rounded to complex64, the passes run in FP32
 *                       with the FP32 spectrum, y is widened back.
 *   precision ORI_DF:   x is split into paired floats, the passes run in
 *                       paired-FP32 arithmetic, y is widened back.
 * x_dev and y_dev may not overlap.  Asynchronous on `stream`.
 */
ori_status ori_matvec(ori_plan_t plan, const double* x_dev, double* y_dev,
                      int form, int precision, void* stream);

/*
 * ori_matvec32 - the FP32 operator on complex64 device vectors (2*n^3 floats
 * each), B or A form.  This is the matvec the mixed solver iterates with.
 * Asynchronous on `stream`.
 */
ori_status ori_matvec32(ori_plan_t plan, const float* x_dev, float* y_dev,
                        int form, void* stream);

/*
 * ori_matvec_noalloc - y = A x, the operator of ori_matvec(ORI_FORM_A,
 * ORI_FP64), for grids of at most ORI_NOALLOC_MAX_N cells per axis, without
 * a plan and without allocating any device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate —
 * code whose device memory belongs to another framework's pool, where a raw
 * cudaMalloc is not allowed; latency-critical code that must not risk the
 * device-wide synchronisation cudaMalloc and cudaFree can cause; code under a
 * rule that forbids dynamic allocation after start-up.
 *   n, k, dom  as for ori_plan, with 2 <= n <= ORI_NOALLOC_MAX_N.
 *   c_S        surface constant (0 -> 4 pi).
 *   h_dev, N_dev, x_dev  n^3 complex128 / float64 / complex128 device inputs.
 *   y_dev      n^3 complex128 device output; its 16 n^3 bytes must not
 *              overlap those of x_dev (ORI_ERR_INVALID_ARG otherwise).
 * Every intermediate (twiddles, h N, the kernel cube and its spectrum, the FFT
 * work cubes) lives in one static device array of ORI_NOALLOC_SCRATCH_BYTES
 * bytes that each GPU loading the library holds until the process exits.
 * Every call looks up the array's device address on the current device (a
 * host-side query; a context made anew after cudaDeviceReset may move it);
 * the first call on a device, and the first after the address moved, also
 * sets kernel attributes: make those calls before any stream capture.  Each call recomputes the spectrum (cheap at these
 * sizes) and writes every scratch element it reads, so the array keeps the
 * last call's contents without harm.  All calls share the one array: calls
 * that overlap on the GPU (different streams, or threads on one device) race;
 * serialise them.  n beyond the maximum returns ORI_ERR_INVALID_ARG before
 * any device work.  Asynchronous on `stream` after the first call's set-up.
 */
#define ORI_NOALLOC_MAX_N 16
#define ORI_NOALLOC_SCRATCH_BYTES 669184
ori_status ori_matvec_noalloc(int64_t n, double k, const ori_domain* dom, double c_S,
                              const double* h_dev, const double* N_dev,
                              const double* x_dev, double* y_dev, void* stream);

/*
 * ori_cocg_solve - solve A u = rhs (Eq. 2.19).
 *   rhs_dev  n^3 complex128 right-hand side, or NULL for the plane wave
 *            u0 = exp(ik alpha . x_p) with alpha = opts->alpha (Eq. 2.4).
 *   u_dev    n^3 complex128 output (also the best iterate on failure).
 * COCG runs on the complex-symmetric B w = S rhs, and u = w / S; cells with
 * S = 0 get u = rhs - K (S w) (one more FP64 operator application).
 * ORI_FP64 runs COCG in FP64 and checks the true residual b - B w at the end;
 * if the recursive residual met tol but the true one did not, COCG restarts
 * from w (at most max_outer runs).  ORI_MIXED runs FP32 COCG with FP64
 * scalars on the normalised FP64 residual and refines w in FP64 until the
 * FP64-class residual meets tol.  Either way ORI_OK means info->relres <= tol
 * (ORI_MIXED: relres + relres_bound <= tol).  Synchronising: returns after the solve has finished; info (may
 * be NULL) is filled.  Returns ORI_ERR_NOT_CONVERGED / _BREAKDOWN /
 * _NONFINITE with the best iterate in u_dev.
 */
ori_status ori_cocg_solve(ori_plan_t plan, const double* rhs_dev, double* u_dev,
                          const ori_solve_opts* opts, ori_solve_info* info,
                          void* stream);

/*
 * ori_cocg_solve_batch - solve A(k_i) u_{i,j} = u0_{i,j} for every wave number
 * k_i of the plan (ori_plan_opts.ks; i < n_k, or the one k) and every
 * incidence direction alpha_j (j < ndir): the multi-frequency, multi-
 * direction data of the inverse problem (Section 1; Eq. 2.4 per direction).
 * Right-hand side r = i * ndir + j; all n_k * ndir systems (at most 4096) run
 * as one batch: every kernel launch covers all of them (blockIdx.y = r), the
 * FFT passes of systems that share k_i read one spectrum, and a system whose
 * COCG has converged leaves the launches at once while the others go on.
 *   ndir        directions per wave number, >= 1.
 *   alphas_host 3 * ndir doubles (x, y, z per direction; normalised here,
 *               (0,0,0) -> (0,0,1)), host memory; NULL -> opts->alpha for
 *               every j.  Ignored when rhs_dev is given.
 *   rhs_dev     NULL for plane waves, else n_k * ndir complex128 n^3 vectors,
 *               system r at offset r * n^3.
 *   u_dev       n_k * ndir complex128 n^3 outputs, system r at offset r * n^3.
 *   infos       NULL or n_k * ndir entries, filled per system (ms: the
 *               whole batch).
 * Each system is solved as by ori_cocg_solve with the same opts (the mixed
 * solver refines every system until it meets tol; a step whose residual is
 * updated with the FP32 operator does so only when every unconverged system
 * allows it).  Scratch grows with the batch and stays with the plan: per
 * system, the FFT work cubes (n^2 L + n L^2 points, in complex64 and in
 * complex128) and ten solver vectors, about 17 n^3 complex128 when L = 2n.
 * Synchronising.  Returns ORI_OK when every system met tol, else the status
 * of the first that did not (its outputs still the best iterates).
 */
ori_status ori_cocg_solve_batch(ori_plan_t plan, int ndir, const double* alphas_host,
                                const double* rhs_dev, double* u_dev,
                                const ori_solve_opts* opts, ori_solve_info* infos,
                                void* stream);

/*
 * ori_adjoint_solve - gradient of J = sum_obs |u_o - t_o|^2 with respect to
 * h and N, where u solves A(h, N) u = u0.  The paper has no gradient; this
 * follows from Eq. 2.19: with psi = A^-T conj(e) (e = u - t on observation
 * cells, 0 elsewhere) and A^T psi = conj(e):
 *     grad_h_p = -2 conj((conj(e_p) - psi_p) u_p / h_p)   (dJ/dRe h + i dJ/dIm h)
 *     grad_N_p = -2 Re((conj(e_p) - psi_p) u_p / N_p)
 * Because A^T = S B S^-1, psi = S z with B z = S^-1 conj(e): one more COCG
 * solve on the same plan.
 *   u_dev       the converged forward solution (n^3 complex128).
 *   econj_dev   conj(u - t) on observation cells, 0 elsewhere (n^3 complex128).
 *   grad_h_dev  n^3 complex128 output.  grad_N_dev: n^3 float64 output.
 * Needs h_p != 0 and N_p != 0 in every cell (else ORI_ERR_UNSUPPORTED).
 * Synchronising, like ori_cocg_solve.
 */
ori_status ori_adjoint_solve(ori_plan_t plan, const double* u_dev,
                             const double* econj_dev, double* grad_h_dev,
                             double* grad_N_dev, const ori_solve_opts* opts,
                             ori_solve_info* info, void* stream);

/*
 * Launch schedules.  The FP32 Y-forward, Z and Y-inverse passes (L >= 64) each have two
 * kernels: a persistent one that streams the next tile into shared memory
 * with cp.async while it transforms the current one, and one CTA per tile of
 * columns.  Which is faster depends on n, the batch size and the GPU; so does
 * the grid of the vector kernels, and the tile width and radix split of the
 * persistent kernels (the launch variants).  The paper relied on its FFT
 * library's planner (Section 3).  Paired-FP32 and FP64 passes have one
 * schedule each.
 */
enum { ORI_SCHED_PERSISTENT = 0, ORI_SCHED_TILES = 1 };

typedef struct {
  int yfwd;             /* FP32 Y forward pass: ORI_SCHED_PERSISTENT (default) or
                           ORI_SCHED_TILES                                         */
  int zconv;            /* FP32 Z pass (forward FFT, spectrum product, inverse)   */
  int ctas_per_sm;      /* persistent kernels: resident CTAs per SM to launch,
                           0 (default) = as many as fit, else at most this many    */
  int vec_ctas_per_sm;  /* vector kernels (updates, norms): CTAs per SM, 1..16;
                           0 -> 8 (default)                                        */
  int yinv;             /* FP32 Y inverse pass                                     */
  int yfwd_variant;     /* persistent FP32 Y-forward, Z and Y-inverse kernels at padded
                           lengths L = 256 .. 1024 (ori_plan_info): 0 (default) tiles
                           of 16 columns with the transform split L = L1 * L2,
                           L1 = 2^ceil(log2(L) / 2); 1: tiles of 8 columns;
                           2: 16 columns, split (2 L1) * (L2 / 2).  Other lengths
                           have variant 0 only                                     */
  int zconv_variant;
  int yinv_variant;
} ori_schedule;

/* The plan's current schedule. */
ori_status ori_plan_get_schedule(ori_plan_t plan, ori_schedule* out);

/* Use schedule *s from now on (drops the plan's captured graphs).  Out-of-range
 * fields return ORI_ERR_INVALID_ARG.  Synchronises the plan's stream. */
ori_status ori_plan_set_schedule(ori_plan_t plan, const ori_schedule* s);

/*
 * ori_plan_autotune - time the candidate schedules on this plan for a batch of
 * nrhs systems (1..4096) and keep the fastest.  Starting from the plan's
 * schedule, each field in turn (Y-forward, Z and Y-inverse kernels, their
 * launch variants 1 and 2 where the length has them and the kernel is the
 * persistent one, then the persistent CTA cap 1 or 2) takes the alternative
 * that lowers the time of
 * `reps` (1..100) FP32 operator applications y = B x on the plan's scratch
 * vectors (each timing after one warm-up); then the vector grid (4, 8 or 16
 * CTAs per SM) is timed on the FP32 COCG update.  Grows the plan's batch scratch to nrhs like
 * ori_cocg_solve_batch; overwrites the scratch vectors (not the medium or
 * spectra); leaves ori_plan_stats unchanged.  *best (may be NULL) receives the
 * chosen schedule, *best_ms (may be NULL) its operator time for the whole
 * batch in milliseconds.  Synchronising.  A cache of results keyed by GPU,
 * n, nrhs and arithmetic belongs to the caller (the Python binding keeps one
 * as JSON).
 */
ori_status ori_plan_autotune(ori_plan_t plan, int nrhs, int reps, ori_schedule* best,
                             float* best_ms, void* stream);

/*
 * ori_field - the field away from the grid points, Eq. 2.10:
 *     out_i = [exp(ik alpha.x_i)] + sum_m G(x_i, x_m) Q_m,
 *     Q_m   = -c_S h_m N_m |Delta| u_m            (Eq. 2.13 summed over cell m:
 *             the particles of a cell carry a^(2-kappa) #(Delta_m) = N_m |Delta|)
 * for a solution u of the plan's system (its first wave number), by direct
 * summation in FP64: O(npts n^3) work.
 *   u_dev       n^3 complex128 solution (device).
 *   npts        number of points, 0 .. 2^30 (0: nothing to do).
 *   points_dev  3*npts doubles (x, y, z of each point), device.
 *   alpha_host  incidence direction (normalised here; (0,0,0) -> (0,0,1)) to add
 *               the incident wave, or NULL for the scattered part alone.
 *   out_dev     npts complex128, device.
 * A point within 1e-9 d of a cell point leaves that cell out, so at the cell
 * points the value is the effective field of Eq. 2.14, which a converged
 * solution equals.  Overwrites the plan's solver scratch (not the medium or
 * the spectra).  Asynchronous on `stream`.
 */
ori_status ori_field(ori_plan_t plan, const double* u_dev, int64_t npts, const double* points_dev,
                     const double* alpha_host, double* out_dev, void* stream);

/* Device-time accounting of a plan's kernels (for profiling and benchmarks). */
enum {
  ORI_PASS_XFWD = 0,   /* X forward FFT pass with its prologue                  */
  ORI_PASS_YFWD = 1,   /* Y forward FFT pass                                    */
  ORI_PASS_ZCONV = 2,  /* Z forward FFT, spectrum multiply, Z inverse FFT       */
  ORI_PASS_YINV = 3,   /* Y inverse FFT pass                                    */
  ORI_PASS_XINV = 4,   /* X inverse FFT pass with its epilogue and reduction    */
  ORI_PASS_UPDATE = 5, /* COCG vector update and reductions                     */
  ORI_PASS_VECTOR = 6, /* other elementwise / reduction kernels of a solve      */
  ORI_PASS_FP64 = 8,   /* added to the kind for launches in FP64 arithmetic     */
  ORI_PASS_DF = 16,    /* added to the kind for launches in paired-FP32 math    */
  ORI_PASS_KINDS = 24
};

typedef struct {
  uint64_t kernel_launches;        /* kernels this plan launched (graph nodes
                                      counted at each replay) since the reset */
  double   pass_ms[ORI_PASS_KINDS];   /* summed device time per kind (FP32 kinds
                                         0..6, FP64 8..14, paired FP32 16..22)  */
  uint64_t pass_count[ORI_PASS_KINDS];/* launches timed per kind               */
  uint64_t fp32_matvecs;           /* FP32 operator applications            */
  uint64_t fp64_matvecs;           /* FP64 operator applications            */
  uint64_t df_matvecs;             /* paired-FP32 operator applications     */
  uint64_t fp32_bulk_matvecs;      /* FP32 applications whose Z pass staged its
                                      tiles by bulk copies (TMA)            */
} ori_plan_stats;

/* Turn per-kernel CUDA-event timing on (1) or off (0).  With timing on, every
 * launch of the plan is bracketed by events on the plan's stream (inside
 * captured graphs too); times are summed into ori_plan_stats.pass_ms at the
 * solver's synchronisation points, and at ori_plan_get_stats.  Timing adds
 * an event record between kernels; leave it off outside measurements. */
ori_status ori_plan_set_timing(ori_plan_t plan, int on);
/* Copy the counters (synchronises the plan's stream).  Returns ORI_ERR_CUDA
 * (counters still copied) when a kernel gave up waiting for a bulk copy since
 * the last check; solver calls check the same at their synchronisation points. */
ori_status ori_plan_get_stats(ori_plan_t plan, ori_plan_stats* out);
/* Zero the counters. */
ori_status ori_plan_reset_stats(ori_plan_t plan);

/*
 * ori_plan_residual_history - the residual estimates of the last solve that ran
 * with opts->history = 1: for system `system` of that solve (0 for
 * ori_cocg_solve), COCG's recursive residual ||r|| / ||RHS|| after every
 * iteration, the refinement steps of a mixed solve one after another (the
 * first 512 iterations of each step).  Copies min(count, max) values to
 * out_host (may be NULL when max = 0); *count receives the number recorded.
 */
ori_status ori_plan_residual_history(ori_plan_t plan, int system, double* out_host, int max,
                                     int* count);

/* Static description of a status code. */
const char* ori_status_string(int status);
/* Message of the last failure on the calling thread ("" if none). */
const char* ori_last_error(void);
/* ORI_ABI_VERSION of the loaded library. */
int ori_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ORI_H_ */
