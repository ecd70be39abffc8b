/*
 * ls.h -- C ABI of the GB300 Lippmann-Schwinger Nystrom library (2-D).
 *
 * The library applies and solves the discretised Lippmann-Schwinger operator
 *
 *     (A u)(x) = u(x) + kappa^2 int G_kappa(x, y) m(y) u(y) dy,   m = 1 - n^2,
 *     G_kappa(x, y) = (i/4) H_0^(1)(kappa |x - y|)                  (2-D)
 *
 * (arXiv:1509.05063, Eq. Lippmann and Eq. G, Section 1) on a Nystrom grid made
 * of one periodic boundary chart ("collar") and one Cartesian interior patch
 * blended by a partition of unity (Section 2), with the localised singular
 * quadratures of Section 3.1 and the equivalent-source / lattice-FFT
 * acceleration of Section 3.2.  All compute runs in hand-written CUDA kernels
 * for sm_103a; plan construction runs on the host (C++) and on the device.
 *
 * Conventions
 *  - Complex vectors are interleaved (re, im): complex128 (double2) for
 *    LS_FP64 entry points, complex64 (float2) where a call says so.
 *  - Node order is the plan's order (nodes grouped by accelerator cell); see
 *    ls_plan_nodes for coordinates and canonical ids.  Several right-hand
 *    sides are stored one after another (column-major over RHS): rhs r of a
 *    vector occupies elements [r N, (r+1) N).
 *  - The caller owns every buffer it passes; the plan owns the device memory it
 *    allocates (weights, matrices, spectra, work space) until ls_plan_destroy.
 *  - Calls never exit or abort.  Every entry point returns an ls_status; the
 *    message of the last failure of a plan is available from ls_last_error.
 *  - Device entry points are asynchronous with respect to the host unless
 *    stated; they run on the given CUDA stream (cudaStream_t passed as void*,
 *    NULL = legacy default stream).  A plan is not re-entrant: calls on one
 *    plan must not overlap (they share the plan's work space).
 */
#ifndef LS_GB300_H
#define LS_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LS_OK = 0,
  LS_ERR_INVALID = 1,      /* bad argument or unsupported geometry/options     */
  LS_ERR_NOMEM = 2,        /* host or device allocation failed                 */
  LS_ERR_CUDA = 3,         /* a CUDA call or kernel launch failed              */
  LS_ERR_NOCONV = 4,       /* GMRES / refinement did not reach the tolerance   */
  LS_ERR_TIMEOUT = 5,      /* a bounded device wait gave up                    */
  LS_ERR_UNSUPPORTED = 6   /* entry point not available for this plan           */
} ls_status;

/* LS_FP64: complex128 throughout.  LS_MIXED: complex64 apply inside FP64
 * iterative refinement (Arnoldi vectors of the correction solves in FP64).
 * LS_MIXED32 (ls_solve and ls_batch_solve only): as LS_MIXED with the
 * correction solves' Arnoldi vectors in complex64 too -- faster where the
 * Arnoldi step costs as much as the apply (many right-hand sides in lock-step),
 * slower to converge on problems whose correction solves stagnate. */
typedef enum { LS_FP64 = 0, LS_MIXED = 1, LS_MIXED32 = 2 } ls_precision;

typedef enum { LS_DISC = 0, LS_KITE = 1, LS_FOURIER_STAR = 2 } ls_shape;

typedef struct ls_plan_s* ls_plan;

/* Scatterer and Nystrom grid (Section 2).  The boundary curve is
 *   disc : gamma(s) = (cx, cy) + a (cos s, sin s),              params = {a, cx, cy}
 *   kite : gamma(s) = (cx, cy) + c (cos s + 0.65 cos 2s - 0.65, 1.5 sin s), params = {c, cx, cy}
 *   star : gamma(s) = (cx, cy) + r(s) (cos s, sin s), r(s) = a0 + sum_{k=1..5} c_k cos(k s),
 *          params = {a0, cx, cy, c1, c2, c3, c4, c5}; r must stay positive (LS_ERR_INVALID
 *          otherwise) and collar_w below the smallest radius of curvature of the convex parts
 * The collar chart is X(a, b) = gamma(2 pi a / n1) - (b / (n2 - 1)) collar_w nu(s),
 * 0 <= a < n1 (periodic), 0 <= b <= n2 - 1, nu the outward normal; the interior
 * chart is the Cartesian grid (cart_x0 + i h, cart_y0 + j h), 0 <= i < cart_nx,
 * 0 <= j < cart_ny, of which the points with omega_I > 0 are nodes.  The
 * partition of unity is omega_B = S((t - tau0) / (tau1 - tau0)) with S the
 * C-infinity step 1 -> 0 and t = b / (n2 - 1) (the collar coordinate of a point),
 * omega_I = 1 - omega_B. */
typedef struct {
  int dim;               /* must be 2                                           */
  int shape;             /* ls_shape                                            */
  double params[8];      /* shape parameters, see above                         */
  double collar_w;       /* collar width along the inward normal                */
  int n1, n2;            /* collar grid: tangential (periodic) x transverse      */
  double tau0, tau1;     /* partition-of-unity transition, 0 < tau0 < tau1 < 1   */
  double h;              /* Cartesian spacing                                   */
  double cart_x0, cart_y0;
  int cart_nx, cart_ny;
} ls_geometry;

/* Quadrature (Section 3.1) and accelerator (Section 3.2) parameters.  Radii
 * are in grid-index units.  The accelerator uses L x L cells of side H whose
 * lower-left corner is (box_x0, box_y0) (L <= 0: the plan chooses the box to
 * cover all nodes, faces half a Cartesian spacing off the grid lines, and
 * ignores box_x0 / box_y0), N_eq lattice intervals per cell side,
 * a Fourier-Bessel local expansion of order n_fb and n_coll collocation points
 * (0 = 16 (N_eq + 1)).  eta must vanish outside the 3 x 3 cell block of every
 * target (checked; LS_ERR_INVALID otherwise). */
typedef struct {
  int Q;                 /* Newton-Cotes points across the collar (2..5)        */
  int p;                 /* Lagrange interpolation degree                       */
  double R_a, R_b;       /* collar cut-off semi-axes (along / across)           */
  double R_cart;         /* Cartesian cut-off radius                            */
  int M;                 /* varrho(tau) = R_a tau^(M+1)                         */
  int N_tau;             /* trapezoid points of the tau rule                    */
  int q_polar;           /* polar rule radial map rho = s^q                     */
  int n_rho, n_theta;    /* polar rule points                                   */
  double chi_s0;         /* cut-off plateau: chi = 1 on [0, chi_s0]             */
  double box_x0, box_y0, H;
  int L, N_eq, n_fb, n_coll;
  double rcond;          /* SVD truncation of the FP64 fits (0 = 1e-13)          */
  double rcond_mixed;    /* SVD truncation of the complex64 fits (0 = 1e-7)     */
  int n_threads;         /* host threads for plan construction (0 = all)        */
} ls_options;

/* n^2 at n points xy[2 i], xy[2 i + 1] -> n2[i]; called on the host during
 * ls_plan_create only.  Returns 0 on success. */
typedef int (*ls_n2_fn)(int64_t n, const double* xy, double* n2, void* ctx);

typedef struct {
  int64_t N;             /* Nystrom nodes                                       */
  int64_t n_collar, n_cart;
  int64_t nnz_near;      /* stored near-field weights                           */
  int L, N_eq, n_es, n_loc, n_fb, fft_M;
  int n_cells_occupied;
  double plan_seconds;   /* host wall time of ls_plan_create                    */
  int64_t device_bytes;  /* device memory held by the plan                      */
  double stage_seconds[4]; /* of plan_seconds: nodes and weights, near-field
                            * weights (singular rules, adjacent part),
                            * accelerator fits and tables, device setup
                            * (uploads, device-built spectra and tiles)       */
} ls_plan_info_t;

typedef struct {
  int iterations;        /* total GMRES iterations (inner ones for LS_MIXED)     */
  int refinements;       /* outer FP64 refinement steps (LS_MIXED)               */
  double residual;       /* final ||b - A x|| / ||b|| (FP64 operator), max over RHS */
  double seconds;        /* wall time of the call                               */
} ls_solve_info;

/* Build a plan: nodes, weights, near-field matrix (singular and regular
 * adjacent quadrature), equivalent-source projections, local expansions and
 * the kernel spectra; uploads them to the current CUDA device.  Host-blocking.
 * Section 2 (charts, POU, nodes), Section 3.1 (singular rules), Section 3.2
 * (acceleration).  Errors: LS_ERR_INVALID (bad geometry/options, eta support
 * outside the 3 x 3 block, nodes outside the box), LS_ERR_NOMEM, LS_ERR_CUDA.
 * On failure *out is NULL; the message is in ls_last_error(NULL). */
ls_status ls_plan_create(const ls_geometry* geom, ls_n2_fn n2, void* ctx, double kappa,
                         const ls_options* opt, ls_plan* out);

ls_status ls_plan_info(ls_plan plan, ls_plan_info_t* info);

/* Cheap check of a cell layout without building the plan (used by the
 * autotuner): builds the nodes, checks the lattice size and kappa H, and that
 * every node's cut-off support lies in its 3 x 3 cell block (Section 3, the
 * condition supp eta in N(x)).  out (7 doubles): N, occupied cells, near-field
 * block entries streamed per apply, lattice FFT size M, L, box_x0, box_y0.
 * LS_ERR_INVALID with the reason in ls_last_error(NULL) when the layout is
 * not usable. */
ls_status ls_check_cells(const ls_geometry* geom, ls_n2_fn n2, void* ctx, double kappa,
                         const ls_options* opt, double* out);

/* Node coordinates (host array of 2 N doubles, x then y per node) and the
 * canonical id of every node (host array of N int64, may be NULL): collar node
 * (i, j) -> i n2 + j; Cartesian nodes follow in increasing (ix cart_ny + iy)
 * order of the kept grid points. */
ls_status ls_plan_nodes(ls_plan plan, double* xy_host, int64_t* canon_host);

/* Au = A u for nrhs right-hand sides (Eq. Lippmann; Eq. VolInt-Adj-NonAdj).
 * LS_FP64: u, Au complex128; LS_MIXED: u, Au complex64 (the accelerated apply
 * in complex FP32 with FP32 near-field weights).  u and Au must not overlap.
 * Device pointers, async on stream. */
ls_status ls_apply(ls_plan plan, const void* u_dev, void* Au_dev, int nrhs,
                   ls_precision prec, void* stream);

/* Solve A u = uinc by GMRES (Section 2, matrix-free, complex arithmetic).
 * uinc, u: complex128 device arrays (u: initial guess in, solution out).
 * LS_FP64: restarted GMRES with the FP64 apply.  LS_MIXED: FP64 iterative
 * refinement r = uinc - A_64 u whose correction equations are solved by GMRES
 * with the complex64 apply (Arnoldi vectors in FP64; LS_MIXED32: in complex64).
 * Stops when ||uinc - A u|| / ||uinc|| <= tol for every RHS (the FP64 residual
 * whatever the precision).  Right-hand sides are solved in lock-step batches
 * (4 for LS_FP64, 16 for the mixed precisions); a right-hand side of
 * a later batch whose initial guess is zero starts from the least-squares
 * combination of the earlier batches' solutions.  Synchronises the stream.
 * Errors: LS_ERR_NOCONV if max_iter is reached (u holds the last iterate). */
ls_status ls_solve(ls_plan plan, const void* uinc_dev, void* u_dev, int nrhs, double tol,
                   int max_iter, int restart, ls_precision prec, ls_solve_info* info,
                   void* stream);

/* Far-field pattern A(x_hat_j) = e^{i pi/4} / sqrt(8 pi kappa) kappa^2
 *   sum_l w_l omega_l (n^2_l - 1) u_l exp(-i kappa x_hat_j . y_l)
 * for ndir unit directions (dirs_host: 2 ndir doubles) and nrhs complex128
 * fields u_dev; A_dev receives ndir x nrhs complex128 (direction fastest).
 * Not in the paper (it reports near fields); standard asymptotics of Eq. G. */
ls_status ls_farfield(ls_plan plan, const void* u_dev, int nrhs, const double* dirs_host,
                      int ndir, void* A_dev, void* stream);

ls_status ls_plan_destroy(ls_plan plan);

/* ---- multi-instance batches -------------------------------------------------
 * Many scatterers of different shape, size and kappa, each with its own plan,
 * applied and solved together: the paper solves one scatterer at a time with
 * GMRES (Section 2) and the accelerated apply (Section 3); a batch runs that
 * apply for every instance in one launch sequence and that GMRES for every
 * instance in lock-step.
 * A batch refers to its plans and does not own them: destroy the batch before
 * them, and do not use its plans on another stream while a batch call runs
 * (they share the plans' work arrays).  All plans must live on the current
 * device.  Vectors of a batch are the instances' node vectors (ls_plan_nodes
 * order) concatenated in plan order; instance i starts at element off[i]
 * (ls_batch_offsets).  ls_batch_apply runs the projection, the local expansion
 * and the near-field correction of all instances as ONE kernel each, walking
 * (instance, projection piece / cell / row block) work lists, and the lattice
 * convolution per instance; each instance sums exactly as ls_apply does for it
 * alone; repeated calls with the same buffers replay a CUDA graph.
 * Errors: LS_ERR_INVALID for null or empty arguments or a plan listed twice
 * (its instances would share the plan's work arrays), LS_ERR_NOMEM / LS_ERR_CUDA
 * from allocation or upload; the message is in ls_batch_last_error (or, for a
 * failed ls_batch_create, ls_batch_last_error(NULL)). */
typedef struct ls_batch_s* ls_batch;
ls_status ls_batch_create(const ls_plan* plans, int n_plans, ls_batch* out);
/* off_host receives n_plans + 1 int64 offsets; the last is the total length. */
ls_status ls_batch_offsets(ls_batch b, int64_t* off_host);
/* Au = A_i u_i for every instance (one right-hand side each).  LS_FP64:
 * complex128, LS_MIXED: complex64; device pointers, async on stream; u and Au
 * must not overlap. */
ls_status ls_batch_apply(ls_batch b, const void* u_dev, void* Au_dev, ls_precision prec, void* stream);
/* Solve A_i u_i = uinc_i for all instances as ls_solve does for one plan
 * (FP64 GMRES, or FP64 refinement around complex64 GMRES), one batched apply
 * per iteration.  uinc, u: complex128 concatenated vectors (u: initial guess
 * in, solution out).  info: totals (iterations summed over instances, residual
 * = the largest); per: n_plans entries (iterations and final residual of each
 * instance) or NULL.  Synchronises the stream.  LS_ERR_NOCONV if max_iter is
 * reached before every instance meets tol. */
ls_status ls_batch_solve(ls_batch b, const void* uinc_dev, void* u_dev, double tol, int max_iter, int restart,
                         ls_precision prec, ls_solve_info* info, ls_solve_info* per, void* stream);
/* Synchronises the device, then frees the batch (not its plans); NULL is a no-op. */
ls_status ls_batch_destroy(ls_batch b);
const char* ls_batch_last_error(ls_batch b);

/* Allocation-free apply (this entry point has no counterpart in the paper; it
 * serves callers that must not allocate device memory when they apply the
 * operator -- e.g. inside a CUDA stream capture, under an external memory pool
 * or in a loop that may never call the allocator).  Same result as ls_apply
 * for ONE right-hand side (u, Au: N complex128 for LS_FP64, complex64 for
 * LS_MIXED; device pointers, async on stream), but the work arrays live in a
 * fixed 16 MiB device array inside the library instead of plan memory; every
 * GPU that loads the library holds that array until the process exits.
 * Limit: 256-byte-rounded sizes of (occupied cells x n_es) + 2 (R x M) +
 * (occupied cells x (2 n_fb + 1)) complex values, R = max(2 (L + 1), L N_eq + 1),
 * must fit 16 MiB (e.g. every plan with FFT size M <= 1024; M = 2048 does not
 * fit); larger plans get LS_ERR_INVALID with the required size in ls_last_error.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  All calls
 * share the array: calls whose GPU work overlaps race and corrupt each other.
 * Nothing in the array needs to start at zero.  It allocates nothing (no
 * cudaMalloc / cudaFree).  The plan's device (current when the plan was
 * created) must be current: otherwise LS_ERR_INVALID. */
ls_status ls_apply_noalloc(ls_plan plan, const void* u_dev, void* Au_dev, ls_precision prec, void* stream);

/* Device-side failure detection.  The tensor-core near field (8 and 16
 * complex64 right-hand sides per apply) waits on shared-memory barriers
 * (mbarrier) inside the kernel; every such wait gives up after a bounded
 * number of polls, records the time-out in a plan-owned device flag, frees
 * its tensor memory and leaves the rows of its work item unwritten, so that
 * the context stays usable.  ls_plan_device_status synchronises the device,
 * returns LS_ERR_TIMEOUT (message in ls_last_error) if a time-out was
 * recorded since the last call, and clears the flag; ls_solve and
 * ls_batch_solve check it before returning.  ls_set_wait_limit sets the polls
 * per wait (default 4194304, a few milliseconds); 0 makes every wait give up
 * at once, which exercises the failure path without a stuck device.  It
 * synchronises the device and drops the plan's captured applies. */
ls_status ls_plan_device_status(ls_plan plan);
ls_status ls_set_wait_limit(ls_plan plan, int polls);

/* Measurement aid with no counterpart in the paper: the throughput of the
 * current GPU's FP64 fused multiply-add (CUDA cores, independent FMA chains
 * on every SM) and of its TF32 tensor-core MMA (tcgen05, M = 128, N = 256,
 * K = 8, operands in shared memory, one issuing thread per SM), in TFLOP/s
 * counting 2 per multiply-add, timed with CUDA events (about 0.5 s in all).
 * The FP64 figure is the roofline denominator of the FP64 kernels; the TF32
 * one is reported beside the tensor-core near field (which runs kind::f16).  Host pointers; blocking; LS_ERR_CUDA on a
 * CUDA error and LS_ERR_TIMEOUT if a (bounded) wait of the tensor-core probe
 * gave up, with the message in ls_last_error(NULL). */
ls_status ls_measure_peaks(double* fp64_tflops, double* tf32_tflops);

/* Kernel-variant autotuner of a 2-D plan (measurement on the plan's GPU, no
 * counterpart in the paper; the cell layout is chosen before plan creation,
 * see the Python autotune module).  It times, with CUDA events on a private
 * stream and scratch vectors it allocates and frees, the variants of the
 * apply that give the same result up to rounding, and keeps the fastest in
 * the plan:
 *   - columns per block of the lattice column pass (1, 2, 4, 8), FP64 and
 *     complex64 separately (FP64: one apply of min(nrhs, 4) right-hand sides);
 *   - for a complex64 apply of nrhs right-hand sides: the right-hand-side
 *     group per near-field launch (16, 8 or 4) and, for groups of 8 or more,
 *     tensor cores or CUDA cores for each of the near field (split FP16), the
 *     local-expansion coefficients and the equivalent-source projection
 *     (3xTF32);
 *   - then, for the chosen variants, the radix of the complex64 lattice
 *     transforms: 16 (two radix-16 passes and one of radix M / 256) or 4.
 * The plan's device must be current (LS_ERR_INVALID otherwise); 3-D plans
 * return LS_ERR_UNSUPPORTED; nrhs in [1, 64].  Blocking; drops the plan's
 * captured applies.  report (host, may be NULL) receives the choice and the
 * default and best times in milliseconds. */
typedef struct {
  int nrhs;                     /* complex64 right-hand sides timed per apply */
  int conv_cols64, conv_cols32; /* chosen columns per block of the lattice column pass */
  int group32;                  /* chosen complex64 right-hand-side group */
  int near_cuda32;              /* 1: CUDA-core complex64 near field for groups >= 8; 0: tensor cores */
  int n_candidates;             /* variants timed */
  int local_cuda32;             /* 1: CUDA-core complex64 local coefficients for groups >= 8; 0: tensor cores */
  int proj_cuda32;              /* 1: CUDA-core complex64 projection for groups >= 8; 0: tensor cores */
  int fft_radix32;              /* radix of the complex64 lattice transforms: 16 or 4 */
  double ms64_default, ms64_best;
  double ms32_default, ms32_best;
} ls_tune_report;
ls_status ls_plan_autotune(ls_plan plan, int nrhs, ls_tune_report* report);

/* Sets the kernel variants of a 2-D plan from a report (host, read only):
 * conv_cols64 and conv_cols32 in {1, 2, 4, 8}, group32 in {4, 8, 16},
 * near_cuda32, local_cuda32 and proj_cuda32 in {0, 1}, fft_radix32 in
 * {4, 16} (0: 16); the other fields are ignored.  The radix applies to the
 * plan's own applies (a batch's multi-instance lattice passes use radix 16).
 * It re-applies a choice ls_plan_autotune made earlier (for
 * instance in another process on the same kind of GPU) and pins variants for
 * tests.  Every variant gives the same result up to rounding.  A plan whose
 * tables do not fit a tensor-core unit (2 n_fb + 1 > 32 for the local
 * coefficients, n_es > 64 for the projection) keeps the CUDA-core kernel
 * there.  LS_ERR_INVALID on a null argument, a value outside these sets or a
 * column width the plan's lattice size does not fit (shared memory or the
 * column pass's launch bound), LS_ERR_UNSUPPORTED for 3-D plans; drops the
 * plan's captured applies. */
ls_status ls_plan_set_variants(ls_plan plan, const ls_tune_report* variants);

/* Per-stage device timing of ls_apply with CUDA events recorded on the call's
 * stream (measurement aid; enabling it makes ls_apply wait for each apply).
 * Stages: 0 equivalent-source projection, 1 lattice fill, 2 lattice FFT
 * convolution (two forward transforms, spectral product, inverse), 3 local
 * expansion coefficients, 4 near-field correction + evaluation + assembly.
 * ls_set_stage_timing(enable) also resets the accumulators; ls_get_stage_times
 * returns the summed milliseconds per stage (5 doubles) and the number of
 * timed applies for the given precision. */
ls_status ls_set_stage_timing(ls_plan plan, int enable);
ls_status ls_get_stage_times(ls_plan plan, ls_precision prec, double* ms /* 5 */, int64_t* calls);

/* ---- host-only inspection of plan construction (no device work) ----------
 * Builds nodes, near-field matrix and accelerator matrices on the host exactly
 * as ls_plan_create does, for validation and for callers that want the
 * discretisation without a GPU.  Arrays are copied out into caller buffers
 * sized from ls_host_plan_sizes: sizes[0] N, [1] nnz of the near field,
 * [2] occupied cells, [3] n_es, [4] 2 n_fb + 1, [5] (N_eq + 1)^2, [6] FFT size M,
 * [7] total length of the projections P.  Complex arrays are interleaved
 * doubles.  Layouts: near field CSR (rowptr N + 1, col nnz, val nnz); P_c is
 * n_es x n_c row-major at P_off[k] for occupied cell k (w m omega folded in);
 * Bpinv (2 n_fb + 1) x n_loc; BT 9 x (2 n_fb + 1) x n_es with offset index
 * (oi + 1) 3 + (oj + 1); Phi N x (2 n_fb + 1); Gtab, Dtab M x M kernel tables. */
typedef struct ls_host_plan_s* ls_host_plan;
ls_status ls_host_plan_create(const ls_geometry* geom, ls_n2_fn n2, void* ctx, double kappa,
                              const ls_options* opt, ls_host_plan* out);
ls_status ls_host_plan_sizes(ls_host_plan h, int64_t* sizes /* 8 */);
ls_status ls_host_plan_nodes(ls_host_plan h, double* xy, int64_t* canon, double* wfac);
ls_status ls_host_plan_near(ls_host_plan h, int64_t* rowptr, int32_t* col, double* val);
ls_status ls_host_plan_accel(ls_host_plan h, int32_t* occ_cells, int64_t* P_off, double* P,
                             double* Bpinv, double* BT, double* Phi, double* Gtab, double* Dtab);
ls_status ls_host_plan_destroy(ls_host_plan h);

/* ---- 3-D accelerator setup (Section 5), host only -------------------------
 * The dense pieces of the three-dimensional accelerator: two-face equivalent
 * sources on cube cells and a 3-D lattice FFT, the extension of Section 3.2
 * that Section 5 names.  Input: N nodes xyz (N x 3 row-major) with per-node
 * factors wfac = w m omega (quadrature weight x contrast x partition of
 * unity), the wavenumber kappa, the cell box (corner box0[3], side H, L cells
 * per axis; every node must fall inside, LS_ERR_INVALID otherwise), N_eq
 * lattice intervals per cell side (delta = H / N_eq), the local-expansion
 * degree p (0 = 2 N_eq + 1; (p + 1)^2 must not exceed (N_eq + 1)^3), the
 * collocation points per face side m_coll (0 = the smallest m with
 * 6 m^2 >= 2 n_es, plus one), the SVD truncation rcond (0 = 1e-13) and the
 * host threads (0 = all).  kappa sqrt(3) H / 2 must stay below pi.
 *
 * Contents (complex arrays interleaved doubles; the caller sizes its buffers
 * from ls_host_accel3_sizes: [0] occupied cells, [1] n_es = 4 (N_eq + 1)^2,
 * [2] nb = (p + 1)^2, [3] n_loc = (N_eq + 1)^3, [4] FFT size M (power of two
 * >= 2 (L N_eq + 1) - 1, at most 512), [5] total length of P, [6] N):
 *   occ_cells  occupied cell ids (k L + j) L + i, increasing;
 *   node_order the nodes grouped by cell (stable within a cell);
 *   P          per occupied cell c, P_c (n_es x n_c, row-major) at P_off[c];
 *              column j acts on node node_order[start + j] and carries wfac;
 *              rows: monopoles on face x_1 = 0 then x_1 = H, (b, c) row-major,
 *              then the dipoles (d/dz_1) in the same order;
 *   Bpinv      nb x n_loc, the least-squares inverse of the spherical-wave
 *              basis j_l(kappa r) Ybar_l^m / j_l(kappa sqrt(3) H / 2) on the
 *              cell's lattice points (a, b, c) in 0..N_eq, row-major;
 *   BT         27 x nb x n_es, B^+ T_o for neighbour offset
 *              (oi + 1) 9 + (oj + 1) 3 + (ok + 1);
 *   Phi        N x nb, the basis at each node (input order) about its cell
 *              centre;
 *   Gtab, Dtab M^3 lattice tables of G and dG/dz_1 at offsets delta (a, b, c)
 *              (indices wrap at M / 2), zero at the origin.
 * Any output pointer may be NULL (that array is skipped).  The handle owns
 * its memory until ls_host_accel3_destroy. */
typedef struct ls_host_accel3_s* ls_host_accel3;
ls_status ls_host_accel3_create(const double* xyz, const double* wfac, int64_t N, double kappa,
                                const double* box0, double H, int L, int N_eq, int p, int m_coll,
                                double rcond, int n_threads, ls_host_accel3* out);
ls_status ls_host_accel3_sizes(ls_host_accel3 h, int64_t* sizes /* 7 */);
ls_status ls_host_accel3_get(ls_host_accel3 h, int32_t* occ_cells, int64_t* P_off, int64_t* node_order,
                             double* P, double* Bpinv, double* BT, double* Phi, double* Gtab, double* Dtab);
ls_status ls_host_accel3_destroy(ls_host_accel3 h);

/* ---- 3-D ball discretisation and interior singular rule (Section 5) ------
 * The Nystrom nodes of a ball of radius a (host only).  Shell of thickness w:
 * the six faces of a cubed sphere in equiangular coordinates (xi, eta) in
 * [-pi/4 - delta, pi/4 + delta]^2 (face frames (e1, e2, e3), direction
 * normalise(e3 + tan(xi) e1 + tan(eta) e2); faces +x, -x, +y, -y, +z, -z with
 * e1, e2 = (y, z), (z, y), (z, x), (x, z), (x, y), (y, x)), blended on the
 * sphere by the C-infinity partition psi_F (normalised products of cut-offs
 * that vanish at the extended edges); n_f x n_f trapezoid points on each face,
 * n_s depth lines s = 0..1 (r = a - s w) under composite Q-point Newton-Cotes
 * (n_s - 1 a multiple of Q - 1); omega_B(s) = S((s - tau0) / (tau1 - tau0)).
 * Interior: the grid h (i, j, k), |i|, |j|, |k| <= ceil(a / h), with
 * omega_I = 1 - omega_B(depth / w) and weight h^3, kept where omega_I > 0.
 * Shell nodes come first (face, then i, j, k), then the interior grid
 * (lexicographic).  Per node: xyz (N x 3), quadrature weight w (Jacobian x
 * rule x psi_F on the shell), omega, psi (0 on the interior), face (-1 on the
 * interior), grid (N x 3: face-grid (i, j, k) on the shell, (i, j, k) +
 * ceil(a / h) on the interior).  A smooth f integrates as sum w omega f.
 * sizes: [0] N, [1] shell nodes, [2] interior nodes, [3] ceil(a / h).
 * Invalid parameters return LS_ERR_INVALID with a message. */
typedef struct {
  double a, w;           /* radius, shell thickness (0 < w < a)                  */
  int n_f, n_s, Q;       /* face points per side, depth lines, Newton-Cotes points */
  double delta;          /* angular overlap of the faces (0 < delta < pi / 4)    */
  double h;              /* interior grid spacing                               */
  double tau0, tau1;     /* partition-of-unity transition, 0 < tau0 < tau1 < 1   */
} ls_ball3;
typedef struct ls_host_ball3_s* ls_host_ball3;
ls_status ls_host_ball3_create(const ls_ball3* ball, ls_host_ball3* out);
ls_status ls_host_ball3_sizes(ls_host_ball3 h, int64_t* sizes /* 4 */);
ls_status ls_host_ball3_nodes(ls_host_ball3 h, double* xyz, double* w, double* omega, double* psi, int8_t* face,
                              int32_t* grid);
ls_status ls_host_ball3_destroy(ls_host_ball3 h);

/* ---- 3-D device plan (Section 5) -------------------------------------------
 * A plan for the penetrable ball: the discretisation of ls_host_ball3_create,
 * the singular rules of ls_host_ball3_row with its adjacent part stored for
 * the device (ls_host_ball3_near over every node, the contrast of the source
 * node folded in), and the 3-D accelerator of ls_host_accel3_create for the
 * far part (two-face equivalent sources on cube cells, a zero-padded M^3
 * lattice FFT with the G and dG/dz_1 tables, 27-neighbour subtraction and a
 * spherical-wave local expansion).  The complex64 apply uses the same fits
 * rounded to complex64, with the neighbours subtracted on the lattice and the
 * local fit folded into the evaluation (E = Phi B^+ per node, formed in FP64):
 * B^+ of the spherical-wave basis is ill-conditioned and would magnify the
 * complex64 rounding of the lattice field.  n2 receives the nodes as xyz triples
 * (3 n doubles).  The returned ls_plan works with ls_plan_info (n_collar =
 * shell nodes, n_cart = interior nodes, n_fb = local-expansion terms
 * (p + 1)^2), ls_plan_nodes (xyz: 3 N doubles in plan order; canon: the
 * ball's node id), ls_apply, ls_solve (any number of right-hand sides, applied
 * one after another), ls_farfield (dirs: 3 ndir doubles; A(x_hat) = kappa^2 /
 * (4 pi) sum w omega (n^2 - 1) u exp(-i kappa x_hat . y), the standard 3-D
 * asymptotics, not in the paper) and ls_plan_destroy; ls_apply_noalloc and
 * ls_batch_create return LS_ERR_UNSUPPORTED for it.  Every node must lie in
 * the cell box and every cut-off inside its 3 x 3 x 3 cell block
 * (LS_ERR_INVALID otherwise); kappa sqrt(3) H / 2 < pi.  Host-blocking. */
typedef struct {
  double box0[3];        /* corner of the cell box                               */
  double H;              /* cube cell side                                      */
  int L;                 /* cells per axis                                      */
  int N_eq;              /* lattice intervals per cell side                     */
  int p;                 /* local-expansion degree (0 = 2 N_eq + 1)             */
  int m_coll;            /* collocation points per face side (0 = automatic)    */
  double rcond;          /* SVD truncation of the fits (0 = 1e-13)              */
  int n_threads;         /* host threads (0 = all)                              */
} ls_accel3;
/* One row of the 3-D operator K (Section 5) at node q of a ball:
 * K[u](x_q) = sum_n row[n] u[n] with u the density at the nodes (the contrast
 * m = 1 - n^2 is applied by the caller: the discrete equation is
 * u + kappa^2 K[m u] = u^i).  The row is the sum of
 *  - the interior patch's spherical rule about x_q (as ls_interior_window3,
 *    at any position), when its cut-off ball reaches interior nodes;
 *  - on every shell face whose extended chart holds x_q's direction: for a
 *    shell target, polar coordinates (rho = rc sigma^q, n_sig - 1 trapezoid
 *    points in sigma, n_th in the angle) in the face parameters about the
 *    target, times the split Newton-Cotes rule across the depth over the lines
 *    within rs of the target's line; for an interior target above the chart's
 *    bottom, an ellipsoidal spherical rule in the face's index space (semi-axes
 *    rc, rc, min(rs, tau0 (n_s - 1))), points past the bottom line dropped;
 *    degree-p Lagrange interpolation along the surface and degree
 *    min(p, n_s - 1) (clamped stencil) across the depth;
 *  - the regular sum w omega G (1 - eta) over every node, eta the product
 *    cut-offs of the rules applied.
 * rules NULL selects the defaults R = 3, p = 5, q = 3, n_rho = 16, n_mu = 16,
 * n_phi = 32, rc = rs = 6, n_sig = 20, n_th = 32, chi_s0 = 0.1.  row: N
 * complex (interleaved doubles); eta: N doubles or NULL. */
typedef struct {
  double R;              /* interior cut-off radius (grid units)                */
  int p, q;              /* Lagrange degree, radial map rho = r s^q             */
  int n_rho, n_mu, n_phi;
  double rc, rs;         /* shell cut-off: along the surface / across the depth  */
  int n_sig, n_th;
  double chi_s0;         /* cut-off plateau                                     */
} ls_rules3;
ls_status ls_host_ball3_row(ls_host_ball3 h, double kappa, const ls_rules3* rules, int64_t q, double* row,
                            double* eta);

/* The 3-D device plan (see ls_accel3 above): ball, rules (NULL: defaults),
 * n^2 callback (xyz triples), kappa and the accelerator options.  On failure
 * *out is NULL and the message is in ls_last_error(NULL). */
ls_status ls_plan_create3(const ls_ball3* ball, const ls_rules3* rules, ls_n2_fn n2, void* ctx, double kappa,
                          const ls_accel3* acc, ls_plan* out);

/* Adjacent part of the 3-D operator (Section 5 with the adjacency of
 * Section 3.2) for the rows listed (rows NULL: every node, in node order):
 * every singular rule of the row plus the regular (1 - eta) terms of the
 * nodes in the 3 x 3 x 3 block of cube cells (side H, L per axis from corner
 * box0[3]) around the target's cell.  The far part (every node outside that
 * block, weight w omega m G) is the accelerator's (ls_host_accel3_*).  Every
 * cut-off eta must vanish outside the block: LS_ERR_INVALID otherwise, as
 * when a node lies outside the cell box.  The result is kept in the handle
 * (replacing an earlier one) as a CSR matrix over the listed rows with sorted
 * columns; *nnz receives its entry count.  ls_host_ball3_near_get copies it:
 * rowptr (n_rows + 1), col (nnz), val (nnz complex, interleaved doubles);
 * any pointer may be NULL.  stencils_only != 0 stores instead only the
 * singular parts and the sparse correction -eta w omega G (entries where a
 * cut-off is positive): the adjacent part is then that matrix plus the plain
 * sum of w omega G over the block's other nodes, which a caller computes on
 * the fly. */
ls_status ls_host_ball3_near(ls_host_ball3 h, double kappa, const ls_rules3* rules, const double* box0, double H,
                             int L, const int64_t* rows, int64_t n_rows, int stencils_only, int n_threads,
                             int64_t* nnz);
ls_status ls_host_ball3_near_get(ls_host_ball3 h, int64_t* rowptr, int32_t* col, double* val);

/* Coefficients c[o] of the interior singular rule for a target on a uniform
 * grid of spacing h: int G(x, y) eta(|y - x| / (R h)) phi(y) dy is
 * sum_o c[o] phi(x + o h) over offsets o in [-Wn, Wn]^3, Wn = ceil(R) + p/2 + 2,
 * G = exp(i kappa r) / (4 pi r).  Spherical coordinates about x: radius
 * rho = R s^q (grid units), n_rho - 1 trapezoid points s = 1..n_rho-1 / n_rho
 * weighted by the cut-off chi(s^q) (1 up to chi_s0), n_mu Gauss-Legendre
 * points in cos(theta), n_phi trapezoid points in the azimuth; phi at the
 * rule's points by degree-p tensor Lagrange interpolation on the grid
 * (stencil starting floor(t) - p/2 per axis).  win: (2 Wn + 1)^3 complex
 * (interleaved doubles, [di][dj][dk]) or NULL to query Wn only. */
ls_status ls_interior_window3(double kappa, double h, double R, int p, int q, int n_rho, int n_mu, int n_phi,
                              double chi_s0, double* win, int* Wn);

const char* ls_status_string(ls_status s);

/* Message of the last failure of this plan (or of the last failed
 * ls_plan_create when plan is NULL).  Valid until the next call on the plan. */
const char* ls_last_error(ls_plan plan);

#ifdef __cplusplus
}
#endif
#endif /* LS_GB300_H */
