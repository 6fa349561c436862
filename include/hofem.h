/*
 * hofem.h -- C ABI of a GB300 (sm_103a) fast direct solver for n-th order Lagrange
 * finite-element Dirichlet Poisson problems on 2D/3D boxes, after Zlotnik & Zlotnik,
 * "A direct fast FFT-based implementation for high order finite element method on
 * rectangular parallelepipeds for PDE" (arXiv:1609.07758).
 *
 * The discrete problem (Eq. bvp glob 2):
 *     ( sum_i 4 h_i^-2 A_i (x) prod_{m!=i} C_m  +  alpha C_1 (x) ... (x) C_N ) v = f,
 * with A_i, C_i the scaled global stiffness / mass matrices of axis i (Eq. eig_glob),
 * h_i = X_i / K_i, and f = f^h the load vector in the same scaling (the "FEM average").
 * It is solved by algorithm (a) of Sect. 2 par. 4: direct F_n-transforms (Theorem 2,
 * part 2) along every axis, division by sum_i 4 h_i^-2 lambda_i + alpha (Eq. decomp v 2),
 * inverse F_n-transforms (Theorem 2, part 1).
 *
 * Conventions shared by every entry point
 *  - Arrays are FP64, C-order, shape (nrhs, M_1, ..., M_N), M_i = n K_i - 1.  Along an
 *    axis, unknown p = (j-1) n + (i-1) is local point i (1..n) of element j (1..K);
 *    i = n is the mesh node x_j.  So p sits at coordinate (p + 1) h / n.
 *  - Pointers named f, u, r, in, out are DEVICE pointers owned by the caller; the
 *    plan owns its tables and workspace.  `stream` is a cudaStream_t (NULL = legacy
 *    default stream); every call is asynchronous on it and returns after enqueueing.
 *  - Every call returns a status and never aborts.  On error nothing is enqueued
 *    unless the status is HOFEM_ERR_CUDA (a launch failed part-way).
 *    hofem_last_error() gives a one-line message for the calling thread.
 *  - A plan may be used from one host thread at a time.
 */
#ifndef HOFEM_H
#define HOFEM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hofem_plan_s* hofem_plan_t;
typedef struct hofem_batch_s* hofem_batch_t;

typedef enum {
  HOFEM_OK = 0,
  HOFEM_ERR_INVALID_ARG = 1,
  HOFEM_ERR_UNSUPPORTED = 2,
  HOFEM_ERR_OOM = 3,
  HOFEM_ERR_CUDA = 4,
  HOFEM_ERR_NOT_CONVERGED = 5,
  HOFEM_ERR_TIMEOUT = 6
} hofem_status;

/* Arithmetic of the transform sweeps.  *_REFINED: low-precision solves corrected by
 * iterative refinement with an FP64 matrix-free residual r = f - A u (Eq. bvp glob 2).
 * BF16 / FP16: the arrays written after the eigenvalue division (by the fused sweep and
 * the inverse sweeps) are stored in that format, half the bytes of FP32; the forward
 * sweeps' arrays stay FP32 (rounding them would be amplified by the division); the
 * transforms and the per-frequency mixing compute in FP32 with FP32 tables.
 * FP16 solves scale each right-hand side by an exact power of two (max near 2^10) and
 * store the intermediate lines multiplied by the eigenvalue sum of the axes not yet
 * inverted, so that their values stay inside FP16's exponent range.
 * Relative L2 error of one unrefined solve: FP32 ~1e-6, BF16 and FP16 ~1e-2. */
typedef enum {
  HOFEM_FP64 = 0,
  HOFEM_FP32 = 1,
  HOFEM_BF16 = 2,
  HOFEM_FP16 = 3,
  HOFEM_FP32_REFINED = 4,
  HOFEM_BF16_REFINED = 5,
  HOFEM_FP16_REFINED = 6
} hofem_dtype;

typedef struct {
  int N;                    /* dimensions */
  int n;                    /* element order */
  int K[3];                 /* elements per axis */
  int M[3];                 /* unknowns per axis, n K - 1 */
  int dtype;                /* hofem_dtype of the plan */
  int refine_iters;         /* most correction steps of a solve (tolerance mode) or its fixed
                               count (refined dtypes; see hofem_set_refinement) */
  int iterations;           /* correction steps actually run by the last solve */
  int converged;            /* 1 if the last solve met its tolerance (or ran a fixed count) */
  double last_rel_update;   /* ||delta||_2 / ||u||_2 of the last correction, max over RHS
                               (valid after the caller synchronises the stream) */
  double plan_ms;           /* host wall time of hofem_plan */
  size_t table_bytes;       /* device bytes of eigen / twiddle tables */
  size_t workspace_bytes;   /* device bytes of solve workspace currently reserved */
  int lines_per_cta[3];     /* launch configuration chosen per axis (W) */
  int threads_per_cta;
  long long kernel_launches; /* kernels this plan has launched since it was created */
  long long tuned_shapes;   /* launch-shape candidates measured by hofem_autotune */
  int orders[3];            /* element order per axis (n above is their maximum) */
  int fft_len[3];           /* per axis, the length of the FFTs its DSTs run at the plan's sweep
                               precision: K for a power of two or direct mixed-radix passes
                               over the prime factors of K, else the power-of-two length of
                               the Bluestein (chirp-z) convolution chosen for K with large
                               prime factors */
} hofem_info;

/* One problem of a batch: N = 2 or 3 axes with K[i] elements of length X[i] (entries
 * i >= N are ignored), order n, alpha, and nrhs right-hand sides (same rules as
 * hofem_plan). */
typedef struct {
  int N;
  int K[3];
  int n;
  double X[3];
  double alpha;
  int nrhs;
} hofem_problem;

typedef struct {
  int count;                /* problems */
  int streams;              /* parallel branches of the captured solve graph */
  long long unknowns;       /* sum over problems of nrhs x prod_i M_i */
  long long graph_nodes;    /* nodes of the captured solve graph (0 before the first solve) */
  int captures;             /* times the solve graph was captured */
  double plan_ms;           /* host wall time of hofem_batch_plan */
  double tune_ms;           /* host wall time of hofem_batch_tune (0 if not tuned) */
  size_t table_bytes;       /* device bytes of all eigen / twiddle tables */
  size_t workspace_bytes;   /* device bytes of all solve workspaces */
} hofem_batch_info;

/* Per-kernel-kind device time, from CUDA events recorded on the launching stream around
 * every kernel while profiling is enabled (see hofem_profile). */
typedef struct {
  char name[32];            /* "sweep_{fwd,fsi,inv}_{f64,f32}" (general sweep kernel, FP64 or FP32
                               work), "sweep_{fwd,fsi,inv}_reg" (register-resident FP32 sweep),
                               "apply_f64" (operator sweep), "banded_f64" (the banded solves
                               of algorithm (b)) */
  int launches;
  double total_ms;
} hofem_kernel_time;

/* Build a plan: N = 2 or 3 axes, 2 <= K[i] <= 8192 elements (any K; powers of two take
 * the fastest FFT path, other K mixed-radix passes costing the sum of K's prime factors
 * per point) and length X[i] > 0 per axis, order 1 <= n <= 16, alpha > -pi^2 sum_i X_i^-2
 * (Sect. 2 par. 4).  A line of n K - 1 unknowns and one DST job must fit a CTA's shared
 * memory at the sweeps' precision (FP64 for FP64 plans, FP32 otherwise), else
 * HOFEM_ERR_UNSUPPORTED.  Largest K, powers of two / other K: FP32 8192 / 6081 (n = 1),
 * 4096 / 3260 (n = 9), 2048 / 2318 (n = 16); FP64 4096 / 2879 (n = 1), 2048 / 1560
 * (n = 9), 1024 / 1114 (n = 16).
 * Computes, on the GPU in double-double arithmetic, the 1D eigen-data of every axis:
 * for k = 1..K-1 the n eigenpairs of the theta-family of Theorem 1 part 3, for k = 0 the
 * element eigenpairs of Lemma 1 (Theorem 1 part 2).  Synchronous; allocates tables. */
hofem_status hofem_plan(int N, const int* K, int n, const double* X, int dtype, double alpha,
                        hofem_plan_t* out);

/* hofem_plan with an element order n[i] per axis (the paper allows n_i per axis, Sect. 2
 * par. 4): M_i = n_i K_i - 1, each axis' eigen-data, transforms and operator products of
 * its own order. */
hofem_status hofem_plan_orders(int N, const int* K, const int* n, const double* X, int dtype, double alpha,
                               hofem_plan_t* out);

/* Refined dtypes only: iters = most residual/correction steps after the first
 * low-precision solve (0..100); tol > 0 stops once ||delta||_2 / ||u||_2 <= tol for every
 * right-hand side, reading two doubles per right-hand side on the host after each step
 * (one stream synchronisation per step), and a solve that ends above tol returns
 * HOFEM_ERR_NOT_CONVERGED; tol = 0 runs exactly iters steps.
 * Default: tol = 1e-12 with iters = 10 (FP32) or 16 (BF16, FP16).  The error after a
 * step measured below its update norm, while the steps needed depend on the right-hand
 * side (2D n = 9, K = 1024: 2 for a smooth one, 4 for N(0,1)).  Orders n <= 11 converge
 * (3-4 steps at K = 8..64); equispaced n >= 12 elements are too ill-conditioned for an
 * FP32 solve to contract to 1e-12, so their default refined solves end with
 * HOFEM_ERR_NOT_CONVERGED (u then holds the last iterate; use HOFEM_FP64).
 * A solve issued into a capturing stream (CUDA graph capture) cannot synchronise: with
 * tol > 0 it runs the plan's fixed capture count, by default FP32 2 when every K is a
 * power of two, else 3, BF16 and FP16 8 (set by a call with tol = 0, which also fixes the
 * count of uncaptured solves). */
hofem_status hofem_set_refinement(hofem_plan_t plan, int iters, double tol);

/* The (n+1)-point Gauss-Legendre quadrature points of the load vector along `axis`
 * (Sect. 2 par. 5): x[e (n+1) + g] = e h + (1 + xi_g) h / 2 for the elements e = 0..K-1,
 * xi_g ascending on [-1, 1], h = X / K.  x: HOST array of K (n+1) doubles.  Synchronous. */
hofem_status hofem_quadrature_points(hofem_plan_t plan, int axis, double* x);

/* The FEM average f^h of Sect. 2 par. 4, f^h_p = prod_i (2/h_i) int f phi_p, by the
 * (n+1)-point Gauss-Legendre rule on every element along every axis (Sect. 2 par. 5),
 * from samples of f at the tensor product of the quadrature points:
 * fq: device FP64 (nrhs, K_1(n+1), .., K_N(n+1)), C-order, axis i indexed e (n+1) + g as in
 * hofem_quadrature_points; fh: device FP64 (nrhs, M_1..M_N), ready for hofem_solve.
 * Two plan-owned intermediate arrays are allocated on first use (or when nrhs grows).
 * Asynchronous on stream; fq != fh. */
hofem_status hofem_load(hofem_plan_t plan, const double* fq, double* fh, int nrhs, void* stream);

/* Inhomogeneous Dirichlet data u = b on the boundary (the remark after Eq. bvp glob 2 in
 * Sect. 2 par. 4: the problem reduces to Eq. bvp glob 2 with a modified f^h):
 *   f <- f - (L^ vb)|interior,  L^ = sum_i 4 h_i^-2 A^_i (x) prod_{m != i} C^_m + alpha prod C^_m,
 * A^_i, C^_i the 1D matrices of axis i with its two boundary nodes kept (same local A, C).
 * vb: device FP64 (nrhs, M_1 + 2, .., M_N + 2), the full grid with the boundary nodes at index
 * 0 and M_i + 1 of every axis (interior dof p at p + 1); only its boundary entries are read
 * (values of b at the boundary Lagrange points, or any other boundary coefficients).
 * f: device FP64 (nrhs, M_1..M_N), updated in place (e.g. the f^h of hofem_load); then
 * hofem_solve gives the interior values of the solution.  Asynchronous on stream; vb != f. */
hofem_status hofem_lift_dirichlet(hofem_plan_t plan, const double* vb, double* f, int nrhs, void* stream);

/* Algorithm (b) of Sect. 2 par. 4 in FP64: the direct F_n-transforms along x_2..x_N, then
 * for every mode of those axes the banded SPD system (4 h_1^-2 A_1 + sigma C_1) v = f
 * along x_1 (sigma = the mode's eigenvalue sum + alpha), solved by static condensation of
 * the element interiors and a tridiagonal nodal Schur system, then the inverse transforms.
 * One correction with the FP64 matrix-free residual follows (the interior blocks of
 * high-order elements are ill-conditioned).  The same discrete solution as hofem_solve
 * (algorithm (a)); f, u as for hofem_solve (f != u).  Orders n_1 <= 9 (HOFEM_ERR_UNSUPPORTED
 * above: at n = 16 the condensed solve is no longer a contraction in FP64).
 * Asynchronous on stream. */
hofem_status hofem_solve_banded(hofem_plan_t plan, const double* f, double* u, int nrhs, void* stream);

/* r = A_a u for the variable-coefficient problem -div(a grad u) = f on the plan's 2D mesh
 * (one order n <= 9 on both axes), in the scaling of Eq. bvp glob 2: per element
 * (2/h_1)(2/h_2) int a grad phi_p . grad phi_q by the (n+1)-point Gauss-Legendre rule per
 * direction (Sect. 2 par. 5).  aq: device FP64 (K_1 (n+1), K_2 (n+1)), the values of a > 0
 * at the points of hofem_quadrature_points; u, r: device FP64 (M_1, M_2), distinct.  For
 * a = 1 this is hofem_apply with alpha = 0.  Asynchronous on stream. */
hofem_status hofem_apply_varcoef(hofem_plan_t plan, const double* aq, const double* u, double* r, void* stream);

/* The solver as a preconditioner (Sect. 1): conjugate gradients on A_a u = f (see
 * hofem_apply_varcoef) preconditioned by the plan's constant-coefficient solve (build
 * the plan with alpha = 0).  u: initial guess in, solution out; stops when
 * ||f - A_a u||_2 <= tol ||f||_2 or after maxit steps (HOFEM_ERR_NOT_CONVERGED).  iters and
 * relres (HOST, may be NULL) receive the steps taken and the final relative residual.
 * Synchronises the stream three times per step (dot products). */
hofem_status hofem_pcg(hofem_plan_t plan, const double* aq, const double* f, double* u, double tol, int maxit,
                       int* iters, double* relres, void* stream);

/* out = (C_1 x .. x C_N) u, the matrix-free mass operator of Eq. bvp glob 2 (its alpha
 * term with alpha = 1).  u, out: distinct device FP64 arrays (nrhs, M_1..M_N). */
hofem_status hofem_mass(hofem_plan_t plan, const double* u, double* out, int nrhs, void* stream);

/* Implicit (backward Euler) steps of the heat equation u_t - Lap u = g, the paper's stated
 * application of the solver (Sect. 1; closing remarks of Sect. 2): with a plan built for
 * alpha = 1/tau > 0, each step solves (A + alpha C x .. x C) u_new = alpha (C x .. x C) u
 * + g^h (Eq. bvp glob 2) and overwrites u.  g: device FP64 (nrhs, M_1..M_N) in the f^h scaling, or NULL (g = 0).
 * Refined plans run their fixed correction count per step (capturable in a CUDA graph
 * after a first call has allocated the plan's step buffer).  Asynchronous on stream. */
hofem_status hofem_heat_steps(hofem_plan_t plan, double* u, const double* g, int steps, int nrhs, void* stream);

/* Autotuner: time every candidate launch shape of this plan's solve and apply for nrhs
 * right-hand sides (sweeps: lines per CTA W and DST batch J, from the largest J that fits
 * down to a quarter of it; operator sweeps: elements per CTA E) on its own workspace,
 * and keep the fastest per shape in a process-wide table that
 * later launches of any plan consult (written to / read from the file named by the
 * environment variable HOFEM_TUNE_CACHE when set).  Synchronous; reserves workspace. */
hofem_status hofem_autotune(hofem_plan_t plan, int nrhs, void* stream);

/* Reserve workspace for nrhs right-hand sides (solve allocates on demand otherwise;
 * call this before capturing a solve in a CUDA graph). */
hofem_status hofem_reserve(hofem_plan_t plan, int nrhs);

/* u = A^{-1} f for nrhs right-hand sides (algorithm (a), Sect. 2 par. 4).  f, u: device
 * FP64 arrays (nrhs, M_1..M_N); u is overwritten; f is not modified.  f == u (in place)
 * is allowed for unrefined dtypes only.  Refined dtypes follow hofem_set_refinement (by
 * default one stream synchronisation per correction step outside graph capture). */
hofem_status hofem_solve(hofem_plan_t plan, const double* f, double* u, int nrhs, void* stream);

/* r = A u: the matrix-free FP64 operator of Eq. bvp glob 2 (stiffness applied to
 * differences so that constants stay in its kernel exactly).  u, r: device FP64. */
hofem_status hofem_apply(hofem_plan_t plan, const double* u, double* r, int nrhs, void* stream);

/* r = A u exactly as hofem_apply, but allocating nothing: for callers that must not
 * allocate device memory when they call (a framework allocator that forbids raw
 * cudaMalloc, or a real-time loop that cannot take cudaMalloc's device-wide
 * synchronisation).  The paper has no counterpart to this entry point.
 * The operator's intermediate arrays (2 for N = 2, 4 for N = 3, each nrhs x unknowns
 * doubles) live in one fixed 32 MiB device array inside the library, resident on every
 * GPU that loads it until the process exits; nrhs x unknowns above 2,097,152 (N = 2) or
 * 1,048,576 (N = 3) returns HOFEM_ERR_INVALID_ARG.  Every call outside stream capture
 * looks up that array's device address (cudaGetSymbolAddress) with the device current, so
 * a context re-created after cudaDeviceReset is picked up; a captured call reuses the
 * address of the last uncaptured call on the device: make a first call before any capture.  All calls share the array, so calls whose
 * work overlaps on the GPU race on it; nothing in it needs clearing between calls.
 * u, r: device FP64, distinct.  The plan must have been created on the current device. */
hofem_status hofem_apply_static(hofem_plan_t plan, const double* u, double* r, int nrhs, void* stream);

/* r = f - A u, the FP64 residual used by iterative refinement.  f, u, r: device FP64. */
hofem_status hofem_residual(hofem_plan_t plan, const double* f, const double* u, double* r,
                            int nrhs, void* stream);

/* Test hook: the 1D F_n-transform of `lines` contiguous lines of length M_axis.
 * inverse = 0: direct transform (Theorem 2 part 2) of y: out_q = (y, s_q) / K, with the
 * eigenvectors s_q normalised to ||s_q||_C^2 = K (so for y = C w it returns the
 * coefficients of w).  inverse = 1: out = sum_q in_q s_q (Theorem 2 part 1).
 * Spectral order q = (k-1) n + (l-1) for k = 1..K-1, l = 1..n (ascending lambda within
 * k), then q = n (K-1) + (l-1), l = 1..n-1 for k = 0.  Signs: the nodal amplitude of
 * s_q is positive for k >= 1; e^(l) has its first component of magnitude >= 1e-3 max|e|
 * positive.  Runs in the plan's transform precision.  in, out: device FP64. */
hofem_status hofem_transform1d(hofem_plan_t plan, int axis, int inverse, const double* in,
                               double* out, long lines, void* stream);

/* Sweep kinds of hofem_sweep. */
enum { HOFEM_SWEEP_FORWARD = 0, HOFEM_SWEEP_FUSED = 1, HOFEM_SWEEP_INVERSE = 2 };

/* One sweep of algorithm (a) (Sect. 2 par. 4) along `axis` on a block of lines that need
 * not be the plan's whole grid -- the building block of one problem split over several
 * GPUs by slabs of x_1 (each GPU transforms the axes it holds whole, an all-to-all
 * exchange makes x_1 whole, and so on).  in, out: device FP64 arrays laid out as
 * [outer][M_axis][inner] (C order; in == out allowed): `outer` blocks of `inner` lines.
 *   HOFEM_SWEEP_FORWARD: the direct F_n-transform of every line (Theorem 2 part 2, as
 *     hofem_transform1d with inverse = 0);
 *   HOFEM_SWEEP_INVERSE: the inverse one (Theorem 2 part 1);
 *   HOFEM_SWEEP_FUSED (axis 0 only): direct transform, division of coefficient q of line
 *     l by lam_1[q] + sum_{i>=2} lam_i[q_i(c)] + alpha (Eq. decomp v 2), where the line's
 *     column c = line_offset + l indexes the x_2..x_N plane in C order (c = q_2 for N = 2,
 *     c = q_2 M_3 + q_3 for N = 3), then the inverse transform.  line_offset + inner must
 *     not exceed the plane's size; nrhs > 1 is outer = nrhs with the same columns.
 * FP64 plans run it in FP64; every other dtype in FP32 arithmetic (a refined plan's correction
 * sweeps) with FP64 input and output.  Asynchronous on stream. */
hofem_status hofem_sweep(hofem_plan_t plan, int axis, int mode, const double* in, double* out,
                         long long outer, long long inner, long long line_offset, void* stream);

/* The FP64 residual r = f - A u (Eq. bvp glob 2, as hofem_residual) of one slab of a problem
 * split over GPUs by x_1: the slab owns elements e0 .. e1 - 1 along x_1, i.e. the dof rows
 * e0 n .. min(e1 n, M_1) - 1 ("rows"), with every x_2..x_N index.  Two stages with an exchange
 * of halo rows between them:
 *   stage 0: a = u of the slab, [nrhs][rows][M_2..M_N]; the operator's sweeps along x_N .. x_2
 *     write its two intermediate arrays out0, out1, laid out [nrhs][ext][M_2..M_N] with
 *     ext = pre + rows + post (pre = 1 if e0 > 0, post = n if e1 < K_1), into rows
 *     pre .. pre + rows - 1.  The caller then fills row 0 (when pre = 1) with the previous
 *     slab's last row and the last `post` rows with the next slab's first n rows, of both
 *     arrays.
 *   stage 1: a, b = the filled intermediates; the sweep along x_1 over the slab's elements
 *     writes out0 = f - A u on the slab's rows, [nrhs][rows][M_2..M_N], FP64 or, with
 *     out_fp32, FP32 values (f: [nrhs][rows][..] FP64, may be NULL for out0 = A u).
 * All device pointers; b, f, out1 unused where not named.  The stage-0 scratch of a 3D plan
 * is the plan's workspace (reserved on first use).  Asynchronous on stream. */
hofem_status hofem_residual_slab(hofem_plan_t plan, int stage, long long e0, long long e1, const double* a,
                                 const double* b, const double* f, double* out0, double* out1, int out_fp32,
                                 int nrhs, void* stream);

/* y += c x over count FP64 values (device pointers; the correction u += delta of a refined
 * solve driven from outside the library, e.g. over several GPUs).  Asynchronous on stream. */
hofem_status hofem_axpy(double* y, double c, const double* x, long long count, void* stream);

/* dst[b][r][c] = src[b][r][c] for b < batch, r < rows, c < cols, with element offsets
 * b src_bs + r src_ld + c (and the dst_* ones): the packing and unpacking of the blocks an
 * all-to-all exchange moves between GPUs.  Device FP64 pointers, not overlapping.
 * Asynchronous on stream. */
hofem_status hofem_copy_block(const double* src, double* dst, long long batch, long long rows, long long cols,
                              long long src_ld, long long dst_ld, long long src_bs, long long dst_bs,
                              void* stream);

/* Test hook: copy axis `axis`'s eigen-data to HOST buffers (any may be NULL):
 * lam[M] true eigenvalues 4 h^-2 lambda_q in spectral order; mix[(K-1) n n]: row l of
 * block k-1 is (q_1..q_{n-1}, c) of mode (k, l) (interior values then the nodal
 * amplitude, ||s||_C^2 = K); evec[(n-1)(n-1)]: row l is e^(l).  Synchronous. */
hofem_status hofem_get_eigen(hofem_plan_t plan, int axis, double* lam, double* mix, double* evec);

hofem_status hofem_get_info(hofem_plan_t plan, hofem_info* out);

/* enable != 0: record a CUDA event pair around each kernel the plan launches (adds two
 * event records per launch); enable == 0 stops recording.  Either call clears the totals. */
hofem_status hofem_profile(hofem_plan_t plan, int enable);

/* Synchronise the recorded events and return up to max_entries per-kind totals since the
 * last hofem_profile call; *count receives the number of kinds.  out is a HOST array. */
hofem_status hofem_get_profile(hofem_plan_t plan, hofem_kernel_time* out, int max_entries, int* count);
void hofem_destroy(hofem_plan_t plan);

/* Batched solves of independent problems of uneven K, n, X and nrhs: one plan per problem
 * with its workspace reserved up front.  The first hofem_batch_solve captures every
 * problem's solve (refined dtypes with the plan's fixed capture count: FP32 2 when every
 * K is a power of two, else 3; BF16 and FP16 8; see hofem_set_refinement) into one CUDA graph
 * whose branches spread the problems over up to 16 streams, so independent problems run
 * concurrently; later calls with the same pointer arrays relaunch that graph (other
 * pointers recapture it).  Synchronous plan; errors of one problem name its index in
 * hofem_last_error. */
hofem_status hofem_batch_plan(int count, const hofem_problem* probs, int dtype, hofem_batch_t* out);

/* hofem_autotune for every problem (shapes shared between problems are measured once). */
hofem_status hofem_batch_tune(hofem_batch_t batch, void* stream);

/* u_i = A_i^{-1} f_i for every problem i.  f, u: HOST arrays of count device pointers,
 * each an FP64 array (nrhs_i, M_1..M_N) as for hofem_solve (f_i != u_i).  Asynchronous
 * on stream: one graph launch. */
hofem_status hofem_batch_solve(hofem_batch_t batch, const double* const* f, double* const* u, void* stream);

hofem_status hofem_batch_get_info(hofem_batch_t batch, hofem_batch_info* out);

/* Split a batch over `parts` GPUs (one process each, no data exchange: the problems are
 * independent).  part_of[i] receives the part of problem i; cost[i] (if non-NULL) its
 * predicted work: nrhs x prod_i M_i x ((corrections + 1) (2N - 1)/N sum_i (log2 L_i + n)
 * + corrections x 2 n N), L_i the FFT length of axis i, corrections the fixed capture count
 * of `dtype` (0 for unrefined dtypes).  Longest processing time first: problems in
 * decreasing cost, each to the part with the least predicted work so far, so the parts'
 * totals differ by at most one problem's cost.  Host only and deterministic (ties by index),
 * so every rank computes the same split.  part_of, cost: HOST arrays of count entries. */
hofem_status hofem_batch_partition(int count, const hofem_problem* probs, int dtype, int parts, int* part_of,
                                   double* cost);

/* The plan of problem i (owned by the batch; for hofem_get_info / hofem_apply). */
hofem_status hofem_batch_get_plan(hofem_batch_t batch, int i, hofem_plan_t* out);
void hofem_batch_destroy(hofem_batch_t batch);

const char* hofem_status_string(int status);
const char* hofem_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HOFEM_H */
