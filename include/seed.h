/*
 * seed.h -- C ABI of the GB300 (sm_103a) implementation of the improved seed
 * method of Abdel-Rehim, Morgan and Wilcox for Hermitian (or real symmetric)
 * positive definite systems with several right-hand sides,
 *
 *     A x^j = b^j,  j = 1..nrhs                                  (Sec. 1)
 *
 * The method (Sec. 2.2 and Sec. 3): the first system is solved by the Lanczos
 * form of CG with periodic reorthogonalization against the stored Lanczos
 * basis V; while that basis grows, every other right-hand side receives the
 * Galerkin projection over it ("single seeding"); the seeded systems are then
 * finished with plain CG.
 *
 * Conventions for every entry point:
 *  - All vector and matrix pointers are DEVICE pointers on the device that was
 *    current when the context was created; the caller owns them.  The library
 *    never frees, reallocates or retains them past the call, except the
 *    operator arrays given to seed_create_* which must stay valid until
 *    seed_destroy.
 *  - Blocks of vectors are column-major: column j starts at ptr + j*ld
 *    elements, ld >= n.  Complex data (SEED_C128) is interleaved (re, im)
 *    doubles, the layout of C99 double complex / numpy complex128.
 *  - Work is enqueued on the stream given at creation.  Calls that return
 *    seed_info synchronise that stream once before returning; the others do
 *    not synchronise.
 *  - Errors are reported only through the returned status; nothing aborts,
 *    throws or prints.  seed_last_error() gives a one-line reason.  Inputs are
 *    validated on the host before any kernel is launched.
 *  - A context is not thread-safe; different contexts are independent.
 */
#ifndef SEED_H_
#define SEED_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SEED_ABI_VERSION 2

typedef struct seed_ctx seed_ctx;
typedef struct CUstream_st *seed_stream; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  SEED_OK = 0,
  SEED_EINVAL = 1,   /* bad argument (size, ld, NULL pointer, malformed operator; from
                        seed_solve_first also a NaN or infinite initial residual of system 1) */
  SEED_ENOMEM = 2,   /* device allocation failed */
  SEED_ECUDA = 3,    /* a CUDA runtime call failed (including no usable device) */
  SEED_ENOTSPD = 4,  /* the LU of the Lanczos tridiagonal met delta_i <= 0 or NaN:
                        A is not positive definite in floating point (Sec. 3
                        uses an LU factorization, which needs a definite T) */
  SEED_ENOTCONV = 5, /* an iteration cap was reached before the tolerance */
  SEED_ESTATE = 6,   /* call out of order (e.g. seed_project without a kept basis) */
  SEED_ETIMEOUT = 7  /* a grid barrier of a persistent kernel waited longer than its limit (2 s);
                        the kernel left without hanging, the results are not valid */
} seed_status;

/* Element types.  The caller's operator arrays, right-hand sides and
 * solutions are always SEED_F64 (CSR) or SEED_C128 (Wilson): the paper's
 * method is stated for one precision (Sec. 3), and the precision the solver
 * computes in is a solver parameter (seed_params.precision), not a property
 * of the operator.  SEED_F32 / SEED_C64 name the element type of the FP32
 * operator copy and Krylov vectors a mixed-precision context keeps, which
 * seed_apply ops 3-7 read and write (SEED_F32 for CSR, SEED_C64 for Wilson). */
typedef enum {
  SEED_F64 = 0,      /* real double */
  SEED_C128 = 1,     /* complex double, interleaved */
  SEED_F32 = 2,      /* real float (mixed-precision CSR vectors) */
  SEED_C64 = 3       /* complex float, interleaved (mixed-precision Wilson vectors) */
} seed_dtype;

/* Real symmetric positive definite matrix in CSR form (device arrays).
 * row_ptr[n+1] (row_ptr[0] = 0, nondecreasing, row_ptr[n] = nnz),
 * col_idx[nnz] in [0, n), vals[nnz].  Symmetry is the caller's promise. */
typedef struct {
  int64_t n;
  int64_t nnz;
  const int32_t *row_ptr;
  const int32_t *col_idx;
  const double *vals;
} seed_csr;

/* Wilson-Dirac operator on a 4-d lattice; the library solves with the normal
 * operator A = D^H D (Sec. 4 turns the non-Hermitian system into a Hermitian
 * one by multiplying it with D^H: two applications of D per iteration).
 *   (D psi)(n) = psi(n) - kappa sum_mu [ (1 - gamma_mu) U_mu(n) psi(n+mu)
 *                                       + (1 + gamma_mu) U_mu(n-mu)^H psi(n-mu) ]
 * Wilson parameter r = 1, gamma matrices in the DeGrand-Rossi (chiral) basis
 * (gamma_5 = diag(1,1,-1,-1)); D^H = gamma_5 D gamma_5.  The paper names D but
 * does not define it; this is the textbook form.
 * Site index s = x + X*(y + Y*(z + Z*t)); spinor [site][spin 0..3][colour 0..2]
 * complex (n = 12 * sites); links [mu 0..3][site][row][col] complex, U_mu(s).
 * bc_t = 1 makes the t direction antiperiodic, 0 periodic (all others periodic).
 * Each dims[k] >= 2. */
typedef struct {
  int32_t dims[4];
  double kappa;
  int32_t bc_t;
  int32_t reserved;
  const void *links;   /* device, complex double, 4*sites*9 elements */
} seed_wilson;

/* Parameters (the inputs of the Sec. 3 algorithm: m, the frequency of
 * reorthogonalization; tolerances for the seed and the remaining systems). */
typedef struct {
  int32_t m_max;          /* m: maximum Lanczos steps kept in V (>= 1) */
  int32_t reorth_freq;    /* reorthogonalize at steps i with i % freq == 0 (i >= 2); 0 = never */
  int32_t reorth_passes;  /* classical Gram-Schmidt passes per reorthogonalization (1 or 2) */
  int32_t extra_iters;    /* Lanczos steps taken after the seed tolerance is first met (Sec. 3) */
  int32_t keep_basis;     /* 1: keep V and T after seed_solve_first for seed_project */
  int32_t x0_zero;        /* 1: X is overwritten with zeros and r_0 = b (no mvp) */
  int32_t maxit_rest;     /* CG iteration cap per remaining system */
  int32_t max_restarts;   /* CG restarts from the true residual if it exceeds 1.5 tol */
  double tol_seed;        /* stop the seed when beta_i |zeta_i| / delta_i <= tol_seed ||b^1|| */
  double tol_rest;        /* CG stops when ||r|| <= tol_rest ||b^j|| */
  double breakdown_rel;   /* lucky breakdown when beta_i <= breakdown_rel * max row sum of |T| */
  int32_t kernel_path;    /* How the steps are issued (same method either way):
                             0 (default): the seed's runs of Lanczos steps between
                             reorthogonalizations in one persistent cooperative kernel (when the
                             frequency is 0 or >= 8), everything else as step kernels
                             replayed from CUDA graphs, the lockstep CG in up to three concurrent
                             column branches; small real CSR problems in FP64 (n <= 9728) run
                             the whole seed run as one cooperative kernel when the frequency is
                             1 to 7 and nrhs <= 16, and their lockstep CG as one cooperative
                             kernel when at most 16 systems remain;
                             1: step kernels only;
                             2: as 0, and FP64 CG in one persistent kernel as well (nrhs <= 33).
                             With two or more systems and a frequency of 0 or >= 8 the seeding of
                             systems 2..p (Sec. 3) is folded into x^2..x^p once per
                             block of at most 128 steps instead of every step (same vectors, other
                             summation order). */
  int32_t precision;      /* 0 (default): FP64 throughout.
                             1: mixed.  Operator applies and Krylov vectors (V included) in FP32
                             (the context keeps an FP32 copy of the operator); every scalar of the
                             recurrences and every reduction in FP64.  The FP32 seed Lanczos seeds
                             all systems (the Sec. 3 algorithm, same stopping rule), the corrections
                             are added to X in FP64, then each system is finished by CG with FP32
                             iterations and FP64 reliable updates (x += the FP32 correction,
                             r = b - A x recomputed with the FP64 operator) until the FP64 true
                             residual meets its tolerance: tol_seed for system 1 (inside
                             seed_solve_first), tol_rest for the others.  The paper runs FP64 only;
                             this is the GPU extension.  seed_project and seed_get_basis use the
                             FP64 path only (SEED_ESTATE after a mixed seed solve). */
  int32_t autotune;       /* CSR contexts: 1 = time the sparse matrix-vector kernel's launch shapes
                             (threads per row 1/2/4/8, block size) on the matrix at creation and
                             keep the fastest (cached per process by size); 0 = one thread per row,
                             256-thread blocks.  Results are reproducible for a given shape. */
  double reliable_delta;  /* mixed only: a reliable update is made when the FP32 recursive residual
                             has fallen below reliable_delta times its value at the last update
                             (checked every 16 iterations), and whenever it meets the tolerance;
                             0 selects 0.001.  Range [0, 1). */
} seed_params;

/* Per right-hand side results. */
typedef struct {
  int32_t iters;          /* Lanczos steps (system 1) or CG iterations (systems 2..); mixed
                             precision: system 1 adds its refinement CG iterations */
  int32_t mvps;           /* applications of A, including true-residual checks (FP32 and FP64) */
  int32_t restarts;       /* CG restarts (systems 2..); mixed precision: FP64 reliable updates */
  int32_t converged;      /* 1 if the tolerance was met */
  double est_relres;      /* recursive residual estimate / ||b^j|| */
  double true_relres;     /* ||b^j - A x^j|| / ||b^j|| computed at the end */
} seed_info;

/* Counters over the life of a context. */
typedef struct {
  int64_t kernel_launches;   /* kernels of this library launched (including those inside CUDA graphs) */
  int64_t graph_launches;
  int64_t mvps;              /* operator applications */
  int64_t reorth_events;
  double ms_seed, ms_project, ms_rest;   /* device time of the last call of each kind */
  int32_t csr_tpr, csr_block;            /* CSR launch shape in use (threads per row, block size) */
} seed_stats;

int32_t seed_abi_version(void);

/* Fill p with defaults: m_max 1000, reorth_freq 0, passes 2, extra 0,
 * keep_basis 0, x0_zero 1, maxit_rest 100000, max_restarts 3, tol_seed 1e-12,
 * tol_rest 1e-8, breakdown_rel 1e-14, kernel_path 0, precision 0, autotune 0,
 * reliable_delta 0.  Returns SEED_EINVAL if p is NULL. */
seed_status seed_params_default(seed_params *p);

/* Create a context for a real CSR operator (dtype SEED_F64): the matrix A of
 * the systems A x^j = b^j, symmetric positive definite (Sec. 1).  Allocates
 * the Lanczos basis V (n x (m_max+1) doubles; Sec. 3 keeps the Lanczos vectors
 * of the seed system for reorthogonalization and notes that this storage can
 * be allocated and freed at run time) and work space on the current device.
 *   out: receives the context (NULL on failure).  A: host struct whose arrays
 *   are device pointers that must stay valid until seed_destroy.  p: host
 *   struct, copied.  stream: every later call on the context is ordered on it.
 * Returns SEED_OK, SEED_EINVAL (NULL argument, malformed CSR, bad parameter:
 * checked on the host before any device work), SEED_ENOMEM, SEED_ECUDA. */
seed_status seed_create_csr(seed_ctx **out, const seed_csr *A, const seed_params *p,
                            seed_stream stream);

/* Create a context for the Wilson normal operator A = D^H D (dtype SEED_C128):
 * Sec. 4 makes the non-Hermitian lattice system Hermitian positive definite by
 * multiplying it with D^H, so each iteration applies D twice.  Builds the
 * site -> 8 neighbour table on the device and allocates V and the work space
 * as seed_create_csr does (Sec. 3: basis storage allocated at run time).
 *   out, p, stream: as for seed_create_csr.  A: host struct; A->links is a
 *   device pointer that must stay valid until seed_destroy.
 * Returns SEED_OK, SEED_EINVAL (dims < 2, bc_t not 0/1, kappa not finite, bad
 * parameter), SEED_ENOMEM, SEED_ECUDA. */
seed_status seed_create_wilson(seed_ctx **out, const seed_wilson *A, const seed_params *p,
                               seed_stream stream);

/* Sec. 3, the Lanczos form of single-seed CG with periodic reorthogonalization,
 * on the first column of B, seeding columns 2..nrhs as the basis grows.
 *   B: n x nrhs (ldb), X: n x nrhs (ldx).  X in: initial guesses (ignored if
 *   x0_zero); X out: x^1 solved, x^2..x^nrhs seeded.  B and X must not overlap.
 *   info: NULL or nrhs entries; entry 0 receives the seed system's results
 *   (its true residual costs one mvp), the others are zeroed.
 * Returns SEED_OK (also for a lucky breakdown or when m_max is reached before
 * the tolerance, then info[0].converged = 0), SEED_ENOTSPD, SEED_EINVAL, ...
 * With keep_basis = 0 the basis is only valid until the next call. */
seed_status seed_solve_first(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx,
                             int32_t nrhs, seed_info *info);

/* Galerkin projection of further right-hand sides over the kept basis of the
 * last seed_solve_first (Sec. 2.1: seeding projects onto the Krylov subspace
 * built for the first system):  x += V T^{-1} V^H (b - A x).
 * Requires keep_basis = 1 (else SEED_ESTATE).  Costs ncols mvps unless
 * x0_zero, in which case X is overwritten. */
seed_status seed_project(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx,
                         int32_t ncols);

/* Plain CG (Sec. 1, Sec. 2.2: once seeded, the remaining systems are finished
 * by CG) on columns 2..nrhs of B from the seeded X, run
 * in lockstep with per-column scalars.  Column 1 (the seed system) is left
 * untouched.  Stops each column at ||r|| <= tol_rest ||b^j||, then checks the
 * true residual and restarts from it if it exceeds 1.5 tol_rest.
 * info: NULL or nrhs entries; entries 1..nrhs-1 are filled.
 * Returns SEED_OK, or SEED_ENOTCONV if some column hit maxit_rest. */
seed_status seed_solve_rest(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx,
                            int32_t nrhs, seed_info *info);

/* Sec. 2.3 (single seeding for related right-hand sides), after
 * seed_solve_first (which solves and seeds system 1) on the same B and X: the remaining systems are
 * projected over x^1 (x^1_bcg = 0, r^1_bcg = b^1); then for j = 2..nrhs, CG
 * runs on system j from its current approximation x^j_bcg (residual r^j_bcg)
 * to tol_rest, and every later system i receives the Galerkin projection over
 * the CG correction x_cg = x^j - x^j_bcg:
 *   delta = (x_cg^H r^i) / (x_cg^H r^j_bcg),  x^i += delta x_cg,  r^i -= delta r^j_bcg.
 * The systems are solved one after another (not in lockstep).  FP64 contexts
 * with x0_zero = 1 only (the paper assumes no initial guesses): SEED_EINVAL
 * otherwise; SEED_ESTATE before seed_solve_first.
 *   info: NULL or nrhs entries; entries 1..nrhs-1 are filled as by seed_solve_rest.
 * Returns SEED_OK or SEED_ENOTCONV. */
seed_status seed_solve_related(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx, int32_t nrhs,
                               seed_info *info);

/* Multiple seeding, the seed CG that Sec. 2.1 compares single seeding with:
 * the systems are solved in order by CG from zero (tol_rest); every CG step of
 * system j, with direction p and q = A p, also projects each later system i:
 *   eta = (p^H r^i) / (p^H q),  x^i += eta p,  r^i -= eta q  (r^i tracked).
 * Each system's CG starts from its projected x^j with the residual recomputed
 * (one mvp) and ends with a true-residual check (one mvp, no restart).  Kept
 * as the comparison baseline; FP64 contexts only.  X: out, all solutions;
 * info: NULL or nrhs entries (iters, mvps, converged, true_relres per system).
 * Returns SEED_OK or SEED_ENOTCONV. */
seed_status seed_solve_multiple(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx, int32_t nrhs,
                                seed_info *info);

/* Lockstep CG (Sec. 1; the iteration of seed_solve_rest) on ALL ncols columns
 * of B from the initial guesses in X, to ||b^j - A x^j|| <= tol_rest ||b^j||
 * (mixed-precision contexts: FP32 iterations with FP64 reliable updates).
 * This finishes systems whose guesses come from elsewhere, e.g. seed_project
 * over a kept basis (the backward solves of an adjoint, Sec. 2.1's projection
 * reused for new right-hand sides).  The paper has no separate entry for it.
 *   B, X: device, column-major n x ncols; X in = guesses, out = solutions.
 *   info: NULL or ncols entries.  Returns SEED_OK or SEED_ENOTCONV. */
seed_status seed_solve_cg(seed_ctx *ctx, const void *B, int64_t ldb, void *X, int64_t ldx, int32_t ncols,
                          seed_info *info);

/* Adjoint helper for Wilson contexts (no counterpart in the paper):
 *   *out = sum_j Re <Lambda_j, (dA/dkappa) X_j>,   A = D^H D, D = 1 - kappa H,
 * so dA/dkappa = -(H^H D + D^H H).  With x^j = A^{-1} b^j, a real loss L and
 * lambda^j = A^{-1} (dL/dx^j) (the conjugate-Wirtinger gradient convention),
 * dL/dkappa = -(*out).  Lambda, X: device, column-major n x ncols (complex
 * double).  Synchronises.  SEED_EINVAL on a CSR context. */
seed_status seed_grad_kappa(seed_ctx *ctx, const void *Lambda, int64_t ldl, const void *X, int64_t ldx,
                            int32_t ncols, double *out);

/* Y = op(X) for ncols columns: op 0 = A; for Wilson contexts op 1 = D and
 * op 2 = D^H (used e.g. to form normal-equation right-hand sides b = D^H eta,
 * Sec. 4).  On a mixed-precision context ops 3 = A, 4 = D, 5 = D^H apply the
 * FP32 copy of the operator to FP32 data (float, or interleaved complex float
 * for Wilson), the arithmetic of the mixed solver's iterations.  On a
 * mixed-precision Wilson context ops 6 = D and 7 = D^H take X and Y in the
 * solver's own tiled FP32 layout, the layout and launch of its iterations and
 * of seed_time_operator: component k = 3*spin + colour of site s at complex
 * index ((s / 32) * 12 + k) * 32 + s % 32 of a column of length
 * 384 * ceil(sites / 32) (ldx, ldy >= that length); the padding sites of the
 * last tile are written as zeros.  X and Y must not overlap.  Not
 * synchronising. */
seed_status seed_apply(seed_ctx *ctx, int32_t op, const void *X, int64_t ldx, void *Y, int64_t ldy,
                       int32_t ncols);

/* Failure detection, tested without a GPU fault.
 *
 * seed_inject_alloc_failure: host-side fault injection.  The k-th device
 * allocation the library makes from now on (k = 1: the next one) fails as if
 * cudaMalloc had run out of memory, without calling it; the call that needed
 * it returns SEED_ENOMEM.  A failed seed_create_* frees what it had
 * allocated; a failed call on a context leaves the context valid, and a later
 * call allocates what is still missing.  k <= 0 disarms.  Process-wide (all
 * threads and contexts).  Returns the previous countdown.
 *
 * seed_check_barrier_timeout: self-test of the bounded wait of the persistent
 * kernels' grid barriers.  Launches two blocks at a barrier that can never
 * complete (its arrival target is one epoch ahead), so that every wait runs
 * out after its limit (2 s) and the kernel returns with the error flag set --
 * the flag the persistent solves turn into SEED_ETIMEOUT.  On SEED_OK,
 * *timed_out = 1 when the wait gave up as designed (0 would mean a barrier
 * completed that cannot complete) and *ms = the kernel's device time.  Enqueued
 * on `stream`, synchronises it; the device stays usable afterwards.
 * SEED_ECUDA without cooperative launch support. */
int32_t seed_inject_alloc_failure(int32_t k);
seed_status seed_check_barrier_timeout(seed_stream stream, int32_t *timed_out, double *ms);

/* Build the site -> neighbour table for a lattice on the device:
 * nbr[8*s + 2*mu] = s + mu-hat, nbr[8*s + 2*mu + 1] = s - mu-hat (periodic
 * wrap), s = x + X*(y + Y*(z + Z*t)).  nbr: device, 8*sites int32.
 * Synchronises the stream.  This is the table the Wilson kernels use. */
seed_status seed_wilson_neighbors(const int32_t dims[4], int32_t *nbr, seed_stream stream);

/* Tridiagonal T of the last seed solve (the Lanczos coefficients of Sec. 3):
 * alpha[0..m-1] = alpha_1..alpha_m, beta[0..m] = beta_0..beta_m (beta_0 =
 * ||r_0^1||), host arrays of capacity cap >= m+1; *m receives the number of
 * Lanczos steps.  With alpha and beta both NULL only *m is returned.
 * SEED_ESTATE before the first seed_solve_first. */
seed_status seed_get_tridiag(const seed_ctx *ctx, double *alpha, double *beta, int32_t cap,
                             int32_t *m);

/* Copy the first ncols Lanczos vectors (column-major, ld = n, host memory).
 * SEED_ESTATE on a mixed-precision context (its basis is FP32). */
seed_status seed_get_basis(const seed_ctx *ctx, void *V_host, int32_t ncols);

seed_status seed_get_stats(const seed_ctx *ctx, seed_stats *out);

/* Batched uneven problems (no counterpart in the paper): for each problem i,
 * seed_solve_first then seed_solve_rest on ctxs[i] with B[i], X[i] (ldb[i],
 * ldx[i], nrhs[i] columns, info[i] NULL or nrhs[i] entries), all problems
 * concurrently on the GPU.  Every context has its own stream; a pool of
 * `workers` host threads (0 = min(nprob, 32)) drives the solves, largest
 * problem (n x nrhs) first, so the launches and CUDA graphs of many small
 * problems overlap on the GPU instead of running one after another.  The
 * contexts must be distinct and must not be used by other threads meanwhile.
 * Each problem runs the arithmetic of a solo solve on its context: the
 * persistent seed runs of kernel_path 0 and 2 and the one-launch CG of small
 * CSR problems run side by side (each waits only on its own blocks), while
 * the persistent FP64 CG of kernel_path 2 is replaced inside a batch by the
 * CG of kernel_path 0.  So each problem's results are bitwise those of a solo
 * solve with its kernel_path (0 for a kernel_path 2 context).  Returns SEED_OK, or the
 * status of the first failing problem (in problem order; the others still
 * run), with seed_last_error(NULL) naming it. */
seed_status seed_batch_solve(seed_ctx *const *ctxs, const void *const *B, const int64_t *ldb, void *const *X,
                             const int64_t *ldx, const int32_t *nrhs, int32_t nprob, int32_t workers,
                             seed_info *const *info);

/* Measurement helper (not part of the method): launch op(X) (op as in
 * seed_apply; on a mixed-precision context also 3 = A, 4 = D, 5 = D^H with the
 * FP32 copy of the operator on FP32 columns filled with the byte 0x3F, floats
 * near 0.75) reps times back to back on the context's internal stream over
 * ncols library-owned columns (filled with the byte 0x3F, i.e. normal
 * doubles near 4.8e-4), with CUDA events on that stream
 * around the launches; *ms_per_apply receives the mean device time of one
 * application.  Synchronises.  reps in [1, 100000], ncols in [1, 64]. */
seed_status seed_time_operator(seed_ctx *ctx, int32_t op, int32_t ncols, int32_t reps, double *ms_per_apply);

/* Measurement helper (no counterpart in the paper): the FMA rate of the FP64
 * (dtype SEED_F64) or FP32 (SEED_F32) pipe of the current device, the
 * roofline denominator of the kernels bound by that pipe (the FP64 Wilson
 * operator).  Every thread of a grid of 8 blocks of 256 threads per SM runs 8
 * independent chains of 4096 fused multiply-adds; *tflops = 2 x FMAs / time
 * of the fastest of five launches (CUDA events on `stream`, after one
 * warm-up); *ms (may be NULL) that launch's time.  Allocates no device
 * memory; synchronises `stream`.  SEED_EINVAL for another dtype or a NULL
 * tflops, SEED_ECUDA without a usable device. */
seed_status seed_time_fma(int32_t dtype, seed_stream stream, double *tflops, double *ms);

/* Measurement helper (no counterpart in the paper): whether the FP64 matrix
 * instructions (mma.sync f64, "DMMA") offer FP64 throughput beyond the FMA pipe
 * that bounds the FP64 Wilson operator (Sec. 4) and the FP64 contractions of
 * Sec. 3.  Fills out[7] (host):
 *   out[0] FP64 FMA chains, TFLOP/s; out[1] DMMA m8n8k4, TFLOP/s;
 *   out[2] DMMA m16n8k16, TFLOP/s (all warps of a full grid in one role);
 *   out[3] t_mix / (t_fma + t_mma): the launch with half the warps on FMA
 *     chains and half on m8n8k4 against the two halves launched alone --
 *     about 0.5 if the two run on separate units, about 1 if they share one;
 *   out[4..6] t_fma, t_mma, t_mix in ms (fastest of five after a warm-up).
 * Allocates no device memory; synchronises `stream`.  SEED_EINVAL for a NULL
 * out, SEED_ECUDA without a usable device. */
seed_status seed_time_fp64_paths(seed_stream stream, double *out);

/* Validation and measurement helper (no counterpart in the paper as an entry
 * point): the products of the mixed-precision seeding, G = V^H R (Sec. 3: each
 * Lanczos vector projected onto every other right-hand side), computed the way
 * a mixed-precision Wilson context folds a block of steps -- on the tensor cores
 * (tcgen05, TF32 with each FP32 operand split into a rounded part and its
 * remainder, FP32 accumulation over 512 elements, FP64 above), operands staged
 * by TMA, partials summed over CTAs in a fixed order.
 *   V: device, FP32 complex (SEED_C64), n x k column-major (ldv); R: n x nr
 *   (ldr); both 16-byte aligned, ldv and ldr even and >= n; n a positive
 *   multiple of 128; k in [1, 128], nr in [1, 63].
 *   G: host, k x nr complex double, row-major (G[2*(q*nr + j)] = Re g_qj).
 *   reps: timed launches of the product kernel after one untimed one; *ms (may
 *   be NULL): mean device time of one launch (CUDA events on `stream`).
 * Allocates its scratch (the per-CTA partials), synchronises `stream`.
 * SEED_EINVAL for bad sizes, SEED_ECUDA without a usable device or TMA,
 * SEED_ETIMEOUT if a wait of the kernel ran past its 2 s limit. */
seed_status seed_block_products(const void *V, int64_t ldv, int32_t k, const void *R, int64_t ldr, int32_t nr,
                                int64_t n, double *G, int32_t reps, double *ms, seed_stream stream);

/* Y = D^H D X (the Wilson normal operator, as seed_apply op 0 on a Wilson
 * context) WITHOUT allocating any device memory.  The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc while they
 * run -- a host loop being captured into a CUDA graph, a service whose device
 * memory is fixed at start-up, a plug-in in a framework that owns the device
 * heap -- and therefore cannot create a context.
 *   A: operator description (links: device pointer); X, Y: device, column-major
 *   n x ncols (n = 12 * sites), ld >= n, must not overlap.  Work is enqueued on
 *   `stream`; the call does not synchronise.
 * Scratch: the neighbour table and the intermediate D X live in one fixed
 * 8 MiB (8388608-byte) device array that every GPU loading this library holds
 * until the process exits.  A call needs 256-byte-rounded 32*sites bytes plus
 * 16*n*ncols bytes and is rejected with SEED_EINVAL beyond 8 MiB (e.g. an 8^4
 * lattice allows up to 10 columns).  The array is shared by all calls and keeps
 * the last call's contents (each call overwrites what it reads, so nothing
 * needs clearing); calls whose work overlaps on the GPU (other streams, or
 * other host threads) race on it -- serialise them.  The call runs in the
 * CUDA context current on the calling thread (the device's primary context
 * unless the caller made another one current); the first call on each device
 * and context looks up the array's device address there
 * (cudaGetSymbolAddress, with that device current) and keeps it, and a later
 * call from another context (after cudaDeviceReset, or a driver context of the
 * caller's) looks it up again.  Make that first call before any stream
 * capture.  Never calls cudaMalloc, cudaFree or any allocating routine. */
seed_status seed_wilson_apply_noalloc(const seed_wilson *A, const void *X, int64_t ldx, void *Y, int64_t ldy,
                                      int32_t ncols, seed_stream stream);

/* One-line reason for the last failure on ctx (or of the last failed
 * seed_create_* / context-free call on this thread when ctx is NULL).  The
 * paper has no counterpart: this is the library's error reporting.  The
 * string is owned by the library and valid until the next call on ctx (or,
 * for NULL, on this thread); never NULL. */
const char *seed_last_error(const seed_ctx *ctx);

/* Free V, the work space and the context (Sec. 3: the Lanczos vectors are
 * needed only while the seed system is solved and seeds the others, and their
 * storage can be released at run time; keep_basis = 1 keeps it until here).
 * Never frees the caller's arrays.  NULL-safe.  Synchronises the context's
 * stream; no status (nothing can be reported after the context is gone). */
void seed_destroy(seed_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* SEED_H_ */
