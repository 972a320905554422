/*
 * slrf.h -- C ABI of the GB300 (sm_103a) shifted Laplace rational-filter
 * eigensolver for the symmetric-definite pencil A x = lambda B x
 * (A, B real, sparse, symmetric positive definite; eigenpairs wanted in
 * (0, gamma]; Section 1, Eq. (1)).
 *
 * General conventions
 * -------------------
 * - Every function returns an slrf_status; nothing aborts or exits.
 * - Dense blocks are ROW-MAJOR n x m: element (i, c) of V lives at
 *   V[i * ldv + c], ldv >= m.  (A torch tensor of shape [n, m] is exactly
 *   this with ldv = m.)
 * - "device" pointers are CUDA global-memory pointers on the handle's device;
 *   "host" pointers are ordinary CPU memory.  Each argument says which.
 * - The caller owns every buffer it passes.  The handle owns its device copy
 *   of the pencil and all workspace (released by slrf_destroy).
 * - Work is enqueued on the CUDA stream given to slrf_create.  Functions that
 *   return results to host memory synchronise that stream before returning;
 *   functions that write device outputs return after enqueuing, and outputs
 *   are valid once the stream has been synchronised.
 * - A filter is given by N poles sigma_j in the upper half plane and weights
 *   w_j; the conjugate poles and weights are implied (Section 3, conjugate
 *   pair reduction), so the filter is
 *       Phi(A, B) = sum_{j=1}^{N} 2 Re( w_j (A - sigma_j B)^{-1} B ).
 *   Any pole set may be passed: the shifted-Laplace (SLRF) design of
 *   Section 3.1 and the circle quadrature rules of Section 3.2 are
 *   interchangeable.
 */
#ifndef SLRF_H
#define SLRF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SLRF_OK = 0,
    SLRF_EINVAL = 1,              /* invalid argument (sizes, pointers, NaN input)   */
    SLRF_ENOMEM = 2,              /* device allocation failed                        */
    SLRF_EBUDGET = 3,             /* workspace would exceed opts.mem_budget          */
    SLRF_ECUDA = 4,               /* a CUDA call failed (see slrf_last_error)        */
    SLRF_ETIMEOUT = 5,            /* a bounded device wait gave up                   */
    SLRF_NOT_CONVERGED = 6,       /* outer iteration cap reached; outputs written    */
    SLRF_STAGNATION = 7,          /* residuals stopped decreasing; outputs written   */
    SLRF_BREAKDOWN = 8,           /* Krylov breakdown in every remaining column      */
    SLRF_SUBSPACE_TOO_SMALL = 9,  /* all L Ritz values lie in (0, gamma]             */
    SLRF_CHOLQR_FAIL = 10,        /* B-Gram matrix not numerically positive definite */
    SLRF_PENDING = 11             /* server request not finished yet                 */
} slrf_status;

typedef struct slrf_handle slrf_handle;

/* Sparse pencil in CSR form on ONE shared (union) pattern; explicit zeros
 * allowed.  Column indices sorted within each row.  A = stiffness, B = mass.
 * Pointers are host memory if on_device == 0, device memory if 1.  The data
 * is copied into the handle by slrf_create; the caller may free it after. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const int32_t *row_ptr;   /* n + 1 */
    const int32_t *col_idx;   /* nnz   */
    const double *a_val;      /* nnz   */
    const double *b_val;      /* nnz   */
    int32_t on_device;
} slrf_pencil;

/* Upper-half-plane poles and weights, host arrays of length n_poles
 * (1 <= n_poles <= SLRF_MAX_POLES).  Im(sigma_j) must be nonzero. */
#define SLRF_MAX_POLES 16
typedef struct {
    int32_t n_poles;
    const double *sigma_re;
    const double *sigma_im;
    const double *w_re;
    const double *w_im;
} slrf_filter;

enum { SLRF_PREC_FP64 = 0,  /* plain: FP64 Krylov to inner_tol relative to ||B v||        */
       SLRF_PREC_MIXED = 1  /* FP32 Krylov on the FP64 residual R = B X Theta - A X      */ };
/* COCG: conjugate-orthogonal CG (unconjugated bilinear form; needs a complex
 * symmetric preconditioner), one shifted product and one preconditioner
 * application per iteration.  BICGSTAB: right-preconditioned BiCGStab with
 * Hermitian products (the paper's solver, Section 4.2.1), two of each per
 * iteration; slrf_report.spmv counts both products. */
enum { SLRF_KRYLOV_COCG = 0, SLRF_KRYLOV_BICGSTAB = 1 };
/* Preconditioner of the shifted solves.  JACOBI: diag(A - sigma_j B).  MG:
 * smoothed-aggregation multigrid cycle (one hierarchy for all poles, built
 * from A; Galerkin pencils (P^T A P, P^T B P) on every level; damped Jacobi
 * smoothing; exact coarsest solve by the eigendecomposition of the coarsest
 * pencil).  AUTO: MG for scalar pencils, JACOBI for 3-dof node-block
 * (elasticity) pencils, where the hierarchy's translation-only aggregates do
 * not pay off for shifts deep inside the spectrum.  The paper's own solver
 * is ILU-preconditioned BiCGStab (Section 4.2.1); every option keeps the
 * preconditioner complex symmetric, as COCG requires. */
enum { SLRF_PRECOND_NONE = 0, SLRF_PRECOND_JACOBI = 1, SLRF_PRECOND_MG = 2, SLRF_PRECOND_AUTO = 3,
       SLRF_PRECOND_ILU = 4 };
/* ILU: incomplete factorisation of each shifted matrix A - sigma_j B on the
 * pencil's own pattern (no fill), in the symmetric form L D L^T (L unit lower
 * triangular, unconjugated transpose), built on the GPU per solve by
 * ilu_sweeps fixed-point (Chow-Patel) sweeps from L = strict lower part
 * scaled by the diagonal, D = diag; applied as z = P^T D^{-1} P r with
 * P = I - N + N^2 - ... (ilu_tri_sweeps Jacobi sweeps of each triangular
 * solve, N = L - I), a fixed complex symmetric operator.  The paper's solver
 * is BiCGStab with ILU (drop tolerance 1e-4, RCM order; Section 4.2.1);
 * this is its GPU-native no-fill form (no sequential triangular solves). */
enum { SLRF_RULE_MIDPOINT = 0, SLRF_RULE_GAUSS_LEGENDRE = 1, SLRF_RULE_GAUSS_CHEBYSHEV = 2,
       SLRF_RULE_SLRF = 3 };

typedef struct {
    int32_t precision;      /* SLRF_PREC_*                                     (MIXED) */
    int32_t krylov;         /* SLRF_KRYLOV_*                                    (COCG) */
    int32_t precond;        /* SLRF_PRECOND_*                                   (AUTO) */
    int32_t inner_maxit;    /* Krylov iteration cap per outer step, Section 4.2.1 (1000) */
    double inner_tol;       /* FP64: rel. to ||B v||, Section 4.2.1 (1e-13);
                               MIXED: rel. to ||R column||                      (1e-5) */
    double lock_tol;        /* MIXED: columns with rho_i below this skip the solve
                               (their correction is below the outer tolerance) (1e-9) */
    int32_t check_every;    /* Krylov iterations between host polls of the
                               active-column count                               (4) */
    int32_t eig_refine;     /* small eigensolver of the projected problem (m <= 160;
                               larger m always take 0): 2 = FP32 Jacobi, then
                               three FP64 refinement steps X <- X (I + E) built
                               from the products X^T X and X^T S X (Ogita-Aishima),
                               and FP64 Jacobi inside groups of nearly equal
                               eigenvalues; 1 = FP32 Jacobi, FP64 re-orthonormal-
                               isation and an FP64 Jacobi polish of the whole
                               matrix; 0 = FP64 Jacobi                          (2) */
    int64_t mem_budget;     /* workspace byte cap, 0 = none                       (0) */
    int32_t profile;        /* 1: time kernel classes with CUDA events around
                               each launch (those selected by profile_mask)      (0) */
    int32_t spmm_rows;      /* rows per group of the shifted SpMM (1..4); 0 = auto:
                               3 for 3-dof node-block patterns, else 2             (0) */
    int32_t gram_ozaki;     /* Grams and tall products (Q1 = U T1, X = Q1 M) of the
                               projection step, FP64-accurate from exact integer
                               digit products (Ozaki splitting): 2 = Grams on the
                               tcgen05 tensor cores (bf16 digits, FP32 TMEM
                               accumulators), tall products as with 1; 1 = int8
                               mma.sync digits for both; 0 = FP64 CUDA cores    (2) */
    int32_t mg_nu;          /* MG: Jacobi sweeps per side on the levels below the
                               finest (the finest always takes one); 0 = one when
                               the FP32 cycle ends at the mg_exact level, else
                               two                                                 (0) */
    int32_t mg_cycle;       /* MG: coarse visits per level, 1 = V-, 2 = W-cycle    (1) */
    int32_t mg_coarse;      /* MG: coarsening stops at or below this size         (256) */
    int32_t mg_block;       /* MG: dofs per node for aggregation, 0 = auto (3 for
                               3-dof node-block patterns, else 1)                   (0) */
    double mg_omega;        /* MG: Jacobi damping relative to the spectral radius:
                               level l smooths with mg_omega / rho(D_l^-1 A_l),
                               0 < mg_omega < 2                                  (4/3) */
    double mg_theta;        /* MG: strength-of-connection threshold of the
                               aggregation, 0 = 0.08                                (0) */
    double mg_shift_limit;  /* MG: a level is smoothed only while
                               max_j |sigma_j| max_i b_ii / a_ii <= this; the first
                               level beyond it is solved exactly (its eigen-
                               decomposition is computed on first use, up to 768
                               unknowns; beyond that AUTO falls back to Jacobi
                               for the solve)                                    (0.8) */
    int32_t stagnation_window; /* outer steps without a 10% drop of the largest
                               wanted residual (of all Ritz pairs while none is
                               wanted) after which slrf_subspace_iterate stops
                               with SLRF_STAGNATION; 0 = never                  (8) */
    uint32_t profile_mask;  /* profile == 1: bit c times kernel class c
                               (slrf_kernel_class_name), 0 = every class; timing
                               fewer classes records fewer events               (0) */
    int32_t spmm_kernel;    /* FP32 shifted product kernel: 1 = row groups gathered
                               through L1/L2 by every warp; 2 = staged: a producer
                               warp moves the gathered rows into shared memory by
                               bulk copies (TMA engine) and consumer warps only
                               multiply; 3 = node blocks (3-dof pencils whose
                               nodes' rows share one pattern of whole neighbour
                               nodes and whose mass couples equal dofs only, as
                               consistent vector-element mass does): one index
                               and one 3 x 3 stiffness block per neighbour node,
                               the zero off-dof mass entries skipped; a pencil
                               not of that form runs kernel 1; 4 = SELL-C-sigma
                               (sell_c, sell_sigma): one warp per permuted row
                               walking its chunk's slot-major entries; 0 = chosen per
                               pattern and column count by timing the available
                               kernels on the first solve (the choice is kept
                               for the process; the kernels differ only in the
                               rounding order of their sums)                 (0) */
    int32_t mg_exact;       /* MG, FP32 Krylov: the first level below the finest with
                               at most this many unknowns (above the coarsest) ends
                               the cycle and is solved exactly by its dense shifted
                               inverses (A_l - sigma_j B_l)^{-1}, formed per solve on
                               the GPU (N n_l^2 complex FP32 values); 0 = off, the
                               cycle then descends to the coarsest level     (1536) */
    int32_t ilu_sweeps;     /* ILU: fixed-point sweeps building the factors     (3) */
    int32_t ilu_tri_sweeps; /* ILU: Jacobi sweeps of each triangular solve      (3) */
    int32_t sell_c;         /* SELL-C-sigma form of the pencil (spmm_kernel 4):
                               rows per chunk, one of 4, 8, 16, 32, 64; 0 = 32 */
    int32_t sell_sigma;     /* SELL-C-sigma: rows are sorted by length within
                               windows of this many rows (1 = natural order);
                               0 = 256                                         */
    int32_t mg_exact_tc;    /* mg_exact level: 1 = apply the inverses on the
                               tcgen05 tensor cores (three-way bf16 split of both
                               operands, FP32 accumulation: FP32-accurate; needs
                               subspace size <= 256), 0 = cuBLAS FP32 complex
                               GEMM                                           (1) */
    int32_t mg_n_null;      /* MG: columns of mg_near_null, 0..16; 0 = none  (0) */
    const double *mg_near_null; /* MG: host n x mg_n_null row-major near-null
                               space of A for the aggregation (e.g. the six
                               rigid-body modes of a 3-dof elasticity pencil,
                               with mg_block 3 or auto): each aggregate's block
                               of the tentative prolongator is the Q factor of
                               its rows, and the next level has mg_n_null dofs
                               per node.  Read and copied by the call that takes
                               the options (create, set_opts, server submit,
                               mg_describe, mg_transfer): it need not outlive
                               it.  Entries must be finite.  Used only where the
                               preconditioner resolves to multigrid (AUTO keeps
                               Jacobi on 3-dof node-block pencils).   (NULL) */
} slrf_opts;

/* Counters of one call.  Krylov iteration counts follow Table 4/5 of the
 * paper: spmv counts one shifted product per (pole, column). */
#define SLRF_NKERNEL_CLASSES 15
typedef struct {
    int32_t outer_iters;          /* filter applications                         */
    int32_t n_wanted;             /* Ritz values in (0, gamma]                   */
    int32_t n_conv;               /* of those, rho_i <= tol                      */
    int32_t status_detail;
    double max_resid;             /* max rho_i over wanted Ritz pairs            */
    double max_resid_ax;          /* max ||A x - theta B x|| / ||A x|| (wanted)  */
    int64_t krylov_iters;         /* Krylov iterations summed over outer steps   */
    int64_t spmv;                 /* shifted SpMV column-products (Table 5)      */
    double iters_per_pole[SLRF_MAX_POLES]; /* mean iterations per column (Table 4) */
    int64_t kernel_launches;      /* kernels launched by this call               */
    double ms_total;              /* device time of the call (events)            */
    double ms_krylov;             /* device time inside the Krylov phases        */
    double ms_rr;                 /* device time inside orthonormalisation + RR  */
    /* per kernel class (profile == 1): launches, summed device ms, algorithmic
     * bytes and flops per class; class names from slrf_kernel_class_name(). */
    int64_t k_launches[SLRF_NKERNEL_CLASSES];
    double k_ms[SLRF_NKERNEL_CLASSES];
    double k_bytes[SLRF_NKERNEL_CLASSES];
    double k_flops[SLRF_NKERNEL_CLASSES];
    int32_t mg_levels;            /* multigrid levels of the last Krylov solve
                                     (0: Jacobi or no preconditioner)           */
    int32_t krylov_fp64;          /* MIXED: 1 if the solve switched its Krylov
                                     solves to FP64 after the FP32 ones stagnated */
    int32_t spmm_kernel;          /* FP32 shifted product kernel used (the value
                                     of slrf_opts.spmm_kernel, resolved when 0) */
} slrf_report;

/* ---- library -------------------------------------------------------- */

/* Human-readable name of a status. Never NULL. */
const char *slrf_status_str(slrf_status s);
/* Text of the last CUDA error seen by this thread ("" if none). */
const char *slrf_last_error(void);
/* Device memory of handles comes from one pool per device that keeps what
 * destroyed handles release reserved for later handles of the process (so
 * creating the next handle maps no new memory).  This returns the unused
 * part of device `device`'s pool to the driver; memory held by live handles
 * stays.  SLRF_OK also when the pool was never created; SLRF_ECUDA if the
 * trim fails. */
slrf_status slrf_release_cached_memory(int32_t device);
/* Name of a kernel class index of slrf_report.k_*; NULL if out of range. */
const char *slrf_kernel_class_name(int32_t k);
/* Fill *o with the defaults listed in slrf_opts. */
slrf_status slrf_opts_default(slrf_opts *o);

/* ---- handle ---------------------------------------------------------- */

/* Create a handle: validate the pencil (n >= 1, CSR monotone, indices in
 * range, finite values), copy it to the current CUDA device in the layouts the
 * kernels use, and bind `cuda_stream` (a cudaStream_t, NULL = legacy default
 * stream).  When the preconditioner resolves to multigrid (MG, or AUTO on a
 * scalar pencil) the hierarchy is built here (host) and uploaded.  Problem statement: Section 1, Eq. (1). */
slrf_status slrf_create(slrf_handle **h, const slrf_pencil *p, const slrf_opts *o,
                        void *cuda_stream);
/* Replace the handle's options (workspace is resized lazily; switching to
 * SLRF_PRECOND_MG or changing mg_coarse / mg_block / mg_theta / the near-null
 * space rebuilds the multigrid hierarchy on the next solve). */
slrf_status slrf_set_opts(slrf_handle *h, const slrf_opts *o);
/* Release the handle and all its device memory.  NULL is ignored. */
void slrf_destroy(slrf_handle *h);

/* ---- the hot path ----------------------------------------------------- */

/* U = sum_j 2 Re(w_j (A - sigma_j B)^{-1} B V)  (Section 3; Algorithm 1, the
 * solve loop and the accumulation).  V, U: device, n x m row-major.  The N*m
 * shifted systems are solved by preconditioned COCG (opts.precond) in the
 * handle's precision to opts.inner_tol relative residual (FP64: Section 4.2.1 uses
 * 1e-13).  In MIXED precision the solves run in FP32, so U is accurate to
 * about kappa(A - sigma B) * max(inner_tol, 1e-7); slrf_subspace_iterate
 * recovers FP64 accuracy by filtering the FP64 residual instead.  Returns
 * SLRF_NOT_CONVERGED (with U written) if some system missed its tolerance. */
slrf_status slrf_filter_apply(slrf_handle *h, const slrf_filter *f, const double *V, int64_t ldv,
                              int32_t m, double *U, int64_t ldu, slrf_report *rep);

/* Algorithm 1: rational-filter subspace iteration from the start block V0
 * (device, n x L row-major) until every Ritz value in (0, gamma] has
 * rho_i = ||A x_i - theta_i B x_i|| / (|theta_i| ||B x_i||) <= tol, or
 * max_outer filter applications.  Outputs (device): theta[L] ascending,
 * X (n x L, B-orthonormal), resid[L] = rho_i; host: *n_conv.  Each outer step
 * is filter -> B-orthonormalisation (Cholesky-QR2) -> Rayleigh-Ritz ->
 * residuals.  MIXED runs the filter on R = B X Theta - A X (FP64) with FP32
 * Krylov, using U = X Phi(Theta) + sum_j 2 Re(w_j (A - sigma_j B)^{-1} R D_j),
 * D_j = (Theta - sigma_j)^{-1}, an identity of the filter operator.
 * Returns SLRF_OK, or NOT_CONVERGED / SUBSPACE_TOO_SMALL / CHOLQR_FAIL /
 * STAGNATION (opts.stagnation_window) with the outputs of the last completed
 * step written. */
slrf_status slrf_subspace_iterate(slrf_handle *h, const slrf_filter *f, double gamma, int32_t L,
                                  const double *V0, int64_t ldv, double tol, int32_t max_outer,
                                  double *theta, double *X, int64_t ldx, double *resid,
                                  int32_t *n_conv, slrf_report *rep);

/* Same as slrf_subspace_iterate with HOST buffers for V0, theta, X, resid:
 * copies V0 in and the results out on the handle's stream (synchronised). */
slrf_status slrf_subspace_iterate_host(slrf_handle *h, const slrf_filter *f, double gamma,
                                       int32_t L, const double *V0, int64_t ldv, double tol,
                                       int32_t max_outer, double *theta, double *X, int64_t ldx,
                                       double *resid, int32_t *n_conv, slrf_report *rep);

/* ---- individual steps (each row of the hot path, for testing/measuring) -- */

/* Q_j = (A - sigma_j B) P_j for every pole j and column: P, Q device complex
 * blocks of n x (N*ldp) interleaved (re, im) in the handle's precision
 * (float pairs if prec == SLRF_PREC_MIXED, double pairs if FP64), pole j
 * occupying columns [j*ldp, j*ldp + m).  ldp must be even.  Also returns
 * mu[j*m + c] = sum_i P_j[i,c] Q_j[i,c] (unconjugated, device complex, same
 * precision) if mu != NULL.  (Eq. (2) operator; the Krylov matrix product.) */
slrf_status slrf_shifted_spmm(slrf_handle *h, const slrf_filter *f, int32_t prec, int32_t m,
                              int32_t ldp, const void *P, void *Q, void *mu);

/* Z_j = C_j R_j for every pole j and column, where C_j is the preconditioner
 * of the shifted system (A - sigma_j B) y = f (Section 4.2.1 preconditions
 * the Krylov solves of Eq. (2)) that the handle's Krylov solves use with its
 * options: one multigrid cycle (SLRF_PRECOND_MG, and AUTO where it picks
 * multigrid; the deep-shift truncation applies), Jacobi
 * diag(A - sigma_j B)^{-1} (JACOBI, and AUTO otherwise) or the identity
 * (NONE).  R, Z: device complex blocks in the layout of slrf_shifted_spmm
 * (prec, m, ldp as there); only the columns c < m of each pole are defined
 * in Z on return.
 * mu[j*m + c] = sum_i R_j[i,c] Z_j[i,c] (unconjugated, device) if mu != NULL.
 * *mg_levels (if not NULL) receives the number of levels the cycle used
 * (0: no multigrid).  Synchronous.  SLRF_EINVAL for bad sizes or filter,
 * SLRF_BREAKDOWN if the hierarchy cannot be built. */
slrf_status slrf_precond_apply(slrf_handle *h, const slrf_filter *f, int32_t prec, int32_t m,
                               int32_t ldp, const void *R, void *Z, void *mu, int32_t *mg_levels);

/* Y = A X and/or Z = B X (FP64, device, row-major n x m; either output may be
 * NULL).  Algorithm 1 products A U, B U, A X, B X. */
slrf_status slrf_spmm_ab(slrf_handle *h, int32_t m, const double *X, int64_t ldx, double *Y,
                         int64_t ldy, double *Z, int64_t ldz);

/* G = X^T Y (m x m row-major, device), X, Y device n x m row-major FP64.
 * The projected matrices A_hat = U^T A U, B_hat = U^T B U of Algorithm 1. */
slrf_status slrf_gram(slrf_handle *h, int32_t m, const double *X, int64_t ldx, const double *Y,
                      int64_t ldy, double *G);

/* C = A B (device, row-major): A n x k with n = the handle's pencil size, B
 * k x m, C n x m; FP64-accurate (the Ozaki digit products of opts.gram_ozaki:
 * 2 = tcgen05 for k <= 512, else int8 mma.sync; 0 = FP64 GEMM).  The tall
 * products Q1 = U T1 and X = Q1 M of Algorithm 1's orthonormalisation and
 * Ritz vectors.  SLRF_ETIMEOUT if a bounded device wait gave up. */
slrf_status slrf_tall_product(slrf_handle *h, int32_t k, int32_t m, const double *A, int64_t lda, const double *B,
                              int64_t ldb, double *C, int64_t ldc);

/* Symmetric eigendecomposition of the m x m row-major device matrix S:
 * S = Q diag(lam) Q^T, lam ascending (device), Q device row-major (columns are
 * eigenvectors).  The small eigenproblem of Algorithm 1 after
 * B-orthonormalisation (m <= 1024). */
slrf_status slrf_syev(slrf_handle *h, int32_t m, const double *S, double *lam, double *Q);

/* Rayleigh-Ritz of span(U) (device n x m): B-orthonormalise by Cholesky-QR2,
 * project A, solve the small eigenproblem; returns theta (device, ascending),
 * X = U S (device, B-orthonormal), and resid = rho_i (device).  Algorithm 1,
 * projection, small eigenproblem and residual steps. */
slrf_status slrf_rayleigh_ritz(slrf_handle *h, int32_t m, const double *U, int64_t ldu,
                               double *theta, double *X, int64_t ldx, double *resid);

/* ---- many problems ---------------------------------------------------------- */

/* Algorithm 1 for nprob independent problems at once.  Problem i uses handle
 * h[i] (all distinct; create each on its own CUDA stream so that the problems'
 * kernels overlap), filter f[i], interval (0, gamma[i]], subspace size L[i] and
 * the device buffers V0[i] (ld ldv[i]), theta[i], X[i] (ld ldx[i]), resid[i],
 * with the layouts of slrf_subspace_iterate.  n_threads host threads drive
 * the problems (<= 0: one per problem).  status[i] and n_conv[i] (and rep[i]
 * if rep != NULL) receive each problem's outcome.  Returns SLRF_OK if every
 * problem returned SLRF_OK, else the first other status.  All reductions run
 * in a fixed order, so each problem's outputs are bit-identical to solving it
 * alone.  With the environment variable SLRF_DEBUG set, the error text of
 * every problem that did not return SLRF_OK is printed to stderr (the text of
 * slrf_last_error() belongs to the worker thread).  (Many independent
 * pencils solved concurrently on one GPU; the paper solves one pencil at a
 * time, Section 4.) */
slrf_status slrf_batch_iterate(int32_t nprob, slrf_handle *const *h, const slrf_filter *f,
                               const double *gamma, const int32_t *L, const double *const *V0,
                               const int64_t *ldv, double tol, int32_t max_outer,
                               double *const *theta, double *const *X, const int64_t *ldx,
                               double *const *resid, int32_t *n_conv, slrf_status *status,
                               slrf_report *rep, int32_t n_threads);

/* A request server: eigen-solve requests of any size and interval are queued,
 * admitted in arrival order as soon as their device-memory estimate
 * (slrf_request_bytes) fits in the free part of the server's budget, and run
 * by n_workers worker threads, each on its own stream and handle, so that
 * requests arriving while others run overlap with them on the GPU. */
typedef struct slrf_server slrf_server;
typedef struct {
    slrf_pencil pencil;   /* host CSR (on_device must be 0); copied at submit   */
    slrf_filter filter;   /* host arrays; copied at submit                      */
    double gamma;         /* interval (0, gamma]                                */
    int32_t L;            /* subspace size                                      */
    const double *V0;     /* host n x L row-major start block; copied at submit */
    double tol;           /* outer tolerance on rho_i                           */
    int32_t max_outer;
    slrf_opts opts;       /* per-request options (slrf_opts_default)            */
} slrf_request;

/* Device bytes a request is admitted with (pencil + workspace + staging). */
int64_t slrf_request_bytes(const slrf_request *r);
/* Create a server on the current device with n_workers (1..64) workers and a
 * device-memory budget in bytes (0: 90 % of the currently free memory). */
slrf_status slrf_server_create(slrf_server **s, int32_t n_workers, int64_t mem_budget);
/* Queue a request; *ticket identifies it.  SLRF_EBUDGET if it can never fit. */
slrf_status slrf_server_submit(slrf_server *s, const slrf_request *r, int64_t *ticket);
/* Fetch a finished request: with wait = 0 returns SLRF_PENDING if it is still
 * queued or running; otherwise (or once done) copies theta[L], X (n x L, ld L),
 * resid[L] (any may be NULL), n_conv, rep, latency_ms (submit to completion)
 * and the request's own status into *result, forgets the ticket and returns
 * SLRF_OK. */
slrf_status slrf_server_poll(slrf_server *s, int64_t ticket, int32_t wait, double *theta, double *X,
                             double *resid, int32_t *n_conv, slrf_report *rep, double *latency_ms,
                             slrf_status *result);
/* Queue length, running requests, finished requests, admitted bytes. */
slrf_status slrf_server_stats(slrf_server *s, int64_t *queued, int64_t *running, int64_t *finished,
                              int64_t *bytes_in_use);
/* Finish queued and running requests, then stop the workers and free the server. */
void slrf_server_destroy(slrf_server *s);

/* ---- allocation-free variant ---------------------------------------------- */

/* G = X^T Y (m x m row-major, device) for X, Y device n x m row-major FP64,
 * like slrf_gram but with no handle and no device allocation.  The paper has
 * no counterpart: this exists for callers that may not allocate device memory
 * themselves (code whose device memory is owned by another allocator or a
 * fixed pool, or that cannot afford cudaMalloc's implicit synchronisation).
 * Its split-K scratch is a static device array of SLRF_NOALLOC_SCRATCH_BYTES
 * held by every GPU that loads the library; m*m*8 must fit in it (m <= 724),
 * larger m returns SLRF_EINVAL (message in slrf_noalloc_last_error()).
 * The first call on a device looks up that array's device address (with that
 * device current), so make the first call before any stream capture: a first
 * call on a capturing stream returns SLRF_EINVAL.  The address is that of the
 * device's primary context (the CUDA runtime's), so call from that context
 * only, and not after cudaDeviceReset in the same process.  All
 * calls share the scratch: calls that overlap on the GPU (concurrent streams)
 * race.  Work is enqueued on cuda_stream (a cudaStream_t); returns after
 * enqueuing. */
#define SLRF_NOALLOC_SCRATCH_BYTES (4u << 20)
slrf_status slrf_gram_noalloc(int64_t n, int32_t m, const double *X, int64_t ldx, const double *Y,
                              int64_t ldy, double *G, void *cuda_stream);
/* Text of the last error of slrf_gram_noalloc on this thread ("" if none). */
const char *slrf_noalloc_last_error(void);

/* ---- measurement ----------------------------------------------------------- */

/* Measured fused multiply-add throughput of the current device in flop/s
 * (2 flops per FMA), FP32 for precision = SLRF_PREC_MIXED, FP64 for
 * SLRF_PREC_FP64: the peak against which kernels bound by plain ALU
 * arithmetic are reported (the paper has no counterpart; it reports no
 * timings).  Runs a register-only FMA kernel that fills every SM on
 * cuda_stream (a cudaStream_t), best of three timed repetitions after one
 * warm-up; synchronises the stream.  *flops_per_s is written on SLRF_OK.
 * SLRF_EINVAL for a NULL output or another precision, SLRF_ECUDA if a CUDA
 * call fails. */
slrf_status slrf_fma_peak(int32_t precision, double *flops_per_s, void *cuda_stream);

/* ---- multigrid hierarchy (inspection) -------------------------------------- */

/* The multigrid hierarchy is built on the host with up to 16 threads per
 * step (the environment variable SLRF_HOST_THREADS, read once, sets another
 * cap, e.g. when many handles are created at once); every value it produces
 * is formed in a fixed order, so the hierarchy does not depend on the count. */

#define SLRF_MG_MAX_LEVELS 16
/* Build the SLRF_PRECOND_MG hierarchy of a HOST pencil (p->on_device must be
 * 0) with the mg_* fields of *o (NULL = defaults), on the host only, and
 * report it: *n_levels, level_n[l] and level_nnz[l] (arrays of
 * SLRF_MG_MAX_LEVELS) the size and stored entries of each level pencil,
 * *setup_ms the host time.  Optional outputs of the coarsest level (size
 * n_c = level_n[*n_levels - 1]), NULL to skip: coarse_lam[n_c], the
 * eigenvalues of the coarsest pencil ascending, and coarse_a / coarse_b
 * (n_c x n_c row-major, dense) the coarsest pencil itself.  No device work.
 * Returns SLRF_EINVAL for invalid input, SLRF_BREAKDOWN if the setup fails
 * (message in slrf_last_error()). */
slrf_status slrf_mg_describe(const slrf_pencil *p, const slrf_opts *o, int32_t *n_levels, int64_t *level_n,
                             int64_t *level_nnz, double *setup_ms, double *coarse_lam, double *coarse_a,
                             double *coarse_b);

/* Prolongator P_l (level l to l + 1, n_l x n_{l+1}, CSR with sorted
 * columns, FP64) of the hierarchy slrf_mg_describe builds, and rho_l, the
 * spectral radius of diag(A_l)^{-1} A_l that scales level l's Jacobi
 * damping (omega_l = mg_omega / rho_l).  First call with ptr = col = val =
 * NULL for *n_rows, *n_cols, *nnz and *rho; then with host arrays
 * ptr[n_rows + 1], col[nnz], val[nnz].  0 <= level <= n_levels - 2.  Host
 * only.  SLRF_EINVAL for invalid input or a level out of range,
 * SLRF_BREAKDOWN if the setup fails. */
slrf_status slrf_mg_transfer(const slrf_pencil *p, const slrf_opts *o, int32_t level, int32_t *n_rows,
                             int32_t *n_cols, int64_t *nnz, double *rho, int32_t *ptr, int32_t *col,
                             double *val);

/* ---- pole/weight sets (host) -------------------------------------------- */

/* Fill N upper-half poles/weights (host arrays of length N) for a rule:
 * SLRF_RULE_MIDPOINT / _GAUSS_LEGENDRE / _GAUSS_CHEBYSHEV on the circle with
 * centre gamma/2 and radius gamma/2 (Section 3.2; alpha, beta ignored), or
 * SLRF_RULE_SLRF: poles gamma x_j (1 + i alpha) with weights minimising the
 * delta-weighted least-squares distance to the step function on [0, 10 gamma]
 * (Section 3.1, the SLRF design).  Poles ordered by real part. */
slrf_status slrf_design_poles(int32_t rule, int32_t N, double alpha, double beta, double gamma,
                              double *sigma_re, double *sigma_im, double *w_re, double *w_im);

/* phi[k] = Phi(x[k]) = sum_j 2 Re(w_j / (x[k] - sigma_j)) for real x (host).
 * Eq. of Phi(lambda), Section 3. */
slrf_status slrf_filter_eval(const slrf_filter *f, const double *x, int64_t count, double *phi);

#ifdef __cplusplus
}
#endif
#endif /* SLRF_H */
