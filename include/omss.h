/*
 * omss -- steady states of driven, damped optomechanical systems on GB300.
 *
 * C ABI of the CUDA library (libomss.so) that implements the iterative
 * steady-state solve of Nation, Johansson, Blencowe & Rimberg, "Iterative
 * solutions to the steady state density matrix for optomechanical systems"
 * (arXiv:1411.4356):
 *
 *   om_build_liouvillian  Eq. 1 (Hamiltonian), Eq. 3 (Lindblad form), Eq. 4
 *                         (column stacking), Eq. 5 (trace augmentation)
 *   om_permute            Sec. III: reverse Cuthill-McKee order of the
 *                         structure of L~ + L~^T, applied to rows and columns
 *   om_ilu_factor         Sec. II: incomplete LU with dual threshold (d, p)
 *   om_steady_state_solve Sec. IV: restarted GMRES with the ILU preconditioner
 *                         (Eq. 6), trace normalisation, rho in natural order
 *   om_steady_state_adjoint  gradients of Tr(O rho) by the adjoint equation
 *                         L~^H mu = dF/drho with the same permuted ILU
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex numbers are complex128 stored as interleaved (re, im) doubles
 *   ("c128"); complex64 as interleaved floats ("c64").
 * - Device pointers are CUDA device addresses on the current device; host
 *   pointers are ordinary host memory.  Each argument states which.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  All device work is ordered on it.  Entry points that return
 *   host-side scalars synchronise the stream before returning.
 * - Handles (om_matrix, om_ilu, om_nojump) own device memory allocated by the
 *   library -- through the hook of om_set_allocator when one is set, else with
 *   cudaMallocAsync on the given stream -- and are released with the matching
 *   *_free call.  Vectors (rho, perm, x0, gradients of rho) are caller-owned.
 * - No C++ exception crosses the ABI.  Every call returns an om_status;
 *   OM_OK is 0 and every error is negative.  om_last_error() returns a
 *   human-readable message for the calling thread's most recent error.
 * - Vectorisation (Eq. 4): rho_ij sits at k = i + j n (column stacking);
 *   Hilbert index of |c, m> is h = c N_m + m (a = a (x) I_b, Sec. III).
 */
#ifndef OMSS_H
#define OMSS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OM_OK = 0,
    OM_EINVAL = -1,      /* bad argument (null pointer, size out of range, ...) */
    OM_ENOMEM = -2,      /* device or host allocation failed */
    OM_ECUDA = -3,       /* a CUDA runtime call failed */
    OM_EZEROPIVOT = -4,  /* ILU produced a zero pivot that the guard could not fix */
    OM_ENOCONV = -5,     /* GMRES hit max_iters; the best iterate is still written */
    OM_EBREAKDOWN = -6,  /* Arnoldi breakdown before convergence */
    OM_ENUMERIC = -7,    /* NaN or Inf met in a residual or a factor */
    OM_ETIMEOUT = -8     /* a device-side wait exceeded wait_timeout_ns */
} om_status;

/* Parameters of Eq. 1 and Eq. 3 (units of omega_m) and the Fock cutoffs of
 * Sec. III.  Gamma_m = omega_m / Q_m.  g2 and lam add the Hamiltonian variants
 * that Sec. VI names, g2 (b + b^dag)^2 a^dag a (quadratic, "membrane in the
 * middle" coupling) and lam (b + b^dag)^4 (anharmonic oscillator term), with
 * the powers of b + b^dag taken in the truncated N_m-level space; zero gives
 * Eq. 1 exactly.  Every entry point that takes om_params honours them. */
typedef struct {
    int32_t Nc, Nm;
    double omega_m, Delta, kappa, g0, E, Q_m, n_th;
    double g2, lam;
} om_params;

typedef struct {
    int32_t trace_mode; /* 0: row 0 of L~ is w T alone ("replace");
                           1: L~ = L + w T as printed in Eq. 5 ("add") */
    double nth_floor;   /* if n_th == 0, use this occupation instead (Sec. IV
                           uses 1e-15); 0 keeps n_th = 0 */
} om_build_opts;

typedef struct {
    int32_t restart;        /* GMRES restart length m (Sec. IV restarts at 10) */
    int32_t max_iters;      /* cap on inner iterations over all cycles */
    int32_t precision;      /* 0: complex128 throughout;
                               1: complex64 inner GMRES / ILU / SpMV inside an
                                  FP64 iterative-refinement loop */
    int32_t precond_fp64;   /* 0: triangular sweeps with the complex64 copy of the
                               factors (default: GB300's FP64 pipe runs at 1/64 of
                               FP32, and the ILU is an approximation far coarser
                               than FP32 rounding); 1: complex128 sweeps */
    double tol;             /* target of eta = ||L x||_inf / (||L||_inf ||x||_inf) */
    int64_t wait_timeout_ns;/* bound on each device-side spin-wait of the solve's
                               kernels (mbarrier phases of the sweeps and of the
                               tensor-core products, the split sweep's cross-block
                               flags); a wait that runs out aborts its kernel and
                               the solve returns OM_ETIMEOUT.  <= 0: 2 s */
} om_solve_opts;

typedef struct {
    int32_t iterations;     /* inner GMRES iterations, all cycles */
    int32_t cycles;         /* restarts + 1 (FP64 path) or refinement steps (mixed) */
    double eta;             /* final normwise backward error (see om_solve_opts.tol) */
    double trace_before;    /* Tr(x) before normalisation */
    double seconds;         /* wall time of the call */
    double residual_history[64]; /* eta at the end of each cycle (first 64) */
} om_solve_info;

/* ---- device memory --------------------------------------------------------
 * om_set_allocator routes every device allocation of the library (handles and
 * the work space of each call) through alloc(bytes, stream, ctx) and
 * free(ptr, stream, ctx), stream being the cudaStream_t of the call that
 * allocates or frees (as void*).  The buffer may be used on that stream as
 * soon as alloc returns, and free is called once the library has enqueued its
 * last use of it on that stream (stream-ordered, as cudaFreeAsync).  Both
 * functions must be thread-safe (the batched solve allocates from several host
 * threads) and alloc returns NULL on failure (the call then fails with
 * OM_ENOMEM).  A framework's caching allocator fits here, so that the factors
 * and Krylov bases (several GB) are counted in its pool.  NULL, NULL restores
 * cudaMallocAsync / cudaFreeAsync.  cuSOLVER's own internal work space, in the
 * set-up of om_nojump_factor, is not routed.  Change the hook only while no
 * handle is alive: a buffer is always freed through the hook current at that
 * time.  No counterpart in the paper.
 * Errors: OM_EINVAL if exactly one of alloc and free is NULL. */
typedef void *(*om_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*om_free_fn)(void *ptr, void *stream, void *ctx);
om_status om_set_allocator(om_alloc_fn alloc, om_free_fn free, void *ctx);
/* Number of allocations made through the hook since the library was loaded
 * (instrumentation). */
int64_t om_allocator_hook_calls(void);

typedef struct om_matrix om_matrix; /* complex CSR on the device */
typedef struct om_ilu om_ilu;       /* ILU factors + sweep schedule on the device */

/* ---- Eq. 1-5: assemble L~ ------------------------------------------------
 * Builds the trace-augmented Liouvillian L~ (N = (Nc*Nm)^2 rows) in CSR with
 * int64 row pointers, int32 columns sorted within each row and c128 values,
 * exact zeros dropped.  w = mean of diag(L) (Sec. IV) is kept in the handle,
 * as are ||L||_inf and the unmodified row 0 of L (for the residual eta).
 * Errors: OM_EINVAL if a pointer is NULL, Nc or Nm < 1, N > 2^31 - 1 or the
 * nonzero count exceeds 2^31 - 1. */
om_status om_build_liouvillian(const om_params *params, const om_build_opts *opts,
                               void *stream, om_matrix **out);

/* Row k of L (Eq. 3 in the basis of Eq. 4, without the trace row), from the
 * closed form the assembly kernels evaluate, computed on the host with no
 * device involved: its count (<= 21) columns (HOST int64) in increasing
 * order and values (HOST interleaved complex128 doubles); exact zeros are
 * left out.  opts->nth_floor as for om_build_liouvillian.  Errors: OM_EINVAL. */
om_status om_liouvillian_row_host(const om_params *params, const om_build_opts *opts, int64_t k, int64_t *cols,
                                  double *vals, int32_t *count);

/* Host-side description of a matrix handle; any out pointer may be NULL. */
om_status om_matrix_info(const om_matrix *A, int64_t *nrows, int64_t *nnz, double *w,
                         double *norm_inf);

/* Copies the CSR arrays to caller-owned HOST buffers of sizes nrows+1, nnz,
 * 2*nnz doubles (any may be NULL to skip).  Synchronises `stream`. */
om_status om_matrix_export(const om_matrix *A, int64_t *rowptr, int32_t *col, double *val,
                           void *stream);

/* ---- Sec. III: reverse Cuthill-McKee ----------------------------------------
 * perm_dev (caller-owned DEVICE int32[N]) receives perm[new] = old, the RCM
 * order of the structure of A + A^T (degree = nonzeros of a row of that
 * structure; each component starts at the unvisited node of least (degree,
 * index); neighbours are queued in increasing (degree, index); the
 * Cuthill-McKee order is reversed).  *A_rcm = P A P^T with
 * A_rcm[r, c] = A[perm[r], perm[c]].  Errors: OM_EINVAL on NULL arguments. */
om_status om_permute(const om_matrix *A, void *stream, int32_t *perm_dev, om_matrix **A_rcm);

/* om_permute computes the order on the device; om_permute_ex chooses: flags
 * bit 0 set, on the device, level by level (each breadth-first level is the
 * previous level's unplaced neighbours sorted by (position of the earliest
 * neighbour in the previous level, degree, index), which is the serial order
 * above) on the union pattern built on the device, with about 40 bytes of
 * device memory per nonzero of A; bit 0 clear, the serial walk on the host
 * cores.  Both give the same permutation.  Errors: OM_EINVAL (also, on the
 * device, for a node of degree >= 2^20 in the union pattern), OM_ENOMEM,
 * OM_ECUDA. */
om_status om_permute_ex(const om_matrix *A, int32_t flags, void *stream, int32_t *perm_dev, om_matrix **A_rcm);

/* The serial order of om_permute_ex (bit 0 clear) alone, on HOST CSR arrays
 * (rowptr int64[N+1], col int32, rows sorted by column), with no device
 * involved: perm (HOST int32[N]) = perm[new] = old.  Errors: OM_EINVAL,
 * OM_ENOMEM. */
om_status om_rcm_order_host(int64_t N, const int64_t *rowptr, const int32_t *col, int32_t *perm);

/* ---- Sec. II: ILUT(d, p) ----------------------------------------------------
 * Row-wise incomplete LU of A (unit L, no pivoting).  In row i every entry
 * of modulus below droptol * ||row i of A||_inf is dropped (the diagonal is
 * kept); the strict-L part keeps at most floor(fill * nnz_i / 2) entries and
 * the U part, diagonal included, at most as many (largest moduli, ties to
 * the smaller column), so NNZ(L) + NNZ(U) <= fill * NNZ(A).  A pivot below
 * 1e-14 ||row i||_inf is replaced by that value and counted.
 * flags bit 0: add the moduli of the entries dropped from row i to |u_ii|
 * (diagonal compensation); bit 1: also store the conjugate transposes U^H,
 * L^H needed by the adjoint; bit 2: also keep complex128 sweep data (the
 * sweeps use complex64 otherwise); bit 3: equilibrate first, as the iLUTP of
 * Sec. II does when SuperLU runs it -- r_i = 1 / max_j |a_ij|, then
 * c_j = 1 / max_i |r_i a_ij| -- and factor diag(r) A diag(c) (the drop rule
 * then reads the scaled rows); every application of the handle is
 * M^{-1} = diag(c) (L U)^{-1} diag(r) (M^{-H} = diag(r) (L U)^{-H} diag(c));
 * bit 4: read the fill cap as a total, NNZ(L) + NNZ(U) <= fill * NNZ(A),
 * held as a running budget over the rows in order -- row i keeps every entry
 * that survives the drop rule while the entries kept by rows 0..i (diagonals
 * apart from row i's own) stay within floor(fill * NNZ(rows 0..i of A)), and
 * beyond that the largest moduli that fit (ties to the smaller column); where
 * the budget never binds this is threshold ILU(droptol).  Not with bit 0.
 * Rows are factored in parallel on the
 * host cores (OMSS_ILU_THREADS caps the thread count); the factors are
 * identical to those of the serial row order.  On the device the factors are
 * stored in the tiled form of the sweeps: per tile of 32 rows, the dense
 * inverse of the diagonal block and the entries that reach earlier tiles.
 * Errors: OM_EINVAL, OM_ENOMEM. */
om_status om_ilu_factor(const om_matrix *A_rcm, double droptol, double fill, int32_t flags,
                        void *stream, om_ilu **out);

/* ILUTP(d, p, permtol): the ILUT above with threshold column pivoting, the
 * "P" of the iLUTP of Sec. II.  Rows are eliminated in the order of the
 * current column positions; after the drop rule and the fill cap, if
 * permtol * (largest kept off-diagonal modulus of U row i) > |u_ii|, that
 * entry's column moves to position i (ties: the smaller position) and the
 * old diagonal column takes its place.  The factors satisfy A Q ~ L U; every
 * application of the handle is M^{-1} = Q U^{-1} L^{-1} (with the
 * equilibration scalings of flag bit 3 outside).  permtol in (0, 1] (0.1
 * keeps the diagonal while it is at least a tenth of the largest entry, the
 * threshold SuperLU's incomplete LU uses); flags as for om_ilu_factor except
 * bit 0 (compensation), which is rejected.  The rows are factored in parallel
 * on the host cores as for om_ilu_factor, each row deciding its pivot once
 * every earlier row has, so the factors are those of the serial order (the
 * pivots lengthen the dependency chain: expect it to be slower than ILUT).
 * The handle keeps work vectors for the permutation: applications of one
 * pivoted handle must not overlap on the GPU.  Errors: OM_EINVAL, OM_ENOMEM. */
om_status om_ilutp_factor(const om_matrix *A_rcm, double droptol, double fill, double permtol, int32_t flags,
                          void *stream, om_ilu **out);

/* The host factorisation of om_ilu_factor / om_ilutp_factor alone, on HOST
 * arrays, with no device involved (A in CSR: rowptr int64[N+1], col int32,
 * val interleaved complex128 doubles; rows sorted by column).  flags bits 0
 * (compensation), 3 (equilibration) and 4 (total fill budget) as for
 * om_ilu_factor; permtol > 0 pivots as om_ilutp_factor (not with bits 0 or
 * 4).  The handle holds the strict L and strict U parts in CSR (position
 * space), the diagonal of U, the column at each position (the identity
 * without pivoting) and the scalings r, c (ones without equilibration):
 * om_host_ilu_sizes gives the entry counts, om_host_ilu_export copies them
 * to caller-owned HOST arrays of sizes N+1, nnz_l, 2 nnz_l, N+1,
 * nnz_u_strict, 2 nnz_u_strict, 2N, N, N, N (any may be NULL).  Errors:
 * OM_EINVAL, OM_ENOMEM. */
typedef struct om_host_ilu om_host_ilu;
om_status om_ilu_factor_host(int64_t N, const int64_t *rowptr, const int32_t *col, const double *val,
                             double droptol, double fill, double permtol, int32_t flags, om_host_ilu **out);
om_status om_host_ilu_sizes(const om_host_ilu *F, int64_t *nnz_l, int64_t *nnz_u_strict, int64_t *n_guarded,
                            int64_t *n_swaps);
om_status om_host_ilu_export(const om_host_ilu *F, int64_t *lp, int32_t *li, double *lx, int64_t *up,
                             int32_t *ui, double *ux, double *diag, int32_t *q, double *r, double *c);
void om_host_ilu_free(om_host_ilu *F);

/* Pivoting of a factor: *pivoted = 1 for an om_ilutp_factor handle, the
 * number of column swaps, and the column at each position (HOST int32[N],
 * the identity without pivoting; synchronises the stream).  Any out pointer
 * may be NULL.  Errors: OM_EINVAL, OM_ECUDA. */
om_status om_ilu_pivots(const om_ilu *M, int32_t *pivoted, int64_t *n_swaps, int32_t *colperm_host, void *stream);

/* Statistics of a factorisation (any out pointer may be NULL). */
om_status om_ilu_info(const om_ilu *M, int64_t *nnz_l, int64_t *nnz_u, int64_t *n_guarded,
                      int64_t *levels_l, int64_t *levels_u);
/* Host wall-clock seconds of the phases of om_ilu_factor (HOST double[4]):
 * copy of A to the host, ILUT, dependency depths, tiled layout and upload.
 * Instrumentation; no counterpart in the paper. */
om_status om_ilu_timings(const om_ilu *M, double seconds[4]);

/* ---- Sec. IV: the steady state ----------------------------------------------
 * Solves L~_rcm x = P (w, 0, ...)^T by restarted GMRES(m) with right
 * preconditioning M = L U (the system of Eq. 6), stops when eta <= tol,
 * divides x by its trace and scatters it back to natural order:
 * rho_dev (caller-owned DEVICE c128[n*n], column-major n x n) receives rho.
 * perm_dev is the DEVICE permutation written by om_permute.  x0 (DEVICE c128
 * [N] in permuted order) may be NULL.  info (HOST) may be NULL.
 * Errors: OM_EINVAL, OM_ENOMEM, OM_ENOCONV (rho still written),
 * OM_ENUMERIC, OM_ETIMEOUT, OM_ECUDA. */
om_status om_steady_state_solve(const om_matrix *A_rcm, const om_ilu *M, const int32_t *perm_dev,
                                const om_solve_opts *opts, const double *x0, double *rho_dev,
                                om_solve_info *info, void *stream);

/* ---- adjoint ------------------------------------------------------------------
 * For a real loss F(rho) with gradient G = dF/dRe(rho) + i dF/dIm(rho)
 * (DEVICE c128[n*n], column-major), solves L~^H mu = G (GMRES with the
 * preconditioner (L U)^H, i.e. sweeps with U^H then L^H) and writes
 * grad_out (HOST double[4]) = dF/d(Delta, E, g0, kappa) = -Re(mu^H dL~/dtheta rho),
 * dL~/dtheta being dL/dtheta in the rows of L and zero in a replaced trace
 * row.  params must be those A_rcm was built from.  rho_dev is the solution
 * written by om_steady_state_solve.  Errors as om_steady_state_solve. */
om_status om_steady_state_adjoint(const om_matrix *A_rcm, const om_ilu *M, const int32_t *perm_dev,
                                  const om_solve_opts *opts, const om_params *params,
                                  const double *rho_dev, const double *grad_rho_dev,
                                  double grad_out[4], om_solve_info *info, void *stream);

/* ---- batched steady states --------------------------------------------------
 * Solves `count` independent systems (a parameter sweep, Sec. IV) with
 * om_steady_state_solve semantics.  A_rcm[i], M[i], perm_dev[i], rho_dev[i]
 * are as for om_steady_state_solve (x0 is not taken; systems may differ in
 * size); opts applies to all.  status[i] (HOST, count entries) receives each
 * solve's status and info[i] (HOST, may be NULL) its statistics
 * (info[i].seconds is the time of the whole batch).
 * concurrency <= 0: lock-step engine.  One flexible GMRES(m) advances all
 * systems together: each Krylov step is one launch per kernel over every
 * system still iterating, the preconditioner kernel running one thread block
 * per system (complex64 L and U sweeps), and systems retire as they converge.
 * Requires opts->precision == 0, opts->precond_fp64 == 0, restart <= 64.
 * concurrency > 0: up to `concurrency` calls of om_steady_state_solve at a
 * time, each on its own stream driven by its own host thread (any opts).
 * Inputs written on `stream` before the call are honoured, and the results
 * are ordered before later work on `stream`.
 * Returns OM_OK if the batch ran (check status[]), else OM_EINVAL, OM_ENOMEM
 * or OM_ECUDA. */
om_status om_steady_state_solve_batched(int32_t count, const om_matrix *const *A_rcm,
                                        const om_ilu *const *M, const int32_t *const *perm_dev,
                                        const om_solve_opts *opts, double *const *rho_dev,
                                        om_solve_info *info, om_status *status, int32_t concurrency,
                                        void *stream);

/* ---- the no-jump preconditioner ----------------------------------------------
 * Eq. 3 splits as L rho = K rho + rho K^dag + sum_O gamma_O O rho O^dag with
 * K = -i H - (kappa a^dag a + Gm (1 + n_th) b^dag b + Gm n_th b b^dag) / 2
 * (H of Eq. 1, Gm = omega_m / Q_m, b b^dag taken in the truncated space).  In
 * the basis of Eq. 4 the first two terms are S = I (x) K + conj(K) (x) I.  The
 * paper does not use S; this library offers S^{-1} as a second preconditioner
 * of the GMRES of Sec. IV beside the ILUT of Sec. II: applied exactly (four
 * dense n x n products after the eigendecomposition K = V diag(lambda) V^{-1})
 * it leaves GMRES a few tens of iterations on the systems of this library,
 * and the steady state is the same (Eq. 5 fixes it).
 *
 * om_nojump_factor: builds K from params (n_th floored as in
 * om_build_liouvillian when opts->nth_floor > 0), computes the
 * eigendecomposition and V^{-1} on the device (cuSOLVER geev, getrf/getrs,
 * complex128) and keeps the operands of the products.  flags bit 0: also keep
 * the operands of S^{-H} (adjoint); bit 1: complex64 SIMT products instead of
 * the TF32 tensor-core products.  Errors: OM_EINVAL (NULL, n*n > 2^31, non-
 * finite parameters, or lambda_i + conj(lambda_j) = 0 for some i, j, i.e. an
 * undamped mode), OM_ENUMERIC (the eigendecomposition or the inverse failed),
 * OM_ENOMEM, OM_ECUDA.  The handle owns device memory (about 4 n^2 x 8 B, twice
 * that with bit 0, plus the tensor-core operands of 16 n_pad^2 B each) and is
 * released with om_nojump_free. */
typedef struct om_nojump om_nojump;
om_status om_nojump_factor(const om_params *params, const om_build_opts *opts, int32_t flags, void *stream,
                           om_nojump **out);
/* n (Hilbert dimension), whether the tensor-core products are in use,
 * min |lambda_i + conj(lambda_j)| and the host wall time of the set-up phases
 * (HOST double[3]: K and its eigendecomposition, V^{-1}, operand layout); any
 * out pointer may be NULL. */
om_status om_nojump_info(const om_nojump *M, int32_t *n, int32_t *tensor_cores, double *min_abs_d,
                         double seconds[3]);
/* z = S^{-1} v (flags bit 1: S^{-H} v, the handle must keep the adjoint
 * operands), DEVICE c128 vectors of n*n entries in the column-stacked order of
 * Eq. 4; z and v may alias.  The products run in complex64 or TF32 (flexible
 * GMRES keeps the solve exact whatever the precision of the preconditioner).
 * The handle's work matrices are used: calls on one handle must not overlap.
 * Synchronises the stream.  Errors: OM_EINVAL, OM_ECUDA. */
om_status om_nojump_apply(const om_nojump *M, int32_t flags, const double *v, double *z, void *stream);
/* om_steady_state_solve with the no-jump preconditioner: A is the UNPERMUTED
 * matrix of om_build_liouvillian (natural order, trace row 0), x0 (DEVICE c128
 * [N], natural order) may be NULL, rho_dev as for om_steady_state_solve.
 * precision 1 runs complex64 inner GMRES (complex64 SpMV and products) inside
 * FP64 refinement.  Errors as om_steady_state_solve, plus OM_EINVAL for a
 * permuted matrix or a handle of another size. */
om_status om_steady_state_solve_nojump(const om_matrix *A, const om_nojump *M, const om_solve_opts *opts,
                                       const double *x0, double *rho_dev, om_solve_info *info, void *stream);
/* om_steady_state_adjoint with the no-jump preconditioner (S^{-H}) on the
 * unpermuted matrix; the handle must keep the adjoint operands (flag 1) and
 * opts->precision must be 0.  Arguments and errors as om_steady_state_adjoint. */
om_status om_steady_state_adjoint_nojump(const om_matrix *A, const om_nojump *M, const om_solve_opts *opts,
                                         const om_params *params, const double *rho_dev,
                                         const double *grad_rho_dev, double grad_out[4], om_solve_info *info,
                                         void *stream);
void om_nojump_free(om_nojump *M);

/* ---- single kernels, exposed for parity tests -------------------------------
 * y = A x (DEVICE c128 vectors of length nrows). */
om_status om_spmv(const om_matrix *A, const double *x, double *y, void *stream);
/* The parameter sweep on the no-jump path (Sec. IV: independent solves of
 * different parameter sets run side by side).  For each of the `count`
 * systems params[i] the whole path runs -- om_build_liouvillian with bopts,
 * om_nojump_factor with factor_flags, om_steady_state_solve_nojump with
 * sopts -- and rho_dev[i] (caller-owned DEVICE c128 n_i x n_i, column-major)
 * receives the steady state; status[i] (HOST) is the first non-OK status of
 * that system's calls, info[i] (HOST, may be NULL) its solve statistics.
 * `concurrency` (1..64) host threads with their own non-blocking streams take
 * the systems in the order given; the work is joined onto `stream` before
 * the call returns, and each system's handles are freed when it is done.  A
 * failing system does not stop the others.  Errors (of the call itself):
 * OM_EINVAL, OM_ECUDA. */
om_status om_steady_state_sweep_nojump(int32_t count, const om_params *params, const om_build_opts *bopts,
                                       int32_t factor_flags, const om_solve_opts *sopts, double *const *rho_dev,
                                       om_solve_info *info, om_status *status, int32_t concurrency, void *stream);

/* y = L~ x for an UNPERMUTED matrix of om_build_liouvillian, computed from the
 * closed-form stencil of Eq. 3 (at most 13 terms per row, coefficients from
 * per-level tables) and the trace row of Eq. 5 instead of the stored CSR
 * values: the operator of the no-jump solves.  DEVICE c128 vectors of N
 * entries, x and y must not alias.  Errors: OM_EINVAL (NULL, aliasing or a
 * permuted matrix), OM_ECUDA. */
om_status om_liouvillian_apply(const om_matrix *A, const double *x, double *y, void *stream);
/* z = M^{-1} v, or M^{-H} v, with DEVICE c128[N] vectors (z and v may alias);
 * M = L U, or diag(r)^{-1} L U diag(c)^{-1} for equilibrated factors.  flags bit 0: sweep with the complex128 data (the factor must have
 * been built with it), else complex64; bit 1: apply the conjugate transpose
 * (the factor must keep the transposes); bit 2: run the complex64 sweeps in
 * one thread block even where the split sweep over all SMs applies (the two
 * differ only in the order of the complex64 sums).  The split sweep takes
 * scratch from the stream-ordered allocator.  Errors: OM_EINVAL, OM_ECUDA. */
om_status om_ilu_apply(const om_ilu *M, int32_t flags, const double *v, double *z,
                       void *stream);
/* Sec. IV's estimate of how the preconditioner amplifies errors, read as
 * ||M^{-1} e||_inf with e the vector of ones (one forward and one backward
 * sweep, with the scalings of equilibrated factors).  flags as for om_ilu_apply (bit 0: complex128 sweeps; bit
 * 2: one-block sweeps; bit 1 is ignored).  out: HOST double.  A NaN or Inf
 * result marks an unstable factorisation.  Errors: OM_EINVAL, OM_ECUDA. */
om_status om_ilu_condest(const om_ilu *M, int32_t flags, double *out, void *stream);
/* Allocation-free variant of om_ilu_apply.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory --
 * code whose device memory belongs to another allocator (a framework's
 * caching pool), and latency-critical code that must not enter the allocator
 * or risk the implicit device synchronisation of cudaMalloc/cudaFree.  It
 * computes the same z as om_ilu_apply with flag bit 2 (one-block sweeps; same
 * flags otherwise, same DEVICE c128 vectors,
 * z and v may alias) but takes its scratch -- a complex64 work vector of at
 * most 1,048,576 rows -- from a static device array that every GPU loading
 * the library holds (8 MiB) until the process exits, and calls no allocator.
 * Factors with more rows are rejected with OM_EINVAL.  The first call on each
 * device looks up the array's device address (with that device current).
 * Every call synchronises its stream before returning.  All calls share the
 * array: calls whose work overlaps on the GPU (two host threads on two
 * streams, say) race.  Errors: OM_EINVAL, OM_ECUDA. */
om_status om_ilu_apply_noalloc(const om_ilu *M, int32_t flags, const double *v, double *z,
                               void *stream);
/* Phonon number distribution of Sec. V (Fig. 5): P[m] = <m| Tr_cavity(rho) |m>
 * (HOST double[Nm]) of a DEVICE rho (c128 n x n column-major, n = Nc Nm), and
 * moments (HOST double[3]) = <N_b>, <N_b^2> and the Fano factor
 * F = <(Delta N_b)^2> / <N_b> (0 when <N_b> = 0).  Synchronises the stream.
 * Errors: OM_EINVAL, OM_ECUDA. */
om_status om_phonon_distribution(int32_t Nc, int32_t Nm, const double *rho_dev, double *P, double moments[3],
                                 void *stream);
/* <a^dag a>, <b^dag b> of a DEVICE rho (c128 n x n column-major); out HOST double[2]. */
om_status om_observables(int32_t Nc, int32_t Nm, const double *rho_dev, double out[2],
                         void *stream);

/* ---- instrumentation (no counterpart in the paper) -------------------------
 * om_kernel_launches: number of kernels the library has launched since it was
 * loaded.  om_profile(1) starts recording CUDA events around every one-block
 * triangular sweep (category 0), SpMV (category 1), split sweep over all
 * SMs (category 2), no-jump preconditioner application (category 3: its
 * four products), Gram-Schmidt step of GMRES (category 4: the two CGS2 passes)
 * and stencil application of L~ (category 5) launch, om_profile(0) stops, both
 * discard earlier records; om_profile_read returns the summed device time
 * (milliseconds, HOST out) and launch count of a category, synchronising on
 * the recorded events. */
int64_t om_kernel_launches(void);
om_status om_profile(int32_t enable);
om_status om_profile_read(int32_t category, double *total_ms, int64_t *count);

void om_matrix_free(om_matrix *A);
void om_ilu_free(om_ilu *M);
const char *om_status_str(om_status s);
const char *om_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* OMSS_H */
