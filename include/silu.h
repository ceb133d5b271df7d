/*
 * silu: scaled-ILU Richardson smoothers on GB300 (sm_103a).
 *
 * C ABI of libsilu.so.  The library applies an incomplete-LU smoother whose
 * upper factor is row-scaled to unit diagonal, with the two triangular solves
 * replaced by a fixed number of Richardson sweeps, each one CSR SpMV, as in
 * Thomas, Carr, Mullowney, Swirydowicz and Day, "Scaled ILU Smoothers for
 * Navier-Stokes Pressure Projection" (arXiv 2111.09512), and wraps it in a
 * flexible GMRES solve.
 *
 * Conventions that hold for every call:
 *  - Matrices are CSR with int64 row pointers (n+1 entries), int32 column
 *    indices and FP64 values, all in HOST memory; the library copies them
 *    (the caller keeps ownership).  Rows need not be sorted; duplicate
 *    entries are summed.  n and nnz must be below 2^31.
 *  - Vectors are DEVICE pointers owned by the caller, FP64, row-major
 *    n x nrhs: the nrhs values of one row are adjacent (right-hand sides
 *    interleaved).  8-byte alignment is required.
 *  - Device calls are asynchronous and ordered on the context's stream,
 *    except where a call says it blocks.  A context is used by one host
 *    thread at a time; separate contexts may run concurrently.
 *  - Every call returns a status; silu_last_error() gives the message of the
 *    last failure on a context.  No call aborts, traps or leaves the device
 *    in an error state on bad input: arguments are checked on the host first.
 *  - Handles are freed by the matching *_destroy call; a silu_ilu refers to
 *    the silu_mat it was built from, which must outlive it.
 */
#ifndef SILU_H
#define SILU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SILU_OK = 0,
  SILU_ERR_INVALID_ARG = 1,   /* bad argument, malformed CSR, NaN/Inf input  */
  SILU_ERR_ZERO_PIVOT = 2,    /* zero or non-finite pivot (pivoting is off)  */
  SILU_ERR_NOT_CONVERGED = 3, /* FGMRES hit maxit; best iterate is written   */
  SILU_ERR_OOM = 4,           /* host or device allocation failed            */
  SILU_ERR_CUDA = 5,          /* a CUDA runtime call failed                  */
  SILU_ERR_TIMEOUT = 6,       /* a bounded device wait gave up               */
  SILU_WARN_DIVERGED = 7,     /* iterate grew beyond a bound (not an error)  */
  SILU_ERR_NO_DEVICE = 8,     /* device call on a host-only context          */
  SILU_ERR_TOO_LARGE = 9,     /* problem exceeds a fixed-capacity entry point */
  SILU_ERR_BUSY = 10,         /* server queue full, or request already running */
  SILU_ERR_CANCELLED = 11     /* request cancelled before it started         */
} silu_status;

/*
 * Factorisation kinds.  ILU0 / ILUK / ILUT are the incomplete factorisations
 * of Sec. 1, Sec. 4.2 and Sec. 5.1.  GS and SGS are the Gauss-Seidel
 * splittings of Sec. 3.1 written as factors, with A = D + L_A + U_A:
 *  SILU_GS   M = D + L_A = (I + L_A D^{-1}) D: L_s = L_A D^{-1}, U = D.
 *            ilu_smooth with sweeps_L = p + 1 and sweeps_U = 1 is the
 *            polynomial Gauss-Seidel smoother of Sec. 3.1,
 *            x <- x + sum_{j=0}^{p} (-D^{-1} L_A)^j D^{-1} (b - A x).
 *  SILU_SGS  M = (D + L_A) D^{-1} (D + U_A) = (I + L_A D^{-1}) D (I + D^{-1} U_A):
 *            the same with a backward half (symmetric Gauss-Seidel), row-
 *            scaled upper factor Utilde_s = D^{-1} U_A.
 * For GS / SGS `tau` and `fill` are ignored and direct_trisolve performs
 * exact Gauss-Seidel.
 */
typedef enum { SILU_ILU0 = 0, SILU_ILUK = 1, SILU_ILUT = 2, SILU_GS = 3, SILU_SGS = 4 } silu_kind;

/*
 * How the upper factor is iterated (Sec. 5.1-5.2):
 *  SILU_SCALE_ROW        Utilde = D^{-1} U, D = diag(U) (Eq. extractD,
 *                        Eq. newD); Richardson v <- D^{-1} y - Utilde_s v
 *                        (Eq. richard).  The method of the paper.
 *  SILU_SCALE_NONE       raw U; Jacobi v <- v + D^{-1} (y - U v), iteration
 *                        matrix G_U = I - D_U^{-1} U (Eq. LUiterMat).
 *  SILU_SCALE_NONE_RICH  raw U; plain Richardson v <- y - (U - I) v, which
 *                        the paper reports as failing to converge.
 *  SILU_SCALE_ROWCOL     row/column scaling (Sec. 5.1, Eq. rowcolScale):
 *                        Uhat = D_r U D_c with D_c from Ruiz equilibration
 *                        of U (at most 20 steps, each dividing every row and
 *                        column by the square root of its largest magnitude,
 *                        stopping once all are within 1e-2 of one) and
 *                        D_r = (D D_c)^{-1}, which makes diag(Uhat) = 1;
 *                        Richardson w <- D_r y - Uhat_s w, then x += D_c w.
 *                        Uhat = D_c^{-1} (D^{-1} U) D_c, so the smoother's
 *                        result equals SILU_SCALE_ROW's up to rounding; the
 *                        factor's departure from normality and the norms of
 *                        the powers of Uhat_s differ (Table dep, Fig. Up).
 */
typedef enum { SILU_SCALE_NONE = 0, SILU_SCALE_ROW = 1, SILU_SCALE_NONE_RICH = 2, SILU_SCALE_ROWCOL = 3 } silu_scale;

/* Precision of the stored factors and of the sweeps (the residual
 * r = b - A x, FGMRES and the solution vector stay FP64). */
typedef enum { SILU_FP64 = 0, SILU_FP32 = 1 } silu_prec;

/* Preconditioner inside fgmres_solve.  SILU_PRECOND_AMG: one AMG V-cycle
 * from zero whose finest level is smoothed by sweeps_L + sweeps_U Richardson
 * sweeps; SILU_PRECOND_AMG_DIRECT: the same cycle smoothed by the exact
 * level-scheduled triangular solves of the same factors (the comparison of
 * Sec. 6).  Both need silu_amg_setup on the factor object. */
typedef enum {
  SILU_PRECOND_SWEEPS = 0,
  SILU_PRECOND_DIRECT = 1,
  SILU_PRECOND_NONE = 2,
  SILU_PRECOND_AMG = 3,
  SILU_PRECOND_AMG_DIRECT = 4,
  SILU_PRECOND_SCHUR = 5, /* one application of the Schur complement smoother (silu_schur_setup) */
  SILU_PRECOND_AMG_SCHUR = 6 /* one AMG V-cycle whose finest level is smoothed by the Schur complement
                                smoother (silu_amg_setup and silu_schur_setup; Sec. 3.1) */
} silu_precond;

typedef struct silu_ctx_s* silu_ctx;
typedef struct silu_mat_s* silu_mat;
typedef struct silu_ilu_s* silu_ilu;
typedef struct silu_batch_s* silu_batch;
typedef struct silu_server_s* silu_server;

/*
 * Create a context on CUDA device `device` whose work is ordered on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream; it may be
 * a stream owned by PyTorch).  device = -1 makes a host-only context: setup,
 * statistics and export work, device calls return SILU_ERR_NO_DEVICE.
 */
silu_status silu_ctx_create(int device, void* cuda_stream, silu_ctx* out);
void silu_ctx_destroy(silu_ctx ctx);

/* Kernel classes for launch counting and timing. */
typedef enum {
  SILU_K_RESIDUAL = 0,    /* r = b - A x and w = A z (CSR SpMV with A)          */
  SILU_K_SWEEP_L = 1,     /* Richardson sweep on L_s                            */
  SILU_K_SWEEP_U = 2,     /* Richardson / Jacobi sweep on the upper factor      */
  SILU_K_LEVEL = 3,       /* level-scheduled substitution (direct_trisolve)     */
  SILU_K_KRYLOV = 4,      /* FGMRES dots, Gram-Schmidt, Givens, update          */
  SILU_K_ELEMENTWISE = 5, /* scaling, casts, x updates                          */
  SILU_K_FUSED = 6,       /* a whole smoother application in one launch         */
  SILU_K_NCLASS = 7
} silu_kclass;

/*
 * Timing of the library's own kernels: with enable = 1 every later launch on
 * ctx is bracketed by two CUDA events recorded on the context's stream (the
 * launching stream), except that the consecutive L sweeps (and U sweeps) of
 * one smoother application share one pair around all of them, so that no
 * event separates one sweep from the next; enable = 0 stops recording.
 * Enabling clears earlier records.  silu_ctx_profile_read blocks on the
 * stream and returns, for one class, the launches recorded and the sum of
 * their event-timed durations.
 */
silu_status silu_ctx_profile(silu_ctx ctx, int enable);
silu_status silu_ctx_profile_read(silu_ctx ctx, int kclass, int64_t* launches, double* total_ms);
/*
 * Sweep overlap (default on): each staged sweep launch is a programmatic
 * dependent of the kernel before it in the stream, so its CTAs start as the
 * previous kernel's CTAs leave the SMs and copy their first factor tiles
 * (which no sweep writes) before waiting for that kernel to complete; every
 * read or write of a vector still waits for it.  Results are the same bits
 * either way.  Applies to launches (and graph captures) made after the call.
 * No counterpart in the paper: it concerns only how consecutive sweeps are
 * launched.
 */
silu_status silu_ctx_set_overlap(silu_ctx ctx, int enable);
/*
 * L2 reuse of staged sweeps (bit flags, default 1; applies to launches and
 * graph captures made after the call).  Bit 0: consecutive staged launches on the
 * context alternate their direction (every other launch walks the row tiles
 * last to first), so a launch starts on the rows the previous one touched
 * last -- vector entries, and factor tiles when both sweep the same factor --
 * while they are still in L2.  Bit 1: factor
 * copies at normal L2 priority (else evict-first).  Bit 2: vector loads and
 * stores at normal L2 priority (else evict-last).  Every row is still
 * computed by one lane from the same tile, so results are the same bits for
 * every setting.  flags outside [0, 7] -> SILU_ERR_INVALID_ARG.  No
 * counterpart in the paper: it concerns only the order in which a sweep
 * visits rows.
 */
silu_status silu_ctx_set_l2_reuse(silu_ctx ctx, int flags);
/* Kernels launched on ctx since creation (all classes; always counted). */
silu_status silu_ctx_launch_count(silu_ctx ctx, int64_t* launches);
/*
 * Block on the context's stream and read (and clear) its device error word.
 * Returns SILU_ERR_TIMEOUT if a kernel's bounded wait gave up since the last
 * check (the results of the calls in between are invalid), else the status
 * of the synchronisation.  fgmres_solve performs this check itself.
 */
silu_status silu_ctx_check(silu_ctx ctx);
/*
 * Self-test of the bounded-wait error path: one GPU thread waits, for at
 * most timeout_ms (1..10000) of the device's global timer, on a device flag
 * that nothing sets, then records the timeout in the context's error word
 * and returns.  The next silu_ctx_check returns SILU_ERR_TIMEOUT; the context
 * stays usable.  Nothing faults, traps or hangs.  Asynchronous.
 */
silu_status silu_ctx_selftest_timeout(silu_ctx ctx, int timeout_ms);
/* Message of the last failed call on ctx ("" if none); valid until the next call. */
const char* silu_last_error(silu_ctx ctx);
/* Library version string. */
const char* silu_version(void);

/*
 * Copy the host CSR matrix A (n rows, nnz entries) into the library:
 * validated (row pointers monotone, columns in range, values finite),
 * columns sorted, duplicates summed, and uploaded to the device on a device
 * context.  A is the pressure matrix of the paper's projection step
 * (Sec. 2, Eq. nodalP, Eq. press); any square matrix with a nonzero diagonal is accepted.
 */
silu_status silu_mat_create(silu_ctx ctx, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                            const double* val, silu_mat* out);
void silu_mat_destroy(silu_mat A);

/*
 * Launch shape of the staged kernel on A (the residual r = b - A x and the
 * FGMRES products): lanes per row (0 = from the mean row length, else 1, 2
 * or 4), rows per lane (0 = automatic, else 1, 2 or 4; more than one only
 * with one lane per row), gather width (8 or 16 entries in flight per lane;
 * 10: the narrow configuration -- tiles of at most 352 entries swept by 24
 * warps per SM with 10 gathers in flight, for one lane and one row per lane
 * and rows of at most 10 entries, 9 on average, else SILU_ERR_INVALID_ARG;
 * 0: automatic, the narrow configuration where it fits, else 16).  The
 * automatic shape (lanes 0, passes 0, chunk 0) is what silu_mat_create
 * chooses.  Results change only by summation order across lanes.  Blocks (the new
 * tiles are uploaded); captured FGMRES iterations of factor objects on A are
 * rebuilt on their next use.
 */
silu_status silu_mat_set_shape(silu_mat A, int lanes, int passes, int chunk);
/*
 * Time r = b - A x (one right-hand side) for each launch shape of the staged
 * kernel (lanes 1/2/4, rows per lane 1/2/4 with one lane, gather width 8/16,
 * the narrow configuration, and the automatic choice), keep the fastest (as silu_mat_set_shape), and
 * return it with its time per product.  Blocks.  Results change only by
 * summation order across lanes.  Device context only; an empty matrix keeps
 * the automatic shape and reports 0 ms.  Any output pointer may be NULL.
 */
silu_status silu_mat_autotune(silu_mat A, int* lanes, int* passes, int* chunk, double* ms);

/*
 * r = b - A x on the device (the residual of Eq. ILUsplit), ordered on A's
 * context stream.  r, x, b: device n x nrhs FP64 (row-major, right-hand sides
 * interleaved); r must not overlap x or b.  Device context only.
 */
silu_status silu_mat_residual(silu_mat A, double* r, const double* x, const double* b, int nrhs);

/*
 * Host factorisation + scaling + packing, then one upload (blocks).
 *  kind  SILU_ILU0: pattern of A (Sec. 5.1, Matlab ilu 'nofill').
 *        SILU_ILUK: level-of-fill k = `fill` (Sec. 1).
 *        SILU_ILUT: dual threshold, drop tolerance `tau` relative to the row's
 *        2-norm and at most `fill` entries per row in each of L and U
 *        (droptol / lfill, Sec. 4.2, Sec. 6.1); the paper does not define
 *        the rule and this is Saad's ILUT.
 *  Pivoting is off; a zero or non-finite pivot gives SILU_ERR_ZERO_PIVOT.
 *  L is unit lower, stored as its strict part L_s.  The level sets of L_s and
 *  of the upper factor (Sec. 4) are built for direct_trisolve.
 */
silu_status ilu_setup(silu_ctx ctx, silu_mat A, silu_kind kind, double tau, int fill, silu_scale scale,
                      silu_prec prec, silu_ilu* out);

/*
 * Numeric refactorisation with new values of A on the SAME pattern (nnz
 * values in the sorted, duplicate-free order of the silu_mat), reusing the
 * symbolic phase (Sec. 3.1: the pattern of the pressure matrix does not change
 * during a fluid step).  ILU0, ILUK, GS and SGS (ILUT's pattern depends on
 * the values): SILU_ERR_INVALID_ARG otherwise.  Blocks.  An AMG hierarchy or
 * a Schur complement smoother already attached to F keeps the operators it
 * was built from (the finest level's residual uses the new values): reusing
 * it is a valid, possibly weaker, preconditioner; silu_amg_setup /
 * silu_schur_setup again rebuild it from the new values.
 */
silu_status ilu_refactor(silu_ilu F, const double* new_val);

/*
 * Save the factors of F (L_s and U as factored, with kind, scaling,
 * precision, tau and fill) to a binary file, and build a factor object for
 * the matrix A from such a file without factoring again (checkpoint /
 * resume of the setup; scaling, level sets and upload are redone).  The file
 * is host-endian; silu_ilu_load checks its header against A (row count) and
 * its CSR structure (L strictly lower, U with its diagonal first) and
 * returns SILU_ERR_INVALID_ARG for a file that does not fit.  Both block.
 */
silu_status silu_ilu_save(silu_ilu F, const char* path);
silu_status silu_ilu_load(silu_ctx ctx, silu_mat A, const char* path, silu_ilu* out);

/*
 * One smoother application (Eq. ILUsplit with M = L D Utilde, Alg. ILUJac):
 *   r = b - A x;  y = r after sweeps_L sweeps y <- r - L_s y from y = 0;
 *   v after sweeps_U sweeps on the upper factor from v = 0 (see silu_scale);
 *   x <- x + v.
 * x (in/out) and b are device n x nrhs FP64 and must not overlap.  A factor
 * with 0 sweeps is skipped (identity; with SILU_SCALE_ROW and sweeps_U = 0
 * the D^{-1} scaling is skipped too).  nrhs >= 1, sweeps >= 0.
 */
silu_status ilu_smooth(silu_ilu F, double* x, const double* b, int nrhs, int sweeps_L, int sweeps_U);

/*
 * The comparison path: the same update with exact triangular solves,
 * x <- x + Utilde^{-1} D^{-1} L^{-1} (b - A x), in the order of the level
 * sets (Sec. 4: rows of one level are independent; a level needs only rows
 * of earlier levels).  Always FP64 arithmetic on FP64 copies of the factors.
 * Two schedules (silu_ilu_set_direct); by default the library times both
 * once per factor object and column count (on its workspace, when the exact
 * solves are first set up or first used with that many columns) and keeps
 * the faster:
 *   persistent (mode 2): both solves and the update of x in one persistent
 *     launch after the residual.  Rows are stored in level order and taken
 *     in items of at most 32 rows of one level, in level order, by whichever
 *     warp is free; a row waits only for the entries it reads.  Each
 *     published intermediate entry carries a readiness tag in the lowest bit
 *     of its FP64 significand (a relative change of at most 2^-52 per entry),
 *     so one store publishes value and readiness; readers use the entry
 *     with that bit cleared, so results do not depend on the tag.  An item
 *     first waits for one row a few levels back, so items far ahead of the
 *     finished levels do not flood L2 with reads.  Every wait is bounded
 *     (2 s); one that gives up makes the next silu_ctx_check return
 *     SILU_ERR_TIMEOUT.  Capturable in CUDA graphs.
 *   per level (mode 1): one kernel per level, as one captured CUDA graph per column
 *     block; the first one built on F is captured twice, with and without
 *     each level launched as a programmatic dependent of the previous one
 *     (see silu_ctx_set_overlap), and both are timed once; the faster form
 *     is kept for F (same bits either way).
 */
silu_status direct_trisolve(silu_ilu F, double* x, const double* b, int nrhs);

/* Schedule of the exact solves (direct_trisolve, SILU_PRECOND_DIRECT and the
 * AMG cycle with exact solves): 0 automatic (default: the faster of the two,
 * timed once), 1 one launch per level, 2 one persistent launch.  Other
 * values -> SILU_ERR_INVALID_ARG. */
silu_status silu_ilu_set_direct(silu_ilu F, int mode);

/*
 * Fused smoother application (no counterpart in the paper; it concerns only
 * how the steps of Alg. ILUJac are launched).  With row or row/column
 * scaling and 1, 2 or 4 right-hand sides per column block, ilu_smooth (and
 * the smoother inside fgmres_solve) can run the whole application -- the
 * residual, the sweeps on L_s and on the scaled upper factor and the update
 * of x -- in one cooperative launch whose steps are separated by grid-wide
 * barriers, instead of one launch per sweep.  Same step sequence, same
 * per-row summation order.  mode 0 (default): fused for 2 or 4 columns of
 * systems of at most 131072 rows, where launches dominate (one column runs
 * as fast through the staged sweeps, each launched as a programmatic
 * dependent of the one before); 1 never; 2 always.  Every barrier
 * wait is bounded (2 s); one that gives up makes the next silu_ctx_check
 * return SILU_ERR_TIMEOUT.  Other modes -> SILU_ERR_INVALID_ARG.
 */
silu_status silu_ilu_set_fused(silu_ilu F, int mode);

/*
 * Right-preconditioned flexible GMRES(restart) on A x = b for one right-hand
 * side (Sec. 6: FGMRES with modified Gram-Schmidt; stop on the relative
 * residual of Eq. relres, with the true residual recomputed before
 * returning, since the paper warns of false convergence).  x holds the
 * initial guess and receives the solution; b is device FP64 length n.
 * precond: SILU_PRECOND_SWEEPS (the smoother with sweeps_L / sweeps_U from a
 * zero guess), SILU_PRECOND_DIRECT, SILU_PRECOND_NONE.  maxit bounds the
 * total inner iterations.  Blocks until done; writes the iteration count and
 * the true relative residual.  SILU_ERR_NOT_CONVERGED when maxit is reached
 * above tol (x holds the last iterate).  Each inner iteration runs as a CUDA
 * graph captured on its first use (per iteration index, restart, sweeps and
 * preconditioner), and the device runs one inner iteration ahead of the
 * host's stopping test; the iteration queued past the one that ends a cycle
 * touches nothing the update of x reads, so results do not depend on it.
 */
silu_status fgmres_solve(silu_ilu F, double* x, const double* b, double tol, int restart, int maxit, int sweeps_L,
                         int sweeps_U, int precond, int* iters_out, double* relres_out);

/* Preallocate the device workspace for nrhs right-hand sides and a restart
 * length (0 = none), so that later calls do not allocate. */
silu_status silu_ilu_reserve(silu_ilu F, int nrhs, int restart);

/* Sizes: rows, stored entries of L_s and of the stored upper factor
 * (Utilde_s for SILU_SCALE_ROW, U with its diagonal otherwise), level counts. */
silu_status silu_ilu_stats(silu_ilu F, int64_t* n, int64_t* nnz_L, int64_t* nnz_U, int32_t* levels_L,
                           int32_t* levels_U);

/*
 * Copy the host factors out (parity tests).  Any pointer may be NULL.
 *  Lp[n+1], Lc, Lv: strict lower L_s.   Up[n+1], Uc, Uv: U with the diagonal
 *  first in each row (as factored, before scaling).  Sp[n+1], Sc, Sv:
 *  Utilde_s = strict part of D^{-1} U.  dinv[n] = 1 / diag(U).
 *  levL[n], levU[n]: level of each row in L_s and in the upper factor.
 */
silu_status silu_ilu_export(silu_ilu F, int64_t* Lp, int32_t* Lc, double* Lv, int64_t* Up, int32_t* Uc, double* Uv,
                            int64_t* Sp, int32_t* Sc, double* Sv, double* dinv, int32_t* levL, int32_t* levU);
/* Row/column scaling only: D_c (n doubles) and the number of Ruiz steps
 * taken (the Sv / dinv arrays of silu_ilu_export then hold Uhat_s and D_r).
 * SILU_ERR_INVALID_ARG for another scaling.  Either pointer may be NULL. */
silu_status silu_ilu_export_colscale(silu_ilu F, double* dcol, int32_t* ruiz_steps);
/*
 * Numerical nilpotence of a sweep factor (Sec. 5.2, Fig. Up): estimates of
 * ||T^p||_2 for p = 1..pmax, where T = L_s (which = 0) or the strict part of
 * the unit-diagonal upper factor (which = 1: Utilde_s, or Uhat_s under
 * SILU_SCALE_ROWCOL), always in FP64 from the host copy of the factor.  For
 * each p: v = v0 / ||v0||, then `iters` times s = ||T^p v||,
 * v = (T^T)^p T^p v / ||(T^T)^p T^p v||; out[p-1] = the last s, a lower bound
 * that rises to ||T^p||_2 (0 once T^p v vanishes, as it must for p at or
 * beyond the factor's number of levels).  v0: host array of n finite values,
 * not all zero.  out: host array of pmax doubles.  Allocates device copies of
 * T and of its transpose for the call; blocks.  Device context only.
 */
silu_status silu_ilu_power_norms(silu_ilu F, int which, int pmax, int iters, const double* v0, double* out);
/*
 * Departure from normality (Eq. depB, Table dep) of the factors, computed on
 * the host: dep(T) = sqrt(||T||_F^2 - sum |lambda_i|^2), which for a
 * triangular T is the Frobenius norm of its off-diagonal part.  dep_L: the
 * unit lower factor L; dep_U: U as factored; dep_scaled: the unit-diagonal
 * upper factor the sweeps use (D^{-1} U, or D_r U D_c under
 * SILU_SCALE_ROWCOL).  Any pointer may be NULL; host-only contexts work.
 */
silu_status silu_ilu_dep(silu_ilu F, double* dep_L, double* dep_U, double* dep_scaled);
/* Entry counts of U with diagonal (for export buffer sizing). */
silu_status silu_ilu_export_sizes(silu_ilu F, int64_t* nnz_L, int64_t* nnz_Ufull, int64_t* nnz_Us);

void silu_ilu_destroy(silu_ilu F);

/*
 * Kernel launch shape of the sweeps: lanes per row (power of two, 1..32) for
 * L_s, the upper factor and A; 0 restores the library's choice.  Used by the
 * autotuner; results do not depend on it beyond rounding order.
 */
silu_status silu_ilu_set_lanes(silu_ilu F, int lanes_L, int lanes_U, int lanes_A);

/*
 * Sweep kernel variant: 0 = automatic (the staged kernel for one right-hand
 * side; for 2 or 4 interleaved right-hand sides the staged kernel on
 * factors tiled one lane per row when the factor has at least 16 tiles per
 * multiprocessor, the lanes-per-row kernel otherwise), 1 = always the
 * lanes-per-row kernel, 2 = the staged kernel wherever it applies, 3 = as 2
 * but on length-sorted copies of the factors for one right-hand side (built
 * on first selection, for the factors where silu_ilu_layout shows sorting
 * pays; device memory for one more copy of those factors).  The staged
 * kernel streams nnz-balanced row tiles of the factor into shared memory
 * with bulk asynchronous copies; it needs rows of at most 416 entries.  With
 * R right-hand sides each staged factor entry feeds R FMAs, so the factor is
 * read once per sweep for all of them.  A sorted copy keeps each row's
 * entries in order, so with one lane per row variants 2 and 3 give the same
 * bits.
 */
silu_status silu_ilu_set_kernel(silu_ilu F, int variant);

/*
 * Storage layout of the sweep factors (no counterpart in the paper, whose
 * performance model of Sec. 6.3 charges one read of each factor per sweep
 * and no arithmetic).  The staged kernel gives each row of a 32-row warp
 * tile one lane and spends, per tile, as many FP64 multiply-adds as the
 * tile's longest row has entries; rows of uneven length (ILUT factors) waste
 * some of that work.  At setup the library measures it for L_s (index 0) and
 * the upper sweep factor (index 1): pad_natural[k] = FMA slots per stored
 * entry with rows in their natural order, pad_sorted[k] = the same after
 * sorting the rows of every 512-row window by length (row numbers then
 * travel with each tile so results land in their rows).  Sorting pays where
 * pad_natural >= 1.08 and it saves at least 0.05; variant 3 of
 * silu_ilu_set_kernel (or the autotuner) then sweeps a sorted device copy,
 * and in_use[k] = 1.  Fewer FMA slots do not always mean a faster sweep:
 * lanes of one warp then gather from rows further apart.
 * Pads are 0 for an empty factor or one with a row too long to stage.
 * Works on host-only contexts (in_use = 0 there).  Any pointer may be NULL.
 */
silu_status silu_ilu_layout(silu_ilu F, double* pad_natural, double* pad_sorted, int32_t* in_use);

/*
 * Algebraic multigrid (Sec. 3, Alg. mgcycle): the paper's solver
 * configuration, a V-cycle whose finest level is smoothed by the scaled-ILU
 * smoother.
 *
 * silu_amg_setup builds the hierarchy of A (the silu_mat F was set up from)
 * on the host and uploads it; it is attached to F and freed with it (a second
 * call replaces it).  Strength of connection (Sec. 3): j strongly influences
 * i when |a_ij| >= theta max_{k != i} |a_ik|.  Coarse points: the
 * Ruge-Stueben first pass (largest number of strongly influenced points
 * first, smallest index on ties).  Interpolation: Stueben's direct
 * interpolation from the strong coarse neighbours.  Coarse operators:
 * A_{l+1} = P^T A_l P.  Coarsening stops at max_levels levels, at
 * coarse_size rows or fewer, or when no further split is possible; the
 * coarsest level (at most 4096 rows, else SILU_ERR_INVALID_ARG) is solved by
 * its dense inverse.  Levels below the finest are smoothed, before and after
 * their coarse-grid correction, by jacobi_sweeps steps of
 *   SILU_AMG_L1_JACOBI: x <- x + D^{-1}(b - A x) with d_i = sum_j |a_ij|, or
 *   SILU_AMG_POLY_GS:   x <- x + sum_{j<gs_terms} (-D^{-1} L)^j D^{-1} (b - A x)
 *                       (polynomial Gauss-Seidel, Sec. 3.1; the mixed V-cycle
 *                       of Sec. 6.3), D = diag(A), L its strict lower part.
 * ilu_levels > 1 smooths levels 1 .. ilu_levels - 1 (those above the
 * coarsest) with the ILU smoother instead (Sec. 6: ILU smoothing from the
 * finest level down, up to all levels): each gets its own incomplete
 * factorisation of A_l of F's kind, drop tolerance and fill (ILU(0), ILU(k)
 * or ILUT; a Gauss-Seidel kind -> SILU_ERR_INVALID_ARG), row-scaled, in F's
 * precision, and is smoothed once before and once after its correction with
 * the cycle's sweep counts (or its exact triangular solves when the cycle
 * uses them on the finest level).  0 or 1: the finest level only.
 * params NULL = {0.25, 25, 400, 1, SILU_AMG_L1_JACOBI, 2, 1}.  Blocks.
 */
typedef enum { SILU_AMG_L1_JACOBI = 0, SILU_AMG_POLY_GS = 1 } silu_amg_smoother;
typedef struct {
  double theta;         /* strength threshold, 0 < theta <= 1 */
  int max_levels;       /* >= 1 */
  int coarse_size;      /* stop coarsening at this many rows or fewer, >= 1 */
  int jacobi_sweeps;    /* smoothing steps before and after the correction below the finest level, >= 0 */
  int coarse_smoother;  /* silu_amg_smoother */
  int gs_terms;         /* Neumann terms of each polynomial Gauss-Seidel step, >= 1 */
  int ilu_levels;       /* levels from the finest smoothed by the ILU smoother, >= 0 (0 and 1: the finest only) */
} silu_amg_params;
silu_status silu_amg_setup(silu_ilu F, const silu_amg_params* params);
/*
 * One V-cycle on A x = b (device, one right-hand side, x in/out, stream-
 * ordered): the finest level is smoothed before and after the coarse-grid
 * correction by ilu_smooth's update with sweeps_L / sweeps_U sweeps of F's
 * smoother, or, with sweeps_L and sweeps_U both negative, by
 * direct_trisolve's update (exact triangular solves); the levels that
 * silu_amg_params.ilu_levels gives the ILU smoother the same way on their own
 * factors.  A one-level hierarchy is the direct solve x = A^{-1} b.
 */
silu_status silu_amg_vcycle(silu_ilu F, double* x, const double* b, int sweeps_L, int sweeps_U);
/*
 * The same V-cycle with the finest level smoothed, before and after the
 * coarse-grid correction, by one application of the ILUT Schur complement
 * smoother (silu_schur_setup; Sec. 3.1 uses it as the smoother of one level of
 * the V-cycle), its interior blocks swept sweeps_L + sweeps_U
 * times; coarser levels as in silu_amg_vcycle (ILU levels with sweeps).  x (n FP64, device) is updated
 * in place from its current value; b is read.  Requires silu_amg_setup and
 * silu_schur_setup on F (else SILU_ERR_INVALID_ARG), negative sweep counts
 * -> SILU_ERR_INVALID_ARG.  Stream-ordered on F's context.
 */
silu_status silu_amg_vcycle_schur(silu_ilu F, double* x, const double* b, int sweeps_L, int sweeps_U);
/*
 * The factor object that smooths AMG level `level` with the ILU smoother
 * (Sec. 6: ILU smoothing from the finest level down): F itself for level 0,
 * the row-scaled factorisation of A_l for levels 1 .. ilu_levels - 1
 * (silu_amg_params).  *out is borrowed: valid until the
 * next silu_amg_setup on F or F's destruction, never passed to
 * silu_ilu_destroy.  Queries (silu_ilu_stats, silu_ilu_export) work on it.
 * A level without one, or no hierarchy -> SILU_ERR_INVALID_ARG.
 */
silu_status silu_amg_level_ilu(silu_ilu F, int level, silu_ilu* out);
/* Levels and, for l < cap, rows, entries of A_l and of P_l (0 on the coarsest level). */
silu_status silu_amg_stats(silu_ilu F, int cap, int* levels, int64_t* rows, int64_t* nnz_A, int64_t* nnz_P);
/* Host copies of level l (parity tests): A_l (row pointers n_l + 1), P_l
 * (row pointers n_l + 1) and the coarse-point marks (n_l), the last two only
 * below the coarsest level.  Any pointer may be NULL. */
silu_status silu_amg_export_level(silu_ilu F, int level, int64_t* Ap, int32_t* Ac, double* Av, int64_t* Pp,
                                  int32_t* Pc, double* Pv, int32_t* cf);

/*
 * ILUT Schur complement smoother (Sec. 3.1, Eq. schur), attached to F (freed
 * with it; a second call replaces it).  The rows are split into `parts`
 * contiguous blocks, the single-device stand-in for the paper's MPI ranks
 * (block k holds rows [k n / parts, (k+1) n / parts)); a row with an entry in
 * another block is an interface row.  With A permuted to [B E; F C] (interior
 * rows first, each group in ascending order), B (block diagonal) is factored
 * by ILUT(tau, fill) with row scaling in F's precision.  One application
 * z = M^{-1} r:  s = r_G - F B^{-1} r_I;  one GMRES iteration on S y = s,
 * S = C - F B^{-1} E, from y = 0 (the minimal-residual step, no residual of
 * the full system formed);  z_I = B^{-1} (r_I - E y), z_G = y.  Every B^{-1}
 * is sweeps_L + sweeps_U Richardson sweeps on B's row-scaled factors.
 * Blocks; works on host-only contexts (setup and statistics only).
 */
silu_status silu_schur_setup(silu_ilu F, int parts, double tau, int fill);
/* x <- x + M^{-1} (b - A x) with the Schur complement smoother (device, one
 * right-hand side, stream-ordered). */
silu_status silu_schur_smooth(silu_ilu F, double* x, const double* b, int sweeps_L, int sweeps_U);
/*
 * The right preconditioner of the smoother's single interface GMRES
 * iteration: SILU_SCHUR_IFACE_NONE (the default, the paper's unpreconditioned
 * iteration) or SILU_SCHUR_IFACE_DIAG, M = diag(C): the step becomes
 * y = ((S q).s / (S q).(S q)) q with q = M^{-1} s, which takes the scale of
 * each interface row into account (not in the paper; it makes the smoother
 * converge where the interface rows' scales vary over orders of magnitude).
 * Requires silu_schur_setup (else SILU_ERR_INVALID_ARG); a zero c_kk ->
 * SILU_ERR_ZERO_PIVOT for SILU_SCHUR_IFACE_DIAG; other modes ->
 * SILU_ERR_INVALID_ARG.  Applies to every later application on F (the
 * stand-alone smoother, SILU_PRECOND_SCHUR and SILU_PRECOND_AMG_SCHUR).
 */
typedef enum { SILU_SCHUR_IFACE_NONE = 0, SILU_SCHUR_IFACE_DIAG = 1 } silu_schur_iface;
silu_status silu_schur_set_interface_prec(silu_ilu F, int mode);
/* Interior and interface counts, and the interface mark of every row (n
 * int32, may be NULL). */
silu_status silu_schur_stats(silu_ilu F, int64_t* n_interior, int64_t* n_interface, int32_t* iface);

/*
 * Batches of independent systems (many pressure solves of uneven size).
 *
 * silu_batch_setup factors `count` host CSR systems (arrays as for
 * silu_mat_create, system k with n[k] rows) independently and in parallel on
 * the host, with the same kind / tau / fill / scale / prec for all, and
 * packs them as one block-diagonal system on the device: the incomplete
 * factors of a block-diagonal matrix are the block-diagonal of the systems'
 * factors, so one sweep launch over the concatenation performs every
 * system's sweep (Alg. ILUJac applied to each system).  Vectors of a batch
 * are the systems' vectors concatenated: system k occupies rows
 * [offsets[k], offsets[k+1]) (silu_batch_info).  Blocks.
 */
silu_status silu_batch_setup(silu_ctx ctx, int count, const int64_t* n, const int64_t* const* row_ptr,
                             const int32_t* const* col_idx, const double* const* val, silu_kind kind, double tau,
                             int fill, silu_scale scale, silu_prec prec, silu_batch* out);
/* Count, offsets[count + 1], and the silu_ilu of the concatenated system
 * (owned by the batch; usable with ilu_smooth, silu_ilu_set_kernel, ...). */
silu_status silu_batch_info(silu_batch B, int* count, int64_t* offsets, silu_ilu* factors);
/* One smoother application on every system (ilu_smooth on the concatenation). */
silu_status silu_batch_smooth(silu_batch B, double* x, const double* b, int sweeps_L, int sweeps_U);
/*
 * Flexible GMRES(restart) on every system at once, each with its own Krylov
 * basis, Hessenberg matrix, Givens rotations, iteration count and stopping
 * test (Sec. 6, Eq. relres): dot products are reduced per system in a fixed
 * order; a system stops updating once its estimate reaches tol * |b_k|, and
 * every restart recomputes every true residual.  precond is
 * SILU_PRECOND_SWEEPS or SILU_PRECOND_NONE.  Each inner iteration runs as a
 * captured CUDA graph.  iters[count] and relres[count] (may be NULL) receive
 * each system's inner iterations and true relative residual.  Blocks;
 * SILU_ERR_NOT_CONVERGED if some system is still above tol at maxit.
 */
silu_status silu_batch_fgmres(silu_batch B, double* x, const double* b, double tol, int restart, int maxit,
                              int sweeps_L, int sweeps_U, int precond, int* iters, double* relres);
/*
 * Autotuner: times one smoother application (sweeps_L, sweeps_U) with each
 * candidate launch shape of the sweep kernels and keeps the fastest:
 * rows per warp (staged kernel: 8, 16, 32, 64 or 128 rows per warp tile,
 * i.e. four or two lanes per row, one, or one lane taking two or four rows;
 * or the lanes-per-row kernel with 2, 4 or 8 lanes) and gather width (8 or
 * 16 entries in flight per lane; 0 = the automatic configuration: narrow
 * tiles swept by 24 warps with 10 gathers in flight for FP64 factors whose
 * rows fit them, see silu_mat_set_shape, else 16).  Writes the chosen
 * candidate's index and its time per application.  Blocks.
 */
silu_status silu_ilu_autotune(silu_ilu F, int sweeps_L, int sweeps_U, int* choice, double* ms);
/*
 * The autotuner's candidates and their times from the last silu_ilu_autotune
 * on F: *count = number of candidates (0 before any tuning); for the first
 * min(cap, *count) candidates, shape[4 k .. 4 k + 3] = {variant (1 lanes-per-
 * row kernel, 2 staged kernel, 3 staged kernel on sorted copies), lanes per
 * row (0 = from the mean row length), rows per lane (0 = automatic), gather
 * width (0 = automatic)} and ms[k] = time per application (-1 for a candidate not run: a
 * sorted-copy candidate when no factor has one).  shape and ms may be NULL.
 */
silu_status silu_ilu_tune_table(silu_ilu F, int cap, int32_t* shape, double* ms, int* count);
void silu_batch_destroy(silu_batch B);

/*
 * Solve server: continuous batching of pressure solves on one GPU.
 *
 * Requests arrive at any time (silu_server_submit copies the host CSR system
 * and right-hand side) and wait in a FIFO queue.  The head of the queue is
 * admitted when one of `workers` slots is free and its device-memory
 * estimate fits in what is left of hbm_budget_bytes; a request larger than
 * the whole budget is refused (SILU_ERR_OOM) and so is any request while
 * `max_queue` requests wait (SILU_ERR_BUSY).  Each slot has its own host
 * thread, CUDA stream and context: it factors the system on the host
 * (ilu_setup, row scaling; with precond SILU_PRECOND_AMG or
 * SILU_PRECOND_AMG_DIRECT also silu_amg_setup with the default parameters),
 * runs fgmres_solve from x = 0 on its stream and
 * copies the solution back, so admitted requests overlap on the device and
 * memory is released as each finishes.  Results do not depend on what else
 * runs.  device = -1 makes a host-only server for testing the admission
 * logic: requests are set up and finish with SILU_ERR_NO_DEVICE.
 */
typedef struct {
  int kind;             /* silu_kind */
  double tau;           /* ILUT drop tolerance */
  int fill;             /* ILU(k) level / ILUT fill per row */
  int prec;             /* silu_prec of the factors and sweeps */
  double tol;           /* relative residual (Eq. relres) */
  int restart, maxit;
  int sweeps_L, sweeps_U;
  int precond;          /* silu_precond: SWEEPS, DIRECT, NONE, AMG or AMG_DIRECT */
} silu_request_params;

typedef struct {
  int status;           /* silu_status of the request */
  int iterations;       /* FGMRES inner iterations */
  double relres;        /* true relative residual at return */
  double t_submit;      /* seconds since the server was created */
  double t_admit;
  double t_setup_done;
  double t_done;
  int64_t device_bytes; /* HBM reserved while it ran */
} silu_result;

silu_status silu_server_create(int device, int64_t hbm_budget_bytes, int workers, int max_queue, silu_server* out);
silu_status silu_server_submit(silu_server S, int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                               const double* val, const double* b, const silu_request_params* params,
                               uint64_t* ticket);
/* Cancel a request that has not been admitted (SILU_ERR_BUSY once it runs). */
silu_status silu_server_cancel(silu_server S, uint64_t ticket);
/*
 * done = 1 once the request finished; then res and (if non-NULL) the
 * solution x[n] are written and the ticket is released.  wait = 1 blocks
 * until it finishes.
 */
silu_status silu_server_poll(silu_server S, uint64_t ticket, int wait, int* done, silu_result* res, double* x);
silu_status silu_server_stats(silu_server S, int64_t* queued, int64_t* running, int64_t* completed,
                              int64_t* refused, int64_t* bytes_in_use);
/* Stop: requests not yet admitted finish as SILU_ERR_CANCELLED; running ones complete. */
void silu_server_destroy(silu_server S);

/*
 * Allocation-free smoother application (the paper has no counterpart; it
 * exists for callers that cannot allocate device memory when they apply
 * the smoother: applications whose device memory is owned up front by their
 * own pool or another framework's allocator, and latency-critical loops
 * that must not pay the implicit synchronisation of cudaMalloc / cudaFree).
 *
 * Computes the same update as ilu_smooth with row scaling, FP64, one
 * right-hand side:  x <- x + v,  v from sweeps_U sweeps on Utilde_s after
 * sweeps_L sweeps on L_s applied to r = b - A x.  All arrays are DEVICE
 * arrays owned by the caller, with int32 row pointers (n+1 entries), int32
 * column indices and FP64 values: A, the strict lower factor L_s, the
 * strict scaled upper factor Utilde_s (as silu_ilu_export's Sp/Sc/Sv), and
 * dinv = 1 / diag(U); x (in/out) and b have n entries.  Work is ordered on
 * cuda_stream of `device` and is asynchronous.
 *
 * Nothing is allocated: the working vectors live in a fixed array compiled
 * into the library (four vectors of 524288 doubles, 16 MiB, held by every
 * device that loads the library until the process exits).  n above 524288
 * returns SILU_ERR_TOO_LARGE before any work.  The first call on a device
 * looks up that array's device address (with the device made current, the
 * caller's current device restored afterwards); under CUDA's default lazy
 * module loading this lookup is what loads the array onto the device, so
 * the 16 MiB are taken by that first call, which returns SILU_ERR_OOM if
 * they are not free.  Make the first call before a memory pool claims the
 * device (and before any stream capture); later calls need no memory.  The
 * address is kept for the life of the process: calls after cudaDeviceReset
 * are not supported.  All calls share the array and it keeps the last
 * call's contents (every vector is written before it is read); calls whose
 * work overlaps on the GPU race on it.
 * Returns SILU_ERR_INVALID_ARG for null pointers or negative counts,
 * SILU_ERR_NO_DEVICE if the device cannot be selected, SILU_ERR_OOM as
 * above, SILU_ERR_CUDA if a launch fails.
 */
silu_status silu_smooth_noalloc(int device, void* cuda_stream, int64_t n, const int32_t* A_rp, const int32_t* A_ci,
                                const double* A_val, const int32_t* L_rp, const int32_t* L_ci, const double* L_val,
                                const int32_t* U_rp, const int32_t* U_ci, const double* U_val, const double* dinv,
                                double* x, const double* b, int sweeps_L, int sweeps_U);

#ifdef __cplusplus
}
#endif

#endif /* SILU_H */
