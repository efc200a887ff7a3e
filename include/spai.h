/*
 * spai.h -- C ABI of libspai.so: global short-recurrence sparse approximate
 * inverses (MR, LOMR, Frobenius-CG) of an SPD matrix A on one GB300 GPU,
 * and the vector PCG that assesses them as preconditioners.
 *
 * Problem (Venkovic & Anzt, Sec. 2, Eqs. (2.3)-(2.4)): find a sparse M with
 * A M ~ I by decreasing f(M) = ||I - A M||_F^2 with global iterations whose
 * sparse matrix iterates are updated as a whole.
 *
 * Conventions for every call:
 *   - return 0 on success, > 0 for a non-fatal outcome, < 0 for an error;
 *     spai_status_string() names each code; the library never aborts or
 *     prints;
 *   - the handle owns all device memory it allocates; pointers passed in are
 *     only read or written during the call (or, for device pointers, by work
 *     the call enqueues on the handle's stream);
 *   - calls are ordered on the handle's CUDA stream and synchronise that
 *     stream only where they return host data;
 *   - a handle is not thread safe; distinct handles are independent;
 *   - no call falls back to CPU computation: every numeric step runs in the
 *     library's CUDA kernels.
 *
 * Storage of A: CSR, int32 row pointers and column indices (rows sorted by
 * column, no duplicates), FP64 values; A must be exactly symmetric with a
 * positive diagonal.  Storage of M on output: CSC (column pointers, row
 * indices sorted within each column, values).
 */
#ifndef SPAI_H
#define SPAI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------- status codes */
#define SPAI_OK 0
#define SPAI_CONVERGED_EARLY 1   /* ||R_i||_F or a step denominator reached 0 */
#define SPAI_LOMR_FALLBACK 2     /* LOMR took at least one MR step (c_i ~ 0) */
#define SPAI_PCG_MAXIT 3         /* PCG stopped at maxit */
#define SPAI_PCG_BREAKDOWN 4     /* PCG: (p,Ap) or (r,z) zero or non-finite */
#define SPAI_ERR_ARG -1          /* bad argument (NULL, negative size, ...) */
#define SPAI_ERR_CSR -2          /* malformed CSR (pointers, order, range) */
#define SPAI_ERR_NOT_SPD_DIAG -3 /* missing or non-positive diagonal entry */
#define SPAI_ERR_NOT_SYMMETRIC -4/* A is not exactly symmetric */
#define SPAI_ERR_NONFINITE -5    /* NaN/Inf in A or in a step coefficient */
#define SPAI_ERR_CUDA -6         /* a CUDA runtime call failed */
#define SPAI_ERR_OOM -7          /* device allocation failed */
#define SPAI_ERR_CAPACITY -8     /* a column outgrew its slab capacity */
#define SPAI_ERR_UNSUPPORTED -9  /* size outside the kernels' limits */
#define SPAI_ERR_STATE -10       /* saved state does not match the handle */

/* --------------------------------------------------------------- options */
enum { SPAI_FP64 = 0, SPAI_MIXED = 1 };           /* MIXED: FP32 values, FP64 reductions */
enum { SPAI_MR = 0, SPAI_LOMR = 1, SPAI_CG = 2, SPAI_MR_PI = 3, SPAI_LOMR_PI = 4, SPAI_CG_PI = 5 };
enum { SPAI_DROP_NONE = 0, SPAI_DROP_TOPK_COL = 1, SPAI_DROP_TOPK_COL_DIAG = 2 };
enum { SPAI_PREC_NONE = 0, SPAI_PREC_JACOBI = 1, SPAI_PREC_SPAI = 2, SPAI_PREC_SPAI_SYM = 3 };

typedef struct spai_ctx *spai_handle;

typedef struct {
  int prec;          /* SPAI_FP64 or SPAI_MIXED */
  double cap_factor; /* per-column capacity and drop cap:
                        cap_j = floor(cap_factor * nnz(A[:,j])), clamped to [1, n] */
} spai_opts;

typedef struct {
  double *resnorm;   /* host, [iters+1] or NULL: ||R_i||_F, i = 0..iters */
  double *coef;      /* host, [2*iters] or NULL: (alpha,0) MR, (delta,gamma) LOMR,
                        (alpha_i, beta_{i+1}) CG */
  int iters_done;    /* out: iterations completed */
  int flags;         /* out: bit0 converged early, bit1 LOMR fallback */
  int64_t *nnz;      /* host, [iters+1] or NULL: nnz(M_i), i = 0..iters, the iterate
                        whose residual resnorm[i] records (spai_run and its
                        shorthands on a single-matrix handle; entries past an
                        early stop are left alone) */
} spai_history;

typedef struct {
  int64_t colpass_launches;   /* column-pass kernels launched since create */
  int64_t colpass_bytes;      /* algorithmic DRAM bytes of those launches */
  double colpass_ms;          /* their summed device time (timing mode only) */
  int64_t pcg_launches;       /* PCG kernels launched since create */
  int64_t other_launches;     /* set-up / transpose / norm kernels */
  int64_t spgemm_columns;     /* column SpGEMMs performed (Table 2 check) */
  int64_t colpass_r_bytes;    /* of colpass_bytes: the R lists CG's pass A stores for the next
                                 pass B (a layout choice of this library, not the method's
                                 own traffic) */
  int64_t colpass_steady_launches; /* of colpass_launches: mid-run passes that ran the kernels
                                      compiled for steady-state flags (same results as the
                                      general kernels; chosen when every column product has
                                      the short DIA form) */
} spai_stats;

/* ------------------------------------------------------------- host only */

/* Validate a CSR matrix on the host without touching the GPU.
 * Checks n >= 1, rowptr monotone with rowptr[0]=0 and rowptr[n]=nnz, column
 * indices in [0,n) strictly increasing per row, finite values, a positive
 * diagonal in every row and, if check_symmetry, exact symmetry.  Returns
 * SPAI_OK or SPAI_ERR_CSR / SPAI_ERR_NOT_SPD_DIAG / SPAI_ERR_NOT_SYMMETRIC /
 * SPAI_ERR_NONFINITE / SPAI_ERR_ARG: with several faults, the code of the
 * one in the smallest row (symmetry is checked after the rest).  Matrices
 * of 2^20 entries or more are checked over row ranges on up to 16 host
 * threads (started and joined within the call). */
int spai_validate_csr(int64_t n, int64_t nnz, const int32_t *rowptr, const int32_t *colind,
                      const double *vals, int check_symmetry);

/* Human-readable name of a status code (static string, never NULL). */
const char *spai_status_string(int code);

/* ---------------------------------------------------------------- handle */

/* Create a handle for the SPD matrix A (n x n, nnz entries).
 * rowptr/colind/vals are host pointers (on_device = 0) or device pointers
 * (on_device = 1); A is validated (symmetry included) and copied, the caller
 * keeps ownership.  stream: a cudaStream_t, or NULL for a stream the handle
 * creates.  M is initialised to diag(A)^{-1} (Algorithm 1 with M_0 = D^{-1}).
 * Column slabs of capacity cap_j are allocated for M and two directions.
 * Limits: n < 2^31, max row length of A <= 64, cap_j * rowlen <= 65534. */
int spai_create(spai_handle *out, int64_t n, int64_t nnz, const int32_t *rowptr,
                const int32_t *colind, const double *vals, int on_device, const spai_opts *opts,
                void *stream);

/* Batched handle (no counterpart in the paper: many independent SPAIs at
 * once).  nmat SPD matrices, each given as its own CSR (host arrays, each
 * validated as in spai_create), are laid block-diagonally, each padded with
 * identity rows to a multiple of 256; every spai_run / PCG step then treats
 * all of them in the same launches, with per-matrix step coefficients, stops
 * and histories, so that each matrix's iterates equal those of a
 * single-matrix handle.  Limits: every matrix n <= 262,144 and has at most 32
 * distinct diagonals for the fast path; the padded total n < 2^26.
 * spai_get_M / spai_apply / pcg_solve see the padded block-diagonal matrix;
 * a call after one matrix converged early restarts every recurrence. */
int spai_create_batched(spai_handle *out, int nmat, const int64_t *n, const int64_t *nnz,
                        const int32_t *const *rowptr, const int32_t *const *colind,
                        const double *const *vals, const spai_opts *opts, void *stream);

/* Number of matrices of a handle (1 for a single-matrix handle) and, if
 * n_each != NULL, their sizes. */
int spai_batch_info(spai_handle h, int *nmat, int64_t *n_each);

/* Per-matrix results of the last spai_run (host arrays, may be NULL):
 * resnorm[m*(iters+1) + i] = ||R_i||_F of matrix m, iters_done[m], flags[m]. */
int spai_batch_history(spai_handle h, double *resnorm, int *iters_done, int *flags);

/* ||I - A_m M_m||_F in FP64 for every matrix m (host out[nmat]). */
int spai_batch_residual_norms(spai_handle h, double *out);

/* CSC of matrix m's M on the host, two-call like spai_get_M. */
int spai_batch_get_M(spai_handle h, int m, int64_t *nnz, int32_t *colptr, int32_t *rowind,
                     double *vals);

/* Free every device and host resource of the handle. */
int spai_destroy(spai_handle h);

/* Re-initialise M := diag(A)^{-1} and forget the method recurrence. */
int spai_reset(spai_handle h);

/* Use another CUDA stream for subsequent calls. */
int spai_set_stream(spai_handle h, void *stream);

/* ---------------------------------------------------------- the methods */

/* Run `iters` iterations of a method from the current M.  A call continues
 * the recurrence of the previous call when it uses the same method (so
 * k + l iterations in two calls equal k + l in one); otherwise the method
 * starts from the current M with empty search directions.
 *   MR   -- Algorithm 1, explicit residual: P_i = D(R_i),
 *           alpha_i = (R_i, A P_i)_F / ||A P_i||_F^2 (Eq. 2.6),
 *           M_{i+1} = D(M_i + alpha_i P_i).
 *   LOMR -- Algorithm 4 / Theorem 3: Z_i = D(R_i), (delta_i, gamma_i) solve the
 *           2x2 normal equations for span{A Z_i, A P_{i-1}} (Eqs. 4.7-4.9),
 *           S_i = delta_i Z_i + gamma_i P_{i-1}, P_i = D(S_i), M_{i+1} = D(M_i + S_i);
 *           a near-singular 2x2 system (c_i <= 64 eps uu vv) takes an MR step.
 *   CG   -- Algorithm 3: alpha_i = ||R_i||^2/(P_i, A P_i), M_{i+1} = D(M_i + alpha_i P_i),
 *           beta_{i+1} = ||R_{i+1}||^2/||R_i||^2, P_{i+1} = D(R_{i+1} + beta_{i+1} P_i).
 *   MR_PI, LOMR_PI, CG_PI -- the left-preconditioned forms of Sec. 5 with
 *           Pi = diag(A)^{-1} (MR_SPD Algorithm 5, LOMR_SPD Algorithm 8, CG
 *           Algorithm 7): the direction is built from Z = Pi R (z_k = r_k / a_kk
 *           as pi_k r_k, pi_k = 1/a_kk in FP64, rounded to the value type) and
 *           every coefficient inner product is weighted, (X, Pi Y)_F with terms
 *           fl(fl(x y) pi_k); CG's (P, A P) stays unweighted.  MR_PI: alpha =
 *           (Pi R, A P)/(A P, Pi A P), P = D(Pi R).  LOMR_PI: the 2x2 system in
 *           the Pi-weighted products, Z = D(Pi R).  CG_PI: alpha =
 *           (R, Pi R)/(P, A P), beta = (R+, Pi R+)/(R, Pi R), P = D(Pi R + beta P).
 *           The history still records ||R_i||_F.
 * D is the per-column hard threshold of Sec. 6.1 (keep the cap_j largest |v|,
 * ties to the smaller row; exact zeros never stored) for SPAI_DROP_TOPK_COL;
 * SPAI_DROP_TOPK_COL_DIAG is the same drop except that row j of column j,
 * when present, is always kept and counts toward cap_j (Appendix A: the
 * diagonal is never dropped), for M and for the directions alike;
 * D is the identity for SPAI_DROP_NONE (a column that outgrows its capacity
 * then fails the call with SPAI_ERR_CAPACITY).  R is always the explicit
 * residual I - A M (Sec. 6.2).  hist may be NULL.  Returns SPAI_OK,
 * SPAI_CONVERGED_EARLY, SPAI_LOMR_FALLBACK or an error.
 * CG keeps the R of each pass A in a device slab for the next pass B, which
 * then reads it instead of forming A M again (Table 2's two products per
 * iteration); when that slab cannot be allocated, or the environment
 * variable SPAI_CG_NO_R_SLAB is 1, pass B forms R itself, with the same
 * results. */
int spai_run(spai_handle h, int method, int iters, int drop_rule, spai_history *hist);

/* Launch-shape autotuner (no counterpart in the paper).  For the column
 * passes that `method` uses, runs `iters` iterations from M_0 and then
 * times `iters` more (continuing from that state) with each
 * distinct candidate shape (the CTA size that lets 1..8 CTAs share an
 * SM's shared memory x 1, 2, 4 or 8 columns per warp) and keeps the
 * fastest for later calls.  Results do not depend on the shape
 * (column sums are order-free and the Frobenius tree runs over column
 * indices), so only the time changes.  Leaves M = diag(A)^{-1} and no
 * recurrence.  *best_ms (may be NULL): the chosen shape's time per
 * iteration. */
int spai_autotune(spai_handle h, int method, int iters, double *best_ms);

/* spai_run with method SPAI_MR, SPAI_LOMR or SPAI_CG (same arguments, same
 * results and return codes). */
int spai_mr(spai_handle h, int iters, int drop_rule, spai_history *hist);
int spai_lomr(spai_handle h, int iters, int drop_rule, spai_history *hist);
int spai_cg(spai_handle h, int iters, int drop_rule, spai_history *hist);

/* ||I - A M||_F computed in FP64 from the stored M (FP32 values promoted
 * exactly), Eq. (2.4); written to *out (host). */
int spai_residual_norm(spai_handle h, double *out);

/* Number of stored nonzeros of M (host *out). */
int spai_get_nnz(spai_handle h, int64_t *out);

/* Export M in CSC.  Two-call use: with colptr == NULL only *nnz is set.
 * Otherwise colptr[n+1], rowind[*nnz], vals[*nnz] (FP64) are filled; they are
 * host arrays (on_device = 0) or device arrays (on_device = 1). */
int spai_get_M(spai_handle h, int64_t *nnz, int32_t *colptr, int32_t *rowind, double *vals,
               int on_device);

/* Replace M by a CSC matrix (host or device arrays, rows sorted per column,
 * column j holding at most cap_j entries) and forget the method recurrence. */
int spai_set_M(spai_handle h, const int32_t *colptr, const int32_t *rowind, const double *vals,
               int on_device);

/* y = M x for nrhs right-hand sides stored column-major with leading
 * dimension ld (>= n); x and y are FP64 device pointers.  Uses the row-wise
 * (transposed) copy of M built on first use after M changes. */
int spai_apply(spai_handle h, const double *x, double *y, int nrhs, int64_t ld);

/* Vector PCG on A x = b (Sec. 7 assessment), x_0 = 0, FP64 vectors and
 * scalars, stop when ||r||_2 <= rtol ||b||_2 (recurrence residual) or after
 * maxit iterations.  precond: SPAI_PREC_NONE, SPAI_PREC_JACOBI,
 * SPAI_PREC_SPAI (z = M r) or SPAI_PREC_SPAI_SYM (z = (M + M^T) r / 2).
 * b, x: n-vectors, host (on_device = 0) or device (on_device = 1); nrhs = 1.
 * *iters (host) = number of A p products; *relres (host, may be NULL) =
 * ||b - A x||_2 / ||b||_2.  Returns SPAI_OK, SPAI_PCG_MAXIT,
 * SPAI_PCG_BREAKDOWN or an error. */
int pcg_solve(spai_handle h, const double *b, double *x, int nrhs, double rtol, int maxit,
              int precond, int on_device, int *iters, double *relres);

/* Arithmetic of the products inside pcg_solve and pcg_solve_block.
 * SPAI_FP64 (the default): A p and M r (or S r) in FP64.  SPAI_MIXED: those
 * products use FP32 values (A rounded once to FP32; M's values, and S's
 * computed in FP64 and then rounded) and an FP32 copy of the operand vector,
 * accumulated by an FP32 fma chain over ascending column and widened to
 * FP64; the vectors x, r, p, z, all inner products, the step scalars and the
 * reported true residual stay FP64 (the mixed path of Sec. 7's assessment:
 * FP32 values, FP64 recurrences).  On GB300 the FP32 products avoid the
 * small FP64 pipe.  The recurrence residual still reaches rtol; the true
 * residual of a mixed solve levels off near FP32 rounding times the
 * conditioning, so report relres beside the iteration count. */
int spai_set_pcg_prec(spai_handle h, int prec);

/* Block PCG (Sec. 7's assessment applied to many right-hand sides; the paper
 * solves one at a time): nrhs (1..32) independent PCG recurrences per matrix
 * of the handle, each one exactly the recurrence pcg_solve runs on that
 * matrix and vector (same stopping rule, same preconditioner choices), all
 * sharing each product with A and with M.  A single-matrix handle counts as
 * one matrix.
 * b, x: host (on_device = 0) or device (on_device = 1) FP64 arrays holding,
 * matrix after matrix, that matrix's nrhs vectors one after another:
 * element i of vector j of matrix m is at off_m + j n_m + i, where
 * off_m = nrhs (n_0 + ... + n_{m-1}) and n_m is the matrix's own size.
 * iters, status (host, [nmat * nrhs], index m nrhs + j): A p products done and
 * SPAI_OK / SPAI_PCG_MAXIT / SPAI_PCG_BREAKDOWN per recurrence; relres (host,
 * may be NULL) = ||b - A x||_2 / ||b||_2 per recurrence.  Returns
 * SPAI_PCG_BREAKDOWN if any recurrence broke down, else SPAI_PCG_MAXIT if any
 * hit maxit, else SPAI_OK; or an error (SPAI_ERR_UNSUPPORTED for a matrix of
 * more than 4,194,304 rows).  The iterations are replayed from a captured
 * CUDA graph of 8 iterations on the handle's stream (launched directly if
 * that stream cannot be captured). */
int pcg_solve_block(spai_handle h, int nrhs, const double *b, double *x, double rtol, int maxit,
                    int precond, int on_device, int *iters, int *status, double *relres);

/* Definiteness diagnostic (the paper's motivation: an SPAI of an SPD matrix
 * should keep a positive-definite symmetric part; the spectra of Tables 4-6):
 * `steps` steps of the Lanczos three-term recurrence on S = (M + M^T)/2 (no
 * reorthogonalisation, FP64) from the host start vector v0[n] (nonzero,
 * finite; the caller draws it).  S v is an fma chain over ascending column
 * per row, inner products and norms the pairwise trees of the PCG,
 * w = fma(-beta_{j-1}, v_{j-1}, fma(-alpha_j, v_j, w)), v_{j+1} = w / beta_j;
 * the recurrence stops early when beta_j is 0 or not finite.  Host outputs:
 * alpha[steps], beta[steps] (may be NULL), *steps_done, and *lmin / *lmax
 * (may be NULL): the extremal eigenvalues of the tridiagonal T of the done
 * steps (bisection on its Sturm sequence), which approach lambda_min(S) and
 * lambda_max(S) from inside as the steps grow; lmin < 0 shows an indefinite
 * symmetric part.  Single-matrix handles only (SPAI_ERR_UNSUPPORTED for a
 * batch). */
int spai_sym_lanczos(spai_handle h, int steps, const double *v0, double *alpha, double *beta,
                     int *steps_done, double *lmin, double *lmax);

/* The best approximate inverse on the fixed pattern supp(A^k) (the paper's
 * Exp. 09 and Figs. 1-2, the classic Frobenius-norm SPAI it contrasts with):
 * replaces M by the matrix whose column j minimises ||e_j - A m_j||_2 over
 * supp(m_j) = supp(A^k e_j) (k >= 0; k = 0 is the diagonal), and forgets the
 * method recurrence.  Column j solves its normal equations
 * (A^2)[J,J] m = A[J,j] in FP64 (Cholesky); M is stored in the handle's
 * precision, so spai_residual_norm, spai_get_M, spai_sym_lanczos and the PCG
 * apply to it.  Errors: SPAI_ERR_CAPACITY if some |supp(A^k e_j)| exceeds
 * cap_j (create the handle with a larger cap_factor), SPAI_ERR_UNSUPPORTED
 * if the largest pattern does not fit a warp's shared memory (about 160
 * rows), SPAI_ERR_NONFINITE if a Gram matrix was not numerically positive
 * definite. */
int spai_fixed_pattern(spai_handle h, int k);

/* ------------------------------------------------ global dropping */

/* Hard thresholding with a global density cap (Sec. 6.1, Eq. 6.2): if the
 * stored M (which = 0) or direction P (which = 1) holds more than m entries,
 * keep the m of largest |v| (ties: smaller column, then smaller row) and
 * drop the rest, in place.  The per-column dropping of spai_run caps each
 * column instead; this is the paper's global form, applied between calls.
 * Forgets the method recurrence.  Single-matrix handles only. */
int spai_drop_global(spai_handle h, int which, int64_t m);

/* The dropping heuristic for the main iterate (Appendix A), in place:
 * (1) M := (M + M^T)/2 (s_kl = 0.5 (m_kl + m_lk) in FP64, rounded to the
 * value type); (2) off-diagonal entries with |m_kl| < u dropped, u the unit
 * round-off of the value type (2^-53 FP64, 2^-24 FP32); (3) if more than m
 * entries remain, the off-diagonal entries of smallest score
 * s_kl = m_kl^2 ||A e_k||^2 + 2 m_kl (A R)_kl (Eq. 435 with the m^2 of
 * Eq. 430: the change of ||R||_F^2 when that entry alone is dropped;
 * R = I - A M after steps 1-2, in the method's arithmetic; ||A e_k||^2 and
 * (A R)_kl FP64 fma chains over row k of A; s = fma(2m, ar, (m m) nrm)) are
 * dropped until m remain (the diagonal is always kept; ties: smaller column,
 * then smaller row).  SPAI_ERR_CAPACITY if a symmetrised column exceeds
 * cap_j.  Forgets the method recurrence.  Single-matrix handles only. */
int spai_drop_heuristic(spai_handle h, int64_t m);

/* MR (Algorithm 1), LOMR (Algorithm 4) or CG (Algorithm 3), or their
 * Pi forms (Algorithms 5, 8, 7; methods SPAI_*_PI), with the paper's
 * global dropping inside every iteration, where its dropping experiments
 * place it (Sec. 7.2).  R_i = I - A M_i is formed explicitly.  Every
 * direction candidate is kept whole, then cut to the m_dir entries of
 * largest |v| over the whole matrix (Sec. 6.1, Eq. 6.2).  The candidates
 * are: MR: P_i from (Pi) R_i; LOMR: Z_i from (Pi) R_i and
 * P_i from S_i = delta_i Z_i + gamma_i P_{i-1}; CG: P_i from
 * (Pi) R_i + beta_{i-1} P_{i-1}.  The step coefficients come from those
 * directions, with spai_run's arithmetic.  M_i + alpha_i P_i (MR, CG) or
 * M_i + S_i (LOMR) is kept whole, then cut by Appendix A's heuristic with
 * density cap m_M (see spai_drop_heuristic).  CG's beta_i uses the R of the
 * dropped M_{i+1}.  The column capacities cap_j (from cap_factor) must hold
 * the whole candidate columns, else SPAI_ERR_CAPACITY.  hist as for
 * spai_run: resnorm[i] = ||R_i||_F of the dropped iterates;
 * coef[2i], coef[2i+1] = (alpha_i, 0), (delta_i, gamma_i) or
 * (alpha_i, beta_i).  Returns SPAI_OK, SPAI_CONVERGED_EARLY,
 * SPAI_LOMR_FALLBACK or an error, and forgets any method recurrence.
 * Single-matrix handles only. */
int spai_run_global(spai_handle h, int method, int iters, int64_t m_dir, int64_t m_M,
                    spai_history *hist);

/* ------------------------------------------------ differentiation */

/* Gradient of fixed-pattern MR (no counterpart in the paper, which gives the
 * objective of Sec. 2 and its gradient -2 A^T R in Sec. 3): K steps
 *   M_0 = diag(A)^{-1}, R_i = I - A M_i, P_i = mask_S(R_i), Q_i = A P_i,
 *   alpha_i = (R_i, Q_i)_F / (Q_i, Q_i)_F, M_{i+1} = M_i + alpha_i P_i,
 * S = supp(A), loss L = ||I - A M_K||_F^2, differentiated with respect to the
 * stored values of A taken as independent entries (through M_0, alpha_i,
 * R_i, P_i and Q_i).  spai_fpmr_create takes A's pattern (host CSR, rows
 * strictly ascending, symmetric, full diagonal; else SPAI_ERR_CSR /
 * SPAI_ERR_NOT_SYMMETRIC / SPAI_ERR_NOT_SPD_DIAG) and builds, once, the
 * patterns S and T = supp(A S) + I and the product lists of the forward and
 * adjoint passes.  spai_fpmr_forward takes A's values (nnz FP64, CSR order,
 * host or device) and returns L on the host, keeping M_0..M_K on the device
 * (one checkpoint per step; R, P, Q are recomputed in the backward pass);
 * SPAI_ERR_NONFINITE if some (Q_i, Q_i) is zero.  spai_fpmr_backward writes
 * dloss * dL/dvals (nnz, CSR order, host or device) for the values of the
 * last forward call (SPAI_ERR_STATE without one).  prec: SPAI_FP64, or
 * SPAI_MIXED (values and the products' fma chains in FP32; inner products,
 * step scalars and the axpy/accumulation arithmetic in FP64, each stored
 * value rounded once to FP32).  The handle owns its device memory: about
 * (K + 6) nnz(A) + 5 nnz(T) values and 6 int32 per product-list entry. */
typedef struct spai_fpmr_ctx *spai_fpmr_handle;
int spai_fpmr_create(spai_fpmr_handle *out, int64_t n, int64_t nnz, const int32_t *rowptr,
                     const int32_t *colind, int K, int prec, void *stream);
int spai_fpmr_forward(spai_fpmr_handle h, const double *vals, int on_device, double *loss);
int spai_fpmr_backward(spai_fpmr_handle h, double dloss, double *dvals, int on_device);
/* Choose the steps the handle differentiates: SPAI_MR (the default, above)
 * or SPAI_LOMR, K steps of LOMR on the same fixed pattern (Algorithm 4 with
 * the 2-D minimiser of Theorem 3):
 *   P_{-1} = 0, Z_i = mask_S(R_i), U = A Z_i, V = A P_{i-1},
 *   (delta_i, gamma_i) solving the 2x2 normal equations in (U,U), (V,V),
 *   (U,V), (U,R_i), (V,R_i) -- or the MR step delta_i = (U,R_i)/(U,U),
 *   gamma_i = 0 when (V,V) = 0 (i = 0) or the system is near singular, as in
 *   spai_run --, S_i = delta_i Z_i + gamma_i P_{i-1}, M_{i+1} = M_i + S_i,
 *   P_i = S_i.
 * The gradient flows through delta_i, gamma_i (the derivatives of the 2x2
 * solution), U, V, Z_i, R_i and P_{i-1}.  LOMR keeps one more checkpoint per
 * step (P_{i-1}) and 5 more arrays on S or T (allocated here: SPAI_ERR_OOM if
 * they do not fit).  Clears the last forward call (SPAI_ERR_STATE for a
 * backward call before the next forward).  SPAI_ERR_ARG for another method. */
int spai_fpmr_set_method(spai_fpmr_handle h, int method);
/* nnz(T), product-list entries and kernel launches so far (any may be NULL). */
int spai_fpmr_info(spai_fpmr_handle h, int64_t *nnz_t, int64_t *list_entries, int64_t *launches);
int spai_fpmr_destroy(spai_fpmr_handle h);

/* Checkpoint of the iteration state (M, directions, scalars, method and
 * iteration index).  Two-call: with buf == NULL only *bytes is set. */
int spai_save_state(spai_handle h, void *buf, size_t *bytes);
int spai_load_state(spai_handle h, const void *buf, size_t bytes);

/* Residual norms of a linear system without allocating: out[0] = ||b - A x||_2
 * and out[1] = ||b||_2, both FP64, written to the device array `out` (2
 * doubles) in stream order on `stream` (NULL: the legacy default stream); the
 * call does not synchronise.  The paper has no counterpart: this is a
 * utility for callers that cannot allocate device memory, such as code whose
 * GPU memory belongs to another allocator, or latency-critical loops that
 * cannot pay for cudaMalloc/cudaFree.  A (CSR int32/int32/FP64, n x n), b
 * and x are device pointers owned by the caller; the rows are summed in the
 * same order as pcg_solve's residual, so out[0]/out[1] equals its *relres.
 * Workspace: a fixed ~1 MB array inside the library (every GPU that loads the
 * library holds it until exit); n above 16,777,216 returns
 * SPAI_ERR_UNSUPPORTED.  The first call on each device looks up that array's
 * device address, so make it before starting any stream capture; the address
 * is kept for the life of the process, so cudaDeviceReset after that first
 * call is not supported (the reloaded library image gets a new one).  All calls
 * share the array: calls that overlap on the GPU race; order them on one
 * stream.  No cudaMalloc, cudaFree or allocating library routine is called. */
int spai_true_residual_noalloc(int64_t n, const int32_t *rowptr, const int32_t *colind,
                               const double *vals, const double *b, const double *x, double *out,
                               void *stream);

/* Launch / byte / time counters; timing (CUDA events around each column
 * pass, on the handle's stream) is recorded only while enabled. */
int spai_set_timing(spai_handle h, int enable);
int spai_get_stats(spai_handle h, spai_stats *out);

#ifdef __cplusplus
}
#endif
#endif /* SPAI_H */
