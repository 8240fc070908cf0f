/*
 * lobpcg.h -- C ABI of the GB300 robust LOBPCG library.
 *
 * Computes the k algebraically smallest eigenpairs of a sparse symmetric-
 * definite pencil (A, B): A X = B X Lambda, X^T B X = I (Duersch, Shao, Yang,
 * Gu, "A robust and efficient implementation of LOBPCG", 2018: Sec. 2, Eq. 1),
 * with the robust iteration of Algorithm 8 of that paper.
 *
 * Conventions for every entry point:
 *   - Return value: a lobpcg_status.  Nothing is thrown across the ABI.  After a
 *     failure lobpcg_last_error() returns a message owned by the handle.
 *   - Dense blocks are row-major with an explicit leading dimension (elements
 *     between consecutive rows, >= the number of columns).  Small dense
 *     matrices passed to the kernel-level entry points are column-major.
 *   - Device pointers must point to memory of the current CUDA device.  Host
 *     pointers may be pageable.  `stream` is a cudaStream_t (NULL: legacy
 *     default stream); all device work of a call is ordered on that stream.
 *   - Inputs are borrowed for the duration of the call; the handle copies what
 *     it keeps.  Outputs go to caller-allocated buffers.
 *   - A handle may be used by one host thread at a time.
 *   - CSR matrices: int32 row pointers and column indices (nnz < 2^31), columns
 *     sorted within a row, float64 values (float32 values are accepted by
 *     lobpcg_set_operator_ex and widened on entry); A and B must be symmetric.
 */
#ifndef GB300_LOBPCG_H
#define GB300_LOBPCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lobpcg_ctx* lobpcg_t;

typedef enum {
  LOBPCG_OK = 0,
  LOBPCG_ERR_ARG = 1,            /* invalid argument (sizes, pointers, options) */
  LOBPCG_ERR_NOT_CONVERGED = 2,  /* maxit reached; outputs hold the current iterate */
  LOBPCG_ERR_BREAKDOWN = 3,      /* initial block numerically rank deficient (Alg. 2) */
  LOBPCG_ERR_CUDA = 4,           /* a CUDA, cuBLAS or cuSOLVER call failed */
  LOBPCG_ERR_OOM = 5,            /* device allocation failed */
  LOBPCG_ERR_TIMEOUT = 6,        /* wall-clock limit of the options exceeded, or a bounded
                                    wait inside a tensor-core kernel ran out (its outputs are
                                    then not valid; the context stays usable) */
  LOBPCG_ERR_CALLBACK = 7,       /* the preconditioner callback returned non-zero */
  LOBPCG_ERR_DEGENERATE = 8      /* lobpcg_eig_adjoint: two wanted eigenvalues coincide */
} lobpcg_status;

typedef enum { LOBPCG_MEM_HOST = 0, LOBPCG_MEM_DEVICE = 1 } lobpcg_mem;

/* Arithmetic used for the n-scaled dense contractions (Gram S^T Y and basis
 * update S C).  F64 rounds like any FP64 dot product.  The emulated modes cut
 * each FP64 input into `slices` exact BF16 digits against the exponent bound
 * shared by its block of the contraction (64 long for mma.sync, 256 for
 * tcgen05); each product is then exact to about 2^-44 (6 slices) or 2^-56 (7)
 * relative to those bounds.  The mma.sync form sums the blocks in
 * double-float, the tcgen05 form in int64 fixed point with one final
 * rounding.  Everything else (projected pencils, Algorithm 7, norms, Eq. 9)
 * runs in FP64 in every mode. */
typedef enum {
  LOBPCG_GEMM_F64 = 0,      /* plain FP64 fused multiply-add on the CUDA cores */
  LOBPCG_GEMM_OZAKI = 1,    /* FP64 emulated by exact BF16 splits, warp-level mma.sync */
  LOBPCG_GEMM_OZAKI_TC = 2  /* same splits; Grams and updates on tcgen05, TMEM accumulators */
} lobpcg_gemm_mode;

/* Options; zero-initialise and set what you need, zeros select the defaults
 * noted.  eps below is 2^-52. */
typedef struct {
  int64_t block_width;    /* n_x; 0: k + max(ceil(k/10), 2), the paper's ~10 % padding (Sec. 6) */
  int32_t maxit;          /* 0: 6000 iterations (the paper stops its runs at 2000, Sec. 6; the
                             512^2 Laplacian + V, k = 32, needs about 2100 in FP64 here) */
  int32_t implicit;       /* implicit product updates (Sec. 5.2): 0 auto (B = I or diagonal
                             B with cond <= 1e4), 1 never, 2 always */
  int32_t refresh_every;  /* 0: 50; explicit A X, A P recomputation period under implicit updates */
  int32_t omega_rows;     /* 0: 16; rows s of the Gaussian sketch Omega of the norm estimates
                             (Sec. 4.3).  Omega^T is the n x s block whose element (r, c) is
                             normal number r*s + c of Philox stream 5 under the solve's seed */
  int32_t gemm_mode;      /* lobpcg_gemm_mode; 0 selects LOBPCG_GEMM_F64 */
  int32_t ozaki_slices;   /* 0: 6; BF16 slices per operand for the emulated modes (3..7); a
                             solve that stalls at the contraction accuracy continues with 7 */
  int32_t certify;        /* 0: on; 1: off.  Explicit-product re-check of Eq. (9) at exit */
  double tau_ortho;       /* 0: 100 eps; Algorithm 5 orthogonality tolerance */
  double tau_skip;        /* 0: 100 eps; switch to orthogonalisation when cond(R)^-3 < tau_skip (Sec. 5.3) */
  double max_seconds;     /* 0: no limit; host wall-clock limit -> LOBPCG_ERR_TIMEOUT */
  int32_t dense_eig;      /* small dense layer of the projected pencils (Algorithms 2, 4, 6, 7):
                             0 this library's device-resident kernels for pencils of order
                             <= 256 (FP32 eigendecomposition refined to FP64 on the device,
                             Cholesky of the W-block Schur complement, FP32 Householder QR
                             for C_p restored to FP64 orthonormality), cuSOLVER/cuBLAS FP64
                             above that order and when the eigensolver's check fails;
                             1 FP32 cuSOLVER syevd refined to FP64 (Ogita-Aishima steps,
                             Newton-Schulz, cluster Jacobi; FP64 syevd when its residual
                             check fails); 2 cuSOLVER FP64 syevd and cuBLAS throughout */
  int32_t basis;          /* basis selection: 0 Algorithm 8 (orthoDrop when cond(R) demands it,
                             LQ-based C_p, Gram identities (12)-(14));  the comparison variants
                             of Sec. 6, with the Hetmaniuk-Lehoucq basis selection (W
                             B-orthogonalised against [X, P] by Algorithm 3 on every iteration,
                             C_p of Eq. 6 orthonormalised by svqb, standard eigenproblem):
                             1 CHL (no implicit products, every Gram block computed),
                             2 AHL (implicit products, only (12) assumed) */
  int32_t explicit_rr;    /* 0 auto (on in the emulated forms), 1 off, 2 on: on the iteration
                             after each explicit refresh of A X, A P the projected pencil is
                             formed from explicit Grams of every block instead of the
                             identities (12)-(14), which the updates' rounding erodes */
  int32_t criterion;      /* convergence test: 0 or 9 the backward error of Eq. (9); 7 and 8
                             the relative residuals (7), (8) of Sec. 4.3 (contrast studies) */
  int32_t gram_blocks;    /* blocks of the projected pencil taken from identities instead of
                             computed (basis 0): 0 all of (12)-(14) (Algorithm 8); 1 only (12)
                             (X^T A X = Theta, X^T B X = I; the P blocks are computed); 2 none
                             (the versions study of Sec. 6.2) */
  int32_t inject_wait_timeout_at; /* 0 off; i > 0: after the update of iteration i the solver
                             sets bit 0 of its tensor-core status word itself, the bit a
                             Gram or update kernel sets when one of its bounded waits runs
                             out, so that tests follow that error path (LOBPCG_ERR_TIMEOUT,
                             handle still usable) without a failing kernel */
} lobpcg_options_t;

/* Per-solve counters and phase times (Sec. 6.2 breakdown methodology). */
typedef struct {
  int64_t iterations;
  int64_t n_x;            /* block width used */
  int64_t converged;      /* n_c at exit */
  int64_t flip_iteration; /* iteration at which orthogonalisation switched on; -1 never */
  int64_t ortho_calls;
  int64_t svqb_passes;
  int64_t dropped_columns;
  int64_t gpu_launches;   /* kernels of this library launched by the last solve */
  double norm_a, norm_b;  /* Gaussian-sketch norm estimates used in Eq. (9) */
  double max_backward_error;
  /* phase times in ms from CUDA events on the handle's stream, exclusive: time
   * inside a phase nested in another is charged to the inner one only (the
   * Grams of orthoDrop count as ms_gram, its own small kernels and host waits
   * as ms_ortho); ms_other is the stream time of the solve outside every phase
   * (norm sums, exponent kernels, host decisions between phases), so the six
   * phases and ms_other add up to the solve's stream time.  ms_total: host
   * wall-clock time of lobpcg_solve. */
  double ms_spmm, ms_gram, ms_update, ms_residual, ms_small_dense, ms_ortho, ms_other, ms_total;
  /* algorithmic work of the n-scaled kernels over the solve (for roofline figures):
   * SpMM bytes nnz*(8+4) + 4(n+1) + 8 n m (X read) + 8 n m (Y written) [+ 8 n + 16 n m
   * for a fused diagonal B]; Gram flops 2 n p q; update flops 2 n s m. */
  int64_t spmm_calls, gram_calls, update_calls;
  double spmm_bytes, gram_flops, update_flops;
  /* BF16 tensor-core work of the emulated contractions: the FP64-equivalent
   * flops times the S(S+1)/2 digit pairs of an S-slice split (0 in FP64 mode) */
  double gram_tensor_flops, update_tensor_flops;
  /* projected eigenproblems solved by this library's own eigensolvers (the
   * device-resident one of dense_eig 0, or the refined FP32 one of
   * dense_eig 1), and how many of them fell back to cuSOLVER's FP64 syevd */
  int64_t eig_calls, eig_fallbacks;
  /* emulated forms: iteration at which a stall (no column converging and the
   * leading backward error flat over 400 iterations) raised the contractions
   * to 7 slices for the rest of the solve; -1 never */
  int64_t slice_escalation_iteration;
  /* algorithmic HBM bytes of the contractions over the solve, each operand
   * block read once and each output written once (8-byte words): Gram
   * 8 n (p + q); update 8 n (s + m), plus 8 n m when Y0 is read */
  double gram_bytes, update_bytes;
  /* ||X^T B X - I||_F of the first k returned columns, from explicit FP64
   * products after the exit certification (-1 when not computed) */
  double orth_error;
  /* host waits on the stream (device scalars read back) during the solve */
  int64_t host_syncs;
  /* why the device-resident eigensolver (dense_eig 0) fell back: its
   * refined eigenvectors failed the orthonormality check, a group of
   * coupled eigenvalues was wider than its cluster Jacobi takes (32), or a
   * value was not finite (a call may count under several) */
  int64_t eig_check_orthogonality, eig_check_wide_cluster, eig_check_nonfinite;
  /* iterations whose projected pencil came from explicit Grams of every block */
  int64_t explicit_rr_calls;
} lobpcg_stats_t;

/* Preconditioner callback: write W = K^-1 R for an n x ncols row-major block.
 * R and W are device pointers with leading dimensions ldr, ldw; `stream` is the
 * handle's cudaStream_t.  Return 0 on success; non-zero aborts the solve with
 * LOBPCG_ERR_CALLBACK. */
typedef int (*lobpcg_precond_fn)(void* ctx, int64_t n, int64_t ncols, const double* R,
                                 int64_t ldr, double* W, int64_t ldw, void* stream);

/* Chebyshev polynomial preconditioner for the callback slot (Algorithm 1,
 * Eq. 2 admit any preconditioner K).  K^-1 R is `degree` steps of the
 * Chebyshev iteration for A W = R from W = 0 with the Jacobi splitting
 * D = diag(A) and the spectral interval [lmin, lmax] of D^-1 A (Saad,
 * Iterative Methods for Sparse Linear Systems, Algorithm 12.1), i.e.
 * W = p(D^-1 A) D^-1 R for a fixed polynomial p positive on the interval, so
 * K is symmetric positive definite.  rowptr, col, val: device CSR of A,
 * borrowed (they must outlive the object); diag: device diag(A) or NULL
 * (taken from the CSR); max_cols: the widest block it will be applied to
 * (the solver's block width).  Allocates 3 n x max_cols work blocks.
 * lobpcg_chebyshev_apply has the lobpcg_precond_fn signature:
 *   lobpcg_set_precond_callback(h, lobpcg_chebyshev_apply, cheb);
 * Errors: LOBPCG_ERR_ARG (degree outside 1..64, 0 < lmin < lmax violated,
 * ncols > max_cols or n different from the object's), LOBPCG_ERR_OOM. */
typedef struct lobpcg_chebyshev* lobpcg_chebyshev_t;
int lobpcg_chebyshev_create(lobpcg_chebyshev_t* out, int64_t n, const int32_t* rowptr,
                            const int32_t* col, const double* val, const double* diag, int degree,
                            double lmin, double lmax, int64_t max_cols);
int lobpcg_chebyshev_apply(void* ctx, int64_t n, int64_t ncols, const double* R, int64_t ldr,
                           double* W, int64_t ldw, void* stream);
void lobpcg_chebyshev_destroy(lobpcg_chebyshev_t c);

/* Create a handle bound to the current CUDA device and `stream`.  opts may be
 * NULL (defaults).  The handle owns every device buffer it allocates. */
int lobpcg_create(lobpcg_t* out, const lobpcg_options_t* opts, void* stream);

/* Set the pencil.  A: CSR (n, A_nnz).  B: either CSR (B_rowptr != NULL), or a
 * diagonal (B_diag != NULL, n values), or the identity (both NULL).  `mem`
 * says whether the arrays are host or device pointers; they are copied.
 * Resets the preconditioner to Jacobi K = diag(A) (Algorithm 1, Eq. 2); when
 * diag(A) has a zero entry K = I instead, the call returns LOBPCG_OK and
 * lobpcg_last_error says so.
 * Errors: LOBPCG_ERR_ARG for n outside 1..2^31, nnz outside 0..2^31-1, B
 * given both ways, a non-positive diagonal B, and, for host arrays (checked
 * before anything is copied), a CSR whose rowptr does not run monotonically
 * from 0 to nnz or whose column indices leave 0..n-1 (device arrays are
 * trusted).  After any error the handle holds no operator: lobpcg_solve and
 * lobpcg_eig_adjoint return LOBPCG_ERR_ARG until an operator is set.  The one
 * exception is a call made while another CUDA device than the handle's is
 * current: it returns LOBPCG_ERR_ARG and changes nothing. */
int lobpcg_set_operator(lobpcg_t h, int64_t n, const int32_t* A_rowptr,
                        const int32_t* A_col, const double* A_val, int64_t A_nnz,
                        const int32_t* B_rowptr, const int32_t* B_col,
                        const double* B_val, int64_t B_nnz, const double* B_diag,
                        int mem);

/* Value types of lobpcg_set_operator_ex and its flags. */
typedef enum { LOBPCG_F64 = 0, LOBPCG_F32 = 1 } lobpcg_dtype;
enum { LOBPCG_BORROW = 1 };

/* lobpcg_set_operator with the values of A, of a CSR B and of a diagonal B
 * given as FP64 or FP32 (A_dtype, B_dtype, lobpcg_dtype).  FP32 values are
 * widened to FP64 on entry (exactly); the solve computes in the form its
 * options select, as after lobpcg_set_operator.  flags: LOBPCG_BORROW
 * (device arrays only) makes the handle use the caller's CSR arrays in place
 * instead of copying them (row pointers, columns, and FP64 values; FP32
 * values are always widened into the handle's own copy, a diagonal B is
 * always copied).  Borrowed arrays must stay allocated and unchanged until
 * the handle is destroyed or given another operator; the handle never frees
 * them.  Errors: as lobpcg_set_operator, and LOBPCG_ERR_ARG for a dtype
 * other than LOBPCG_F64 / LOBPCG_F32, unknown flags, or LOBPCG_BORROW with
 * host arrays. */
int lobpcg_set_operator_ex(lobpcg_t h, int64_t n, const int32_t* A_rowptr,
                           const int32_t* A_col, const void* A_val, int64_t A_nnz, int A_dtype,
                           const int32_t* B_rowptr, const int32_t* B_col, const void* B_val,
                           int64_t B_nnz, const void* B_diag, int B_dtype, int mem, int flags);

/* Diagonal preconditioner K = diag(kdiag) (n values, `mem` as above);
 * kdiag == NULL restores K = diag(A); a negative `mem` selects K = I.
 * Host values must be positive (LOBPCG_ERR_ARG otherwise). */
int lobpcg_set_precond_diag(lobpcg_t h, const double* kdiag, int mem);

/* General preconditioner through a callback (see lobpcg_precond_fn). */
int lobpcg_set_precond_callback(lobpcg_t h, lobpcg_precond_fn fn, void* ctx);

/* Algorithm 8: k smallest eigenpairs to backward error tol (Eq. 9).
 *   X0      n x n_x initial block (row-major, leading dimension ldx0), or NULL:
 *           standard normal entries from Philox4x32-10 with key `seed` and
 *           stream 1 (element (r, c) is normal number r*n_x + c of the stream).
 *   mem_in  memory kind of X0.
 *   lambda  k eigenvalues, ascending (memory kind mem_out).
 *   X       n x k eigenvectors, row-major with leading dimension ldx, B-
 *           orthonormal, each sign-normalised so its largest-magnitude entry
 *           (lowest index on ties) is positive.
 *   iters   iterations of the main loop (host pointer, may be NULL); also written when the
 *           solve ends with an error inside the loop (the iteration it stopped in).
 *   resnorm k backward errors of Eq. (9) from explicit products (mem_out; may be NULL).
 * Returns LOBPCG_ERR_NOT_CONVERGED (outputs valid) when maxit is reached. */
int lobpcg_solve(lobpcg_t h, int64_t k, double tol, const double* X0, int64_t ldx0,
                 uint64_t seed, int mem_in, double* lambda, double* X, int64_t ldx,
                 int mem_out, int64_t* iters, double* resnorm);

int lobpcg_get_stats(lobpcg_t h, lobpcg_stats_t* out);
const char* lobpcg_last_error(lobpcg_t h);
void lobpcg_destroy(lobpcg_t h);

/* ---------------------------------------------------------------------------
 * Kernel-level entry points: single steps of one iteration on device buffers,
 * ordered on `stream`.  They allocate nothing unless noted.
 * ------------------------------------------------------------------------- */

/* Block sparse product Y = A X for an n x m row-major block X (the A W and
 * B W products of Algorithm 8, Sec. 5.2), optionally also BY = diag(b) X
 * (b != NULL).  All pointers are device pointers. */
int lobpcg_spmm(int64_t n, const int32_t* rowptr, const int32_t* col, const double* val,
                const double* X, int64_t ldx, int64_t m, double* Y, int64_t ldy,
                const double* b, double* BY, int64_t ldby, void* stream);

/* Tall-skinny Gram G = U^T V (the block inner products of Sec. 5.2, Eq. 12-14):
 * U n x p, V n x q row-major; G written column-major with leading dimension
 * ldg (>= p).  mode: lobpcg_gemm_mode; `slices` is the Ozaki slice count (0:
 * 6).  Needs device scratch; `work` of `work_bytes` bytes may be NULL, then
 * the call allocates and frees its own (use lobpcg_gram_workspace to size it). */
int lobpcg_gram(int64_t n, const double* U, int64_t ldu, int64_t p, const double* V,
                int64_t ldv, int64_t q, double* G, int64_t ldg, int mode, int slices,
                void* work, int64_t work_bytes, void* stream);
int64_t lobpcg_gram_workspace(int64_t n, int64_t p, int64_t q, int mode, int slices);

/* Allocation-free Gram.  The paper has no counterpart: this exists for callers
 * that cannot allocate device memory when they need a Gram (code inside a
 * framework that owns the memory pool, callbacks run under an allocator lock,
 * loops that must not call cudaMalloc/cudaFree because those synchronise).
 * Computes G = U^T V exactly as lobpcg_gram with mode LOBPCG_GEMM_OZAKI (same
 * arguments, same accuracy; the row split may differ, so results may differ
 * from lobpcg_gram in the last bits), taking its scratch from a fixed 16 MiB
 * array in the library's device memory that every GPU loading the library
 * holds until the process exits.  It calls no allocator.
 * Limits: p * q * 16 bytes must fit in that array (p * q <= 1,048,576);
 * larger shapes return LOBPCG_ERR_ARG before any device work.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the array and it keeps the last
 * call's contents: calls whose executions overlap on the GPU (different
 * streams, or different host threads) race on it and must be serialised by
 * the caller.  Nothing in it needs to start at zero. */
int lobpcg_gram_noalloc(int64_t n, const double* U, int64_t ldu, int64_t p, const double* V,
                        int64_t ldv, int64_t q, double* G, int64_t ldg, int slices, void* stream);

/* Self-test of the bounded waits of the tensor-core kernels: one CTA waits,
 * with the same bounded mbarrier wait limited to `polls` polls, on a barrier
 * phase that nothing completes, and records the timeout in a status word the
 * way the Gram and update kernels do.  Returns LOBPCG_ERR_TIMEOUT when the
 * wait ran out and was reported (the expected outcome), LOBPCG_ERR_CUDA if the
 * launch failed, LOBPCG_ERR_ARG for polls < 1.  Synchronises the stream. */
int lobpcg_wait_selftest(int32_t polls, void* stream);

/* Basis update Y = beta * Y0 + alpha * S C (Eq. 10-11): S n x s row-major, C
 * s x m column-major (leading dimension ldc), Y and Y0 n x m row-major (Y0 may
 * be NULL when beta == 0; Y must not alias S).  mode/slices as lobpcg_gram. */
int lobpcg_update(int64_t n, const double* S, int64_t lds, int64_t s, const double* C,
                  int64_t ldc, int64_t m, double alpha, double beta, const double* Y0,
                  int64_t ldy0, double* Y, int64_t ldy, int mode, int slices, void* stream);

/* Residual, preconditioner and norms (the residual, W and convergence steps of Algorithm 8):
 * for columns j = c0 .. m-1: r_j = AX_j - theta_j BX_j (BX == NULL: B = I),
 * W(:, j - c0) = r_j / kdiag (kdiag == NULL: K = I), and
 * be_j = ||r_j|| / ((normA + |theta_j| normB) ||x_j||)  (Eq. 9) written to
 * be[j - c0].  theta, kdiag, be: device pointers.  W may be NULL (norms only). */
int lobpcg_residual(int64_t n, const double* X, const double* AX, const double* BX,
                    int64_t ld, int64_t m, int64_t c0, const double* theta,
                    const double* kdiag, double* W, int64_t ldw, double normA,
                    double normB, double* be, void* stream);

/* Gradients of the eigenpairs with respect to the stored values of A and B.
 * The paper computes eigenpairs only; this is first-order perturbation theory
 * of the pencil A x = lambda B x with B-orthonormal, sign-fixed eigenvectors.
 * For a loss L with upstream gradients glam_i = dL/dlambda_i and
 * g_i = dL/dx_i of the k pairs (lambda, X) that lobpcg_solve returned for the
 * handle's current pencil:
 *   w_i   = sum_{j != i} x_j (x_j^T g_i) / (lambda_i - lambda_j)
 *         = w_i^in - u_i, w_i^in over the k given pairs, u_i solving
 *           (A - lambda_i B) u_i = (I - B X X^T) g_i with X^T B u_i = 0 by a
 *           projected conjugate gradient preconditioned with the handle's K
 *           (positive definite there when lambda_{k+1} > lambda_k);
 *   gA[e] = sum_i glam_i x_ri x_ci + (w_ri x_ci + x_ri w_ci) / 2 for each
 *           stored entry e = (r, c) of A (A_nnz values, A's CSR order);
 *   gB    = the same with coefficients -lambda_i glam_i - (g_i^T x_i)/2 and
 *           -lambda_i: B_nnz values on B's CSR pattern, n values for a
 *           diagonal B; not written (may be NULL) when B = I.
 * A symmetric pair (r, c), (c, r) is one parameter: its derivative is
 * gA[(r,c)] + gA[(c,r)].
 *   lambda (k), X (n x k row-major, leading dimension ldx), glam (k; NULL:
 *   zero), G (n x k, ldg; NULL: zero, no linear solve): memory kind mem_in.
 *   gA, gB: memory kind mem_out.  cg_tol (0: 1e-10) is the relative residual
 *   |r_i| <= cg_tol |(I - B X X^T) g_i| of every column; cg_maxit 0: 20000;
 *   *cg_iters (host, may be NULL) gets the iterations run.
 * Returns LOBPCG_ERR_DEGENERATE when two of the k eigenvalues are closer than
 * 1e-10 max(|lambda|, ||A||) (the eigenvector derivative does not exist),
 * LOBPCG_ERR_NOT_CONVERGED (outputs written) when cg_maxit is reached.
 * Allocates its n x k scratch blocks per call; k <= min(n, 2048). */
int lobpcg_eig_adjoint(lobpcg_t h, int64_t k, const double* lambda, const double* X,
                       int64_t ldx, const double* glam, const double* G, int64_t ldg,
                       int mem_in, double* gA, double* gB, int mem_out, double cg_tol,
                       int32_t cg_maxit, int64_t* cg_iters);

/* Symmetric eigendecomposition of a small dense matrix, the eigensolver of
 * the projected pencils of Algorithms 2, 4, 6 and 7 (their "eig" step):
 * A n x n column-major (leading dimension lda, device), symmetric (both
 * triangles read; it is symmetrised first).  On return A holds the
 * orthonormal eigenvectors and w (device, n) the eigenvalues ascending.
 * mode 0: cuSOLVER FP64 syevd; mode 1: FP32 cuSOLVER decomposition refined
 * to FP64 (Ogita-Aishima steps, a Newton-Schulz orthonormalisation, Jacobi on
 * eigenvalue clusters; FP64 syevd when its residual check fails); mode 2:
 * this library's device-resident eigensolver (FP32 Householder
 * tridiagonalisation, bisection and inverse iteration, then FP64
 * Ogita-Aishima refinement, a Newton-Schulz step and Jacobi on clusters,
 * n <= 256), cuSOLVER FP64 syevd when its check fails; mode 3: mode 2
 * without the fallback, returning LOBPCG_ERR_NOT_CONVERGED (outputs written)
 * when the check fails.  n <= 8192.  Allocates its workspace per call and
 * synchronises `stream`. */
int lobpcg_syev(int64_t n, double* A, int64_t lda, double* w, int mode, void* stream);

/* Philox4x32-10 normals: Y(r, c) = normal number r*m + c of stream `stream_id`
 * under key `seed` (Box-Muller of two 52-bit uniforms), n x m row-major. */
int lobpcg_philox_normal(int64_t n, int64_t m, uint64_t seed, uint32_t stream_id,
                         double* Y, int64_t ldy, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GB300_LOBPCG_H */
