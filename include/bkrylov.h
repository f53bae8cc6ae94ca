/*
 * bkrylov — block Krylov solvers for one NVIDIA GB300 (sm_103a), C ABI.
 *
 * Solves the block system  A X = B  with n x s blocks X, B (Dreier 2020,
 * "Hardware-Oriented Krylov Methods for High-Performance Computing",
 * Ch. 3, Eq. "blocklinearsystem": s simultaneous systems A x_i = b_i).
 *
 * Conventions shared by every entry point
 *  - Block vectors are n x s ROW-MAJOR arrays (leading dimension s): the s
 *    right-hand sides of one row are contiguous, as the thesis's SIMD block
 *    vector (Ch. 3.2).  1 <= s <= 32.
 *  - s x s results (Gram matrices, R factors) are dense row-major s x s
 *    arrays of doubles, element (i, j) at [i * s + j].
 *  - Unless a parameter says "host", pointers are device pointers on the
 *    handle's device.  The library never frees memory it did not allocate.
 *  - All GPU work is enqueued on the handle's stream.  Entry points that
 *    return results to the host (solvers filling bkrylov_info) synchronise
 *    that stream before returning; the others return right after enqueueing.
 *  - Every entry point returns a bkrylov_status.  Errors are reported, never
 *    thrown; on BK_ERR_ARG nothing was enqueued.
 *  - A handle is not thread-safe; use one handle per host thread.
 *  - Precision: BK_FP64 blocks are double, BK_FP32 blocks are float.  Gram
 *    matrices and every s x s computation are always double.
 */
#ifndef BKRYLOV_H
#define BKRYLOV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BKRYLOV_VERSION 201
#define BKRYLOV_MAX_S 32

typedef struct bkrylov_ctx* bkrylov_handle;   /* owns workspace + stream binding */
typedef struct bkrylov_op_s* bkrylov_op;      /* operator descriptor             */

typedef enum { BK_FP64 = 0, BK_FP32 = 1, BK_FP32_IR = 2 } bkrylov_prec;

typedef enum {
  BK_OK = 0,
  BK_ERR_ARG = 1,          /* invalid argument; nothing enqueued               */
  BK_ERR_CUDA = 2,         /* a CUDA runtime call failed                       */
  BK_ERR_ALLOC = 3,        /* device allocation of workspace failed            */
  BK_NOT_CONVERGED = 4,    /* maxit reached; X holds the last iterate           */
  BK_BREAKDOWN = 5,        /* an s x s coefficient matrix could not be factored */
  BK_NONFINITE = 6,        /* NaN/Inf appeared in an s x s quantity             */
  BK_TIMEOUT = 7,          /* a bounded device-side wait gave up                */
  BK_ERR_UNSUPPORTED = 8   /* valid request this build does not implement       */
} bkrylov_status;

/* Matrix-free stencil operators (grid numbered x fastest: i = x + nx*(y + ny*z)). */
typedef enum {
  /* 7-point constant coefficients, homogeneous Dirichlet boundary.
     coeffs: HOST array of 7 doubles (centre, -x, +x, -y, +y, -z, +z), copied.
     nz = 1 gives the 2D 5-point stencil (the z coefficients are unused). */
  BK_STENCIL_CONST7 = 0,
  /* -div(k grad u), cell-centred FV, h = 1, Dirichlet u = 0 in ghost cells:
     interior face 2 k_i k_j / (k_i + k_j), boundary face 2 k_i.
     coeffs: DEVICE array of n doubles (k per cell), read once at creation. */
  BK_STENCIL_VAR7 = 1,
  /* 2D per-edge diffusion A = sum_e a_e (e_i - e_j)(e_i - e_j)^T plus a_e e_i e_i^T
     for edges to the Dirichlet ghost.  nz must be 1.  coeffs: DEVICE array of
     ny*(nx+1) horizontal edges (a_x[y][x] joins cells (x-1,y),(x,y)) followed by
     (ny+1)*nx vertical edges (a_y[y][x] joins (x,y-1),(x,y)); BORROWED (the caller
     keeps it alive until bkrylov_op_destroy). */
  BK_STENCIL_EDGE5 = 2,
  /* BK_STENCIL_EDGE5 parameterised by log-coefficients: coeffs holds theta_e in the same
     layout and the operator forms and owns a_e = exp(theta_e) at creation (theta is not
     kept).  The per-edge model of the differentiable solve, a_e = exp(theta_e). */
  BK_STENCIL_EDGE5_LOG = 3
} bkrylov_stencil_kind;

/* Solver options (bkrylov_opts_default fills the defaults noted here).  The tolerance
   and the iteration limit are arguments of the solve calls. */
typedef struct {
  double eta;          /* re-orthonormalisation parameter: 0 never, INFINITY always;
                          otherwise re-orthonormalise when eta*kappa_D > 1/sqrt(eps)
                          (Ch. 4.3, Eq. "reortho_criterion", read as 1/sqrt(eps))   (INFINITY) */
  int restart;         /* BGMRes restart length m                              (30)   */
  int ortho;           /* BGMRes orthogonalisation: 0 = CGS2 (two classical passes, Ch. 9.1),
                          1 = block MGS (Alg. "block-arnoldi"), 2 = localized Arnoldi (Ch. 9.3:
                          the basis kept as a distributed S-QR decomposition over the row
                          tiles, one tree reduction per step; s <= 16, every row tile at least
                          s rows and restart small enough for its tree nodes' shared memory,
                          else BK_ERR_UNSUPPORTED).  The default is block MGS: on one GPU the
                          thesis's reasons for CGS2 and the localized method (fewer global
                          reductions) cost nothing, and MGS does half of CGS2's FP64 work
                          (measured 1.6x faster to 1e-8 on the 96^3 convection-diffusion
                          workload at s = 8)                                     (1)    */
  int prec;            /* bkrylov_prec of the solve: BK_FP64; BK_FP32 (BCG only: FP32 blocks
                          and products, every s x s quantity in FP64, eps = 2^-23 in the
                          criterion); BK_FP32_IR (BCG only: FP32 inner solves inside FP64
                          iterative refinement)                                 (FP64) */
  double ir_inner_tol; /* relative tolerance of each FP32 inner solve          (1e-5)  */
  int ir_max_outer;    /* refinement steps limit                               (30)    */
  const uint8_t* forced_reortho; /* HOST, optional: decision of iteration k (k < n_forced)
                                    replaces the adaptive criterion (replay)    (NULL) */
  int n_forced;
  int sync_every;      /* iterations enqueued between host checks of the stop flag;
                          0 = automatic                                          (0)  */
  int profile;         /* BCG and BGMRes: time every kernel phase of every iteration with
                          CUDA events on the handle's stream (adds one stream
                          synchronisation per iteration); read with
                          bkrylov_profile_get                                      (0)  */
  int subalgebra_p;    /* BCG only: block size p of the block-parallel *-subalgebra
                          S_BP^p (Ch. 3.1, Def. "subalgebras"; Ch. 4.3): every s x s
                          quantity is block diagonal with s/p blocks of p x p, the
                          normaliser is one Householder QR per p-column group.  0 or s:
                          the block case S_B; 1: S_P (s scalar CGs sharing the operator
                          products).  p must divide s; BK_ERR_ARG otherwise, and
                          BK_ERR_UNSUPPORTED for BBiCGStab and BGMRes with p < s  (0) */
  bkrylov_op precond;  /* BCG only: an operator applying M^-1 of Alg. "bcgaro" (Ch. 4.3),
                          M symmetric positive definite (Ch. 4): each iteration forms
                          Z = M^-1 R-bar, rho = <Z, R-bar> and P = Z + P beta; the
                          stopping test stays on the Euclidean ||R_i||.  Any operator
                          of the same n may serve; bkrylov_op_jacobi builds point
                          Jacobi.  Applies to the FP32 inner solves of FP32_IR too.
                          NULL: M = I.  BK_ERR_ARG if its n differs from A's;
                          BK_ERR_UNSUPPORTED for BBiCGStab and BGMRes            (NULL) */
  int norm_mode;       /* stopping measure of the relative residual (Ch. 4.1 "break if ||R||
                          < tol" names no norm): 0 = max_i ||R_i|| / ||R0_i||, a reduction in
                          every column; 1 = ||R||_F / ||R0||_F.  For FP32_IR it is the
                          outer test (relative to ||B||); the inner solves test every
                          column.  Other values: BK_ERR_ARG                      (0)    */
  int one_reduction;   /* BCG only: 1 = the schedule of Alg. "1R-CG" (Ch. 8.1): U = A Z and
                          delta = <Z, U> after the preconditioner, Q = U + Q beta,
                          alpha = delta - beta^T alpha beta, arithmetically equal to the
                          default two-reduction schedule (Alg. "2R-CG") at two more block
                          vectors and one more block update per iteration.  Needs the
                          block case (BK_ERR_UNSUPPORTED with subalgebra_p < s)     (0) */
  int replace_every;   /* one_reduction only: m > 0 forms Q = A P and alpha = <P, Q> directly
                          (one more operator pass, the two-reduction formulas) after every
                          m-th iteration and after any iteration whose recursive alpha has
                          a non-positive Cholesky pivot (residual replacement applied to the
                          recursion of Ch. 8.1); m = 1 gives the iterates of Alg. "2R-CG".
                          In FP32 the recursion's cancellation can lose alpha within one
                          step (the log-normal diffusion workloads: only m = 1 converges).
                          0: never.  Negative: BK_ERR_ARG                        (0)    */
  int qr_mode;         /* normaliser of the re-orthonormalising BCG iterations (Def.
                          "normalizer", Ch. 3.1): 0 = CholeskyQR2 (Fukaya et al. 2014: two
                          passes Y <- Y U^-1 with U the Cholesky factor of the Gram, the first
                          Gram fused into the block update) wherever the first Gram's pivots
                          all keep U_kk^2 > 1e-10 G_kk, the Householder TSQR (Ch. 7.3) for the
                          other blocks (nearly dependent or rank deficient) and when the
                          second factor fails; used by FP64 two-reduction BCG in the block
                          case, the other solves always take the TSQR.  1 = the Householder
                          TSQR in every iteration.  Other values: BK_ERR_ARG       (0)    */
} bkrylov_opts;

/* Solver report.  Pointer members are HOST arrays supplied by the caller (or NULL). */
typedef struct {
  int iters;           /* iterations performed (SpMMs of the loop; Arnoldi steps)    */
  int reorths;         /* residual re-orthonormalisations inside the loop            */
  int converged;       /* 1 if the tolerance was met                                  */
  int status;          /* bkrylov_status of the solve                                */
  int outer;           /* refinement steps (FP32_IR), else 0                          */
  double relres_max;   /* final max_i ||R_i|| / ||R0_i|| as tracked by the method     */
  double* relres;      /* [s]      final per-column relative residuals, or NULL        */
  double* history;     /* [maxit]  stopping measure (norm_mode) after each iteration
                                   (after each outer step for FP32_IR), or NULL        */
  uint8_t* decisions;  /* [maxit]  re-orthonormalised in iteration k?, or NULL          */
  int history_len;     /* capacity of history/decisions (entries written <= this)      */
  double elapsed_ms;   /* device time of the solve (CUDA events)                      */
  int reorths_cholqr;  /* of reorths, those normalised by CholeskyQR2 (qr_mode 0; the
                          others by the Householder TSQR)                             */
  int replacements;    /* 1R-BCG: iterations after which Q and alpha were formed directly */
} bkrylov_info;

/* ---- handle ------------------------------------------------------------------ */
/* Create a handle on `device`, bound to `cuda_stream` (a cudaStream_t; NULL = legacy
   default stream).  The handle owns a workspace grown on demand and freed by destroy. */
int bkrylov_create(bkrylov_handle* h, int device, void* cuda_stream);
int bkrylov_destroy(bkrylov_handle h);
int bkrylov_set_stream(bkrylov_handle h, void* cuda_stream);
const char* bkrylov_status_string(int status);
int bkrylov_version(void);
void bkrylov_opts_default(bkrylov_opts* o);

/* ---- operators (BOP, Ch. 3.3 Table "kernels") ---------------------------------- */
/* CSR matrix, n x n, int32 row_ptr[n+1] and col[nnz] (columns sorted within a row), val[nnz]
   of precision val_prec: BK_FP64 (double) or BK_FP32 (float); all device arrays BORROWED
   until bkrylov_op_destroy.  FP64 values: a float copy (owned) is made the first time an
   FP32 product is asked for.  FP32 values: the FP64 products (FP64 solvers, the outer
   residual of refinement) use an owned double widening made here (exact), so the operator
   is the same matrix in both precisions.  Errors: BK_ERR_ARG (another val_prec, n < 1,
   nnz < 0 or > INT32_MAX, null arrays), BK_ERR_ALLOC. */
int bkrylov_op_csr(bkrylov_handle h, int64_t n, int64_t nnz, const int32_t* row_ptr,
                   const int32_t* col, const void* val, int val_prec, bkrylov_op* A);
/* Matrix-free stencil (see bkrylov_stencil_kind).  n = nx*ny*nz.  VAR7 precomputes the
   3 face coefficients of every cell (owned, 3n doubles); EDGE5 precomputes the diagonal
   (owned, n doubles). */
int bkrylov_op_stencil(bkrylov_handle h, int kind, int nx, int ny, int nz,
                       const double* coeffs, bkrylov_op* A);
/* Diagonal operator (Q = D P, row i scaled by d[i]): DEVICE array of n doubles, copied
   (owned by the operator).  Used as a diagonal preconditioner M^{-1} (bkrylov_opts.precond)
   or as an operator of its own. */
int bkrylov_op_diag(bkrylov_handle h, int64_t n, const double* d, bkrylov_op* M);
/* Point Jacobi preconditioner M = diag(A) (Ch. 2, the Jacobi splitting), returned as the
   diagonal operator M^{-1} = diag(1 / a_ii), computed on the device from any operator
   kind (CSR: the stored entries with column == row, summed).  Synchronises the handle's
   stream; BK_ERR_ARG (nothing kept) when some a_ii is zero or not finite.  Destroy the
   result with bkrylov_op_destroy; it does not borrow A. */
int bkrylov_op_jacobi(bkrylov_handle h, bkrylov_op A, bkrylov_op* M);
/* At = A^T as an operator of its own (the adjoint solve A^T Lambda = dL/dX of a
   differentiable solve needs it for a non-symmetric A).  CSR: the transposed arrays are
   formed on the device and owned by At (columns sorted within every row; synchronises
   the handle's stream); CONST7: the -/+ coefficient of every direction swapped.
   VAR7, EDGE5 and diagonal operators are symmetric by construction (use A itself):
   BK_ERR_UNSUPPORTED.  At does not borrow A. */
int bkrylov_op_transpose(bkrylov_handle h, bkrylov_op A, bkrylov_op* At);
int bkrylov_op_destroy(bkrylov_op A);
int bkrylov_op_size(bkrylov_op A, int64_t* n, int64_t* nnz);

/* Q = A P (BOP).  P, Q: n x s blocks of precision prec (BK_FP64 or BK_FP32). */
int bkrylov_spmm(bkrylov_handle h, bkrylov_op A, int s, const void* P, void* Q, int prec);
/* Q = A P with the block inner product G = P^T Q fused into the same pass over the block:
   the operator product of an iteration with its Gram alpha = P^T A P (Ch. 3.3, Table
   "kernels": BOP followed by BDOT; Ch. 4.1, Eq. "cg_alpha").  sym != 0 computes the upper
   triangle and mirrors it (G exactly symmetric).  P, Q: n x s blocks of precision prec
   (BK_FP64 or BK_FP32), P != Q; G: s x s row-major doubles, device.  FP32 stencil operators
   with s % 4 == 0 and sym != 0 run the pipelined marching kernel (tensor copies of halo
   tiles into a shared-memory ring).  Errors: BK_ERR_ARG (nothing enqueued) for a null
   pointer, P == Q, s outside 1..32 or another prec. */
int bkrylov_spmm_gram(bkrylov_handle h, bkrylov_op A, int s, const void* P, void* Q, double* G, int sym,
                      int prec);
/* R = B - A X (the residual of Alg. "bcg", first line). */
int bkrylov_residual(bkrylov_handle h, bkrylov_op A, int s, const void* B, const void* X,
                     void* R, int prec);

/* ---- block inner product (BDOT, Ch. 3.1/3.3) ----------------------------------- */
/* G = X^T Y (s x s, double, device), summed in a fixed order (bitwise reproducible
   for a given n, s and device).  sym != 0 computes the upper triangle and mirrors it
   (the thesis's alpha and rho, Eqs. "cg_alpha", "cg_rho"). */
int bkrylov_bdot(bkrylov_handle h, int64_t n, int s, const void* X, const void* Y,
                 double* G, int sym, int prec);

/* G = X^T Y as bkrylov_bdot, for callers that cannot allocate device memory (a program
   that runs under a fixed device-memory budget, e.g. a host framework that reserved all
   device memory up front, or a loop where an allocation could block or fail).  The thesis
   has no counterpart: this is a deployment variant of the block inner product above.
   No handle: the call allocates nothing (no cudaMalloc/cudaFree, no allocating library
   routine).  Its scratch (per-CTA partial sums, the reduced matrix, the ticket words)
   is one file-scope device array of 4.2 MB that every GPU loading the library keeps
   until the process exits; the reduction grid is limited to 512 CTAs (any n works).
   X, Y: n x s device blocks (prec BK_FP64 or BK_FP32); G: s x s device doubles.
   Work is enqueued on cuda_stream (NULL = legacy default stream).
   Errors: BK_ERR_ARG for n < 1, s outside 1..32, null pointers or another prec, before
   any work; BK_ERR_CUDA if a CUDA call fails.
   The first call on a device looks up the array's device address (cudaGetSymbolAddress
   on the current device); make that first call before any stream capture.  With lazy
   module loading the first call of each precision on a device may also make the driver
   load the library's kernels and the array itself: make one call per device and
   precision before reserving the device-memory budget; later calls allocate nothing.
   The sums run in a fixed order, so results are reproducible from call to call, but the
   512-CTA grid orders the partial sums differently from bkrylov_bdot: the two agree to
   rounding, not bit for bit.
   All calls share the one array: calls that overlap on the GPU (other streams, other
   host threads) race and must be serialised by the caller. */
int bkrylov_bdot_noalloc(int64_t n, int s, const void* X, const void* Y, double* G, int sym,
                         int prec, void* cuda_stream);

/* ---- normalizer = TSQR (Def. "normalizer", Ch. 3.1; TSQR, Ch. 7.3) --------------- */
/* X = Y sigma with Y^T Y = I, sigma upper triangular s x s (double, device) with
   diag(sigma) >= 0; defined also for rank-deficient X (Householder at every level).
   Y may alias X.  n >= s required. */
int bkrylov_tsqr(bkrylov_handle h, int64_t n, int s, const void* X, void* Y, double* sigma,
                 int prec);

/* ---- solvers --------------------------------------------------------------------- */
/* Solve A X = B for the n x s block X (Ch. 3, Eq. "blocklinearsystem"; the algorithms'
   inputs X0, B, tol, maxit).  B (read) and X (in: X0, out: the solution) are n x s
   row-major blocks of double (prec BK_FP64 and BK_FP32_IR) or float (prec BK_FP32),
   either device pointers or HOST pointers (then the library copies them to and from the
   device inside the call).  tol: the stopping tolerance of the relative residual in the
   measure opts->norm_mode (>= 0); maxit: iteration limit (Arnoldi steps for BGMRes; inner
   iterations of each refinement step for FP32_IR; >= 0).  opts may be NULL (defaults);
   info may be NULL.  Returns BK_OK, BK_NOT_CONVERGED, BK_BREAKDOWN, BK_NONFINITE or
   BK_TIMEOUT (X is the last iterate in those cases), or an error code: BK_ERR_ARG
   (nothing enqueued) for null pointers, B == X, s outside 1..32, n < s, tol < 0,
   maxit < 0, eta < 0 or another norm_mode. */
/* Block CG with adaptive residual re-orthonormalisation, Alg. "bcgaro" (Ch. 4.3)
   scheduled as Alg. "2R-CG" (Ch. 8.1); prec = BK_FP32 solves with FP32 blocks (the
   thesis's single-precision runs, Ch. 4.4), BK_FP32_IR runs FP32 inner solves inside FP64
   iterative refinement (B - A X in FP64).  The block-parallel subalgebra (subalgebra_p
   < s) is FP64 only (BK_ERR_UNSUPPORTED otherwise). */
int bkrylov_solve_bcg(bkrylov_handle h, bkrylov_op A, int s, const void* B, void* X, double tol,
                      int maxit, const bkrylov_opts* opts, bkrylov_info* info);
/* Block BiCGStab with adaptive re-orthonormalisation, Alg. "BlockBiCGStab_with_reortho"
   (Ch. 6.2).  FP64 only. */
int bkrylov_solve_bbicgstab(bkrylov_handle h, bkrylov_op A, int s, const void* B, void* X,
                            double tol, int maxit, const bkrylov_opts* opts, bkrylov_info* info);
/* Restarted block GMRes, Alg. "bgmres" (Ch. 5.1), block MGS (Alg. "block-arnoldi"),
   CGS2 (Ch. 9.1) or localized Arnoldi (Ch. 9.3) and the TSQR normalizer.  FP64 only. */
int bkrylov_solve_bgmres(bkrylov_handle h, bkrylov_op A, int s, const void* B, void* X,
                         double tol, int maxit, const bkrylov_opts* opts, bkrylov_info* info);

/* ---- measurement ----------------------------------------------------------------- */
/* Number of timed phases of a BCG iteration (spmm_alpha, small_1, update_rho,
   tsqr_leaf_factor, tsqr_tree, tsqr_leaf_apply, tsqr_rho_gram, small_2, p_update). */
int bkrylov_profile_count(void);
/* Accumulated device time (ms) and kernel launches of phase i over all profiled
   iterations since the last reset; *name is a static string. */
int bkrylov_profile_get(bkrylov_handle h, int i, const char** name, double* total_ms,
                        long long* launches);
int bkrylov_profile_reset(bkrylov_handle h);
/* Diagonally scaled condition number kappa_D(A) = kappa_2(D^-1/2 A D^-1/2), D = diag(A)
   (Ch. 4.3, Def. "Diagonally scaled condition number"), the quantity of the adaptive
   re-orthonormalisation test, by the solvers' own device routine.  A: DEVICE s x s
   symmetric, row-major; kappa: DEVICE double (+inf when a diagonal entry or the smallest
   eigenvalue of the scaled matrix is <= 0).  Enqueued on the handle's stream. */
int bkrylov_kappa_d(bkrylov_handle h, int s, const double* A, double* kappa);
/* The adaptive re-orthonormalisation decision as the solvers take it: *decision = 1 when
   eta * kappa_D(A) > 1 / sqrt(eps) (Ch. 4.3, Eq. "reortho_criterion"; eta = 0 never, INFINITY
   always).  kappa_D is first bracketed in FP32; where it is below 2^10 and eta kappa_D is more
   than 1 % off the threshold that decides, otherwise the FP64 kappa_D of bkrylov_kappa_d does.
   A: DEVICE s x s symmetric, row-major; decision: DEVICE int.  Enqueued on the stream. */
int bkrylov_reortho_decision(bkrylov_handle h, int s, const double* A, double eta, double eps, int* decision);
/* Kernel launches of one BCG iteration for an n x s block with the options opts (NULL:
   the defaults); host-only, no GPU.  Kernels whose device-side condition is not met
   (the TSQR when the CholeskyQR2 normaliser was taken) are launched and return at once,
   and are counted. */
int bkrylov_bcg_launches_per_iteration(int64_t n, int s, const bkrylov_opts* opts);

/* ---- adjoint (reverse-mode derivative of X = A^{-1} B) ----------------------------- */
/* For a CSR operator: g[e] = -sum_k Lam[i,k] X[j,k] for every stored entry e = (i, j),
   i.e. dL/dA on the sparsity pattern given Lam = A^{-T} dL/dX.  Lam, X: n x s double. */
int bkrylov_adjoint_scatter(bkrylov_handle h, bkrylov_op A, int s, const double* Lam,
                            const double* X, double* g);
/* For an EDGE5 operator with a_e = exp(theta_e): dL/dtheta_e =
   -a_e sum_k (Lam_ik - Lam_jk)(X_ik - X_jk) (boundary edges: -a_e sum_k Lam_ik X_ik).
   gtheta has the layout of the operator's coefficient array. */
int bkrylov_edge_theta_grad(bkrylov_handle h, bkrylov_op A, int s, const double* Lam,
                            const double* X, double* gtheta);

#ifdef __cplusplus
}
#endif
#endif /* BKRYLOV_H */
