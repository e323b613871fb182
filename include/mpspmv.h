/*
 * mpspmv.h -- C ABI of the GB300 (sm_103a) multiple-precision sparse library.
 *
 * Multiple-precision CSR sparse matrix-vector products y = A x in
 * double-double (DD), triple-double (TD) and quad-double (QD) arithmetic for
 * real and complex A (arXiv 2412.17510, Kouya: Sections 2 and 3), the
 * multi-right-hand-side form Y = A X, and the CG / BiCGSTAB loops built on
 * them (Section 4.2).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - A number with L components (L = 1 binary64, 2 DD, 3 TD, 4 QD) is the
 *    unevaluated sum of L binary64 values, leading component first.
 *  - Structure of limbs (Section 3: "allocated independently as binary64
 *    matrices and vectors for each component"): a vector of length n is P
 *    consecutive planes of n binary64 values, plane p holding component p.
 *    Real data: P = L.  Complex data (Eq. complex_expression): P = 2L, planes
 *    0..L-1 the real part's components, planes L..2L-1 the imaginary part's.
 *  - Device pointers are CUDA device addresses on the device that was
 *    current when the handle was created; "host" pointers are ordinary (or
 *    pinned) host memory.  Pointers may not alias unless stated.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Work is enqueued on it and returns before completion unless
 *    stated.
 *  - Every function returns an int status: MPSPMV_OK (0) or a negative code
 *    below.  No exception or CUDA error crosses the ABI; on error the outputs
 *    are unspecified unless stated and the handle stays valid.
 */
#ifndef MPSPMV_H
#define MPSPMV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define MPSPMV_OK 0
#define MPSPMV_EINVAL (-1)     /* bad argument: size, index, precision, flag, NULL, NaN/Inf input */
#define MPSPMV_ENOMEM (-2)     /* device or host allocation failed */
#define MPSPMV_ECUDA (-3)      /* a CUDA runtime call or kernel launch failed */
#define MPSPMV_ENOTSUP (-4)    /* combination of options not supported */
#define MPSPMV_EBREAKDOWN (-5) /* Krylov breakdown: zero or non-finite scalar */
#define MPSPMV_ENOCONV (-6)    /* maxit reached before the stopping test held */
#define MPSPMV_ETIMEOUT (-7)   /* a bounded device-side wait expired */

/* Precision tag = number of binary64 components L. */
typedef enum { MPSPMV_D = 1, MPSPMV_DD = 2, MPSPMV_TD = 3, MPSPMV_QD = 4 } mpspmv_prec;

/* Flags for mpspmv_create_csr. */
#define MPSPMV_COMPLEX 1u   /* A and the vectors are complex (P = 2L planes) */
#define MPSPMV_MIXED 2u     /* "M" mode (Section 4): A kept in binary64, products MP x binary64
                               (Algorithms 3-5); requires val_limbs == 1 */
#define MPSPMV_SYMMETRIC 4u /* triplets hold one triangle (Matrix Market "symmetric"):
                               every off-diagonal (i,j,v) also stands for (j,i,v) */
#define MPSPMV_ONE_BASED 8u /* row/col indices start at 1 (Matrix Market) */
#define MPSPMV_EXACT_ACC 16u /* GB300 arithmetic variant: the error-free products of a stored entry are
                                formed exactly (DD/TD/QD: 106-bit integer products of the mantissas;
                                binary64: TwoProd by FMA), only the products just above the unit
                                roundoff run as one binary64 FMA chain, and the row sum is accumulated
                                exactly in fixed point on the integer pipe, then cut to L components by
                                truncation.  Krylov vector updates and inner products on such a handle
                                are exact in the same way.  Same bound 8 m u (|A||x|)_i, error of the
                                same order; results are not bit-identical to the paper-order
                                arithmetic.  Single-vector products on such handles whose values are
                                binary64 (one stored value plane) first turn x, per product, into one
                                fixed-point number per column (x truncated toward zero to a 4 / 5 / 7
                                word mantissa for DD / TD / QD), so each stored entry is one integer
                                product; the handle then holds 32 bytes per column part for these
                                records and, for real matrices summed over runs, 96 bytes per row for
                                finished row sums that a second pass turns into components. */
#define MPSPMV_TRANSPOSE 32u /* also build A^T (a second internal matrix from the swapped triplets, about
                                doubling the device bytes) for mpspmv_spmtv and mpspmv_bicg */

typedef struct mpspmv_mat* mpspmv_h;

/* Read-only description of a handle. */
typedef struct {
  int64_t nrows, ncols;
  int64_t nnz;          /* stored entries after duplicate merging (and symmetric expansion) */
  int64_t max_row_nnz;  /* longest row: the m of the error bound */
  int64_t nchunks;      /* fixed-size runs of stored entries, one per thread */
  int64_t nsplit_rows;  /* rows whose entries span more than one run */
  int32_t prec;         /* L */
  int32_t planes;       /* P = L or 2L */
  int32_t chunk;        /* entries per run (K): the longest of 128 (exact accumulation) or 64, halved
                           down to 4, that still gives about four waves of threads */
  uint32_t flags;
  int64_t device_bytes; /* device memory owned by the handle */
  int64_t nlong_rows;   /* of nsplit_rows, those spanning more than 32 runs */
  int64_t value_planes; /* binary64 value planes stored per entry (1 or 2 when only leading
                           components are kept: M mode, or MPSPMV_EXACT_ACC on binary64 data) */
  int64_t sell_slots;   /* exact-accumulation handles with short, evenly sized rows: slots of the
                           sliced-ELL copy that single-vector products use (one row per thread);
                           0 when products use the run layout only */
} mpspmv_info;

/*
 * mpspmv_create_csr -- build a device CSR matrix from COO / Matrix Market
 * triplets (Section 3: the COO arrays data/row/col and the CSR arrays
 * data/indices/indptr of the worked 5x5 example).
 *
 *  out        receives the new handle (owned by the caller; release with
 *             mpspmv_destroy).
 *  nrows, ncols, nnz   matrix shape and number of triplets (nnz may be 0).
 *  row, col   host arrays of nnz indices, any order; 0-based unless
 *             MPSPMV_ONE_BASED.  Indices outside the shape -> MPSPMV_EINVAL.
 *  val        host values, structure of limbs: val_limbs planes of nnz
 *             (2*val_limbs planes if MPSPMV_COMPLEX: real components, then
 *             imaginary components).  Components beyond val_limbs are zero
 *             ("P" mode promotes binary64 data with zero lower components).
 *             NaN or Inf -> MPSPMV_EINVAL.
 *  val_limbs  1..prec (exactly 1 with MPSPMV_MIXED).
 *  prec       MPSPMV_DD, MPSPMV_TD or MPSPMV_QD (MPSPMV_D: binary64).
 *  flags      MPSPMV_COMPLEX | MPSPMV_MIXED | MPSPMV_SYMMETRIC | MPSPMV_ONE_BASED |
 *             MPSPMV_EXACT_ACC | MPSPMV_TRANSPOSE.
 *  stream     stream for the uploads and the device-side build.
 *
 * Triplets are ordered by (row, col); duplicates are summed in the working
 * precision in input order.  The library copies what it needs: the caller
 * may free row/col/val when the call returns (it synchronises `stream`).
 */
int mpspmv_create_csr(mpspmv_h* out, int64_t nrows, int64_t ncols, int64_t nnz, const int64_t* row,
                      const int64_t* col, const double* val, int val_limbs, int prec, unsigned flags,
                      void* stream);

/* Release a handle and all device memory it owns (synchronises the device). */
int mpspmv_destroy(mpspmv_h h);

/* Static description of a status code (never NULL). */
const char* mpspmv_strerror(int status);

/* Fill *info (host struct) for handle h. */
int mpspmv_get_info(mpspmv_h h, mpspmv_info* info);

/*
 * mpspmv_spmv -- y = A x in the handle's precision (Section 3; complex by
 * Eq. complex_spmv: re = A_re x_re - A_im x_im, im = A_re x_im + A_im x_re).
 *
 *  x  device, P planes of ncols (read only).
 *  y  device, P planes of nrows (overwritten; must not overlap x).
 *
 * Each stored entry contributes one MP product and one MP addition
 * (Algorithms 2 and 1 for DD; the QD / TD sloppy forms for QD / TD).  The
 * result satisfies |y_i - (Ax)_i| <= 8 m u (|A||x|)_i componentwise, with m
 * the longest row and u = 2^-104, 2^-155, 2^-207 (DD, TD, QD).  Asynchronous.
 */
int mpspmv_spmv(mpspmv_h h, const double* x, double* y, void* stream);

/*
 * mpspmv_spmtv -- y = A^T x (Section 4, "SpTMV"; complex: the transpose, not
 * the conjugate transpose).  Requires a handle created with MPSPMV_TRANSPOSE
 * (MPSPMV_ENOTSUP otherwise).
 *
 *  x  device, P planes of nrows (read only).
 *  y  device, P planes of ncols (overwritten; must not overlap x).
 *
 * A^T is stored as its own matrix, built once at creation from the swapped
 * triplets, so the product is a row sum like mpspmv_spmv and needs no
 * scatter or combining step.  Each y_j adds its products in increasing row
 * of A, the order of the row-oriented scatter (rows of A in order, each
 * entry a_ij adding a_ij x_i into y_j).  Same bound as mpspmv_spmv with m
 * the longest column of A.  Asynchronous.
 */
int mpspmv_spmtv(mpspmv_h h, const double* x, double* y, void* stream);

/*
 * mpspmv_spmv_host -- mpspmv_spmv with host buffers: copies x (P planes of
 * ncols) to device memory owned by the handle, multiplies, copies y (P planes
 * of nrows) back and synchronises `stream` before returning.
 */
int mpspmv_spmv_host(mpspmv_h h, const double* x_host, double* y_host, void* stream);

/*
 * mpspmv_spmv_host_async -- mpspmv_spmv_host without the final
 * synchronisation: the copy of x in, the product and the copy of y out are
 * enqueued on `stream` and the call returns.  x_host and y_host must be
 * pinned (page-locked) host memory and stay valid, unread (y) and unmodified
 * (x), until `stream` has completed.  Products of different handles on
 * different streams then overlap one product's copies with another's
 * kernels.  Two calls on the same handle use the same device buffers: order
 * them on one stream.
 */
int mpspmv_spmv_host_async(mpspmv_h h, const double* x_host, double* y_host, void* stream);

/*
 * mpspmv_spmm -- Y = A X for k right-hand sides (1 <= k <= 32).
 *
 *  X  device, P planes; plane p, row j, column c at X[(p*ncols + j)*ldx + c]
 *     (right-hand sides contiguous, so one stored entry of A serves all k).
 *  Y  device, same layout with nrows and ldy.  ldx, ldy >= k.
 * Column c of Y equals mpspmv_spmv applied to column c of X.  Asynchronous.
 */
int mpspmv_spmm(mpspmv_h h, int k, const double* X, int64_t ldx, double* Y, int64_t ldy, void* stream);

/*
 * mpspmv_cg -- conjugate gradients for real symmetric positive definite A
 * (Section 4.2: CG on nd3k), every vector and scalar in the handle's
 * precision; unpreconditioned Hestenes-Stiefel form.
 *
 *  b       device, L planes of n (right-hand side; n = nrows = ncols).
 *  x       device, L planes of n: initial guess on entry (the paper uses 0),
 *          the last iterate on return (also on MPSPMV_ENOCONV).
 *  rtol, atol  stop when ||r_k||_2 <= rtol ||b||_2 + atol, r_k the recurrence
 *          residual (the paper: rtol = 1e-13, atol = 1e-99).
 *  maxit   iteration limit (>= 0).
 *  iters   host, may be NULL: iterations taken.
 *  relres  host, may be NULL: ||b - A x||_2 / ||b||_2 of the returned x,
 *          recomputed in the working precision.
 * Returns MPSPMV_OK when the test held, MPSPMV_ENOCONV at maxit,
 * MPSPMV_EBREAKDOWN on a zero or non-finite p'Ap / r'r, MPSPMV_ENOTSUP for a
 * complex or M-mode handle.  Synchronises `stream` before returning.
 */
int mpspmv_cg(mpspmv_h h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
              double* relres, void* stream);

/*
 * mpspmv_bicgstab -- BiCGSTAB (van der Vorst) for real or complex A, r_hat =
 * r_0, inner products sum conj(u_i) v_i (Section 4.2: product-type Krylov
 * methods on tub1000).  Arguments and returns as mpspmv_cg; b and x have P
 * planes (complex: 2L).
 */
int mpspmv_bicgstab(mpspmv_h h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
                    double* relres, void* stream);

/*
 * mpspmv_bicg, mpspmv_cgs, mpspmv_gpbicg -- the other product-type Krylov
 * methods of Section 4.2 (BiCG, CGS and GPBiCG on tub1000), real or complex,
 * every vector and scalar in the handle's precision; arguments, stopping
 * test and returns as mpspmv_cg.
 *   BiCG (Fletcher): shadow residual r~_0 = r_0, shadow products with A^H.
 *     Requires a handle created with MPSPMV_TRANSPOSE (MPSPMV_ENOTSUP
 *     otherwise).  Complex data keep the shadow vectors conjugated, so the
 *     shadow product is mpspmv_spmtv of a conjugated vector.
 *   CGS (Sonneveld): r^ = r_0.
 *   GPBiCG (Zhang): r^ = r_0; the iteration also stops, after x += alpha p,
 *     when ||t_k|| = ||r_k - alpha A p_k|| meets the test (t_k is the
 *     residual of that iterate).
 * MPSPMV_EXACT_ACC handles use the exact vector arithmetic of mpspmv_dot /
 * mpspmv_axpy.  Synchronise `stream` before returning.
 */
int mpspmv_bicg(mpspmv_h h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
                double* relres, void* stream);
int mpspmv_cgs(mpspmv_h h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
               double* relres, void* stream);
int mpspmv_gpbicg(mpspmv_h h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
                  double* relres, void* stream);

/*
 * Krylov vector operations in the handle's precision and arithmetic (the
 * inner products and vector updates of Section 4.2's CG and BiCGSTAB, with
 * every vector and scalar in DD / TD / QD).  The handle supplies L, real or
 * complex, and the arithmetic only; n is the vectors' own length (plane
 * stride), n >= 0.  Vectors are device arrays of P planes of n (complex: the
 * L real planes, then the L imaginary planes).
 *   Paper order (default): each product and sum in the MP arithmetic of
 *     Algorithms 1-5; mpspmv_axpy is bit-identical, element by element, to
 *     the same operations done in sequence.
 *   MPSPMV_EXACT_ACC handles: each updated element is formed from the
 *     error-free products in one exact fixed-point sum and rounded (truncated)
 *     to L components once; each thread's share of an inner product is summed
 *     exactly, the shares are added in MP arithmetic.  mpspmv_cg and
 *     mpspmv_bicgstab use the same kernels for such handles.
 *
 * mpspmv_dot -- out (host, 2L doubles) = sum_i conj(u_i) v_i: out[0..L) the
 *   real part's components, out[L..2L) the imaginary part's (zeros for a real
 *   handle).  Synchronises `stream`.
 * mpspmv_axpy -- w = u + alpha v; alpha (host, 2L doubles, same layout as
 *   out; the imaginary part is ignored for a real handle).  w may be u or v
 *   (element-wise in place); other overlaps are undefined.  Asynchronous.
 * Both return MPSPMV_EINVAL for a NULL handle, n < 0, or a NULL vector or
 * scalar with n > 0 (mpspmv_dot: a NULL out always).
 */
int mpspmv_dot(mpspmv_h h, int64_t n, const double* u, const double* v, double* out, void* stream);
int mpspmv_axpy(mpspmv_h h, int64_t n, const double* alpha, const double* u, const double* v, double* w,
                void* stream);

/*
 * MP scalars of a solve whose vectors are split into row blocks, one block
 * per process (the row-parallel CSR product of Section 3 with the inner
 * products of Section 4.2's solvers).  The handle supplies L, real or
 * complex, and the arithmetic only.  Scalars use mpspmv_dot's layout: 2L
 * host doubles, the real part's components, then the imaginary part's.
 *
 * mpspmv_scalar_sum -- out = parts[0] + parts[1] + ... + parts[count-1]
 *   (parts: host, count x 2L doubles, e.g. the blocks' mpspmv_dot results in
 *   rank order; 1 <= count <= 4096).  Paper order: MP additions from left to
 *   right, so every process that sums the same parts gets the same bits,
 *   independent of any collective's own summation order.  MPSPMV_EXACT_ACC
 *   handles: the exact sum of all components, cut to L components once.
 * mpspmv_scalar_div -- out = a / b in the handle's precision (complex:
 *   a conj(b) / |b|^2 after scaling a and b by one power of two).
 *   MPSPMV_EBREAKDOWN when every component of b is zero.
 * Both run one device thread and synchronise `stream`; MPSPMV_EINVAL for a
 * NULL pointer or a count out of range.
 */
int mpspmv_scalar_sum(mpspmv_h h, int count, const double* parts, double* out, void* stream);
int mpspmv_scalar_div(mpspmv_h h, const double* a, const double* b, double* out, void* stream);

/*
 * Batched products and solves over many independent matrices of one
 * precision (real, P mode, nnz > 0 each), each with k_i right-hand sides
 * (1 <= k_i <= 32).  The paper multiplies one matrix at a time (Sections 3
 * and 4); the batch runs hundreds of uneven matrices in one persistent launch.
 */
typedef struct mpspmv_batch* mpspmv_batch_h;

#define MPSPMV_BATCH_AUTOTUNE 1u /* time run lengths K and lanes per run w per matrix at creation */

/*
 * mpspmv_batch_create -- group `count` handles with k[i] right-hand sides.
 * The handles stay owned by the caller and must outlive the batch; with
 * MPSPMV_BATCH_AUTOTUNE each handle may be re-cut into runs of another length
 * (K in {8, 16, 32, 64}, chosen by timing; results stay within the SpMV
 * bound).  Synchronises `stream`.
 */
int mpspmv_batch_create(const mpspmv_h* mats, const int* k, int count, unsigned flags, mpspmv_batch_h* out,
                        void* stream);

/* Release the batch (not its handles). */
int mpspmv_batch_destroy(mpspmv_batch_h b);

/* Host arrays of count entries: the run length K and lanes per run w chosen
 * for each matrix (either may be NULL). */
int mpspmv_batch_get_plan(mpspmv_batch_h b, int* K, int* w);

/*
 * mpspmv_batch_spmm -- Y_i = A_i X_i for every matrix in one CUDA graph
 * launch (queue reset, persistent run kernel, row-boundary combine).
 *  X, Y      host arrays of count device pointers; matrix i's X and Y use the
 *            mpspmv_spmm layout with k[i] columns and leading dimensions
 *            ldx[i], ldy[i] (host arrays; NULL means k[i]).
 * The graph is cached for the last (X, Y, ldx, ldy) set.  Each column of Y_i
 * equals mpspmv_spmv on the same handle except that rows spanning more than
 * 32 runs are combined serially.  Asynchronous.
 */
int mpspmv_batch_spmm(mpspmv_batch_h b, const double* const* X, const int64_t* ldx, double* const* Y,
                      const int64_t* ldy, void* stream);

/*
 * mpspmv_batch_cg -- CG (as mpspmv_cg, Section 4.2) on every (matrix, column)
 * system at once: sum(k) independent solves, each with its own scalars and
 * stopping test, iterations captured in a CUDA graph and replayed until no
 * system is running.
 *  B, X      host arrays of count device pointers; n_i x k_i row-major planes
 *            (ldb, ldx NULL or equal to k[i]).  X holds the initial guesses
 *            and returns the iterates.
 *  iters, relres, status   host arrays of sum(k) entries (may be NULL):
 *            iterations, true relative residual, per-system status.
 * Returns MPSPMV_EBREAKDOWN if any system broke down, else MPSPMV_ENOCONV if
 * any reached maxit, else MPSPMV_OK.  Synchronises `stream`.
 */
int mpspmv_batch_cg(mpspmv_batch_h b, const double* const* B, const int64_t* ldb, double* const* X,
                    const int64_t* ldx, double rtol, double atol, int maxit, int* iters, double* relres, int* status,
                    void* stream);

/*
 * Precision ladder (binary64 -> DD -> TD -> QD) and the learned selector.
 * The paper observes that Krylov iteration counts settle as the precision
 * rises (Section 4.2) and motivates multiple precision by round-off
 * (Section 1); these entry points choose the precision per system.
 *
 * `hs` is a host array of 4 handles of the same real, square, P-mode matrix
 * at L = 1, 2, 3, 4 (hs[L-1]; NULL skips that level).  b is one binary64
 * plane of n (device); x is 4 planes of n (device, QD: a level-L iterate uses
 * the first L planes, the others stay zero, so moving up a level is exact).
 */

/*
 * mpspmv_ladder_solve -- x = 0, then CG (mpspmv_cg) at L = start_L, ... 4:
 * after each level the residual b - A x is recomputed in that level's
 * precision; when it meets rtol ||b|| + atol the solve stops, otherwise CG
 * restarts at the next level from the current x.  maxit applies per level.
 *  final_L  host: last level run.  iters: host array of 4, iterations per
 *  level.  relres: host, the last recomputed relative residual.
 * Returns MPSPMV_OK on success, MPSPMV_ENOCONV if no level met the target.
 * Synchronises `stream`.
 */
int mpspmv_ladder_solve(const mpspmv_h* hs, int start_L, const double* b, double* x, double rtol, double atol,
                        int maxit, int* final_L, int* iters, double* relres, void* stream);

/*
 * mpspmv_cg_history -- ||r_j|| / ||b||, j = 1..k (k <= 16), of the first k
 * CG steps from x = 0 on handle h (recurrence residual, h's precision); b has
 * h's planes.  hist: host array of k.  Synchronises `stream`.
 */
int mpspmv_cg_history(mpspmv_h h, const double* b, int k, double* hist, void* stream);

/*
 * mpspmv_features -- the selector's 32 features of handle h (host floats):
 * row-length statistics, diagonal dominance, log norms, Gershgorin bounds,
 * and (when cg_hist, 8 host doubles from mpspmv_cg_history, is given) the
 * binary64 CG residual history and its slope.  Synchronises `stream`.
 */
int mpspmv_features(mpspmv_h h, const double* cg_hist, float* feat, void* stream);

/*
 * Selector network: float32 MLP 32 -> 128 -> 128 -> C (ReLU hidden layers,
 * softmax cross-entropy), parameters in one device buffer of
 * mpspmv_mlp_param_count(C) floats: W1 (32x128), b1, W2 (128x128), b2,
 * W3 (128xC), b3, row-major, activations h = x W + b.  X: device, B x 32
 * row-major; y: device int labels in [0, C).
 */
int64_t mpspmv_mlp_param_count(int C);
/* logits: device, B x C. Synchronises `stream`. */
int mpspmv_mlp_forward(const float* params, int C, const float* X, int B, float* logits, void* stream);
/* grads: device, same layout as params; loss: host (mean cross-entropy). */
int mpspmv_mlp_grad(const float* params, int C, const float* X, const int* y, int B, float* grads, float* loss,
                    void* stream);
/* `epochs` passes of plain SGD (step lr) over n samples in mini-batches of
 * `batch` (in data order; a final partial batch is skipped); params updated
 * in place; loss_per_epoch: host array of epochs (may be NULL). */
int mpspmv_mlp_train(float* params, int C, const float* X, const int* y, int n, int batch, int epochs, float lr,
                     float* loss_per_epoch, void* stream);

/*
 * Input standardisation of the selector network, on the device.
 * mpspmv_mlp_standardize -- for n feature vectors X (device, n x 32
 *   row-major): mu, sd (device, 32 floats each) = mean and population
 *   standard deviation of every feature (binary64 sums in sample order,
 *   rounded to float; a deviation below 1e-6 becomes 1), and Xs (device,
 *   n x 32) = (X - mu) / sd.  Asynchronous.
 * mpspmv_mlp_fold -- rewrite W1 and b1 of params (device) in place so that
 *   the network takes raw features: W1 / sd (row i divided by sd_i) and
 *   b1 - (mu / sd) W1, in binary64 rounded to float.  A network trained on
 *   mpspmv_mlp_standardize's Xs then gives, on raw X, the logits it gave on Xs
 *   (to float rounding).  Asynchronous.
 */
int mpspmv_mlp_standardize(const float* X, int n, float* mu, float* sd, float* Xs, void* stream);
int mpspmv_mlp_fold(float* params, int C, const float* mu, const float* sd, void* stream);

/*
 * mpspmv_select_precision -- features of (hs[0], b) (binary64 CG history
 * included) -> network -> *prec in 1..4 (classes binary64, DD, TD, QD and
 * "none", which maps to QD).  feat_out: host 32 floats, may be NULL.
 */
int mpspmv_select_precision(const mpspmv_h* hs, const float* params, int C, const double* b, int* prec,
                            float* feat_out, void* stream);

/* mpspmv_solve_auto -- mpspmv_select_precision, then mpspmv_ladder_solve from
 * the chosen level (the ladder is the fallback when the choice falls short). */
int mpspmv_solve_auto(const mpspmv_h* hs, const float* params, int C, const double* b, double* x, double rtol,
                      double atol, int maxit, int* chosen_L, int* final_L, int* iters, double* relres, void* stream);

/*
 * mpspmv_spmv_csr_noalloc -- y = A x for callers that cannot allocate device
 * memory when they multiply: a process that has given all of its device
 * memory to its own pool or arena at start-up, or a latency-bound loop that
 * cannot take the device-wide synchronisation of cudaMalloc / cudaFree.  The
 * paper has no counterpart.  The matrix comes as plain caller-owned CSR
 * arrays and no handle is made; the arithmetic is the paper-order MP
 * multiply and add of mpspmv_spmv, over runs of 16 stored entries summed
 * one per thread.  Results meet the bound of mpspmv_spmv,
 * 8 m u (|A||x|)_i; they equal mpspmv_spmv's bit for bit only on rows that
 * both entry points sum within one run (a handle cuts rows into runs of
 * another length, and MPSPMV_EXACT_ACC handles use another arithmetic).
 *
 *  prec        1..4 (L).   flags  0 or MPSPMV_COMPLEX (P = L or 2L planes).
 *  nrows, ncols, nnz   shape; nnz must equal indptr[nrows] (it is not read
 *              from the device): with a smaller nnz, rows past the first nnz
 *              entries are left unspecified, with no error.
 *  indptr      device, nrows + 1 int64 row offsets, non-decreasing from 0.
 *  indices     device, nnz int32 column indices, each in [0, ncols).
 *  vals        device, P planes of nnz binary64 (CSR order, structure of limbs).
 *  x, y        device, P planes of ncols / nrows; y must not overlap x.
 *
 * No cudaMalloc, cudaFree or allocating library call is made.  The partial
 * sums of rows that cross a run boundary go to a fixed 32 MiB array in the
 * library's device image, so nnz may be at most 2^22 / (2 P) * 16 (DD:
 * 16,777,216; QD complex: 4,194,304); larger problems return MPSPMV_EINVAL.
 *
 * Set-up: CUDA loads the module that holds the array lazily, on the first
 * call on each device; that call places the array (32 MiB, kept until the
 * process exits) and the module's code in device memory, looks up the
 * array's device address (cudaGetSymbolAddress) and caches it.  A call with
 * nrows = 0 (pointers may be NULL) does only this set-up.  Make one such call
 * per device, with that device current, at start-up: before the caller's
 * pool or arena claims the device's memory, and before any stream capture.
 * The cached address belongs to the device's primary context: after
 * cudaDeviceReset this entry point must not be used again in the process.
 *
 * Every call shares the array and leaves its partial sums there; each call
 * writes every slot it reads, so nothing needs clearing, but calls that
 * overlap on the GPU (two streams, or two host threads) race on it and must
 * be ordered by the caller.  Asynchronous on `stream`.
 */
int mpspmv_spmv_csr_noalloc(int prec, unsigned flags, int64_t nrows, int64_t ncols, int64_t nnz,
                            const int64_t* indptr, const int32_t* indices, const double* vals, const double* x,
                            double* y, void* stream);

/*
 * mpspmv_probe_fp64 -- measured binary64 instruction throughput of this GPU
 * at the current clocks (the compute denominator of the SpMV roofline; the
 * paper has no counterpart -- its kernels are CPU SIMD code).
 *
 *  op           0 = DFMA, 1 = DADD, 2 = DMUL.
 *  iters        loop trips per thread (each trip = 8 independent instructions).
 *  instr_per_s  host; receives the best of two timed runs, in instructions/s.
 * Synchronous: allocates a small scratch buffer and synchronises `stream`.
 */
int mpspmv_probe_fp64(int op, int iters, double* instr_per_s, void* stream);


#ifdef __cplusplus
}
#endif

#endif /* MPSPMV_H */
