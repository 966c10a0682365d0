/*
 * feast_gb300.h -- C ABI of the GB300 (sm_103a) oblique-projection FEAST
 * solver for the generalized eigenproblem A x = lambda B x (Yin, Chan &
 * Yeung, "A FEAST algorithm with oblique projection for generalized
 * eigenvalue problems").
 *
 * The solver finds the eigenpairs whose eigenvalues lie strictly inside a
 * closed contour Gamma.  Its hot path is the contour-integral subspace build
 * of eq. 4.1 -- one shifted multi-right-hand-side solve (z_j B - A) X_j = B U1
 * per quadrature node (eq. 4.2), summed as U = sum_j w_j X_j -- followed by
 * the oblique (Petrov-Galerkin) projection onto the test space B K (eq. 3.9
 * to 3.10): A~ = U2^H A U1, B~ = U2^H B U1 with U2 an orthonormal basis of
 * B U1, a small QZ solve of (A~, B~), the residuals of eq. 5.1 and the three
 * stopping tests of Algorithm GFEAST (Section 4.3).
 *
 * Conventions for every entry point:
 *   - Matrices are column-major complex128 (interleaved re, im doubles)
 *     unless stated otherwise, with an explicit leading dimension.
 *   - "device" pointers are CUDA global-memory addresses on the current
 *     device; "host" pointers are ordinary CPU memory.
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as
 *     void*; NULL is the legacy default stream) except where a call says it
 *     synchronises.
 *   - The return value is FEAST_OK (0) or a negative FEAST_E* status.  The
 *     paper's convergence flag (1 / 0 / -1) is a result, not an error.
 *   - No entry point allocates device memory except feast_setup's host-side
 *     context record; all device workspace is caller-provided.
 */
#ifndef FEAST_GB300_H
#define FEAST_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------- status codes */
#define FEAST_OK          0
#define FEAST_EINVAL     -1   /* an argument is out of range or inconsistent      */
#define FEAST_ENOMEM     -2   /* workspace too small or host allocation failed    */
#define FEAST_ECUDA      -3   /* a CUDA runtime call or kernel launch failed      */
#define FEAST_ESINGULAR  -4   /* a shifted matrix z_j B - A has an exact zero pivot */
#define FEAST_ENONFINITE -5   /* NaN or Inf reached a residual                    */
#define FEAST_ETIMEOUT   -6   /* a bounded device wait gave up (after 4 s of device
                                 time); feast_last_cuda_error names the wait      */
#define FEAST_ENOCONV    -7   /* the projected QZ hit its iteration cap, two runs disagree, or SEARCH
                                  outgrew the workspace's width */
#define FEAST_EDONE      -8   /* feast_iterate called after the algorithm stopped */

/* ------------------------------------------------------------- problem types */
typedef enum { FEAST_DENSE = 0, FEAST_BANDED = 1 } feast_kind;
typedef enum { FEAST_CIRCLE = 0, FEAST_ELLIPSE = 1 } feast_contour_kind;
typedef enum { FEAST_TRAPEZOID = 0, FEAST_GAUSS_LEGENDRE = 1 } feast_rule;
typedef enum { FEAST_FP64 = 0, FEAST_C64_REFINE = 1 } feast_precision;

/* Projection of line 5.  FEAST_OBLIQUE: the paper's method, test basis U2
 * with U2 R2 = B U1 (eq. 3.10, Algorithm GFEAST).  FEAST_RAYLEIGH_RITZ: the
 * Rayleigh-Ritz projection of Algorithm FEAST (Section 3), A~ = U1^H A U1,
 * B~ = U1^H B U1 -- made for Hermitian A with Hermitian positive definite B,
 * and failing where U1^H B U1 is singular (Example 3.1: every Ritz pair is
 * then rejected; a projected pencil singular to rounding may instead end
 * the projected solve with FEAST_ENOCONV). */
typedef enum { FEAST_OBLIQUE = 0, FEAST_RAYLEIGH_RITZ = 1 } feast_projection;

/* The regular pencil z B - A of eq. 1.1 (Section 1: only regularity is
 * required).
 *   kind = FEAST_DENSE : A, B are device n x n complex128, leading dim ld.
 *   kind = FEAST_BANDED: A, B are device complex128 in compact band storage,
 *                        entry (i, j) at row ku + i - j of column j,
 *                        ld >= kl + ku + 1.  The band solves stage the
 *                        band in shared memory, which bounds it: about
 *                        kl + ku <= 597 with FEAST_FP64 and <= 1199 with
 *                        FEAST_C64_REFINE (FEAST_EINVAL beyond).
 *   b_is_identity != 0 : B = I and the B pointer is ignored (may be NULL).
 * The matrices are read during feast_setup only (copied into the context). */
typedef struct {
    int kind;
    int64_t n;
    const void *A;
    const void *B;
    int64_t ld;
    int64_t kl, ku;
    int b_is_identity;
} feast_pencil;

/* The contour Gamma.  Circle: centre (center_re, center_im), radius a (b is
 * ignored).  Ellipse: semi-axis a along the real axis, b along the
 * imaginary axis.  q quadrature nodes, rule = trapezoid (theta_j =
 * 2 pi (j - 1/2) / q) or Gauss-Legendre (theta_j = (1 + t_j) pi, eq. 4.1).
 * "Inside" is strict (|lambda - centre| < a for the circle). */
typedef struct {
    int kind;
    double center_re, center_im, a, b;
    int q;
    int rule;
} feast_contour;

/* Collective hook of a node-sharded run (one rank per GPU, each owning a
 * range of quadrature nodes; see feast_options.node_begin).
 *   op = FEAST_COLL_SUM  : buf <- the elementwise sum of every rank's buf
 *                          (in place, on every rank);
 *   op = FEAST_COLL_BCAST: buf <- rank 0's buf on every rank.
 * buf is feast_options.collective_buf (device), ndoubles its used length.
 * The library calls it from the thread of feast_setup / feast_iterate /
 * feast_filter after enqueuing on `stream` the work that wrote buf; the
 * hook must order its collective after that work and make the result
 * visible to work enqueued on `stream` after it returns (an NCCL collective
 * issued on or ordered with `stream`, or a synchronisation, a host copy,
 * a host collective and a copy back).  Every rank makes the same sequence
 * of calls.  Return 0, or non-zero on failure (the library then returns
 * FEAST_ECUDA).  Uses: the partial sums of line 16 and of the first
 * subspace (SUM, 2 n m0 doubles), the set-up's singular-pivot outcome
 * (SUM, 1 double) and each pass's stopping flag (BCAST, 1 double: rank 0's
 * flag is every rank's, so that all ranks stop at the same pass). */
enum { FEAST_COLL_SUM = 0, FEAST_COLL_BCAST = 1 };
typedef int (*feast_collective_fn)(void *user, int op, void *buf, int64_t ndoubles, void *stream);

/* Iteration controls (GFEAST inputs, Section 4.3).
 *   m0        : subspace width t (>= the number of eigenvalues inside).
 *   Y0        : device n x m0 complex128 start block (leading dim n); the
 *               first subspace is U = Q Y0 by the quadrature (Algorithm
 *               EIGENPAIRS, line 2).  Required (no internal RNG).
 *   eps, eta  : accuracy and spurious-detection tolerances of lines 10, 13.
 *   max_iter  : line 15.
 *   prec      : FEAST_FP64 (every step in FP64) or FEAST_C64_REFINE
 *               (complex64 factors and solves on the tensor cores; inside
 *               feast_iterate line 16 runs in defect form on the Ritz pairs,
 *               U = X rho(Lambda) + sum_j w_j M_j^{-1} (R D_j) with
 *               R = A X - B X Lambda, which needs no refinement sweeps).
 *   max_refine, refine_tol : refinement of each shifted solve in
 *               feast_filter under FEAST_C64_REFINE (sweeps until the
 *               relative residual is <= refine_tol, at most max_refine).
 *   stream    : cudaStream_t for every launch of this context.
 *   no_stop   : benchmark aid -- when non-zero, feast_iterate always performs
 *               lines 16-17 and keeps iterating after a stop has fired (the
 *               stopped result stays available through feast_eigs).
 *   converged_only : when non-zero, line 14 (stop with flag 0 when e(k)
 *               grows) is not applied: the run ends only with flag 1 (count
 *               fixed and e(k) < eps, line 13) or -1 (max_iter).  For users
 *               that need converged pairs, e.g. the differentiation form.
 *   projection : FEAST_OBLIQUE (default, zero) or FEAST_RAYLEIGH_RITZ.  Under
 *               Rayleigh-Ritz no test basis is built (feast_get's U2 / R2
 *               are not maintained) and every projected solve starts cold. */
typedef struct {
    int m0;
    const void *Y0;
    double eps, eta;
    int max_iter;
    int prec;
    int max_refine;
    double refine_tol;
    void *stream;
    int no_stop;
    int converged_only;
    int projection;
    /* Node sharding (end of Section 4.3: the q shifted systems of eq. 4.2
     * are independent).  node_begin = node_end = 0: this context owns every
     * node.  Otherwise 0 <= node_begin < node_end <= q: it forms, factors
     * and solves only nodes j in [node_begin, node_end) (the LU memory
     * shrinks accordingly), its line-16 quadrature sum covers those nodes
     * only, and collective (required) combines the ranks: see
     * feast_collective_fn.  collective_buf: device, 256-byte aligned, at
     * least 2 * n * m0 doubles, owned by the caller, handed to every
     * collective call.  Every other step (lines 5-15, 17) runs on every
     * rank on the summed subspace. */
    int node_begin, node_end;
    feast_collective_fn collective;
    void *collective_user;
    void *collective_buf;
} feast_options;

/* Per-pass report.  flag: 2 = continue, 1 = converged (line 13), 0 = no
 * further improvement, previous iterate returned (line 14), -1 = max_iter
 * (line 15).  bad_node: 1-based node whose factor had a zero pivot. */
typedef struct {
    int k, count, flag;
    double err;
    double ms_lu, ms_solve, ms_refine, ms_qr, ms_proj, ms_qz;
    int refine_sweeps_max;
    int bad_node;
    int qz_sweeps;    /* QR sweeps of the projected eigensolve (m0 > 64), this pass */
    int qz_phases;    /* bulge-chase phases of those sweeps */
    int qz_warm;      /* 1: the projected problem was solved warm (only its
                         unconverged trailing block went through the QR) */
    int qz_rows;      /* rows given to the QR this pass (m0 when cold) */
    double qz_warm_resid; /* largest relative eigen-residual of the warm
                         solve's Newton step (0 when not tried) */
    int qz_warm_k;    /* converged leading columns the warm solve found
                         (-1 when it was not tried) */
    double ms_warm_gemm;   /* device time of the warm solve's FP64 product
                              segments (GEMMs and triangular inverses) */
    double warm_gemm_flop; /* their algorithmic flops (complex MAC = 8) */
    double ms_tc_gemm;     /* dense precision form: device time of the
                              tensor-core GEMM launches alone -- the LU's
                              trailing updates (feast_setup) or this pass's
                              shifted solves' off-block updates (feast_iterate) */
    double tc_gemm_flop;   /* their algorithmic flops (complex MAC = 8) */
    int qz_cold_fp32;      /* the projected solve started cold: 1 = its Schur
                              form came from the FP32 QR, polished by the
                              FP64 Newton step and accepted; -1 = that was
                              tried and rejected (the double-single QR ran);
                              0 = not tried */
} feast_iter_info;

typedef struct feast_ctx feast_ctx;

/* Device workspace (bytes, 256-byte aligned start required) that
 * feast_setup needs for this problem.  Returns FEAST_EINVAL on bad sizes. */
int feast_workspace_size(const feast_pencil *pencil, const feast_contour *contour,
                         const feast_options *opts, size_t *bytes);

/* GFEAST lines 1-3 with the start block Y0 in place of SEARCH: nodes and
 * weights (eq. 4.1), z_j B - A for every node, their LU factors (factored
 * once and reused every pass, end of Section 4.3), U = Q Y0 by quadrature,
 * U = U1 R1, B U1 = U2 R2.  workspace: device, >= feast_workspace_size bytes,
 * owned by the caller and used by the context until feast_destroy.
 * Synchronises the stream once (to report singular pivots).  On success
 * *out receives a context; info (may be NULL) receives ms_lu. */
int feast_setup(feast_ctx **out, const feast_pencil *pencil, const feast_contour *contour,
                const feast_options *opts, void *workspace, size_t workspace_bytes,
                feast_iter_info *info);

/* One pass of GFEAST lines 5-17: projection A~, B~ (line 5), projected
 * eigenpairs and Ritz vectors x_i = U1 y_i (line 6), residuals r_i of
 * eq. 5.1 and the selection of line 10, c(k), e(k) and the stopping tests
 * of lines 13-15 (evaluated on the device), then -- unless a test fired --
 * the quadrature of line 16 (eq. 4.1-4.2) and U = U1 R1, B U1 = U2 R2
 * (line 17).  Line 16 is applied to the Ritz vectors X = U1 Y (the same
 * subspace as U1's) when m0 >= 96 (ordered by r_i / |rho(lambda_i)|, most
 * converged first) and always under FEAST_C64_REFINE; from the second pass
 * on, line 6 for m0 >= 96 reuses that order (QR of the unconverged
 * trailing block only, one FP64 Newton step for the rest, accepted against
 * a residual bound, else the full solve).  Synchronises the stream a few
 * times (projected-solve decisions, c(k), e(k) and the flag).  Returns
 * FEAST_EDONE if the algorithm has stopped and no_stop is 0. */
int feast_iterate(feast_ctx *ctx, feast_iter_info *info);

/* Output of lines 13-15 (the previous iterate's pairs when flag = 0).
 *   count  : host, number of pairs returned.
 *   lambda : host, 2 * m0 doubles (re, im) -- at least count pairs written.
 *   X      : device, n x count complex128 (leading dim ldx) or NULL.
 *   resid  : host, m0 doubles (eq. 5.1 residuals) or NULL.
 *   err, flag : host.
 * Synchronises the stream.  Returns FEAST_EINVAL if no stop has fired yet. */
int feast_eigs(feast_ctx *ctx, int *count, double *lambda, void *X, int64_t ldx, double *resid,
               double *err, int *flag);

/* Diagnostic accessor for the test-suite: copies an internal array to the
 * device buffer dst (asynchronous).  what: 0 U1 (n x m0), 1 U2 (n x m0),
 * 2 R2 (m0 x m0), 3 A~ (m0 x m0), 4 B~ (m0 x m0), 5 Ritz vectors (n x m0),
 * 6 Ritz values (m0), 7 A U1 (n x m0), 8 B U1 (n x m0), 9 nodes (q),
 * 10 weights (q), 11 residuals r_i (m0 doubles), 12 selection flags
 * (m0 int32).  All complex128 column-major with leading dim = rows. */
int feast_get(const feast_ctx *ctx, int what, void *dst);

/* Block CIRR (Section 2.1, Algorithm Block_CIRR), the comparison method the
 * paper measures GFEAST against, on this context's pencil, contour and
 * factors (the context must have been set up with FEAST_RAYLEIGH_RITZ):
 *   1. R_i = F_i Y, i = 0..g-1, by the context's quadrature, in the shifted
 *      and scaled form sum_j w_j ((z_j - centre) / max(a, b))^i
 *      (z_j B - A)^{-1} Y (degree by degree the span of the z^i moments);
 *   2. an orthonormal basis U1 of [R_0, ..., R_{g-1}] (QR: the SVD's U of
 *      the algorithm spans the same space);
 *   3-5. one Rayleigh-Ritz pass (feast_iterate with the stop of line 15):
 *      the pairs inside the contour with eq. 5.1 residual below eta are the
 *      result, read with feast_eigs (flag -1: one pass, no convergence test).
 *   Y    : device n x h complex128 (leading dim n), the random block.
 *   h, g : block width and number of moments; t = h g <= the m0 given to
 *          feast_setup, and the context's width becomes t.
 *   info : host out, the pass report of step 3-5.
 * FEAST_EINVAL for a bad argument or an oblique context.  Synchronises the
 * stream. */
int feast_cirr(feast_ctx *ctx, const void *Y, int h, int g, feast_iter_info *info);

/* Sparse pencils onto the banded path.  The paper's pencils are sparse
 * discretisations; a symmetric permutation P A P^T, P B P^T keeps the
 * eigenvalues (eigenvectors are permuted), so a bandwidth-reducing ordering
 * lets such a pencil run as FEAST_BANDED.
 *
 * feast_csr_rcm: reverse Cuthill-McKee ordering of the symmetrised joint
 * pattern of A and B (host arrays; CSR with int64 row pointers rowptr[0..n]
 * from 0 and column indices; B may be NULL for B = I).  perm (host, n):
 * perm[new] = old.  kl, ku (host out): the lower / upper bandwidth of both
 * permuted matrices.  FEAST_EINVAL for malformed CSR.  Host only; no CUDA. */
int feast_csr_rcm(int64_t n, const int64_t *a_rowptr, const int64_t *a_col, const int64_t *b_rowptr,
                  const int64_t *b_col, int64_t *perm, int64_t *kl, int64_t *ku);

/* feast_csr_to_band: writes P M P^T of the CSR matrix M (device rowptr,
 * col, complex128 val) into compact band storage band (device,
 * (kl + ku + 1) x n column-major, entry (i, j) at row ku + i - j), zero
 * elsewhere; duplicate entries are summed.  iperm (device, n): iperm[old] =
 * new.  status: a device int of scratch.  FEAST_EINVAL if an entry falls
 * outside the band or a column index is out of range (those entries are
 * skipped).  Synchronises the stream. */
int feast_csr_to_band(int64_t n, const int64_t *rowptr, const int64_t *col, const void *val, const int64_t *iperm,
                      int64_t kl, int64_t ku, void *band, int *status, void *stream);

/* SEARCH (Section 4.1, Algorithm SEARCH): an upper bound t of the number of
 * eigenvalues inside the contour and a basis of the filtered subspace, which
 * then replaces the start block (Algorithm 6, line 1): on success the
 * context's width becomes t and feast_iterate starts from U1 = that basis.
 *   Ypool   : device n x npool complex128 (leading dim n), the random columns
 *             the algorithm draws, used in order (its first p are Y_0, each
 *             augmentation takes the next ones); the caller draws them.
 *   alpha   : growth factor (> 1) of line 10; p: first sample size (line 1),
 *             1 <= p <= the context's m0.
 *   rank_tol: the numerical rank of line 9 counts R_kk > rank_tol R_00 in the
 *             column-pivoted factorisation (0 < rank_tol < 1; resolved down
 *             to ~1e-7, the factorisation runs on the Gram matrix).
 *   t, s0   : host out: the bound (width) and the trace estimate of line 2.
 * The working width may not exceed the m0 given to feast_setup (its
 * workspace): FEAST_ENOCONV if the search would grow beyond it, or if the
 * filtered block stays of full rank up to n; FEAST_EINVAL if Ypool runs out.
 * Synchronises the stream. */
int feast_search(feast_ctx *ctx, const void *Ypool, int npool, double alpha, int p, double rank_tol, int *t,
                 int *s0);

/* The subspace build alone (GFEAST line 16, eq. 4.1-4.2) with the stored
 * factors: U = sum_j w_j (z_j B - A)^{-1} B V.  V, U: device n x m0
 * complex128, leading dim n.  Asynchronous. */
int feast_filter(feast_ctx *ctx, const void *V, void *U);

/* Replace U1 by the device n x m0 matrix U1 (assumed orthonormal) and
 * recompute U2 R2 = B U1 -- lets a test start a pass from a chosen subspace. */
int feast_set_subspace(feast_ctx *ctx, const void *U1);

void feast_destroy(feast_ctx *ctx);
const char *feast_strerror(int status);

/* Complex64 GEMM on the 5th-generation tensor cores (tcgen05, TF32 inputs
 * with a head/tail split of each operand for ~FP32 accuracy, FP32
 * accumulation in tensor memory): C_b = beta C_b + alpha A_b X_b for b <
 * batch, column-major interleaved complex64, A m x k, X k x n.  This is the
 * update product of the complex64 factorization and solves of eq. 4.2 in the
 * precision form.  scratch: device, >= feast_cgemm_tc_scratch_bytes bytes
 * (operand copies in the tensor-core layout).  err: device int32, set
 * non-zero (a bit per wait site: 0x40 loads, 0x80 MMA issue, 0x100 epilogue,
 * 0x200 final drain) if a bounded pipeline wait (4 s of device time) gave
 * up.  Asynchronous. */
size_t feast_cgemm_tc_scratch_bytes(int64_t m, int64_t n, int64_t k, int batch);
int feast_cgemm_tc(int64_t m, int64_t n, int64_t k, float alpha_re, float alpha_im, const void *A,
                   int64_t lda, int64_t sA, const void *X, int64_t ldx, int64_t sX, float beta_re,
                   float beta_im, void *C, int64_t ldc, int64_t sC, int batch, void *scratch,
                   size_t scratch_bytes, int *err, void *stream);

/* ---------------------------------------------------------- ragged batch */

/* Per-pencil outcome of feast_solve_batch. */
typedef struct {
    int status;      /* FEAST_OK or the first error of this pencil          */
    int flag;        /* GFEAST flag of lines 13-15                          */
    int count;       /* eigenpairs returned                                 */
    int k;           /* passes run                                          */
    double err;      /* Err of lines 13-15                                  */
    double ms_setup; /* device time of the set-up (LU and first subspace)   */
    double ms_pass;  /* device time of all passes (on this pencil's stream;
                        other pencils' kernels run beside it)             */
    double ms_solve; /* of which the subspace-build solves (line 16)        */
    double ms_qz;    /* of which the projected eigensolves (line 6)         */
} feast_batch_item;

/* Device workspace for feast_solve_batch with nworkers concurrent pencils
 * (0 on invalid input). */
size_t feast_batch_workspace_size(int count, const feast_pencil *pencils,
                                  const feast_contour *contours, const feast_options *opts,
                                  int nworkers);

/* Many independent pencils of uneven size, each with its own contour and
 * options (arrays of count entries; the stream fields are ignored): the
 * whole GFEAST run (set-up, passes until a stopping test fires, output) for
 * every pencil.  nworkers host threads each own a CUDA stream and a slice
 * of the workspace and take pencils in index order, so the kernels of up to
 * nworkers pencils overlap on the GPU (the node-parallel and right-hand-side
 * parallel structure noted at the end of Section 4.3, applied across
 * problems).  Outputs (host): items[count]; lambda: 2 * sum(m0) doubles,
 * pencil i's eigenvalues (re, im) starting at 2 * sum_{p<i} m0_p; resid
 * (may be NULL): sum(m0) doubles, same offsets.  Blocks until all pencils
 * are done; returns FEAST_OK or the first error (see items[i].status). */
int feast_solve_batch(int count, const feast_pencil *pencils, const feast_contour *contours,
                      const feast_options *opts, void *workspace, size_t workspace_bytes,
                      int nworkers, feast_batch_item *items, double *lambda, double *resid);

/* Number of CUDA kernels this library has launched in the process so far
 * (host-side counter; every launch site increments it). */
unsigned long long feast_kernel_launches(void);

/* The CUDA error behind the calling thread's last FEAST_ECUDA: the error's
 * name and the library source location that saw it ("" if none yet); after
 * a FEAST_ETIMEOUT, the kernels whose bounded waits gave up.  The string
 * belongs to the library and stays valid until the thread's next failing
 * call. */
const char *feast_last_cuda_error(void);

/* ---------------------------------------------------- standalone kernels */

/* Batched LU with partial pivoting (pivot = largest modulus), the direct
 * solver of eq. 4.2 (Section 5 factors each shifted matrix once).
 *   M    : device, batch blocks of n x n complex128 (leading dim ld, block
 *          stride stride elements), factored in place (unit-lower L below
 *          the diagonal, U on and above).
 *   piv  : device int32, batch x n; piv[b*n + k] = row swapped with k.
 *   info : device int32[1]: 0, or 1 + (first block with an exact zero pivot).
 * Asynchronous. */
int feast_zgetrf_batched(int64_t n, int batch, void *M, int64_t ld, int64_t stride, int *piv,
                         int *info, void *stream);

/* Solve with those factors: X_b = M_b^{-1} X_b (X: device, batch blocks of
 * n x nrhs, leading dim ldx, block stride sx).  Asynchronous. */
int feast_zgetrs_batched(int64_t n, int64_t nrhs, int batch, const void *M, int64_t ld,
                         int64_t stride, const int *piv, void *X, int64_t ldx, int64_t sx,
                         void *stream);

/* Differentiation form: L = sum over the eigenvalues inside the contour of
 * |lambda|^2 and its gradients G_A, G_B for a real loss of complex inputs
 * (dL = Re sum conj(G_A) dA + Re sum conj(G_B) dB).  First-order
 * perturbation of a simple eigenvalue (right vector x, left vector v):
 * d lambda = v^H (dA - lambda dB) x / (v^H B x), hence
 * G_A = sum 2 lambda_i v_i x_i^H / conj(c_i), G_B = -sum 2 |lambda_i|^2
 * v_i x_i^H / conj(c_i), c_i = v_i^H B x_i.  The paper has no gradient; it
 * is built on top of the method.  right: a finished run (flag set) on
 * (A, B); left: a finished run on (A^H, B^H) over the conjugated contour,
 * whose Ritz vectors are the left eigenvectors (its eigenvalues, conjugated,
 * are paired with the right ones by nearness).  Dense pencils only.  gA,
 * gB: device n x n complex128 (leading dim ldg), overwritten; L, count:
 * host.  FEAST_ENOCONV if the two runs found different inside counts.
 * Uses the right run's internal scratch; synchronises its stream. */
int feast_grad_abs2(feast_ctx *right, feast_ctx *left, void *gA, void *gB, int64_t ldg, double *L, int *count);

/* FP64-accurate complex GEMM on the bf16 tensor cores: C = beta C + alpha A B,
 * A m x k, B k x n, C m x n, complex128 column-major (device, leading dims
 * lda, ldb, ldc).  This is the product of the refinement residual
 * R_j = B V - (z_j B - A) X_j of the precision form (the refinement of the
 * shifted solves of eq. 4.2).  Each row of the real form of A and each
 * column of B is scaled by a power of two and written as 8 base-64 digits;
 * digit products and their sums over K-chunks of 2048 are exact in the
 * tensor cores' FP32 accumulators, and the chunk sums are combined in FP64.
 * Error: about 2^-47 times max_k|A_ik| * max_k|B_kj| * k per entry (not
 * relative to |C|).  work: device, >= feast_zgemm_oz_work_bytes bytes, 256-
 * byte aligned (digit planes).  err: device int32, set non-zero (0x400) if
 * a bounded pipeline wait (4 s of device time) gave up (C is then
 * unspecified).  Asynchronous. */
size_t feast_zgemm_oz_work_bytes(int64_t m, int64_t n, int64_t k);
int feast_zgemm_oz(int64_t m, int64_t n, int64_t k, double alpha_re, double alpha_im, const void *A, int64_t lda,
                   const void *B, int64_t ldb, double beta_re, double beta_im, void *C, int64_t ldc, void *work,
                   size_t work_bytes, int *err, void *stream);

/* Batched eigensolve of projected pencils (GFEAST line 6; the paper points
 * to the LAPACK drivers xGGES / xGGEV).  A, B: device, batch blocks of m x m
 * complex128 (B upper triangular -- its strictly lower part is ignored --
 * as the projected B~ = U2^H B U1 = R2 is), both overwritten.  alpha, beta:
 * device m per pencil, eigenvalue alpha/beta; V: device m x m per pencil,
 * unit-norm right eigenvectors (beta A v = alpha B v).
 *   m <= 64: complex QZ (Hessenberg-triangular reduction, single-shift QZ),
 *            one warp per pencil in shared memory.
 *   m >  64: B must be nonsingular; C = B^{-1} A is reduced to Hessenberg
 *            form and QR-iterated by the whole GPU (beta = 1).
 * work: device, feast_zqz_work_bytes(m, batch) bytes.  status: device
 * int32[2]: [0] pencils whose iteration cap was hit, [1] non-zero if a
 * bounded device barrier timed out.  Asynchronous. */
size_t feast_zqz_work_bytes(int m, int batch);
int feast_zqz_batched(int m, int batch, void *A, void *B, void *alpha, void *beta, void *V,
                      void *work, int *status, void *stream);

/* The same eigensolve for callers that cannot allocate device memory (for
 * example code running during CUDA graph capture, inside a callback that
 * must not touch the allocator, or in a process whose device memory belongs
 * to someone else's pool).  The paper has no counterpart: this is a calling
 * convention, not a step of the method.  Scratch comes from a fixed array
 * inside the library (4 MiB per device, held until the process exits), so
 * the caller passes only A, B, alpha, beta, V and status exactly as for
 * feast_zqz_batched.  Limits: m <= 64 and batch * m * m <= 262144; larger
 * requests return FEAST_EINVAL and queue no work.  No device memory is
 * allocated or freed.  All calls on a device share the array: calls that
 * overlap on the GPU (other streams or host threads) race and must be
 * serialised by the caller.  The first call in each CUDA context (per
 * device; a new primary context after cudaDeviceReset, or a context the
 * caller created, counts as new) looks up the array's address in that
 * context and should come before any stream capture.  Asynchronous. */
int feast_zqz_batched_noalloc(int m, int batch, void *A, void *B, void *alpha, void *beta,
                              void *V, int *status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FEAST_GB300_H */
