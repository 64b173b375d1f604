/*
 * nfl -- NFFT-based fast summation for the graph Laplacian of fully
 * connected Gaussian-weighted graphs, on one GB300 GPU (sm_103a).
 *
 * Method: Alfke, Potts, Stoll, Volkmer, "NFFT meets Krylov methods: Fast
 * matrix-vector products for the graph Laplacian of fully connected
 * networks" (2018).
 *
 *   W_ji = exp(-||v_j - v_i||^2 / sigma^2) for j != i, W_jj = 0   (Sec. 2, eq. (W_gaussian))
 *   d = W 1, D = diag(d), A = D^{-1/2} W D^{-1/2}, L_s = I - A     (Sec. 2, eq. (nomlap))
 *
 * W is never formed.  Products with W~ = W + K(0) I use Alg. 1 (adjoint
 * NFFT, multiply by the Fourier coefficients b_l of the regularized kernel,
 * NFFT); products with A use Alg. 2 (Sec. 3.1).  A plan performs Alg. 2's
 * steps 1-4 once; the apply calls perform step 5.
 *
 * Conventions for every call below:
 *   - Pointers named "device" are CUDA device pointers owned by the caller;
 *     the library never frees them.  The plan owns all of its own device
 *     memory (sorted nodes, grids, coefficients, D^{-1/2}).
 *   - Vectors are FP64.  Blocks of r right-hand sides are column-major with
 *     a leading dimension ld >= n (column c starts at x + c * ld).
 *   - Work is ordered on the plan's stream.  Apply calls do not synchronize
 *     the host; plan creation and the solvers do (they read scalars back).
 *   - Inputs and outputs must not alias.
 *   - A plan is not thread-safe: calls on one plan must not run concurrently
 *     from several host threads (a block product switches the plan's
 *     buffer set for the duration of the call).
 *   - Every call returns an nfl_status.  Errors never trap on the device:
 *     arguments are checked on the host, numerical failures are reported by
 *     status, CUDA errors map to NFL_ERR_CUDA.  After NFL_ERR_CUDA the plan
 *     should be destroyed.
 */
#ifndef NFL_H
#define NFL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nfl_plan nfl_plan;
typedef struct nfl_batch nfl_batch;

typedef enum {
    NFL_OK = 0,
    NFL_ERR_INVALID_ARG = 1,        /* an argument is out of range (see each call)          */
    NFL_ERR_NONPOSITIVE_DEGREE = 2, /* min_j d_E,j <= 0: D_E^{-1/2} undefined (Lemma 3.1)  */
    NFL_ERR_BREAKDOWN = 3,          /* Lanczos beta ~ 0: an invariant subspace was found   */
    NFL_ERR_NOT_CONVERGED = 4,      /* iteration limit reached before the tolerance        */
    NFL_ERR_NAN = 5,                /* a NaN or Inf appeared in a solver's scalars          */
    NFL_ERR_TIMEOUT = 6,            /* a bounded device wait gave up                        */
    NFL_ERR_CUDA = 7,               /* a CUDA runtime call failed                           */
    NFL_ERR_OUT_OF_MEMORY = 8       /* a device allocation failed                           */
} nfl_status;

/* Kernels of Sec. 2 (after eq. (W_gaussian)); r = ||v_j - v_i||, shape parameter s:
 *   GAUSSIAN             exp(-r^2 / s^2)        K(0) = 1
 *   LAPLACIAN_RBF        exp(-r / s)            K(0) = 1  (cusp at r = 0: the fast sum
 *                                                          converges slowly in N)
 *   MULTIQUADRIC         (r^2 + s^2)^{1/2}      K(0) = s
 *   INV_MULTIQUADRIC     (r^2 + s^2)^{-1/2}     K(0) = 1/s
 *   GAUSSIAN_DSIGMA      (2 r^2 / s^3) exp(-r^2 / s^2), the s-derivative of the
 *                        Gaussian (for gradients in sigma)  K(0) = 0
 * Alg. 2 step 2 scales s with the nodes (s~ = rho s); for the multiquadrics
 * the fast sum's output is then scaled by 1/rho (multiquadric) or rho (inverse
 * multiquadric), which makes the scaled kernel equal the caller's (reading of
 * Alg. 2 steps 2, 4, 5, whose printed rule c := c/rho does not); likewise by
 * rho for GAUSSIAN_DSIGMA. */
enum {
    NFL_KERNEL_GAUSSIAN = 0,
    NFL_KERNEL_LAPLACIAN_RBF = 1,
    NFL_KERNEL_MULTIQUADRIC = 2,
    NFL_KERNEL_INV_MULTIQUADRIC = 3,
    NFL_KERNEL_GAUSSIAN_DSIGMA = 4
};

/* Arithmetic of the spread / FFT / gather steps.  Epilogues (-K(0) x,
 * D^{-1/2} scaling, x - A x) and all solver scalars are FP64 in every mode.
 *   FP64  : everything in FP64.
 *   FP32  : window weights, spreading grid, FFT and interpolation in FP32.
 *   FP32C : FP32 window weights and products; FP32 partial sums over at
 *           most 2048 nodes are carried into 64-bit fixed point and
 *           accumulated exactly from there on; FFT in FP32; interpolation
 *           on the tensor cores with FP32-accurate (three-term TF32) products.
 *           Results may vary in the last FP32 bits from run to run where a
 *           kernel's partial sums meet in an order that is not fixed.      */
/*   BF16W : FP32, with every window tap rounded to BF16 (round to nearest,
 *           ties to even) where it is produced, i.e. the accuracy of a design
 *           that stores the per-node 1-D window weights phi / phi(0) in BF16
 *           and accumulates in FP32.  The kernels evaluate the taps instead
 *           of storing them, so BF16 storage would save nothing here; the
 *           form exists to report that accuracy (about 1e-3 relative).      */
enum { NFL_PREC_FP64 = 0, NFL_PREC_FP32 = 1, NFL_PREC_FP32C = 2, NFL_PREC_BF16W = 3 };

typedef struct {
    int64_t n;            /* number of nodes                                   */
    int d;                /* dimension 1..3                                    */
    int N, m, p;          /* bandwidth, window cut-off, regularization order   */
    int precision;        /* NFL_PREC_*                                        */
    double sigma;         /* kernel shape parameter in the caller's coordinates */
    double eps_B;         /* regularization width                              */
    double rho;           /* node scale factor (Alg. 2 step 1)                 */
    double sigma_tilde;   /* rho * sigma (Alg. 2 step 2)                       */
    double center[3];     /* bounding-box midpoint subtracted before scaling   */
    int box[3];           /* extent of the active oversampled grid per axis    */
    int64_t tiles;        /* non-empty spreading tiles                         */
    int64_t work_items;   /* tile chunks (<= 8192 nodes) of the gather; the 3-D
                             warp spread takes runs of tiles built from them  */
    double min_degree;    /* min_j d_E,j                                       */
    double max_degree;    /* max_j d_E,j                                       */
    int degree_ok;        /* 1 if min_degree > 0 (A, L_s and solvers usable)  */
    int device_error;     /* 1 if a kernel's bounded wait ran out (results of
                             the products since then are unreliable)          */
    int kernel;           /* NFL_KERNEL_*                                      */
    double k0;            /* K(0) in the caller's coordinates                  */
    double out_scale;     /* factor from the scaled fast sum to the caller's   */
    int fft_lines_cap;    /* FFT passes: grid points per CTA (lines x length)  */
    int slide_tiles;      /* 3-D warp spread: most tiles in one sliding run    */
    int block_cols;       /* columns per launch of a block product (1: none)   */
    int64_t dense_items;  /* 3-D m = 6 FP32 / FP32C: slab pieces (cells of one
                             axis-0 position) of the tiles with at least
                             dense_cell nodes per occupied cell, which
                             one-column products spread and interpolate by
                             Chebyshev moments                                 */
    int chunk;            /* most nodes in one work item                       */
    int dense_cell;       /* nodes per occupied cell from which a tile is dense */
    int dense_chunk;      /* most nodes in one slab piece of the moment spread */
} nfl_info;

/*
 * Alg. 2 steps 1-4 (Sec. 3.1): shift the nodes by their bounding-box
 * midpoint and scale them by rho = (1/4 - eps_B/2) / max_j ||v_j - c||
 * (rho = 1 when all nodes coincide), set sigma~ = rho sigma (the kernel's
 * shape parameter; see the kernel list above), compute the
 * coefficients b_l of the regularized kernel by the trapezoidal rule
 * (Sec. 3, eq. (b_l::K_RF)) and the degrees d_E = W~_E 1 - K(0) 1.
 *
 *   v         device, n x d row-major FP64 node coordinates (read only; may
 *             be freed after the call returns).
 *   n         >= 1.   d in {1, 2, 3}.
 *   kernel    NFL_KERNEL_* (above).
 *   sigma     > 0: the kernel's shape parameter (sigma, or c for the multiquadrics).
 *   N         bandwidth: a power of two in [4, 512].  Sec. 3 and Fig.
 *             tab:fastsum_param allow any even N; this library reads it as a
 *             power of two (its FFT passes are radix-4/2), which covers every
 *             N the paper uses (16, 32, 64 and 512 in Sec. 6).
 *   m         window cut-off, 1 <= m <= 12.
 *   p         regularization smoothness; p <= 0 selects the default p = m.
 *   eps_B     regularization width in [0, 1/2); eps_B < 0 selects p / N.
 *   precision NFL_PREC_FP64, NFL_PREC_FP32, NFL_PREC_FP32C or NFL_PREC_BF16W.
 *   stream    a cudaStream_t (0 = legacy default stream).
 *   out       receives the plan.
 *
 * Returns NFL_OK even when some degree is <= 0; the A / L_s products and the
 * solvers then return NFL_ERR_NONPOSITIVE_DEGREE (nfl_plan_info tells).
 */
nfl_status nfl_plan_create(const double *v, int64_t n, int d, int kernel, double sigma,
                           int N, int m, int p, double eps_B, int precision,
                           void *stream, nfl_plan **out);

/*
 * G plans at once (Alg. 2 steps 1-4 for each of G independent node sets, e.g.
 * many graphs of uneven size): the same work as G calls of nfl_plan_create,
 * but each stage of plan creation is issued for every plan (spread over the
 * library's streams, forked from `stream`) before the host synchronizes once,
 * so the batch costs a handful of host synchronizations in total rather than
 * a handful per plan.
 *   v[g]      device, n[g] x d row-major FP64 node coordinates of graph g.
 *   n[g]      >= 1.   sigma[g] > 0: the kernel parameter of graph g.
 *   d, kernel, N, m, p, eps_B, precision   as in nfl_plan_create, common to all.
 *   stream    every plan's stream on return.
 *   out       host array of G entries receiving the plans.
 * On any failure no plan is returned (all entries NULL) and the first failing
 * plan's status is returned.  Synchronizes the host.
 */
nfl_status nfl_plan_create_batched(int G, const double *const *v, const int64_t *n, int d, int kernel,
                                   const double *sigma, int N, int m, int p, double eps_B, int precision,
                                   void *stream, nfl_plan **out);

/* Release the plan and its device memory (synchronizes its stream). NULL is ignored. */
void nfl_plan_destroy(nfl_plan *plan);

/* Copy the plan's parameters, degree summary and device error flag into *info
 * (synchronizes the plan's stream to read the flag). */
nfl_status nfl_plan_info(const nfl_plan *plan, nfl_info *info);

/*
 * Pick the launch parameters of the plan's products by timing them on the
 * plan's own nodes (not a paper construct: the products stay those of Alg. 1
 * and Alg. 2 step 5; the paper's parameters N, m, p, eps_B are the caller's) (a W product with x = 1, CUDA events on the plan's
 * stream), one parameter at a time, keeping the fastest:
 *   fft_lines_cap  grid points per CTA of the FFT passes (lines of length
 *                  2N per CTA = cap / 2N), from {256, 512, 1024, 2048};
 *   chunk          3-D: most nodes in one work item of the spread and the
 *                  interpolation, from {2048, 4096, 8192};
 *   dense_cell     3-D m = 6 FP32 / FP32C: nodes per occupied cell from which
 *                  a tile goes to the moment kernels (spread and
 *                  interpolation), from {16, 32, 64};
 *   dense_chunk    the same plans: most nodes in one slab piece of the
 *                  moment spread, from {2048, 4096, 8192};
 *   slide_tiles    3-D warp-slice spread: most tiles of one axis-2 run that
 *                  the tile copies slide along (1 = no sliding), from
 *                  {1, 4, 8, 16}.
 * Results are unchanged up to the FP32 summation order of the mixed forms.
 * The chosen values are in nfl_info; best_ms (host, may be NULL) receives
 * the fastest time of one product.  Synchronizes the plan's stream;
 * allocates 2 n FP64 of device scratch for the call.
 */
nfl_status nfl_plan_autotune(nfl_plan *plan, double *best_ms);

/* Move subsequent work of the plan to another stream. */
nfl_status nfl_set_stream(nfl_plan *plan, void *stream);

/* d (device, n FP64, node order of the input) = d_E = W~_E 1 - K(0) 1
 * (Alg. 2 step 4), as computed at plan creation. */
nfl_status nfl_degree(const nfl_plan *plan, double *d);

/*
 * y = W_E x = W~_E x - K(0) x   (Alg. 1 and Sec. 3, W = W~ - K(0) I).
 * x, y: device FP64 blocks of nrhs >= 1 columns, leading dims ldx, ldy >= n.
 * On the 3-D FP32 / FP32C / BF16W path with m in {2, 3, 4, 6} the columns go
 * through each stage in blocks of nfl_info.block_cols per launch: as many
 * (up to 8) as keep a column's staged values, grids and FFT buffers within
 * half of L2 together, 1 for large plans; elsewhere one column at a time.
 * The first block product allocates the plan's block buffers (make it
 * before capturing products into a CUDA graph: under capture it returns
 * NFL_ERR_INVALID_ARG instead of allocating); no buffer of the plan is
 * ever reallocated, so captured products stay valid.  Where columns go one
 * at a time (block_cols 1) on that path, the staging of column c + 1 runs on a
 * second stream of the plan beside column c's FFT and interpolation, into a
 * second set of staging buffers made by the first such call (under capture,
 * before they exist, the columns go one after another instead).  The same
 * holds for nfl_apply_A and nfl_apply_Ls, and for nfl_apply_host.
 */
nfl_status nfl_apply_W(nfl_plan *plan, const double *x, int64_t ldx,
                       double *y, int64_t ldy, int nrhs);

/* y = A_E x = D_E^{-1/2} (W~_E (D_E^{-1/2} x) - K(0) D_E^{-1/2} x)   (Alg. 2 step 5). */
nfl_status nfl_apply_A(nfl_plan *plan, const double *x, int64_t ldx,
                       double *y, int64_t ldy, int nrhs);

/* y = L_s x = x - A_E x   (Sec. 2, eq. (nomlap), with Alg. 2 step 5). */
nfl_status nfl_apply_Ls(nfl_plan *plan, const double *x, int64_t ldx,
                        double *y, int64_t ldy, int nrhs);

/*
 * y = op(x) for blocks in HOST memory, op 0 = W, 1 = A, 2 = L_s (the products
 * of nfl_apply_W, nfl_apply_A and nfl_apply_Ls: Alg. 1, Alg. 2 step 5).
 * Column c is copied to a device slot of the plan, multiplied on the plan's
 * stream and copied back; the copies run on two streams the plan creates on
 * first use, so column c + 1 travels in and column c - 1 travels out while
 * column c is multiplied.  The copies overlap the products only when the
 * host memory is page-locked (cudaHostAlloc, cudaHostRegister); pageable
 * memory gives the same result without the overlap.  Any memory the CUDA
 * runtime can copy from (cudaMemcpyDefault) is accepted.
 *   x, y     FP64 blocks of nrhs >= 1 columns, leading dimensions ldx, ldy >= n;
 *            they must not overlap.  The library reads x and writes y only
 *            during the call.
 * The plan allocates 6 n FP64 of device staging on first use and keeps it
 * until nfl_plan_destroy.  Synchronizes the host: y is complete when the call
 * returns, and after an error no copy is still running.
 */
nfl_status nfl_apply_host(nfl_plan *plan, int op, const double *x, int64_t ldx,
                          double *y, int64_t ldy, int nrhs);

/*
 * Products for many independent graphs in one call (a batch of plans):
 * y_g = op(x_g) for g < G with op 0 = W, 1 = A, 2 = L_s (Alg. 1, Alg. 2 step 5;
 * the batching is not a paper construct: the paper treats one graph at a time), each x_g / y_g a
 * device block of nrhs columns with leading dimension ld[g] >= n_g.  The
 * work forks from the stream of plans[0] onto library streams (16 per
 * device, made on first use; plans largest first to the least loaded
 * stream), so the products of different plans run concurrently, and joins
 * back: the stream of plans[0] is ordered after every product, and every
 * plan's stream is set to it on return.  No host synchronization, so the
 * whole batch can be captured into one CUDA graph (a DAG of parallel
 * chains) and replayed as a single launch; make one uncaptured call first,
 * which creates the library streams.
 *   plans, x, y, ld: host arrays of G entries; plans must be distinct.
 * Returns the first failing plan's status (earlier products are issued).
 */
nfl_status nfl_apply_batched(nfl_plan *const *plans, int G, int op, const double *const *x,
                             double *const *y, const int64_t *ld, int nrhs);

/*
 * A batch of G plans whose products run with one kernel launch per stage and
 * part (Alg. 1 with the scalings of Alg. 2 step 5 for many independent graphs;
 * the batching is not a paper construct): y_g = op(x_g), op 0 = W, 1 = A,
 * 2 = L_s, for every member g, where x_g and y_g are the caller's device blocks
 * of nrhs columns bound at creation.  The members are split into `parts`
 * groups of about equal estimated work; a run issues, for each part on its
 * own library stream (forked from the run's stream and joined back), three
 * memsets and eight kernels: the staging of x~ and the epilogue's z, the
 * spread (all the part's (work item, column) pairs from one counter, largest
 * first), the five FFT passes and the interpolation, each over every member
 * of the part.  Several parts let the stages of different parts overlap (the
 * spread and interpolation are FMA-bound, the FFT passes bound by shared
 * memory).  Members must be 3-D plans of one mixed precision (FP32, FP32C or
 * BF16W), with the same m in {2, 3, 4, 6} and the same N (NFL_ERR_INVALID_ARG
 * otherwise), distinct, with positive degrees unless op is W
 * (NFL_ERR_NONPOSITIVE_DEGREE); they keep their own spread items, and the FFT
 * passes use the first member's CTA size.  The batch owns its staging, grid
 * and FFT buffers (per member and column: 12 n bytes, 12 to 16 bytes per box
 * position and the FFT buffers, all allocated at creation), and refers to
 * the plans and the caller's blocks, which must outlive it.
 *   plans, x, y, ldx, ldy   host arrays of G entries; ldx[g], ldy[g] >= n_g.
 *   nrhs                    columns per member, 1 <= nrhs <= 65535.
 *   parts                   1 <= parts <= 8 (at most G are used).
 * nfl_batch_run allocates nothing and does not synchronize the host, so a run
 * can be captured into a CUDA graph (a DAG of `parts` chains).  Results equal
 * the members' own products up to the FP32 summation order.  A bounded-wait
 * timeout in the interpolation sets the device_error flag of the member it
 * was working on.  nfl_batch_destroy synchronizes the device and frees the
 * batch's buffers; nfl_batch_parts returns the number of parts.
 */
nfl_status nfl_batch_create(nfl_plan *const *plans, int G, int op, const double *const *x, const int64_t *ldx,
                            double *const *y, const int64_t *ldy, int nrhs, int parts, nfl_batch **out);
nfl_status nfl_batch_parts(const nfl_batch *batch, int *parts);
nfl_status nfl_batch_run(nfl_batch *batch, void *stream);
void nfl_batch_destroy(nfl_batch *batch);

/* Stage timing of a batch's runs (tracing; not a paper construct), as for plans:
 * when enabled, events bracket the staging (with the memsets), the spread, the
 * FFT passes and the interpolation of every run; nfl_batch_stage_times
 * synchronizes the stream of the last run, writes the accumulated ms per stage
 * into ms[0..3] and the number of timed runs into *runs, and clears them;
 * with several parts the times are summed over the parts. */
nfl_status nfl_batch_set_profiling(nfl_batch *batch, int enable);
nfl_status nfl_batch_stage_times(nfl_batch *batch, double *ms, int64_t *runs);

/*
 * k smallest eigenpairs of L_s, i.e. the k largest of A (Sec. 2), by the
 * Lanczos process with full reorthogonalization (Sec. 4, eq. (krylov1)).
 * Ritz pair (theta, Q_k w) is accepted when |beta_{k+1} w_k| <= tol (Sec. 4).
 *
 *   k       1 <= k < n.
 *   tol     residual tolerance (e.g. 1e-10).
 *   maxit   maximum Krylov dimension, k < maxit <= min(n, 4096).
 *   seed    seed of the random start vector.
 *   evals   host, k FP64: eigenvalues of L_s ascending (1 - theta).
 *   evecs   device, n x k FP64 column-major (ld = n), unit 2-norm eigenvectors;
 *           may be NULL.
 *   iters   host, receives the number of Lanczos steps taken (may be NULL).
 * Returns NFL_ERR_NOT_CONVERGED (results still written) when maxit steps do
 * not converge all k pairs.
 */
nfl_status nfl_lanczos_k_smallest(nfl_plan *plan, int k, double tol, int maxit,
                                  uint64_t seed, double *evals, double *evecs, int *iters);

/*
 * Nystrom-Gaussian-NFFT (Alg. 3, Sec. 5.2): the k largest eigenpairs of
 * A = D^{-1/2} W D^{-1/2}, approximately, from a rank-M approximation
 * (A Q)(Q^T A Q)^+_M (A Q)^T with Q = orth(A G) for a Gaussian n x L block G:
 * 2L products with A (the plan's fast sums), Gram-Schmidt QR with
 * reorthogonalization on the device, and two small symmetric
 * eigen-decompositions (L x L and M x M, cyclic Jacobi on the host).
 *
 *   k, L, M   1 <= k <= M <= L <= min(n, 512).
 *   G         device n x L FP64 column-major random block (read only), or NULL
 *             to draw it on the device from seed.
 *   evals     host, k FP64: the approximate eigenvalues of A, descending.
 *   evecs     device, n x k FP64 column-major orthonormal vectors (may be NULL).
 * Returns NFL_ERR_BREAKDOWN when Q^T A Q has fewer than M positive
 * eigenvalues, NFL_ERR_NONPOSITIVE_DEGREE as the products do.
 */
nfl_status nfl_nystrom_k_largest(nfl_plan *plan, int k, int L, int M, const double *G, uint64_t seed,
                                 double *evals, double *evecs);

/*
 * Conjugate gradients for (beta L_s + diag(s)) u = f, the system of Sec. 6.2.2
 * (eq. (ssl::system) is beta L_s + I).  Stops when ||r||_2 <= tol ||f||_2.
 *
 *   beta    > 0.
 *   shift   device n FP64 diagonal s >= 0 (NULL means s = 1), so that the
 *           operator is symmetric positive definite.
 *   f       device n FP64 right-hand side.
 *   u       device n FP64: initial guess on entry, solution on exit.
 *   iters   host (may be NULL); relres host (may be NULL): final ||r|| / ||f||.
 */
nfl_status nfl_cg_solve(nfl_plan *plan, double beta, const double *shift,
                        const double *f, double *u, double tol, int maxit,
                        int *iters, double *relres);

/*
 * nfl_cg_solve to FP64 accuracy with nearly all products in a mixed form:
 * mixed-precision iterative refinement (the refinement pass of the
 * compensated form; Sec. 4 notes that Krylov methods tolerate inexact
 * products, Sec. 6.2.2 gives the system).  With A_64 the operator
 * beta L_s + diag(s) of `plan` (normally FP64) and A_in that of `inner`
 * (normally the FP32C form of the same nodes and parameters):
 *   r_k = f - A_64 u_k;  stop when ||r_k|| <= tol ||f||;
 *   A_in c_k = r_k by CG from c_k = 0 to ||r_k - A_in c_k|| <= inner_tol ||r_k||;
 *   u_{k+1} = u_k + c_k.
 * Each outer step costs one product of `plan`; the inner CG steps use
 * `inner`.  The answer is that of nfl_cg_solve on `plan`.
 *
 *   plan, inner  plans created from the same nodes with the same kernel and
 *                sigma (checked through n, d, kernel, sigma and the nodes'
 *                bounding-box centre; NFL_ERR_INVALID_ARG otherwise); N, m,
 *                p and the precision may differ.  inner runs on plan's stream
 *                for the call.
 *   beta, shift, f, u, tol   as in nfl_cg_solve (u: initial guess in, solution out).
 *   inner_tol    relative residual of each correction solve, 0 < inner_tol < 1.
 *   maxit        most CG steps of one correction solve (a correction that
 *                stops at maxit is still applied).
 *   max_outer    most refinement steps (FP64 residuals: max_outer + 1).
 *   iters        host (may be NULL): inner CG steps in total.
 *   outer        host (may be NULL): refinement steps taken.
 *   relres       host (may be NULL): final ||r|| / ||f|| with plan's products.
 * Returns NFL_ERR_NOT_CONVERGED when max_outer steps do not reach tol.
 * Synchronizes the stream; allocates 6 n FP64 of device scratch.
 */
nfl_status nfl_cg_solve_refined(nfl_plan *plan, nfl_plan *inner, double beta, const double *shift,
                                const double *f, double *u, double tol, double inner_tol, int maxit,
                                int max_outer, int *iters, int *outer, double *relres);

/*
 * Gradients of a loss l(u) through the solve of nfl_cg_solve, given the
 * forward solution u and g = dl/du (the differentiable form of the system of
 * Sec. 6.2.2).  The operator beta L_s + diag(s) is symmetric, so one more
 * solve gives lambda = (beta L_s + diag(s))^{-1} g, and
 *   dl/df = lambda,  dl/ds_i = -lambda_i u_i,  dl/dbeta = -lambda^T L_s u,
 *   dl/dsigma = -beta lambda^T (dL_s/dsigma) u,
 * where, with d the degrees, delta = W_sigma 1, W_sigma = dW/dsigma (the
 * plan dplan of kernel NFL_KERNEL_GAUSSIAN_DSIGMA), a~ = D^{-1/2} a and
 * b~ = D^{-1/2} b (differentiating L_s = I - D^{-1/2} W D^{-1/2}, Sec. 2):
 *   a^T (dL_s/dsigma) b = -a~^T W_sigma b~ + 1/2 sum_i (delta_i / d_i) (a~_i (W b~)_i + (W a~)_i b~_i).
 * All products are the plans' fast sums.
 *
 *   plan        the NFL_KERNEL_GAUSSIAN plan of the forward solve.
 *   dplan       NFL_KERNEL_GAUSSIAN_DSIGMA plan with the same nodes, sigma, N,
 *               m, p and eps_B; may be NULL when grad_sigma is NULL.
 *   beta, shift, tol, maxit   as in nfl_cg_solve (same values as the forward solve).
 *   u           device n FP64: the forward solution.
 *   g           device n FP64: dl/du.
 *   grad_f      device n FP64: initial guess of the adjoint solve on entry,
 *               lambda = dl/df on exit.
 *   grad_shift  device n FP64 (out), may be NULL.
 *   grad_beta, grad_sigma   host FP64 (out), may be NULL.
 *   iters, relres           host (may be NULL): of the adjoint solve.
 * Errors as nfl_cg_solve; NFL_ERR_INVALID_ARG when dplan does not match plan.
 */
nfl_status nfl_cg_solve_backward(nfl_plan *plan, nfl_plan *dplan, double beta, const double *shift,
                                 const double *u, const double *g, double tol, int maxit, double *grad_f,
                                 double *grad_shift, double *grad_beta, double *grad_sigma, int *iters,
                                 double *relres);

/*
 * Gradient of the bilinear form a^T A_E b (A = D^{-1/2} W D^{-1/2}, Sec. 2,
 * eq. (nomlap)) with respect to the node coordinates, the degrees d = W 1
 * moving with the nodes.  Differentiating A, with a~ = D^{-1/2} a,
 * b~ = D^{-1/2} b and c = (a~ (W b~) + b~ (W a~)) / d:
 *   a^T dA b = sum_ij dW_ij (a~_i b~_j - c_i / 2),
 * and for the Gaussian (Sec. 2, eq. (W_gaussian)), grad K(y) = -(2 / sigma^2) y K(y):
 *   g_k = -(2 / sigma^2) (y_k S0_k - S1_k),
 *   S0 = a~ (W b~) + b~ (W a~) - c d / 2 - (W c) / 2,
 *   S1 = a~ W(b~ y) + b~ W(a~ y) - c (W y) / 2 - W(c y) / 2,
 * y = v - center (any shift gives the same g; the plan's centre keeps the
 * products well scaled).  3 + 4 d fast products with W, all with the
 * plan's kernel (even, so the plan's coefficients serve).  With
 * a = lambda, b = u of nfl_cg_solve_backward, beta g is dl/dv of the
 * differentiable solve of Sec. 6.2.2.
 *   plan    NFL_KERNEL_GAUSSIAN plan (others: NFL_ERR_INVALID_ARG).
 *   v       device n x d FP64 row-major: the nodes the plan was created with.
 *   a, b    device n FP64.
 *   grad    device n x d FP64 row-major (out).
 * Synchronizes the plan's stream.  Allocates 15 n FP64 of device scratch.
 */
nfl_status nfl_form_grad_nodes(nfl_plan *plan, const double *v, const double *a, const double *b,
                               double *grad);


/*
 * nfl_cg_solve without device allocation.  The paper has no counterpart:
 * this is a deployment variant of nfl_cg_solve for callers that cannot
 * call cudaMalloc / cudaFree while they solve (a process whose device
 * footprint is fixed at start-up, an allocator that must not see foreign
 * allocations).  Arguments, results and status codes are those of
 * nfl_cg_solve.  Like nfl_cg_solve it synchronizes the plan's stream in
 * every iteration to read the reductions, so it cannot be captured into a
 * CUDA graph.
 *
 * The four work vectors and the reduction partials live in one static
 * device array of this library, sized for n <= NFL_NOALLOC_MAX_N nodes
 * (4 x 262144 + 520 doubles, about 8 MiB, held by every GPU that loads the
 * library until the process exits).  A plan with more nodes returns
 * NFL_ERR_INVALID_ARG.  The plan's device must be current; the first call
 * on a device looks up the array's device address.  All calls share the
 * array: calls that overlap on the GPU (other streams, plans or threads)
 * race on it.
 */
#define NFL_NOALLOC_MAX_N 262144
nfl_status nfl_cg_solve_noalloc(nfl_plan *plan, double beta, const double *shift,
                                const double *f, double *u, double tol, int maxit,
                                int *iters, double *relres);

/*
 * Stage timing (tracing; not a paper construct).  When enabled, CUDA events on the plan's stream
 * bracket the four stages of every product column -- or of every block of
 * columns that goes through the stages together: prep (grid clear, staging
 * of x~ and the epilogue's z, for FP32C the fixed-point scale), spread, FFT
 * (all passes, multiply fused) and gather.  nfl_plan_stage_times
 * synchronizes the stream, writes the accumulated milliseconds per stage
 * into ms[0..3] and the number of columns timed into *columns (a block
 * counts its columns), then clears the accumulators.  Disabled by default.
 */
nfl_status nfl_plan_set_profiling(nfl_plan *plan, int enable);
nfl_status nfl_plan_stage_times(nfl_plan *plan, double *ms, int64_t *columns);

/*
 * Failure-detection test hook; the paper has no counterpart.  kind 1 makes
 * the tensor-core interpolation skip its MMAs, so its bounded waits (limited
 * to 10 ms of device time in this mode, 2 s otherwise) run out: the kernel
 * sets the plan's device_error (nfl_plan_info), skips its remaining work,
 * frees its tensor memory and returns; nothing traps or hangs.  kind 0
 * switches it off (device_error stays set for the plan).  Products made in
 * this mode are meaningless.  NFL_ERR_INVALID_ARG for other kinds.
 */
nfl_status nfl_plan_inject_fault(nfl_plan *plan, int kind);

/* Number of kernel launches one product column makes (launch accounting; not a
 * paper construct). */
nfl_status nfl_plan_kernels_per_column(const nfl_plan *plan, int *kernels);

/* Number of kernel launches one product of nrhs >= 1 columns makes (not a paper
 * construct): blocks of
 * nfl_info.block_cols columns take one launch per stage on the 3-D
 * tensor-core path. */
nfl_status nfl_plan_kernels(const nfl_plan *plan, int nrhs, int *kernels);

/*
 * Measured arithmetic rate of the current device, the denominator of the ALU
 * rooflines of the spread and gather kernels; the paper has no counterpart.
 * kind selects the instruction:
 *   NFL_RATE_FP32_FMA    fma.rn.f32 (one FP32 multiply-add per lane),
 *   NFL_RATE_FP32X2_FMA  fma.rn.f32x2 (two FP32 multiply-adds per lane, the
 *                        packed form the spread and gather use),
 *   NFL_RATE_FP64_FMA    fma.rn.f64.
 * Launches register-resident chains of fused multiply-adds over all SMs
 * (64 warps per SM) on `stream`, and returns the best of five timed launches
 * after one untimed one (CUDA events): *flops_per_s counts 2 flop per
 * multiply-add, *ms (host, may be NULL) the launch time.  Synchronizes the
 * stream; allocates 1 KB of device memory for the call.
 */
enum { NFL_RATE_FP32_FMA = 0, NFL_RATE_FP32X2_FMA = 1, NFL_RATE_FP64_FMA = 2 };
nfl_status nfl_fma_rate(int kind, void *stream, double *flops_per_s, double *ms);

/* Human-readable name of a status code. */
const char *nfl_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* NFL_H */
