/*
 * feast_gb300.h -- C ABI of the GB300 (sm_103a) non-Hermitian FEAST library.
 *
 * The library finds the eigenpairs (lambda, x) of A x = lambda B x whose
 * eigenvalues lie inside an elliptical domain C (the problem of Sec. 2 of
 * Tang, Kestyn & Polizzi, "A New Highly Parallel Non-Hermitian Eigensolver"),
 * by subspace iteration (Algorithm R-FEAST) or Bauer bi-iteration (Algorithm
 * Bi-FEAST) accelerated by the quadrature filter of Sec. 3:
 *
 *   rho(M) U = sum_k sigma_k (phi_k B - A)^{-1} (B U)                (Eq. Rasp)
 *   left:      sum_k conj(sigma_k) (phi_k B - A)^{-H} (B^H V)         (Eq. quadf_surMconj)
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex numbers are interleaved complex128 (feast_z).  Matrices are
 *   column-major with a leading dimension; n x m blocks passed to or returned
 *   from the library have leading dimension n.
 * - Any matrix/vector pointer may be HOST memory (pageable or pinned) or
 *   DEVICE memory of the current CUDA device (unified addressing: the library
 *   copies every input into its own device buffers and every output back with
 *   cudaMemcpyDefault).  Caller memory is never retained after a call returns.
 * - All GPU work is enqueued on the stream given to feast_create (NULL = the
 *   legacy default stream) and on the handle's own streams, which are joined
 *   to it before anything reads their results.  A call returns after its work
 *   is complete (results in host buffers are valid; device outputs are
 *   complete on that stream); the ||A||_2 estimate started by feast_create
 *   may still run until the first call that needs it (feast_rayleigh_ritz,
 *   feast_solve, feast_get_stats) waits for it.
 * - Errors are returned as feast_status; nothing aborts or traps.  After a
 *   FEAST_ERR_CUDA status the handle should be destroyed.
 * - Not thread-safe per handle; distinct handles are independent.
 */
#ifndef FEAST_GB300_H
#define FEAST_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double re, im; } feast_z;

typedef enum {
  FEAST_OK = 0,
  FEAST_ERR_ARG = 1,            /* invalid size, pointer or option                      */
  FEAST_ERR_ALLOC = 2,          /* device allocation failed                             */
  FEAST_ERR_SINGULAR_SHIFT = 3, /* a shifted matrix phi_k B - A had an exact zero pivot */
  FEAST_ERR_REFINE_NOCONV = 4,  /* per-shift refinement (max_refine > 0) stalled above
                                   refine_tol even after the FP64 refactorisation      */
  FEAST_ERR_M0_TOO_SMALL = 5,   /* every Ritz value of the subspace lies inside C: m0 is
                                   at most the count, so some eigenvalues may be missed;
                                   the outputs of the last iteration are returned      */
  FEAST_ERR_NOCONV = 6,         /* max_iter reached; results are still returned         */
  FEAST_ERR_NONFINITE = 7,      /* NaN or Inf appeared in the input or the iteration    */
  FEAST_ERR_DEVICE_TIMEOUT = 8, /* a bounded device-side wait gave up                   */
  FEAST_ERR_CUDA = 9,           /* a CUDA runtime call failed                           */
  FEAST_ERR_STATE = 10,         /* call out of order (e.g. no factorisation yet)        */
  FEAST_ERR_TOO_LARGE = 11      /* size beyond the fixed scratch of an allocation-free entry point */
} feast_status;

/* Quadrature rules of Sec. 3 (Eq. quadrature_for_pi) and the meaning of N_e:
 *   TRAP_MID : q = N_e nodes at angles 2 pi (j + 1/2) / N_e (composite midpoint
 *              rule; on a circle rho(mu) = 1 / (1 + ((mu - c)/R)^N_e)).
 *   TRAP_END : the paper's trapezoid with t_1 = -1, t_K = 1, K = N_e, q = 2(K-1).
 *   GAUSS    : Gauss-Legendre with K = N_e nodes per half, q = 2K.
 *   CUSTOM   : q = q_custom caller-supplied nodes and weights (host memory),
 *              e.g. piecewise contours glued from several curves (Sec. 5.4). */
typedef enum {
  FEAST_RULE_TRAP_MID = 0,
  FEAST_RULE_TRAP_END = 1,
  FEAST_RULE_GAUSS = 2,
  FEAST_RULE_CUSTOM = 3
} feast_rule;

/* The ellipse of Eq. ellipses: centre c, semi-axes R (real direction) and
 * R * aspect (imaginary direction).  The domain test for candidates uses this
 * ellipse.  With CUSTOM nodes and R = 0 (no ellipse: a piecewise contour of
 * Sec. 5.4, see feast_piecewise_nodes) a value lambda counts as inside when
 * the filter of the nodes gives |rho(lambda)| = |sum_k sigma_k / (phi_k -
 * lambda)| >= 1/2: rho approximates the indicator of the enclosed domain. */
typedef struct {
  feast_z center;
  double R;
  double aspect;
  int rule;               /* feast_rule */
  int N_e;
  const feast_z* nodes;   /* CUSTOM only (host) */
  const feast_z* weights; /* CUSTOM only (host) */
  int q_custom;           /* CUSTOM only */
} feast_contour;

typedef enum { FEAST_ALGO_R = 0, FEAST_ALGO_BI = 1 } feast_algo;

/* FP64: every shifted system factored and solved in complex128 (DMMA tensor path).
 * MIXED: factors in complex64 with the trailing updates on the tensor cores,
 *        solves in low precision, and the FP64 accuracy recovered by
 *        iterative refinement: the correction solve takes the FP64 residual
 *        of the initial iterate X_k0 = U (phi_k - Theta)^{-1}, which every
 *        shift shares (R_k = (A U - B U Theta)(phi_k - Theta)^{-1}). */
typedef enum { FEAST_PREC_FP64 = 0, FEAST_PREC_MIXED = 1 } feast_precision;

typedef struct {
  int algo;          /* feast_algo                                             */
  int precision;     /* feast_precision                                        */
  double tol;        /* stop when every candidate has
                        ||A x - lam B x|| / (||A||_2 ||x||) <= tol (default 1e-10) */
  int max_iter;      /* default 20                                             */
  double cand_tol;   /* candidate test ||A u - lam B u|| / ||u|| <= cand_tol
                        (Sec. 5, default 1e-4)                                 */
  int panel;         /* LU panel width (0 = library default)                   */
  int timing;        /* nonzero: record per-phase CUDA-event times in stats    */
  int symmetric;     /* nonzero: A = A^T and B = B^T (complex symmetric pencil).
                        Then (phi B - A)^{-H} conj(V) = conj((phi B - A)^{-1} V),
                        so Bi-FEAST takes the left block as conj(right block):
                        no left solves, Qhat = conj(Q), Vk = conj(Uk).        */
  int max_refine;    /* MIXED only: 0 (default) = the residual form above; k > 0 =
                        classical per-shift refinement as well, up to k sweeps
                        X_k += S_k^{-1} (R - S_k X_k) with the residual in FP64,
                        until every column has ||r|| <= refine_tol ||R||; a shift
                        that stalls is refactored in FP64 and solved again.    */
  double refine_tol; /* tau of the refinement (default 1e-12)                 */
  int shift_begin;   /* this handle factors and filters the nodes           */
  int shift_end;     /* [shift_begin, shift_end) only (0, 0 = all): the
                        shift-partitioned filter, where each process owns a
                        range of the linear systems (Sec. 6) and the partial
                        sums are added by the caller                           */
  int real_pencil;   /* nonzero: A and B are real and the nodes come in
                        conjugate pairs (any rule on a contour symmetric about
                        the real axis): only the nodes with Im >= 0 are
                        factored, since (conj(phi) B - A) = conj(phi B - A)   */
  const char* tune_cache; /* JSON file of tuned launch parameters written by
                        paper_1404_2891_gb300.autotune (NULL = built-in)       */
  int lu_outer;      /* MIXED: outer block of the two-level LU in columns (a
                        multiple of 64, at most 256); 0 = library default (256
                        for n >= 1024), -1 = one-level LU (every trailing
                        update with K = 64)                                    */
  int panel_cluster; /* MIXED: 0 (default) = panels of 1024 to 8192 rows run
                        on a thread-block cluster of four CTAs per system;
                        k > 0 = from k rows on (k >= 256); -1 = one CTA per
                        system                                                 */
  int deep_solves;   /* MIXED, two-level LU: 0 (default) = the filter's solves
                        in diagonal blocks of lu_outer rows (the stored D^{-1}
                        of each block, K = lu_outer updates); -1 = 64-row
                        blocks                                                 */
  int batch_tc_min;  /* batched path: shifted matrices of pencils of order
                        >= batch_tc_min (at least 512) are padded to a multiple
                        of 256 and factored by the tensor-core LU in classes of
                        equal padded order (two-level from 1024 on), the rest
                        by the persistent launch; 0 (default) = the tuned
                        value of options.tune_cache, else 768; -1 = every
                        matrix in the persistent launch                        */
  int batch_direct;  /* batched path: nonzero = launch the classes'
                        factorisations kernel by kernel instead of replaying
                        the CUDA graph captured at their first use (for tools
                        that cannot follow stream capture)                     */
} feast_options;

typedef struct {
  int iters;
  int m_found;
  double max_res;        /* max normalised residual over candidates, last iteration */
  double normA;          /* ||A||_2 estimate used for normalisation                */
  double t_factor_ms;    /* times are filled only when options.timing != 0          */
  double t_filter_ms;
  double t_rr_ms;
  double t_total_ms;
  double t_update_ms;    /* summed duration of the LU trailing-update launches
                            with K = 64 (panel width)                             */
  int update_launches;   /* number of those launches in the last factorisation     */
  int res_hist_len;
  double res_hist[64];   /* max candidate residual per iteration (inf if none)      */
  int count_hist[64];    /* candidate count per iteration                          */
  int q;                 /* linear systems of this handle                          */
  int shift_info[256];   /* per system: 0, or 1 + the first column whose pivot was
                            exactly zero (FEAST_ERR_SINGULAR_SHIFT); 2^30 + sweeps
                            for a shift whose refinement stalled                   */
  int refine_sweeps;     /* classical refinement sweeps of the last filter          */
  int refactored;        /* shifts refactored in FP64 by the last filter            */
  int lu_outer;          /* outer block of the last factorisation (0 = one-level)   */
  double t_deep_ms;      /* summed duration of its deep (K = lu_outer) updates      */
  int deep_launches;     /* number of those launches                              */
  double deep_flops;     /* their algorithmic flops (8 per complex MAC), all shifts */
  double deep_bytes;     /* their algorithmic HBM bytes (C read + written, L, U)    */
  double update_flops;   /* algorithmic flops of the K = 64 update launches         */
  double update_bytes;   /* and their algorithmic HBM bytes                         */
  int tuned;             /* 1 if lu_outer / panel_cluster came from options.tune_cache */
  double t_rr_phase_ms[8]; /* the last Rayleigh-Ritz step by phase, on the main stream
                            (timing): orthonormal basis of Q; A Q and B Q (and the
                            wait for Qhat's basis); the projections Qhat^H A Q,
                            Qhat^H B Q; Bhat^{-1} and C; Schur form, eigenvectors
                            and W^{-1}; FP64 refinement sweeps; right Ritz vectors
                            and residuals; left ones                               */
} feast_stats;

typedef struct feast_handle feast_handle;

/* Default options: BI, MIXED, tol 1e-10, max_iter 20, cand_tol 1e-4. */
void feast_default_options(feast_options* o);

/* Create a handle for the pencil (A, B) of order n with subspace size m0.
 *   A    : n x n, leading dimension lda >= n, host or device; copied.
 *   B    : n x n (ldb >= n) or NULL for the standard problem B = I.
 *   c    : contour and quadrature rule (Sec. 3); nodes and weights are computed
 *          on the host (Eq. ellipses, Eq. pi, Eq. quadrature_for_pi).
 *   m0   : subspace dimension p of Sec. 4, 1 <= m0 <= n and m0 <= 160.
 *   stream : a cudaStream_t, or NULL.
 * The handle owns the device copies of A and B, the q factorisations and all
 * workspace until feast_destroy.  Its device memory comes from a stream-ordered
 * pool of the library that keeps blocks returned by feast_destroy for later
 * handles (it holds the largest set of handles alive at once until the process
 * exits).  Returns FEAST_ERR_ARG for n < 1, m0 > n, N_e < 1 or a NULL A;
 * FEAST_ERR_ALLOC if device memory runs out. */
feast_status feast_create(feast_handle** h, int64_t n, const feast_z* A, int64_t lda,
                          const feast_z* B, int64_t ldb, const feast_contour* c, int m0,
                          const feast_options* o, void* stream);

void feast_destroy(feast_handle* h);

const char* feast_status_str(feast_status s);

/* Number of linear systems q and their nodes phi_k / weights sigma_k (host
 * arrays of q entries each, either may be NULL). */
feast_status feast_get_quadrature(const feast_handle* h, int* q, feast_z* nodes, feast_z* weights);

/* Form every shifted matrix phi_k B - A and factor it once (Sec. 5.5: one
 * factorisation per linear system for the whole iteration): P_k S_k = L_k U_k
 * by blocked Gaussian elimination with partial pivoting (largest |Re|+|Im|,
 * lowest row on ties).  FEAST_ERR_SINGULAR_SHIFT if some exact pivot is zero
 * (the factor is still stored).  Called implicitly by filter/solve when no
 * factorisation exists yet; an explicit call always forms and factors again. */
feast_status feast_factor(feast_handle* h);

/* Copy out the factorisation of shift k (0 <= k < q) for inspection:
 * LU (n x n complex128, packed unit-L and U, ld n) and piv (n int32, LAPACK
 * style: row i was exchanged with piv[i], 0-based).  Either may be NULL. */
feast_status feast_get_factor(feast_handle* h, int k, feast_z* LU, int32_t* piv);

/* Solve one shifted system with the stored factor: side 0 solves
 * (phi_k B - A) X = R, side 1 solves (phi_k B - A)^H X = R (Eq. Rasp,
 * Eq. Lasp).  R and X are n x nrhs (ld n), nrhs <= m0.  In MIXED precision
 * this is the low-precision solve alone (no refinement). */
feast_status feast_solve_shift(feast_handle* h, int k, int side, const feast_z* R, feast_z* X,
                               int nrhs);

/* The filter (Eq. Rasp and Eq. Lasp):
 *   Q    = sum_k sigma_k (phi_k B - A)^{-1} B Y
 *   Qhat = sum_k conj(sigma_k) (phi_k B - A)^{-H} B^H Yhat   (if Yhat != NULL)
 * Y, Yhat, Q, Qhat are n x m0.  theta (m0 complex, may be NULL) supplies Ritz
 * values for the MIXED refinement's initial iterate; the mathematical result
 * does not depend on it.  Sums over k run in a fixed order (deterministic). */
feast_status feast_filter(feast_handle* h, const feast_z* Y, const feast_z* Yhat,
                          const feast_z* theta, feast_z* Q, feast_z* Qhat);

/* The shift-partitioned filter (Sec. 6: the linear systems are independent,
 * one process may own each).  The q terms of the filter are summed along a
 * fixed tree: the nodes are split into eight leaves [b_g, b_{g+1}),
 * b_g = floor(g q / 8), each leaf summed in order of k, and the leaves
 * added pairwise, ((0+1)+(2+3))+((4+5)+(6+7)), before the residual form's
 * rho(theta) Y term.  A handle created with options.shift_begin/shift_end
 * equal to an aligned run of 1, 2, 4 or 8 leaves ([b_{jL}, b_{(j+1)L}))
 * factors only those systems, and its feast_filter returns the subtree sum of
 * its leaves (no rho(theta) Y term), also when the range is every node (a
 * partition of one process); other ranges are FEAST_ERR_ARG, and feast_solve
 * on such a handle is FEAST_ERR_STATE.
 * feast_filter_combine adds nparts (1, 2, 4 or 8) such partial blocks, given
 * in the order of their ranges, along the top of the same tree and adds the
 * rho(theta) Y term for the Ritz values theta (MIXED; NULL = plain form), so
 * the result has the same bits as feast_filter on one handle that owns every
 * node.  parts[j] (and parts_hat[j] for the left filter, or NULL) are n x m0,
 * host or device; Y/Yhat are the filter's inputs (needed with theta). */
feast_status feast_filter_combine(feast_handle* h, int nparts, const feast_z* const* parts,
                                  const feast_z* const* parts_hat, const feast_z* Y, const feast_z* Yhat,
                                  const feast_z* theta, feast_z* Q, feast_z* Qhat);

/* Stochastic moments of the filter for counting eigenvalues (the count
 * estimation of Sec. 6, in its plain stochastic-trace form):
 *   mu_k = (1/S) sum_s v_s^H [ sum_j sigma_j t_j^k (phi_j B - A)^{-1} B ] v_s,
 *   t_j = (phi_j - c) / R,  k = 0 .. kmax (kmax <= 31),
 * with the stored factorisations.  mu_0 estimates tr rho(M) = sum_i rho(lambda_i),
 * close to the number of eigenvalues inside C.  V: n x S probe block (entries
 * +-1 for the usual estimator), 1 <= S <= m0; mu: kmax + 1 complex values. */
feast_status feast_moments(feast_handle* h, const feast_z* V, int S, int kmax, feast_z* mu);

/* Rayleigh-Ritz (R-FEAST steps 4-5 / Bi-FEAST steps 6-7) on the filtered blocks.
 * Q (and Qhat for Bi-FEAST; NULL selects R-FEAST's one-sided projection) are
 * replaced in FP64 by orthonormal bases of their spans, the reduced pencil
 * (A^, B^) = (V^H A U, V^H B U) is solved for Lambda^, W, Z with
 * Z^H B^ W = I, and the Ritz vectors X = U W (unit 2-norm columns) and
 * Xl = V Z (scaled so Xl^H B X = I) are returned with their eigenvalues
 * lambda (m0) and residuals res[i] = ||A x_i - lambda_i B x_i|| / ||A||_2
 * (m0 doubles).  m_inside counts pairs that are candidates (inside C and
 * ||A x - lambda B x|| <= cand_tol).  Xl, res, m_inside may be NULL. */
feast_status feast_rayleigh_ritz(feast_handle* h, const feast_z* Q, const feast_z* Qhat,
                                 feast_z* lambda, feast_z* X, feast_z* Xl, double* res,
                                 int* m_inside);

/* The candidates of the last Rayleigh-Ritz step (Sec. 5: inside C and
 * ||A x - lambda B x|| <= cand_tol): count, their column indices sorted by
 * (Re lambda, Im lambda) (idx: m0 slots, may be NULL) and the largest
 * normalised residual among them (inf if none; may be NULL).
 * FEAST_ERR_STATE before any Rayleigh-Ritz step. */
feast_status feast_candidates(const feast_handle* h, int* count, int* idx, double* max_res);

/* The whole iteration (Algorithm R-FEAST or Bi-FEAST, with the Sec. 5
 * candidate monitoring).  Y0 (n x m0) is the random starting block; Vrand
 * (n x m0, Bi-FEAST only, may be NULL = Y0) builds V0 = Vrand (Vrand^H B Y0)^{-H}
 * so that V0^H B Y0 = I.  On return the first m_found entries of lambda
 * (m0 slots), columns of X and Xl (n x m0 each; Xl may be NULL) and res are
 * the converged candidates sorted by (Re lambda, Im lambda).  Returns
 * FEAST_ERR_NOCONV if max_iter iterations did not converge (outputs valid).
 * stats may be NULL. */
feast_status feast_solve(feast_handle* h, const feast_z* Y0, const feast_z* Vrand,
                         feast_z* lambda, feast_z* X, feast_z* Xl, double* res, int* m_found,
                         feast_stats* stats);

/* Timings of the last factorisation and of the last feast_solve on this handle
 * (filled when options.timing != 0; normA always).  stats must not be NULL. */
feast_status feast_get_stats(const feast_handle* h, feast_stats* stats);

/* ---- Learned choice of the subspace size m0 --------------------------------
 * The paper leaves p (m0) to experience or to a count estimate (Sec. 6).  This
 * network predicts the eigenvalue count from the pencil's parameter and the
 * stochastic moments of feast_moments; m0 is then chosen from the prediction.
 * Architecture: d_in -> width -> width -> 1, GELU after the two hidden layers,
 * inputs standardised as (x - mean) / scale, BF16 weights in every product with
 * FP32 accumulation, FP32 master weights, Adam (beta1 0.9, beta2 0.999,
 * eps 1e-8), mean-squared-error loss.
 * Parameters are one FP32 vector in the order W1 (width x d_in, row-major),
 * b1 (width), W2 (width x width), b2, W3 (1 x width), b3 (1);
 * feast_mlp_param_count gives its length.  Feature, label and index arrays
 * given to predict/grad/train are row-major FP32 / int32 in DEVICE memory
 * (FEAST_ERR_ARG otherwise); params, mean, scale, outputs may be host or device. */
typedef struct feast_mlp feast_mlp;
size_t feast_mlp_param_count(int d_in, int width);
feast_status feast_mlp_create(feast_mlp** net, int d_in, int width, int max_batch, const float* params,
                              const float* mean, const float* scale, void* stream);
void feast_mlp_destroy(feast_mlp* net);
feast_status feast_mlp_get_params(feast_mlp* net, float* params);
/* y[b] = network(X[b, :]) for b < B (B <= max_batch). */
feast_status feast_mlp_predict(feast_mlp* net, const float* X, int B, float* y);
/* Loss (1/B) sum_b (net(X[b]) - y[b])^2 and its gradient w.r.t. every parameter. */
feast_status feast_mlp_grad(feast_mlp* net, const float* X, const float* y, int B, float* loss, float* grads);
/* `steps` Adam steps with learning rate lr; step s uses the B rows
 * batches[s*B .. s*B+B) of (X, y) (n_rows rows; indices are clamped). */
feast_status feast_mlp_train(feast_mlp* net, const float* X, const float* y, int n_rows, const int* batches,
                             int steps, int B, float lr, float* last_loss);

/* ||A||_2 estimate for callers that cannot allocate device memory (the paper
 * has no counterpart: it is the norm that scales the residual gate).
 * Some callers may not call cudaMalloc -- code running while a host framework
 * owns all device memory and hands out only its own buffers, or a phase whose
 * memory budget is fixed.  This entry point allocates nothing: it runs the same
 * power iteration as feast_create (iters steps on A^H A from the all-ones
 * vector, result sqrt of the last Rayleigh quotient) and keeps its scratch in a
 * fixed device array of 520.5 KiB that every GPU loading this library holds
 * until exit.
 *   A     : DEVICE pointer, n x n column-major, lda >= n (host memory is rejected
 *           with FEAST_ERR_ARG); not modified.
 *   n     : 1 <= n <= 16384; larger orders return FEAST_ERR_TOO_LARGE.
 *   iters : >= 1 (feast_create uses 50).
 *   norm  : receives the estimate (host or device pointer).
 *   stream: cudaStream_t or NULL; the call returns after the stream has drained.
 * The first call on each device looks up the fixed array's address with that
 * device current; make it before any stream capture.  All calls share the one
 * array, which keeps the last call's contents: calls that overlap on the GPU
 * race and must be serialised by the caller.  Calls no cudaMalloc, cudaFree
 * or allocating library routine. */
feast_status feast_norm2_estimate_static(const feast_z* A, int64_t n, int64_t lda, int iters,
                                         double* norm, void* stream);

/* ---- Batched path: many independent standard pencils (B = I) at once.
 * Sec. 6 notes that FEAST's systems are independent across quadrature nodes
 * and across search intervals; the batched path uses that independence
 * across pencils too.  Every pencil p has its own order n[p], subspace size
 * m0[p] and contour, and the pencils are iterated together with Algorithm
 * R-FEAST (Q^ = Q) in mixed precision.
 *
 * On the device, ONE persistent launch factors all sum_p q_p shifted matrices
 * z I - A_p with partial pivoting (complex64, padded to a multiple of 64) and
 * solves them for their pencil's right-hand sides.  A device task queue in an
 * order planned on the host drives it: critical path first, largest pencils
 * first.  Pencils of order >= opts.batch_tc_min (default 768) are instead
 * factored by the tensor-core LU of the single-pencil path, in classes of
 * equal padded order (a multiple of 256), each class on its own stream before
 * the persistent launch, which then only solves them.  The Rayleigh-Ritz
 * steps run as grouped kernels (one launch per step for all pencils), and the
 * steady iterations replay one CUDA graph.
 *
 *   n        : count orders, 1 <= n[p] <= 4096.
 *   A        : count pointers to n[p] x n[p] column-major matrices (host or
 *              device), leading dimensions lda[p] >= n[p] (lda NULL: lda = n);
 *              copied.
 *   contours : count contours (any rule; q_p <= 256 nodes).
 *   m0       : count subspace sizes, 1 <= m0[p] <= min(n[p], 160).
 *   opts     : algo must be FEAST_ALGO_R and precision FEAST_PREC_MIXED
 *              (FEAST_ERR_ARG otherwise); tol, max_iter, cand_tol and timing
 *              as for a handle.
 * The batch owns all device memory until feast_batch_destroy. */
typedef struct feast_batch feast_batch;

typedef struct {
  int iters;                /* lockstep iterations                                  */
  int converged;            /* pencils that met the Sec. 5 test                     */
  int tasks_factor;         /* tasks of the persistent factorisation launch         */
  int grid;                 /* CTAs of the persistent launch                        */
  int graph;                /* 1 if the steady iterations replayed a CUDA graph;
                               -e if capturing them failed with cudaError_t e and
                               they ran as ordinary launches                         */
  double plan_makespan_us;  /* makespan of the host schedule's cost model           */
  double t_factor_ms;       /* first launch (factorisations + first solves), timing */
  double t_iter_ms[64];     /* wall time of each iteration, timing option           */
  int tuned;                /* 1 if the persistent grid and the scheduler's cost
                               model were read from options.tune_cache             */
} feast_batch_stats;

feast_status feast_batch_create(feast_batch** out, int count, const int64_t* n, const feast_z* const* A,
                                const int64_t* lda, const feast_contour* contours, const int* m0,
                                const feast_options* opts, void* stream);
void feast_batch_destroy(feast_batch* b);
/* Factor every shifted matrix (one persistent launch of the factorisation
 * tasks only).  A later call forms and factors them again.
 * FEAST_ERR_SINGULAR_SHIFT if some pivot is exactly zero. */
feast_status feast_batch_factor(feast_batch* b);
/* Q[p] = sum_k w_k (z_k I - A_p)^{-1} Y[p] for every pencil (Eq. Rasp with
 * B = I); Y[p], Q[p] are n[p] x m0[p] (host or device).  Factors first if
 * needed, in the same launch as the solves. */
feast_status feast_batch_filter(feast_batch* b, const feast_z* const* Y, feast_z* const* Q);
/* Iterate every pencil from its starting block Y0[p] (n[p] x m0[p]) until all
 * converge or max_iter.  Per pencil: lambda[p] (m0[p] values, the first
 * m_found[p] valid, sorted by (Re, Im)), X[p] (n[p] x m0[p], unit columns;
 * nullable), res[p] (normalised residuals, nullable).  FEAST_ERR_NOCONV if
 * some pencil did not converge (its outputs are those of the last iteration). */
feast_status feast_batch_solve(feast_batch* b, const feast_z* const* Y0, feast_z* const* lambda, feast_z* const* X,
                               double* const* res, int* m_found, feast_batch_stats* stats);
/* Factor of shift k of pencil p after factorisation: LU (n x n, host or
 * device; L unit lower below the diagonal, U on and above), and the row
 * permutation perm (n entries) with (P S)[r, :] = S[perm[r], :]. */
feast_status feast_batch_get_factor(feast_batch* b, int pencil, int shift, feast_z* LU, int32_t* perm);
/* Shape of the batch: pencils, shifted matrices, CTAs of the persistent
 * launch, tasks of the factorisation, the schedule's model makespan (us), and
 * the algorithmic LU flops sum_i 8/3 n_i^3. Any output may be NULL. */
feast_status feast_batch_info(const feast_batch* b, int* count, int* nmat, int* grid, int* tasks_factor,
                              double* plan_makespan_us, double* lu_flops);
/* The tensor-core classes of the batch: the order from which pencils join
 * them (0 = none), the number of classes (distinct padded orders) and of
 * shifted matrices they hold. Any output may be NULL. */
feast_status feast_batch_tc_info(const feast_batch* b, int* tc_min, int* classes, int* matrices);
/* The host scheduler alone (no GPU): the task order of the persistent launch
 * for nmat matrices with nb[i] = ceil(n_i / 64) block columns and m[i]
 * right-hand sides on `workers` CTAs, with factorisation tasks (with_lu) and/or
 * solve tasks (with_solve).  tasks receives 4 ints per task {kind, matrix, k, j}
 * with kind 0 = panel k, 1 = update of block column j by step k,
 * 2 = interchange fix-up of block column j, 3 = solve of 32-column chunk j.
 * capacity is in tasks; tasks may be NULL to query ntasks. */
feast_status feast_batch_plan(int nmat, const int* nb, const int* m, int with_lu, int with_solve, int workers,
                              int* tasks, int capacity, int* ntasks, double* makespan_us);

/* Diagnostic: C = op(A) X by the emulated-FP64 tensor-core product that the
 * mixed path uses for its n x n x m0 Rayleigh-Ritz products (no paper
 * counterpart).  Each row of the real form of op(A) and each column of X is
 * scaled by a power of two and cut into signed integer digits of beta bits,
 * stored exactly in bfloat16, with n 2^(2 beta + 1) <= 2^24.  Every digit-pair
 * product is then exact in the tensor cores' FP32 accumulators, and the pairs
 * are summed with their weights in FP64 (about 50 significant bits kept).
 *   A : n x n, lda >= n;  X : n x m (1 <= m <= 4096), ldx >= n;  C : n x m, ldc >= n;
 *   column-major complex128, host or device; op = 0 (A) or 2 (A^H).
 * Allocates its own scratch (freed before return); returns after the stream has drained. */
feast_status feast_emulated_zgemm(int64_t n, int64_t m, const feast_z* A, int64_t lda, int op, const feast_z* X,
                                  int64_t ldx, feast_z* C, int64_t ldc, void* stream);

/* Diagnostic: Q (n x m, 1 <= m <= min(n, 256), ldq >= n, column-major
 * complex128, host or device) replaced in place by the orthonormal basis of
 * its columns that the Rayleigh-Ritz step uses (the orthogonalisation of the
 * filtered block recommended at the close of Sec. 4): classical Gram-Schmidt
 * applied twice, column by column, in FP64.  For a block of full numerical
 * rank this is the Q of the QR factorisation with a positive real diagonal in
 * R.  A column that lies numerically in the span of the earlier ones (the
 * second projection takes more than 1 - 1/sqrt(2) of what the first left:
 * Kahan's twice-is-enough test) restarts from a unit vector, so the result
 * stays orthonormal.  Allocates its own scratch (freed before return);
 * returns after the stream has drained. */
feast_status feast_orthonormalize(int64_t n, int64_t m, feast_z* Q, int64_t ldq, void* stream);

/* Number of CUDA kernels this library has launched in this process so far
 * (a diagnostic counter; no paper counterpart). */
uint64_t feast_kernel_launches(void);

/* Diagnostic (no paper counterpart): the time limit of the library's
 * cross-CTA waits -- the grid barriers of the cooperative kernels and the
 * dependency waits of the batched persistent launch.  seconds <= 0 restores
 * the built-in limits (about one to two seconds).  A wait that runs out sets a
 * device flag, the kernel returns, and the call reports
 * FEAST_ERR_DEVICE_TIMEOUT; the context stays usable.  Process-wide; takes
 * effect for launches made after the call. */
void feast_set_wait_limit(double seconds);

/* Nodes and weights of a contour (Sec. 3, Eq. quadrature_for_pi) without a
 * handle, on the host: q receives the number of nodes; nodes and weights
 * (q entries each, host) may be NULL to query q. */
feast_status feast_contour_nodes(const feast_contour* c, int* q, feast_z* nodes, feast_z* weights);

/* ---- General domain shapes (Sec. 5.4): a boundary glued from segments,
 * each parameterised on its own over t in [0, 1] and traversed
 * counter-clockwise, each starting where the previous one ends:
 *   kind 0: the line a + (b - a) t;
 *   kind 1: the arc a + r exp(i (t0 + (t1 - t0) t)).
 * feast_piecewise_nodes computes the nodes phi and weights
 * sigma = w phi'(t) / (2 pi i) (host):
 *   rule FEAST_RULE_TRAP_END: the trapezoidal rule with K >= 2 points per
 *     segment, both ends included; the coinciding end and start nodes of
 *     consecutive segments are merged (weights added), so
 *     q = nseg (K - 1), each vertex once, at the start of the segment that
 *     leaves it;
 *   rule FEAST_RULE_GAUSS: K Gauss-Legendre points per segment, q = nseg K.
 * Pass the result as FEAST_RULE_CUSTOM nodes (R = 0 selects the filter-value
 * domain test).  q <= 256.  nodes/weights may be NULL to query q. */
typedef struct {
  int kind;
  feast_z a, b;
  double r, t0, t1;
} feast_segment;
feast_status feast_piecewise_nodes(const feast_segment* seg, int nseg, int K, int rule, int* q, feast_z* nodes,
                                   feast_z* weights);

/* The filter-quality indicator eta(r) of Sec. 3, a tuning tool for the
 * choice of rule and N_e: on the level curves mu(r, th) = c + r R (cos th +
 * i aspect sin th), th = 2 pi j / ntheta, eta(r) is the minimum of
 * |rho(mu)| = |sum_k sigma_k / (phi_k - mu)| over the curve for r < 1 and
 * its maximum for r > 1 (values near 1 inside and small outside mark a good
 * filter).  Needs an ellipse (R > 0); host only.  r, eta: nr entries. */
feast_status feast_eta_indicator(const feast_contour* c, const double* r, int nr, int ntheta, double* eta);

#ifdef __cplusplus
}
#endif

#endif /* FEAST_GB300_H */
