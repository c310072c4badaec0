/*
 * laker.h -- C ABI of the GB300 (sm_103a) implementation of the LAKER hot path:
 * regularized attention-kernel regression solved by preconditioned conjugate
 * gradients with a CCCP-learned preconditioner (arXiv 2604.25138).
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Array arguments are DEVICE pointers owned by the caller, unless the name
 *   ends in `_host`.  Matrices are row-major and contiguous.  Floating-point
 *   inputs and outputs are float64 whatever precision the library computes in.
 * - Work is issued on the stream given to laker_create(); calls that return
 *   an info struct synchronise that stream before returning, the others are
 *   asynchronous.
 * - Handles (laker_ctx, laker_op, laker_precond) are owned by the library from
 *   their create/build call until the matching destroy call.  All device
 *   workspace is allocated at create/build/fit time and freed by destroy; the
 *   solve, apply and map calls allocate nothing unless noted.
 * - Every call returns a laker_status (0 = success, < 0 = error).  No call
 *   aborts, traps or prints.  laker_last_error() gives a message for the last
 *   failing call on a context.  Errors in device code are reported through a
 *   status word and never by a trap.
 */
#ifndef LAKER_H
#define LAKER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LAKER_OK = 0,
    LAKER_ERR_ARG = -1,          /* invalid argument (sizes, NULL, lambda <= 0) */
    LAKER_ERR_CUDA = -2,         /* a CUDA runtime call failed */
    LAKER_ERR_NOT_SPD = -3,      /* a Cholesky factorisation met a non-positive pivot */
    LAKER_ERR_BREAKDOWN = -4,    /* PCG breakdown: p^T A p <= 0 or r^T z <= 0 or non-finite */
    LAKER_ERR_MAXITER = -5,      /* tolerance not reached; the best alpha is still written */
    LAKER_ERR_NONFINITE = -6,    /* NaN or Inf found in an input */
    LAKER_ERR_TIMEOUT = -7,      /* a bounded device-side wait gave up */
    LAKER_ERR_OOM = -8,          /* device allocation failed */
    LAKER_ERR_UNSUPPORTED = -9   /* combination of options not built */
} laker_status;

/* Arithmetic of the kernel operator (Sec. III-A, Eq. sc-exp-kernel). */
typedef enum {
    LAKER_FP64 = 0,      /* float64 logits, exp and accumulation */
    LAKER_FP32 = 1,      /* float32 storage / arithmetic, float64 PCG scalars */
    LAKER_BF16X3 = 2     /* split-bf16 logits (q = hi + lo, all hi/lo products) on tensor
                            cores, float32 exp2 and sums; matrix-free */
} laker_precision;

/* How the operator v -> (lambda I + G) v is evaluated.  FP64 operators are
 * materialised; BF16X3 operators are matrix-free; FP32 operators whose d
 * rounds up to 16, 32 or 64 (d <= 32 or 49 <= d <= 64) have both variants (the matrix-free one recomputes G with the
 * split-bf16 tensor-core kernel, ~1e-6 relative), and LAKER_AUTO times one
 * product of each after the build and keeps the faster for this n (the
 * choice and both times are reported by laker_op_describe). */
typedef enum {
    LAKER_AUTO = 0,
    LAKER_MATERIALISED = 1,   /* G stored in HBM, streamed each product */
    LAKER_MATRIX_FREE = 2     /* G recomputed tile by tile from Q each product */
} laker_variant;

typedef struct laker_ctx laker_ctx;
typedef struct laker_op laker_op;
typedef struct laker_precond laker_precond;
typedef struct laker_setnet laker_setnet;

typedef struct {
    int iterations;      /* CCCP updates applied */
    int converged;       /* 1 if the relative Frobenius change fell below tol */
    double c;            /* Sigma_* = c I + U diag(D) U^T, isotropic part */
    double rho;          /* shrinkage used */
    double change;       /* last relative Frobenius change |S_{t+1}-S_t|_F/|S_t|_F */
    int status;          /* laker_status of the fit */
    int eig_sweeps;      /* Jacobi sweeps of the eigendecomposition behind Sigma_*^-1/2 */
} laker_fit_info;

typedef struct {
    int iterations;      /* number of operator products (lambda I + G) p */
    int true_residuals;  /* number of float64-accurate residual recomputations */
    int converged;       /* 1 if the stopping test held */
    double rel_res;      /* |r|/|y| of the recursive residual at exit */
    double rel_res_true; /* |y - (lambda I + G) alpha| / |y| (float64 operator) */
    int status;          /* laker_status of the solve */
    int restarts;        /* mixed single solves: roll-backs and direction restarts of the guard */
} laker_solve_info;

/* Context: binds a device and a CUDA stream (cudaStream_t passed as void*).
 * The stream must not be the legacy default stream, because solves capture
 * their iterations into CUDA graphs; NULL makes the library create and own a
 * non-blocking stream, which callers then order against their own work. */
laker_status laker_create(laker_ctx** ctx, int device, void* stream);
laker_status laker_destroy(laker_ctx* ctx);
const char* laker_last_error(const laker_ctx* ctx);
const char* laker_status_string(int status);
/* Number of kernels this context has launched so far (for launch accounting). */
int64_t laker_launch_count(const laker_ctx* ctx);
/* Budget, in SM clock cycles, of each bounded device-side wait of the batched
 * solver's grid barriers on this context (no counterpart in the paper); 0
 * restores the default (~2 s).  A wait that runs out raises LAKER_ERR_TIMEOUT
 * through the kernel's status word; every thread block then leaves at its
 * next barrier and the context stays usable.  Errors: LAKER_ERR_ARG for
 * cycles < 0. */
laker_status laker_set_wait_budget(laker_ctx* ctx, int64_t cycles);

/*
 * Kernel construction (Algorithm 1, kernel-construction stage; Sec. III-A,
 * Eqs. sc-exp-kernel and sc-final):  G_ij = exp(scale * <q_i, q_j>), operator
 * v -> lambda v + G v.
 *   Q       n x d embeddings (device, float64, row-major); copied, the caller
 *           may free it after the call returns.
 *   scale   1.0 reproduces the paper's exp(<e_i,e_j>); 1/sqrt(d) gives the
 *           scaled dot-product form.
 *   lambda  ridge parameter, must be > 0.
 *   precision / variant  see the enums.  FP32 operators keep G as a float32
 *           pair (hi, lo), n x n each, with hi + lo equal to G to ~2^-48: hi
 *           is the float32 operator, hi + lo gives float64-accurate true
 *           residuals.  BF16X3 operators are matrix-free for their products
 *           and keep the pair only for the upper triangle (128 x 128 tiles,
 *           n^2/2 x 8 bytes, built in double-float) for the float64-accurate
 *           product.  FP32 and BF16X3 operators with d <= 64 also keep the
 *           split-bf16 embedding for the tensor-core kernels.
 * Errors: LAKER_ERR_ARG for n < 1, d < 1 or d > 256, lambda <= 0;
 *         LAKER_ERR_UNSUPPORTED for a matrix-free FP64 operator, or a
 *         matrix-free FP32 / BF16X3 one with d > 64; LAKER_ERR_OOM if G does
 *         not fit.
 */
laker_status laker_build_kernel(laker_ctx* ctx, const double* Q, int64_t n, int d,
                                double scale, double lambda, int precision, int variant,
                                laker_op** op);

/*
 * Streaming update (the paper's future work, Sec. VI: measurements that arrive
 * one batch at a time; no counterpart in its experiments): a new operator over
 * the n points of op followed by m new points.
 *   Q_new   m x d embeddings of the new points (device, float64, row-major);
 *           copied.
 *   out     receives the new operator (n + m points, op's scale, lambda,
 *           precision and resolved variant).  op stays valid and unchanged;
 *           the caller destroys each.
 * The stored entries of op are copied; only the tiles whose column block
 * reaches a new point are evaluated (O(m (n + m) d) work plus a copy), by the
 * same kernels as laker_build_kernel, so every product of the result equals
 * that of laker_build_kernel on the concatenated embeddings bit for bit.
 * Errors: LAKER_ERR_ARG for m < 1 or an operator of another device;
 *         LAKER_ERR_NONFINITE for a non-finite Q_new entry; LAKER_ERR_OOM.
 */
laker_status laker_op_append(laker_ctx* ctx, const laker_op* op, const double* Q_new, int64_t m,
                             laker_op** out);
laker_status laker_op_destroy(laker_op* op);
/* The operator's precision and the variant its products use; for an FP32
 * operator built with LAKER_AUTO also the measured time of one product of
 * each variant (ms; 0 when not measured).  Any output pointer may be NULL.
 * Errors: LAKER_ERR_ARG for a NULL operator. */
laker_status laker_op_describe(const laker_op* op, int* precision, int* variant, double* t_materialised_ms,
                               double* t_matrix_free_ms);


/* w = (lambda I + G) x with the operator's inner precision (device n-vectors). */
laker_status laker_op_matvec(laker_ctx* ctx, const laker_op* op, const double* x, double* w);
/* w = (lambda I + G) x with the float64-accurate operator. */
laker_status laker_op_matvec_fp64(laker_ctx* ctx, const laker_op* op, const double* x, double* w);

/*
 * Measurement hook (no counterpart in the paper): average device time in
 * milliseconds of the operator's main kernel alone -- the streamed matvec of a
 * materialised operator, the tensor-core kernel of a matrix-free one -- over
 * `reps` back-to-back launches on x (device, n), timed with CUDA events on the
 * context's stream after one warm-up launch.  Used for roofline reporting.
 */
laker_status laker_op_time_operator(laker_ctx* ctx, const laker_op* op, const double* x, int reps, double* ms);
/*
 * Measurement hook (no counterpart in the paper): average device time in
 * milliseconds of one whole product w = (lambda I + G) x as a PCG solve issues
 * it -- for a matrix-free operator the preparation kernel, the tensor-core
 * kernel and the finishing kernel; for a materialised one the streamed matvec
 * -- over `reps` back-to-back products after one warm-up, timed with CUDA
 * events on the context's stream with no synchronisation between products.
 * Errors: LAKER_ERR_ARG for reps < 1 or NULL pointers; LAKER_ERR_TIMEOUT if a
 * bounded wait of the tensor-core kernel expired.
 */
laker_status laker_op_time_product(laker_ctx* ctx, const laker_op* op, const double* x, int reps, double* ms);

/*
 * Preconditioner learning (Algorithm 1, learning stage; Sec. IV-B Eq.
 * random_directions, Sec. IV-D Eqs. kernel_shrinkage_cccp_F/_Sigma/
 * _normalization, Eq. preconditioner-Sigmma):
 *   u_k = (lambda I + G) z_k, u_k <- u_k/|u_k|;  Sigma_0 = I;
 *   Sigma_{t+1} = normalise((1-rho) F_gamma(Sigma_t) + rho I)  until the
 *   relative Frobenius change is <= tol or max_iter updates;
 *   P = Sigma_*^(-1/2).
 * The iterate is kept exactly as Sigma_t = c I + U diag(D) U^T (N_r directions).
 *   Z       n x n_r Gaussian directions (device, float64, column k = z_k).
 *   rho     < 0 selects the adaptive rule min(1/2, max(1e-3, gamma (1 - n_r/n)))
 *           (1e-3 when n_r >= n).
 *   eps     safeguard of F_gamma (> 0).
 * Precision: float64 throughout for FP64 operators.  For FP32 and BF16X3
 * operators (d <= 64) the directions are z~_k = bf16(z_k) (round to nearest
 * even; still standard-normal to 2^-9) and u_k = (lambda I + G) z~_k comes
 * from a tensor-core kernel that recomputes each 128 x 128 tile of G from
 * the embedding and multiplies it, as bf16 hi + lo, into all directions at
 * once (~1e-5 relative; G is never formed); for d > 64 from the float32 G.
 * P is kept in the orthonormal form c^-1/2 I + U~ diag(phi) U~^T over the
 * eigen-directions
 * of D^1/2 M D^1/2 with eigenvalue > 1e-3 c (float32 U~).
 * Errors: LAKER_ERR_ARG for n_r < 1 or n_r > 2048; LAKER_ERR_NOT_SPD if a
 * factorisation fails; LAKER_ERR_TIMEOUT if a bounded wait of the
 * tensor-core directions kernel expired.
 */
laker_status laker_fit_preconditioner(laker_ctx* ctx, const laker_op* op, const double* Z,
                                      int n_r, double gamma, double rho, double eps,
                                      int max_iter, double tol, laker_precond** P,
                                      laker_fit_info* info);
/*
 * laker_fit_preconditioner with the random directions drawn on the device from
 * a seed instead of passed in (Sec. IV-B, Eq. random_directions: z_k ~ N(0, I_n)).
 * Z is laker_random_directions(seed, n, n_r) in a workspace allocated and freed
 * by the call; all other arguments, the result and the errors are those of
 * laker_fit_preconditioner.
 */
laker_status laker_fit_preconditioner_seeded(laker_ctx* ctx, const laker_op* op, uint64_t seed, int n_r,
                                             double gamma, double rho, double eps, int max_iter, double tol,
                                             laker_precond** P, laker_fit_info* info);

/*
 * laker_fit_preconditioner started from a previous fit (streaming update; the
 * warm start of Sec. IV-C's iteration, which the paper starts from
 * Sigma_0 = I): Sigma_0 = c I + U diag(D) U^T with prev's (c, D) and this
 * fit's normalised directions u_k, scaled to trace n.  The directions must
 * continue prev's: Z is prev's Z with rows appended for the new points (the
 * same n_r columns).  All other arguments, the result and the errors are those
 * of laker_fit_preconditioner; LAKER_ERR_ARG also if prev is not a CCCP
 * preconditioner over n_r directions, or if op or prev belongs to another
 * device than ctx.
 */
laker_status laker_fit_preconditioner_warm(laker_ctx* ctx, const laker_op* op, const double* Z, int n_r,
                                           double gamma, double rho, double eps, int max_iter, double tol,
                                           const laker_precond* prev, laker_precond** P, laker_fit_info* info);

/*
 * Gaussian random directions (Sec. IV-B, Eq. random_directions): Z (device,
 * n x n_r float64, row-major, column k = z_k) with entries N(0, 1) from the
 * counter-based generator Philox4x32-10 (Salmon et al., SC 2011) under the key
 * seed: the pair of entries 2g, 2g + 1 of the row-major array is the
 * Box-Muller transform of the two 53-bit uniforms
 * u = ((x_a >> 6) 2^27 + (x_b >> 5) + 1/2) 2^-53 formed from the words
 * (x0, x1) and (x2, x3) of the block at counter (g mod 2^32, g div 2^32, 0, 0):
 * r cos(2 pi u2), r sin(2 pi u2) with r = sqrt(-2 ln u1).  Asynchronous.
 * Errors: LAKER_ERR_ARG for n < 1, n_r < 1 or Z NULL.
 */
laker_status laker_random_directions(laker_ctx* ctx, uint64_t seed, int64_t n, int n_r, double* Z);

/*
 * The raw generator behind laker_random_directions (no counterpart in the
 * paper; exposed so that its words can be checked bit for bit): out (device,
 * 4 count uint32) receives the Philox4x32-10 blocks of the counters
 * counter0 .. counter0 + count - 1 (64-bit counter in words c0, c1; c2 = c3
 * = 0) under the 64-bit key.  Asynchronous.
 * Errors: LAKER_ERR_ARG for count < 0 or out NULL.
 */
laker_status laker_philox4x32_10(laker_ctx* ctx, uint64_t key, uint64_t counter0, int64_t count, uint32_t* out);

/* Jacobi preconditioner P_J = diag(lambda I + G)^-1 (Sec. V-A baselines). */
laker_status laker_precond_jacobi(laker_ctx* ctx, const laker_op* op, laker_precond** P);
laker_status laker_precond_destroy(laker_precond* P);
/* z = P r (device n-vectors). */
laker_status laker_precond_apply(laker_ctx* ctx, const laker_precond* P, const double* r, double* z);
/* Export the CCCP state: c (1 value), D (n_r values), Ubar (n x n_r), all
 * device float64; any pointer may be NULL. */
laker_status laker_precond_export(laker_ctx* ctx, const laker_precond* P, double* c, double* D,
                                  double* Ubar);

/*
 * PCG solve of (lambda I + G) alpha = y (Sec. IV-E, Algorithm 1, PCG stage):
 *   alpha^0 = 0, r^0 = y, z^0 = P r^0, p^0 = z^0; delta = r.z / p.Ap;
 *   alpha += delta p; r -= delta Ap; stop if |r|/|y| <= tol; z = P r;
 *   beta = r.z_new / r.z_old; p = z + beta p.
 *   P          NULL = identity.
 *   tol        relative residual tolerance.
 *   refine_every  k > 0 (FP32 / BF16X3 operators): every k products, and
 *              whenever the recursive residual passes the test, r is replaced
 *              by y - (lambda I + G) alpha computed with the float64-accurate
 *              operator, and the stop test uses that true residual.  0 = never.
 *              The replacements are guarded: the lowest true residual seen
 *              is kept with its iterate; a non-finite residual, or two
 *              replacements in a row more than 30 times above the best,
 *              roll alpha back to it, restart the direction and halve the
 *              interval (at least 4); a product with p^T A p <= 0 forces a
 *              replacement and restarts the direction.  A roll-back at
 *              interval 4 ends the solve with LAKER_ERR_MAXITER
 *              ("stagnated": the tolerance is below what the operator's
 *              accuracy lets the solve reach).
 * alpha (device, n) receives the last iterate, also on LAKER_ERR_MAXITER
 *              (mixed forms: the iterate with the lowest true residual).
 */
laker_status laker_pcg_solve(laker_ctx* ctx, const laker_op* op, const laker_precond* P,
                             const double* y, double* alpha, double tol, int max_iter,
                             int refine_every, laker_solve_info* info);

/*
 * laker_pcg_solve from a caller-given start (streaming update: the previous
 * solution with zeros for the new points).  alpha (device, n) holds the start
 * alpha^0 on entry and the solution on return; r^0 = y - (lambda I + G)
 * alpha^0 is formed with the float64-accurate product (one product, not
 * counted in info->iterations), and the iteration is Algorithm 1's PCG from
 * there.  A start that already meets tol returns with 0 iterations.
 * Arguments, results and errors otherwise as laker_pcg_solve; also
 * LAKER_ERR_NONFINITE for a non-finite start.
 */
laker_status laker_pcg_solve_warm(laker_ctx* ctx, const laker_op* op, const laker_precond* P,
                                  const double* y, double* alpha, double tol, int max_iter,
                                  int refine_every, laker_solve_info* info);

/*
 * laker_pcg_solve that also records, for every product k = 1 .. min(iterations,
 * trace_cap), four float64 values in trace[4 (k-1) ..] (host memory, owned by
 * the caller; rows past the last product are zeroed):
 *   delta_k          the step of product k;
 *   |r_k|^2 / |y|^2  the recursive residual after it;
 *   R(alpha_k)       |G alpha - y|^2 + lambda alpha^T G alpha (Eq. simu-R-definition),
 *                    from the recursive residual: |r|^2 + lambda (r.alpha + y.alpha);
 *   beta_k           the conjugation coefficient formed after it (0 past the last).
 * These feed the paper's numerical-layer metrics (Sec. V-A): iterations to an
 * objective gap (laker_trace_gap_iterations) and the condition-number
 * estimate from the Lanczos tridiagonal (laker_lanczos_extremes).  For mixed
 * solves the values follow the recursive residual between replacements.
 * Errors: as laker_pcg_solve; LAKER_ERR_ARG for trace_cap < 1 or trace NULL.
 */
laker_status laker_pcg_solve_trace(laker_ctx* ctx, const laker_op* op, const laker_precond* P,
                                   const double* y, double* alpha, double tol, int max_iter,
                                   int refine_every, laker_solve_info* info, double* trace, int trace_cap);

/*
 * laker_pcg_solve that stops on the paper's objective gap (Sec. V-A,
 * Eq. iterations with TAR.TOL = gap): after product k the objective
 * R(alpha_k) = |G alpha_k - y|^2 + lambda alpha_k^T G alpha_k (Eq.
 * simu-R-definition, formed from the recursive residual as in
 * laker_pcg_solve_trace) is compared with the reference R_ref, and the solve
 * stops at the first k with |R(alpha_k) - R_ref| <= gap |R_ref|, or when the
 * residual test with `tol` holds (tol = 0 disables it), or at max_iter.
 * info->iterations is that k.  R_ref comes from a reference solution (the
 * paper's convex-solver solution; a tight PCG solve serves).
 * Errors: as laker_pcg_solve; LAKER_ERR_ARG for gap <= 0 or R_ref zero or
 * not finite.
 */
laker_status laker_pcg_solve_gap(laker_ctx* ctx, const laker_op* op, const laker_precond* P, const double* y,
                                 double* alpha, double R_ref, double gap, double tol, int max_iter, int refine_every,
                                 laker_solve_info* info);

/*
 * Extreme eigenvalues of the Lanczos tridiagonal T_k of k PCG products (host
 * arithmetic on a trace of laker_pcg_solve_trace): T_jj = 1/delta_j +
 * beta_{j-1}/delta_{j-1}, T_j,j+1 = sqrt(beta_j)/delta_j.  Its eigenvalues are
 * the Ritz values of P^1/2 (lambda I + G) P^1/2 on the Krylov space, so
 * lmax / lmin estimates kappa(P (lambda I + G)) from below (Sec. V-A, the
 * condition-number metric), exactly once k reaches the number of distinct
 * eigenvalues.  Bisection on Sturm counts, relative accuracy ~1e-14.
 * Errors: LAKER_ERR_ARG for k < 1, NULL pointers, delta <= 0 or beta < 0.
 */
laker_status laker_lanczos_extremes(const double* trace, int k, double* lmin, double* lmax);

/*
 * The first product k (1-based) of a trace whose objective gap
 * |R(alpha_k) - R_ref| / |R_ref| is <= gap (Eq. iterations with TAR.TOL =
 * gap; R_ref from a reference solution), or -1 if none of the k_max rows
 * reaches it.
 */
int laker_trace_gap_iterations(const double* trace, int k_max, double R_ref, double gap);

/*
 * Gradient descent on R(alpha) (Sec. V-A, the first-order baseline of the
 * numerical-layer comparison; Eq. simu-R-definition):
 *   alpha^0 = 0;  alpha^{k+1} = alpha^k - eta grad R(alpha^k),
 *   grad R(alpha) = 2 G ((lambda I + G) alpha - y),
 * two operator products per step.  The paper selects eta by grid search;
 * eta <= 0 here selects eta = 1 / (2 mu (mu + lambda)) with mu = lambda_max(G)
 * from 50 power-iteration products (laker_op_lambda_max), the largest step
 * that contracts every eigen-component of the error; a caller's grid search
 * passes multiples of it.  *eta_used (host, may be NULL) receives the step.
 * Stops when |y - (lambda I + G) alpha^k| / |y| <= tol (tested every 16
 * steps) or after max_iter steps; alpha (device, n) receives the last iterate.
 * trace (host, 2 trace_cap doubles, may be NULL): for k = 1 .. min(steps,
 * trace_cap), |r_k|^2 / |y|^2 and R(alpha_k) of the iterate after k steps.
 * Errors: LAKER_ERR_ARG for NULL pointers, max_iter < 0, tol < 0;
 * LAKER_ERR_MAXITER if tol was not reached (alpha still written);
 * LAKER_ERR_BREAKDOWN if the iterates overflow.
 */
laker_status laker_gd_solve(laker_ctx* ctx, const laker_op* op, const double* y, double* alpha, double eta,
                            double tol, int max_iter, double* eta_used, laker_solve_info* info, double* trace,
                            int trace_cap);

/* lambda_max(G) (host *mu) by `iters` power-iteration products with the
 * operator's inner precision, from the all-ones start (no counterpart in the
 * paper; the step-size rule of laker_gd_solve).  Errors: LAKER_ERR_ARG for
 * iters < 1 or NULL pointers. */
laker_status laker_op_lambda_max(laker_ctx* ctx, const laker_op* op, int iters, double* mu);

/*
 * Prediction discrepancy (Sec. V-A, Eq. prediction-discrepancy):
 * *out (host) = |G alpha - G alpha_ref| / |G alpha_ref| with the operator's
 * float64-accurate product (G x = (lambda I + G) x - lambda x).  alpha and
 * alpha_ref are device n-vectors.  Synchronous.
 * Errors: LAKER_ERR_ARG for NULL pointers or G alpha_ref = 0.
 */
laker_status laker_prediction_discrepancy(laker_ctx* ctx, const laker_op* op, const double* alpha,
                                          const double* alpha_ref, double* out);

/* One instance of a batched solve: its operator, preconditioner (NULL =
 * identity), right-hand side y (device, n) and output alpha (device, n). */
typedef struct {
    const laker_op* op;
    const laker_precond* P;
    const double* y;
    double* alpha;
} laker_batch_item;

/*
 * Batched PCG (the PCG stage of Algorithm 1, Sec. IV-E, for `count`
 * independent instances of any sizes) in one persistent cooperative launch.
 * Each instance runs the iteration of laker_pcg_solve with its own float64
 * scalars and stops on its own test; instances that stop leave the shared
 * work lists.
 *   items      host array of `count` instances.  Operators must be
 *              materialised and share a precision class: all FP64, or all
 *              FP32 / BF16X3 (these use the float32 G for the product and the
 *              float32 pair for the float64-accurate true residual).  CCCP
 *              preconditioners must come from operators of the same class.
 *   refine_every  as in laker_pcg_solve (mixed instances).
 *   infos      host array of `count` (may be NULL); rel_res_true is the
 *              float64-accurate residual of the returned alpha.
 *   done_ms    host array of `count` (may be NULL): time from the launch
 *              start to each instance's stop, from the device clock.
 * The first call for a batch shape (count, total n) times six candidate work
 * shapes (rows per work item x CTAs per SM) on 8 products each and keeps the
 * fastest.  The call allocates its workspace and synchronises the stream.
 * Errors: LAKER_ERR_ARG / LAKER_ERR_UNSUPPORTED for mixed precision classes or
 * non-materialised operators; LAKER_ERR_BREAKDOWN or LAKER_ERR_MAXITER if any
 * instance failed (its info says which; every alpha is written).
 */
laker_status laker_pcg_solve_batched(laker_ctx* ctx, int count, const laker_batch_item* items,
                                     double tol, int max_iter, int refine_every,
                                     laker_solve_info* infos, double* done_ms);

/*
 * The same independent solves as laker_pcg_solve_batched, run as concurrent
 * single-instance solves (laker_pcg_solve, Algorithm 1's PCG stage, one per
 * instance): `streams` host threads each take the next instance and solve it
 * on a stream of their own, so small instances overlap on the GPU and every
 * instance stops on its own test without waiting for the others at a
 * barrier (no counterpart in the paper).
 *   items      host array of `count` instances, any precisions and variants
 *              (laker_pcg_solve's rules per item).  An operator with a
 *              matrix-free or packed-pair workspace (BF16X3, matrix-free
 *              FP32) may appear in one item only.
 *   streams    1 .. 64 worker threads and streams (at most count are used).
 *   tol, max_iter, refine_every  as in laker_pcg_solve, for every instance.
 *   infos      host array of `count` (may be NULL); done_ms (host, may be
 *              NULL): host time from the call's start to each instance's end.
 * The workers start after the work already queued on the context's stream and
 * the call returns when every solve has ended.  Workspaces for all workers
 * are allocated before the first solve and freed after the last; the solves
 * themselves allocate nothing (an allocation or a free would synchronise the
 * device and serialise the streams).
 * Errors: LAKER_ERR_ARG for bad arguments or a shared workspace operator;
 * LAKER_ERR_NONFINITE for a non-finite y; otherwise the worst instance status
 * (a hard error, then LAKER_ERR_BREAKDOWN, then LAKER_ERR_MAXITER), every
 * alpha written and its info saying which failed.  An instance that no worker
 * thread could run (none could select the device) reports LAKER_ERR_CUDA in
 * its info.
 */
laker_status laker_pcg_solve_concurrent(laker_ctx* ctx, int count, const laker_batch_item* items, double tol,
                                        int max_iter, int refine_every, int streams, laker_solve_info* infos,
                                        double* done_ms);

/*
 * Learned set-to-parameters network (no counterpart in the paper, whose only
 * learning is the CCCP fit of Sec. IV-B..D).  It reads an instance as a set of
 * points x_i = [location / L (2), q_i (d), y_i] and predicts log c and the
 * per-direction log(D_k N_r / n) of Sigma_* = c I + U diag(D) U^T (both
 * targets free of the instance size: tr Sigma_* = n):
 *   h1 = tanh(x W1 + b1), h2 = tanh(h1 W2 + b2), h3 = tanh(h2 W3 + b3);
 *   z = mean over the points of h3;
 *   log c = tanh(z Wg1 + bg1) . wg2 + bg2;
 *   log(D_k N_r / n) = tanh([z, f_k] Wd1 + bd1) . wd2 + bd2 with the
 *   direction features f_k = [log(|u_k| / n), (1/N_r) sum_j M_kj^2]
 *   (laker_precond_direction_features; |u_k| before normalisation).
 * Loss over a batch of B instances:
 *   (1/B) sum_b [(log c_b - t_b)^2 + (1/K_b) sum_k (log D_bk - T_bk)^2].
 * Weights: float32 masters, used in bf16; float32 activations and sums; Adam
 * (beta 0.9 / 0.999, eps 1e-8).  Parameters form one float32 vector laid out
 * as W1, b1, W2, b2, W3, b3, Wg1, bg1, wg2, bg2, Wd1, bd1, wd2, bd2 (matrices
 * row-major, input dimension first); Glorot-uniform from `seed`, zero biases.
 * A batch passes its points as one device array X (P x in_dim float32;
 * instance b owns rows poff[b] .. poff[b+1]-1) and its directions as F
 * (K x 2 float32, rows koff[b] .. koff[b+1]-1); poff and koff are HOST
 * arrays of B + 1 ints starting at 0; every instance needs at least one point.
 */
laker_status laker_setnet_create(laker_ctx* ctx, int in_dim, int hidden, int dir_hidden, uint64_t seed,
                                 laker_setnet** net);
laker_status laker_setnet_destroy(laker_setnet* net);
int64_t laker_setnet_num_params(const laker_setnet* net);
/* host float32 arrays of laker_setnet_num_params entries; set resets Adam */
laker_status laker_setnet_get_params(laker_ctx* ctx, const laker_setnet* net, float* host);
laker_status laker_setnet_set_params(laker_ctx* ctx, laker_setnet* net, const float* host);
/*
 * Checkpoint of a set network (no counterpart in the paper): laker_setnet_save
 * writes the sizes, the Adam step count, the float32 weights and both Adam
 * moments to the file `path` (created or replaced; 8-byte magic "LAKERSN1",
 * int32 in_dim, hidden, dir_hidden, step, int64 parameter count, then three
 * float32 arrays of that count, host byte order); laker_setnet_load creates a
 * network from such a file, so that training resumes exactly where it stopped.
 * Both synchronise the context's stream.
 * Errors: LAKER_ERR_ARG for NULL pointers, a file that cannot be opened,
 * written or read, or one that is not a checkpoint of consistent sizes.
 */
laker_status laker_setnet_save(laker_ctx* ctx, const laker_setnet* net, const char* path);
laker_status laker_setnet_load(laker_ctx* ctx, const char* path, laker_setnet** net);
/* X (device, n x (d + 3) float32) = [loc (n x 2), Q (n x d), y (n)] (device float64 inputs) */
laker_status laker_setnet_point_features(laker_ctx* ctx, int64_t n, int d, const double* loc, const double* Q,
                                         const double* y, float* X);
/* logc (device, B) and logD (device, koff[B]); either may be NULL */
laker_status laker_setnet_forward(laker_ctx* ctx, laker_setnet* net, int B, const float* X, const int* poff,
                                  const float* F, const int* koff, float* logc, float* logD);
/* gradient of the loss (device, num_params) at targets tc (device, B), tD
 * (device, koff[B]); *loss (host) receives the loss; no update */
laker_status laker_setnet_gradient(laker_ctx* ctx, laker_setnet* net, int B, const float* X, const int* poff,
                                   const float* F, const int* koff, const float* tc, const float* tD, float* grad,
                                   float* loss);
/* one Adam step with learning rate lr on the batch; *loss (host) before the step */
laker_status laker_setnet_train_step(laker_ctx* ctx, laker_setnet* net, int B, const float* X, const int* poff,
                                     const float* F, const int* koff, const float* tc, const float* tD, float lr,
                                     float* loss);
/* F (device, n_r x 2 float32) = [log(|u_k| / n), (1/N_r) sum_j M_kj^2] of a CCCP preconditioner's directions */
laker_status laker_precond_direction_features(laker_ctx* ctx, const laker_precond* P, float* F);
/*
 * CCCP fit started from, or replaced by, the network's prediction (Sec. IV-D
 * iteration; the prediction is an extension beyond the paper).  After the
 * directions U and their Gram M are formed, the network predicts (c, D) from
 * the point features X (device, n x in_dim, laker_setnet_point_features) and
 * the direction features; D_k = (n / N_r) exp(prediction), and (c, D) is
 * scaled to tr Sigma = n.
 *   mode 0: CCCP iterations start from the prediction (warm start);
 *   mode 1: the prediction is used as Sigma_* (no CCCP iteration).
 * Other arguments as laker_fit_preconditioner.
 */
laker_status laker_fit_preconditioner_learned(laker_ctx* ctx, const laker_op* op, const double* Z, int n_r,
                                              double gamma, double rho, double eps, int max_iter, double tol,
                                              laker_setnet* net, const float* X, int mode, laker_precond** P,
                                              laker_fit_info* info);

/*
 * Radio-map reconstruction (Sec. III-A, Eq. sc-radio-map-reconstruction;
 * Algorithm 1, reconstruction stage):  out_m = sum_i exp(scale <qg_m, q_i>) alpha_i.
 *   Qg   m x d query embeddings (device float64, row-major);  alpha (n), out (m)
 *   device float64.  Synchronous on the context's stream; allocates scratch.
 * laker_eval_map is laker_eval_map_method with LAKER_MAP_AUTO.
 * Methods:
 *   LAKER_MAP_DOUBLE_FLOAT  float64 kernel for FP64 operators; for FP32 and
 *       BF16X3 operators double-float arithmetic on the float32 pipes (every
 *       kernel value to ~1e-14 relative); d <= 64.
 *   LAKER_MAP_TENSOR  exp(L) = 1 + L + L^2/2 + L^3 g(L) with L = scale <qg, q>:
 *       the first three terms from float64 alpha-weighted moments of the
 *       training embeddings, the remainder from tcgen05 logits of a three-piece
 *       bf16 split and a float32 polynomial for g (map error ~1e-5 relative to
 *       |y| on the benchmark instances, ~1e-4 dB).  Applies when
 *       scale * max|qg_m| * max|q_i| <= 1/2 and d <= 64; otherwise
 *       LAKER_ERR_UNSUPPORTED.
 *   LAKER_MAP_AUTO  FP64 operators: the float64 kernel; FP32 and BF16X3
 *       operators: LAKER_MAP_TENSOR where it applies, else LAKER_MAP_DOUBLE_FLOAT.
 * Errors: LAKER_ERR_ARG for m < 1, null pointers or an unknown method;
 *         LAKER_ERR_TIMEOUT if a bounded wait of the tensor-core kernel expired.
 */
typedef enum {
    LAKER_MAP_AUTO = 0,
    LAKER_MAP_DOUBLE_FLOAT = 1,
    LAKER_MAP_TENSOR = 2
} laker_map_method;
laker_status laker_eval_map(laker_ctx* ctx, const laker_op* op, const double* Qg, int64_t m,
                            const double* alpha, double* out);
laker_status laker_eval_map_method(laker_ctx* ctx, const laker_op* op, const double* Qg, int64_t m,
                                   const double* alpha, double* out, int method);

/*
 * Radio map without device allocation (no counterpart in the paper; a
 * deployment variant of laker_eval_map_method with LAKER_MAP_DOUBLE_FLOAT, same
 * arguments and results).
 * For callers that cannot call cudaMalloc -- services whose device memory is
 * owned and pre-reserved by another allocator, or loops that must not
 * synchronise the device, as cudaMalloc and cudaFree do.  Scratch comes from a
 * static 32 MiB device array that every GPU loading this library keeps until
 * exit; its address is looked up on the first call per device (make that call
 * before any stream capture; first calls from several host threads are
 * serialised by a lock).  Nothing else is set up or uploaded: the kernels
 * build their exp2 table in shared memory.  The call is asynchronous on the
 * context's stream.  All calls on a device share the array: calls that
 * overlap on the GPU race, so serialise them.
 * Errors: LAKER_ERR_ARG if the scratch needed, (m d + n d + n) * 8 bytes for
 * FP32/BF16X3 operators plus 8 m bytes of partial sums, exceeds 32 MiB.
 */
laker_status laker_eval_map_noalloc(laker_ctx* ctx, const laker_op* op, const double* Qg, int64_t m,
                                    const double* alpha, double* out);

#ifdef __cplusplus
}
#endif

#endif /* LAKER_H */
