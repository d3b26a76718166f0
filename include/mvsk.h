/*
 * mvsk.h -- C ABI of the GB300 (sm_103a) YAND-MVSK sample-oracle library.
 *
 * YAND-MVSK (arXiv 2604.25378) minimises the unrestricted sample-moment MVSK
 * objective  f(x) = -c1 mu^T x + c2 m2(x) - c3 m3(x) + c4 m4(x)  over the
 * simplex slice Delta(tau) = {x : 1^T x = 1, x_i >= tau}  (Sec. 2, Eq. mvsk),
 * working only with the centred return matrix A = R - 1 mu^T (Sec. 3.1).
 *
 * Conventions for every entry point:
 *  - All matrices are row-major.  Every vector or matrix argument may be a
 *    host pointer or a device pointer; the library detects which
 *    (cudaPointerGetAttributes) and copies as needed.  The caller keeps
 *    ownership of every pointer it passes; the library never frees them and
 *    never keeps them after the call returns.
 *  - All inputs and outputs are IEEE binary64, whatever the storage precision
 *    of A inside the context.
 *  - Work is issued on the context's stream (mvsk_set_stream; default: a
 *    blocking stream the context creates, which orders with the legacy
 *    default stream) and every call returns after its results are in the
 *    caller's buffers.  PCG solves replay each iteration as a CUDA graph
 *    captured on that stream.
 *  - No C++ exception crosses the ABI and nothing aborts the process; a
 *    failing call returns a non-zero mvsk_status and mvsk_last_error() gives
 *    a message.  Outputs are left untouched on MVSK_EINVAL, MVSK_ESTATE,
 *    MVSK_ENOMEM and MVSK_ECUDA unless stated otherwise.
 *  - A context may be used by one host thread at a time.
 *  - Device kernels never trap: every wait inside a kernel is bounded and a
 *    wait that runs out sets an error word that the call reports as
 *    MVSK_ECUDA.
 */
#ifndef MVSK_H
#define MVSK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mvsk_ctx mvsk_ctx; /* opaque; owns all of its device memory */

typedef enum {
  MVSK_OK = 0,
  MVSK_EINVAL = 1,         /* bad argument: sizes, NaN/Inf data, lambda < 0, w0 outside Delta(tau) */
  MVSK_ENOMEM = 2,         /* device or pinned-host allocation failed */
  MVSK_ECUDA = 3,          /* CUDA runtime error or a bounded in-kernel wait ran out */
  MVSK_ENOTCONVERGED = 4,  /* iteration budget spent before the tolerance; best iterate returned */
  MVSK_ETIMEOUT = 5,       /* max_elapsed reached; best iterate returned */
  MVSK_ESTATE = 6,         /* call out of order (e.g. solve before set_prefs) */
  MVSK_ENUMERIC = 7        /* non-finite value met during the solve */
} mvsk_status;

typedef enum { MVSK_DIRECT = 0, MVSK_PCG = 1 } mvsk_config;

/* Storage precision of A (mvsk_create flags). */
#define MVSK_PREC_FP64 0u        /* A in FP64 only: every pass in FP64 */
#define MVSK_PREC_MIXED_BF16 1u  /* plus a BF16 copy of A for the direction passes (FP32 accumulate) */
#define MVSK_PREC_MIXED_FP32 2u  /* plus an FP32 copy of A for the direction passes */

/* Per-solve report. */
typedef struct {
  int32_t iters;          /* outer YAND iterations, all phases */
  int32_t restarts;       /* stall-recovery restarts taken (PCG) */
  int32_t passes;         /* streaming passes over A issued */
  int32_t hvps;           /* Hessian-vector columns applied */
  int32_t third_calls;    /* third-order back-projections */
  int32_t krylov_iters;   /* PCG iterations summed over columns */
  int32_t free_count;     /* coordinates above tau at the returned point */
  int32_t evals;          /* inner solves spent by the target calibration (1 without target) */
  double f;               /* objective at the returned point */
  double kkt_residual;    /* ||x - Pi_{Delta(tau)}(x - grad f)||_2 (projected-simplex KKT) */
  double kkt0;            /* the same at x0 = 1/n */
  double kkt_rel;         /* kkt_residual / kkt0: the quantity `tol` bounds */
  double c[4];            /* coefficients used (c1 after target calibration) */
  double achieved_mean;   /* mu^T x */
  double seconds;         /* wall time of the call */
  int32_t status;         /* mvsk_status of the solve */
  int32_t batch_iters;    /* mvsk_solve_batch: lockstep iterations the whole batch ran (every
                             request of the call reports the same count); 0 otherwise */
} mvsk_info;

/*
 * mvsk_create -- build a context from RAW returns R (Sec. 2; Alg. 1 set-up).
 *   R: T x n row-major with leading dimension ld >= n (elements); host or
 *      device.  The library computes mu = T^-1 R^T 1 and A = R - 1 mu^T in
 *      FP64 on the GPU and keeps its own padded copies (FP64 master, plus
 *      BF16 or FP32 per flags).  1 <= n <= 6144, T >= 1.
 *   flags: one MVSK_PREC_* value.
 *   *out receives the context.  Errors: EINVAL (sizes, ld < n, non-finite R;
 *   no context is created), ENOMEM, ECUDA.
 */
mvsk_status mvsk_create(const double* R, int64_t T, int64_t n, int64_t ld, uint32_t flags,
                        mvsk_ctx** out);

/* mvsk_set_stream -- issue all later work on `cuda_stream` (a cudaStream_t;
 * NULL restores the context's own stream).  The legacy NULL stream cannot be
 * captured, so PCG solves on it would not use graphs: pass a created stream. */
mvsk_status mvsk_set_stream(mvsk_ctx* ctx, void* cuda_stream);

/*
 * mvsk_set_prefs -- preferences lambda[4] >= 0 (Sec. 2: c_i >= 0) and an
 *   optional return target (Sec. 6: calibrate the mean coefficient).
 *   pref_scaling option 0 (raw): c = lambda; 1 (standardised, default):
 *   c_p = lambda_p / s^p with s^2 = m2(1/n).  target = NaN: c1 from lambda1;
 *   otherwise mvsk_solve finds c1 >= 0 with mu^T x*(c1) = target.
 *   Errors: EINVAL for negative or non-finite lambda.
 */
mvsk_status mvsk_set_prefs(mvsk_ctx* ctx, const double lambda[4], double target);

/*
 * mvsk_set_option -- numeric options (Table yand-core-parameters and the
 *   readings): "tau" (1e-8), "eta" (0.05), "max_iter" (300, direct),
 *   "pcg_max_iter" (40), "restart_iter" (120: iterations of each restart
 *   phase; "restart_iter1" / "restart_iter2" set one phase), "restart_eta1" (0.045),
 *   "restart_eta2" (0.02), "max_elapsed" (60 s), "krylov_tol" (1e-3),
 *   "krylov_maxit" (15), "reg" (NaN: 0 direct / 1e-4 PCG), "probes" (8),
 *   "probe_seed" (24301), "pref_scaling" (1), "release_ratio" (0.5),
 *   "eps_act" (1e-15), "oracle_prec" (0: FP64 A, 1: BF16 A, 2: FP32 A for
 *   the mvsk_oracle_* exports), "cal_rel_tol" (1e-9), "graphs" (1: replay
 *   captured CUDA graphs), "split_products" (1: in mvsk_solve_batch the FP64
 *   products A x, A^T psi'(z) and A d run as split BF16 tensor-core products
 *   with FP64 accuracy, see mvsk_product; 0: FP64 streaming passes),
 *   "batch_lanes" (0: mvsk_solve_batch advances all B requests together; L
 *   with 0 < L < B and split products: L lanes, a lane whose request has
 *   finished takes the next one, so throughput follows the mean iteration
 *   count rather than the slowest request of each batch),
 *   "group_calibration" (1: in mvsk_solve_batch, requests sharing (c2, c3,
 *   c4) with targets start their calibration on a shared c1 grid; 0: each
 *   request alone), "face_products" (1: in mvsk_solve_batch the direction
 *   products run on the union of the instances' working faces; 0: on all
 *   n columns of A), "face_small" (1: when every working face of the batch
 *   has at most 320 coordinates, the direction block forms each face's
 *   Gram matrix and runs the PCG rounds on it, in a narrower launch shape
 *   when every face has at most 128; 2: the same with the 320-coordinate
 *   shape for every small face; 0: always the products),
 *   "line_search" (0: exact quartic step, Prop. quartic exact line search;
 *   1: Armijo backtracking on the same quartic, the paper's Armijo diagnostic
 *   of Table yand-line-search: the largest alpha_max 2^-j, j < 60, with
 *   phi(alpha) - phi(0) <= 1e-4 alpha phi'(0)).
 *   Errors: EINVAL for an unknown key or an out-of-range value.
 */
mvsk_status mvsk_set_option(mvsk_ctx* ctx, const char* key, double value);

/*
 * mvsk_solve -- YAND-MVSK, Alg. 1 (oracle block, affine-normal block, exact
 *   quartic step, boundary block with the projected active-set step of
 *   App. C.3 and face continuation), configuration `cfg` (Table
 *   yand-core-parameters: direct reduced solve, or PCG with stall-recovery
 *   restarts).  Stops when kkt_rel <= tol.
 *   w0: start in Delta(tau) (n values) or NULL for 1/n.
 *   w_out: n values, host or device; written with the best iterate on OK,
 *   ENOTCONVERGED and ETIMEOUT.  info may be NULL.
 *   Errors: ESTATE (no prefs), EINVAL (tol <= 0, w0 outside Delta(tau)),
 *   ENUMERIC, ECUDA.
 */
mvsk_status mvsk_solve(mvsk_ctx* ctx, mvsk_config cfg, double tol, const double* w0,
                       double* w_out, mvsk_info* info);

/*
 * mvsk_solve_batch -- B independent instances (lambda_b, target_b) on the same
 *   A, solved together: every pass over A serves all live instances.
 *   lambdas: B x 4; targets: B (NaN = none); W0: B x n or NULL; W_out: B x n;
 *   infos: B entries or NULL.  Returns OK if every instance converged, else
 *   the first non-OK instance status.
 */
mvsk_status mvsk_solve_batch(mvsk_ctx* ctx, mvsk_config cfg, int32_t B, const double* lambdas,
                             const double* targets, double tol, const double* W0, double* W_out,
                             mvsk_info* infos);

/*
 * mvsk_eval -- exact sample oracle at w (Prop. 1, Eqs. operator-f and
 *   operator-grad): f(w), grad f(w) (n values, may be NULL) and the
 *   projected-simplex KKT residual (may be NULL).  FP64 A.
 */
mvsk_status mvsk_eval(mvsk_ctx* ctx, const double* w, double* f, double* grad, double* kkt);

/*
 * mvsk_eval_noalloc -- f(x), grad f(x) and z = A x for callers that cannot
 *   allocate GPU memory.  The paper has no counterpart: it serves code that
 *   must not call cudaMalloc (a fixed memory budget, a steady-state loop of a
 *   larger framework that owns the allocator) and has only its own buffers.
 *   It runs the value/gradient pass of mvsk_eval; its scratch lives in one
 *   static device array of 8 MiB that every GPU loading the library keeps
 *   until the process exits.  It calls no cudaMalloc/cudaFree and no
 *   allocating library routine.
 *   A: device, centred returns T x ld row-major FP64 (columns n..ld-1 zero),
 *   16-byte aligned, n <= ld <= 6144, ld even; mu: device, n values; c: host,
 *   4 coefficients; x: device, n values.  Outputs (device): z (T values),
 *   g (n values), f (1 value).  Work is issued on `stream` (a cudaStream_t,
 *   NULL = legacy default) and the call returns after it has finished.
 *   The first call on each device fetches the array's device address with
 *   cudaGetSymbolAddress (make that first call before any stream capture).
 *   All calls share the array: calls that overlap on the GPU (other streams
 *   or threads) race and must be serialised by the caller.  Errors: EINVAL
 *   for sizes beyond the limits above (the message says which), ECUDA.
 */
mvsk_status mvsk_eval_noalloc(const double* A, const double* mu, int64_t T, int64_t n, int64_t ld,
                              const double c[4], const double* x, double* z, double* g, double* f,
                              void* stream);

/* Oracle exports (the same kernels as the solver, for parity checks). The
 * copy of A they read is chosen by option "oracle_prec". */

/* Eq. operator-hvp: out = grad^2 f(w) v = T^-1 A^T (psi''(Aw) o Av). */
mvsk_status mvsk_oracle_hvp(mvsk_ctx* ctx, const double* w, const double* v, double* out);

/* Eq. operator-third: out = T3(w; u, v) = T^-1 A^T (psi'''(Aw) o Au o Av). */
mvsk_status mvsk_oracle_third(mvsk_ctx* ctx, const double* w, const double* u, const double* v,
                              double* out);

/* Prop. 2: G = T^-1 A^T Diag(psi''(Aw)) A, n x n row-major (ld = n). */
mvsk_status mvsk_oracle_gram(mvsk_ctx* ctx, const double* w, double* G);

/*
 * mvsk_product -- the sample products z = A v (Prop. 1, Eq. operator-f:
 *   z_t = a_t^T w) and A^T v (Eq. operator-grad), for nvec vectors at once,
 *   with FP64 accuracy on the BF16 tensor cores (error-free splitting of
 *   Ozaki et al.; the paper computes these products in FP64).
 *   transpose = 0: V holds nvec vectors of n values (vector b at V + b*ldv,
 *   ldv >= n) and out vector b (T values) at out + b*ldo (ldo >= T);
 *   transpose = 1: vectors of T values in, n values out.  1 <= nvec <= 64.
 *   Both operands are rounded to 49 significant bits relative to their row
 *   or vector maximum; the product of the rounded operands is then exact up
 *   to terms below 2^-49 of the row maximum times the vector maximum.
 *   V and out are device pointers (EINVAL otherwise); the call returns
 *   after the work has finished.  The first call per context builds the
 *   split copies of A (14 bytes per element of A).  Errors: EINVAL, ECUDA
 *   (also when a bounded wait inside the tensor-core kernel ran out).
 */
mvsk_status mvsk_product(mvsk_ctx* ctx, int32_t transpose, int32_t nvec, const double* V, int64_t ldv,
                         double* out, int64_t ldo);

/*
 * mvsk_batch_hvp -- the direction products of one lockstep iteration of
 *   mvsk_solve_batch, for parity tests, on caller-given operands: B instances
 *   with coefficients C (B x 4, c1..c4) at points X (B x n), working faces
 *   maskF (B x n, 1 free / 0 held; NULL: every coordinate free), each with nc
 *   columns V (B x nc x n, column j of instance b at V + (b*nc + j)*n).
 *   With z_b = A x_b (FP64) and G_b = T^-1 A^T Diag(psi''_b(z_b)) A (Prop. 2):
 *     HV[b][j]  = G_b v_bj  (Eq. operator-hvp), B x nc x n;
 *     Gnu[b]    = G_b nuhat_b, nuhat: B x n;      diagG[b] = diag(G_b), B x n.
 *   They run exactly as in the solve: A in BF16 with FP32 accumulation on the
 *   tensor cores (psi'' in FP32; v, nuhat and the weighted rows rounded to
 *   BF16), the B*nc columns side by side in one product.  With option
 *   "face_products" = 1 (default) the products are restricted, as in the
 *   solve, to the union U of the faces: the caller's v_bj and nuhat_b must
 *   then be zero off face b, and the three outputs are given on U (zero
 *   elsewhere).  path[0] (nullable) receives 1 when the first product A V
 *   took the fused psi''-weighting epilogue, 0 when it took split-K partials
 *   and a separate weighting pass; path[1] the split-K count of the second
 *   product A^T S.  Arguments are host or device pointers.  Needs a
 *   MVSK_PREC_MIXED_BF16 context; 1 <= nc <= 16, 1 <= B <= 4096.  Uses the
 *   batch buffers of mvsk_solve_batch and a scratch allocation released
 *   before returning.  Errors: EINVAL, ENOMEM, ECUDA.
 */
mvsk_status mvsk_batch_hvp(mvsk_ctx* ctx, int32_t B, const double* C, const double* X,
                           const double* nuhat, const double* maskF, int32_t nc, const double* V,
                           double* HV, double* Gnu, double* diagG, int32_t path[2]);

/*
 * mvsk_batch_third -- the Hutchinson correction of the PCG configuration as
 *   mvsk_solve_batch computes it (Eq. operator-third, Sec. 3.2), for parity
 *   tests: for B instances with coefficients C (B x 4) at points X (B x n),
 *   working faces maskF (B x n or NULL, as in mvsk_batch_hvp) and K probe
 *   pairs (U, P) (each B x K x n, pair k of instance b at (b*K + k)*n),
 *     rhat_b = K^-1 sum_k (A u_bk) o (A p_bk),
 *     at[b]  = T^-1 A^T (psi'''_b(z_b) o rhat_b),  z_b = A x_b,  B x n
 *   (on the union of the faces, zero elsewhere, with face_products = 1; the
 *   probe pairs must then be zero off their face).  BF16 A and operands on
 *   the tensor cores, FP32 accumulation, the weighted rows rounded to BF16.
 *   Host or device pointers; MVSK_PREC_MIXED_BF16 context; 1 <= K <= 8.
 *   Errors: EINVAL, ENOMEM, ECUDA.
 */
mvsk_status mvsk_batch_third(mvsk_ctx* ctx, int32_t B, const double* C, const double* X,
                             const double* maskF, int32_t K, const double* U, const double* P,
                             double* at);

/*
 * Prop. quartic exact line search: coef[5] = A0..A4 of f(w + alpha d) from
 * the power sums s_rs, and *alpha_max = alpha_max(w, d; tau) (Lemma cap;
 * +inf when no d_i < 0).  FP64 A.
 */
mvsk_status mvsk_oracle_ls(mvsk_ctx* ctx, const double* w, const double* d, double coef[5],
                           double* alpha_max);

/*
 * YAND direction at w (Sec. 3.2; the formulas of Sec. 3.4) on the face that
 * the boundary block would use, for configuration cfg; `iteration` seeds the
 * Hutchinson probes of the PCG configuration.  d_out: n values, zero on the
 * held face, 1^T d = 0.
 */
mvsk_status mvsk_oracle_direction(mvsk_ctx* ctx, mvsk_config cfg, const double* w,
                                  int32_t iteration, double* d_out);

/* Euclidean projection onto Delta(tau) (App. C.3 projected trial). */
mvsk_status mvsk_project_slice(mvsk_ctx* ctx, const double* v, double tau, double* out);

/* Column means mu (the centring of mvsk_create) and population standard
 * deviations sigma_j = sqrt(T^-1 sum_t (R_tj - mu_j)^2) of the panel, n each
 * (host or device pointers): the panel statistics of the warm-start features
 * (mvsk_mlp.h). */
mvsk_status mvsk_column_stats(mvsk_ctx* ctx, double* mu, double* sigma);

/* Exact minimiser of A0 + A1 a + ... + A4 a^4 on [0, amax] by the device
 * routine the solver uses (candidates: 0, amax, real roots of the cubic). */
mvsk_status mvsk_quartic_argmin(mvsk_ctx* ctx, const double coef[5], double amax, double* alpha);

/*
 * Profiling of the streaming passes over A (tracing, no effect on results).
 * mvsk_profile_enable(ctx, 1) clears the counters and brackets every later
 * kernel launch with CUDA events on the context's stream (launches inside
 * captured CUDA graphs as event nodes, read after each replay); (ctx, 0) stops.
 * mvsk_profile_only(ctx, prefix) restricts the brackets to kinds whose label
 * starts with `prefix`, or with one of the comma-separated prefixes it lists
 * (NULL: all kinds), which keeps the event overhead of a timed run to the
 * kernels of interest.  mvsk_profile_stride(ctx, k) (k >= 1, default 1; reset
 * by mvsk_profile_enable) brackets only every k-th launch of each selected
 * kind, counted per kind in issue order (inside a captured graph, at
 * capture): an event node between two kernels costs the graph part of their
 * overlap, so a timed run samples its kernels.  EINVAL for k < 1.
 * mvsk_profile_read fills up to `max` entries, one per kind: its label
 * (streaming pass, tensor-core product, split FP64 product or named kernel),
 * launches, summed device time (ms) and the average algorithmic work per
 * launch: bytes for streaming passes (one read of A: T * n * element size),
 * FLOPs for tensor-core products, 0 for kernels without a fixed figure.
 * *count receives the number of kinds and *kernel_launches every kernel
 * launch the library issued since enabling.
 */
typedef struct {
  char name[56];
  int64_t launches;
  double total_ms;
  double bytes_per_launch;
} mvsk_prof_entry;

mvsk_status mvsk_profile_enable(mvsk_ctx* ctx, int32_t on);
mvsk_status mvsk_profile_only(mvsk_ctx* ctx, const char* prefix);
mvsk_status mvsk_profile_stride(mvsk_ctx* ctx, int32_t k);
mvsk_status mvsk_profile_read(mvsk_ctx* ctx, mvsk_prof_entry* out, int32_t max, int32_t* count,
                              int64_t* kernel_launches);

/* Thread-local message describing the last failure of any call. */
const char* mvsk_last_error(const mvsk_ctx* ctx);

/* Release every resource of the context.  NULL-safe. */
void mvsk_destroy(mvsk_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MVSK_H */
