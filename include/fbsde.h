/*
 * fbsde.h -- C ABI of the GB300 (sm_103a) library for the localized stochastic
 * FBSDE scheme of Fang, Sheng, Su and Zhou, "A derivative-free localized
 * stochastic method for very high dimensional semilinear parabolic PDEs"
 * (arXiv 2510.02635).
 *
 * The library evaluates u(0, x0) and grad u(0, x0) for semilinear parabolic PDEs
 *     d_t u + 1/2 sigma^2 Lap u + f(t, x, u, sigma^T grad u) = 0,  u(T, .) = g      (Eq. 2.1)
 * with zero drift and a constant scalar diffusion sigma, by the particle scheme of
 * Algorithm 1: an Euler-Maruyama cloud of M particles per query point (Eq. 2.7), a
 * kernel-weighted local linear regression per backward level (Eqs. 2.10-2.15 with the
 * ridge of Remark 2.2 and the Gaussian kernel of Remark 2.3) solved matrix-free on
 * its Schur complement (Lemma 3.7, Eqs. 3.19-3.20), Z = sigma^T alpha_x, and a scalar
 * Newton iteration per particle (Eqs. 2.16-2.17).
 *
 * Conventions (all entry points):
 *  - Plain C types only.  "device" pointers are CUDA global-memory addresses of the
 *    current device; "host" pointers are ordinary host memory.  The caller owns
 *    every buffer, including the workspace; the library allocates no device memory.
 *  - Work is enqueued on the given stream (NULL = the legacy default stream) and
 *    returns before it completes.  Argument errors are returned synchronously and
 *    nothing is enqueued.  Errors found on the device (Newton or CG exhaustion,
 *    non-finite values) are recorded in the workspace and read by
 *    fbsde_diagnostics() after the stream has been synchronised.
 *  - No C++ exception crosses this boundary.
 *  - Deterministic: identical inputs, seed and workspace size give bit-identical
 *    results (every reduction has a fixed order; no floating-point atomics).
 *  - One workspace must not be used by two calls that may overlap in time.
 */
#ifndef FBSDE_H
#define FBSDE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FBSDE_API __attribute__((visibility("default")))
#else
#define FBSDE_API
#endif

typedef struct CUstream_st *fbsde_stream_t; /* the same handle as cudaStream_t */

#define FBSDE_ABI_VERSION 3
#define FBSDE_MAX_D 16384 /* largest dimension d accepted */
#define FBSDE_MAX_D_FP64 10240 /* largest d of the FP64 path (one team of at most 10 warps
                                  of 16 chunks per thread per row in the product kernel) */

typedef enum {
    FBSDE_OK = 0,
    FBSDE_ERR_ARG = 1,        /* invalid argument (synchronous; nothing enqueued)      */
    FBSDE_ERR_WORKSPACE = 2,  /* workspace missing, misaligned or too small           */
    FBSDE_ERR_CUDA = 3,       /* a CUDA call failed (launch or copy)                   */
    FBSDE_ERR_NEWTON = 4,     /* a particle's Newton iteration hit newton_max_iter     */
    FBSDE_ERR_CG = 5,         /* a level's CG solve hit cg_max_iter before cg_tol      */
    FBSDE_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up                    */
    FBSDE_ERR_NONFINITE = 7   /* u(0,x0) or grad u(0,x0) is not finite                 */
} fbsde_status;

/* Problem kinds: terminal condition g and driver f(t, x, y, z) of (2.1). */
typedef enum {
    /* f = y - y^3 + q(t,x), q = u*^3 - (2 - sigma^2/2) u*, g = (1/d) sum cos x_i;
       exact solution u*(t,x) = e^{t-T} (1/d) sum_i cos x_i (Allen-Cahn with a
       manufactured source, the form of Eq. 4.1). */
    FBSDE_AC_MANUFACTURED = 0,
    /* f = (y - (2+d)/(2d)) sum_i z_i, g = 1/(1 + exp(-(T + sum_i x_i/d)));
       exact solution logistic(t + sum_i x_i/d) when sigma = d. */
    FBSDE_LOGISTIC_GRAD = 1,
    /* f = -|z|^2/2, g = log((1 + sum_i theta_i x_i^2)/2); with sigma = sqrt 2,
       exp(-u) solves the heat equation (Cole-Hopf). */
    FBSDE_HJB_LOGQUAD = 2,
    /* f = c0 + c1 y + c2 sum_i z_i + c3 t, g = A + sum_i theta_i x_i (exactly solvable). */
    FBSDE_AFFINE_TEST = 3,
    /* f = y - y^3, g = A (reduces to a scalar backward implicit Euler recursion). */
    FBSDE_CUBIC_TEST = 4,
    /* f = y - y^3, g = 1/(2 + 0.4 |x|^2): Sec. 4.1, case 1 (use sigma = sqrt 2). */
    FBSDE_AC_DOUBLEWELL = 5,
    /* f = c0 + c1 y, g = (1/d) sum_i cos x_i. */
    FBSDE_COS_LINEAR_TEST = 6,
    /* For the forward SDE with drift and state-dependent diffusion (see fbsde_problem), with
       s_i = sigma + sig1 x_i, m_i = mu0 + mu1 x_i: g = (1/d) sum_i cos x_i, f = y - y^3 + q,
       q = u*^3 - 2 u* + e^{t-T} (1/d) sum_i [s_i^2 cos x_i / 2 + m_i sin x_i]; exact
       solution u*(t,x) = e^{t-T} (1/d) sum_i cos x_i for any such coefficients. */
    FBSDE_DRIFT_AC = 7,
    /* The same with g = (1/d) sum_i x_i^2, q = u*^3 - 2 u* - e^{t-T} (1/d) sum_i
       [s_i^2 + 2 m_i x_i]; exact solution u*(t,x) = e^{t-T} (1/d) sum_i x_i^2. */
    FBSDE_DRIFT_QUAD = 8
} fbsde_kind;

typedef enum {
    FBSDE_FP32 = 0, /* particle state, increments and moment sums in FP32; regression
                       combination, CG vectors and Newton in FP64                    */
    FBSDE_FP64 = 1  /* FP64 throughout                                               */
} fbsde_precision;

typedef struct {
    int32_t kind;            /* fbsde_kind                                             */
    int32_t d;               /* dimension, 1 <= d <= FBSDE_MAX_D (FBSDE_MAX_D_FP64 on
                                the FP64 path)                                         */
    int32_t N;               /* number of time steps, dt = T/N, N >= 1                 */
    int32_t precision;       /* fbsde_precision                                        */
    int64_t M;               /* particles per query point, M >= 2                      */
    double sigma;            /* scalar diffusion coefficient, > 0                      */
    double T;                /* terminal time, > 0                                     */
    const double *theta;     /* device, d coefficients for HJB_LOGQUAD and AFFINE_TEST;
                                NULL for the other kinds                               */
    double A, c0, c1, c2, c3;/* parameters of the test kinds (ignored otherwise)       */
    double h;                /* kernel bandwidth: eps_k^2 = h^2 sigma^2 d t_{k+1};
                                h <= 0 or h = inf gives uniform weights                */
    double ridge_rel;        /* ridge lambda = ridge_rel * tr(Gamma_c) / d, >= 0       */
    double cg_tol;           /* CG stops when ||r|| <= cg_tol ||rhs||, > 0             */
    int32_t cg_max_iter;     /* CG iterations per level; 0 selects 200                 */
    int32_t newton_max_iter; /* Newton iterations per particle; 0 selects 50           */
    double newton_tol;       /* Newton stops when |dY| <= newton_tol max(1,|Y|); 0 selects 1e-13 */
    int32_t ctas;            /* CTAs of one streaming pass over all Q queries (tiling of the
                                particle clouds; results depend on it through the order of
                                the partial sums); 0 selects 608; at most M / 32 CTAs
                                per query are used                                       */
    int32_t reserved;        /* must be 0                                               */
    /* Forward SDE dX = mu(t,X) dt + sigma(t,X) dW of Sec. 2.1 with the componentwise affine
       coefficients mu_i(x) = mu0 + mu1 x_i and sigma(x) = diag(sigma + sig1 x_i).  With
       mu0 = mu1 = sig1 = 0 (and kinds 0-6) the driftless scheme: Brownian paths drawn by the
       bridge, fused level step.  Otherwise (and always for kinds 7-8) Euler-Maruyama paths
       (2.7), X_{k+1} = X_k + mu(X_k) dt + sigma(X_k) sqrt(dt) xi_k, kept at checkpoints
       every s = ceil(sqrt N) levels and recomputed segment by segment on the way back; the
       regression of level k is anchored on the drift path a_{k+1} = a_k + mu(a_k) dt of x0,
       its kernel scale is h^2 times the cloud's mean squared distance to that anchor,
       Z_k^j = sigma(X_k^j)^T alpha_x per particle and the prediction is taken at the
       drifted position X_k^j + mu(X_k^j) dt.  HJB_LOGQUAD needs sig1 = 0; fbsde_adjoint and
       the per-anchor entry points accept only the driftless scheme. */
    double mu0, mu1, sig1;
} fbsde_problem;

/* Optional per-level outputs of a solve (all device pointers, each may be NULL).
   Level k (0 <= k < N) is the regression of Y_{k+1} on X_{k+1} - x0 at time t_k. */
typedef struct {
    double *alpha;          /* [Q][N]    intercept alpha of level k                      */
    double *alpha_x;        /* [Q][N][d] slope alpha_x (the grad u estimate) of level k  */
    int32_t *cg_iters;      /* [Q][N]    CG iterations used at level k                   */
    int32_t *newton_iters;  /* [Q][N]    most Newton iterations of any particle, level k */
    double *x_N;            /* [Q][M][d] X_N^j - x0 after the forward sweep              */
    double *y_N;            /* [Q][M]    Y_N^j = g(X_N^j)                                */
} fbsde_trace;

typedef struct {
    int32_t status;         /* first fbsde_status met by any solve (FBSDE_OK if none)    */
    int32_t solves_cg_exhausted;
    int32_t max_newton_iters;
    int32_t cg_iters_total;  /* CG iterations over all levels and queries of the solve    */
} fbsde_diag;

/* Bytes of device workspace that fbsde_solve needs for Q query points of problem P (the
   particle rows, weights and regression vectors of Algorithm 1, laid out per query).
   Returns 0 when the arguments are invalid. */
FBSDE_API size_t fbsde_workspace_bytes(const fbsde_problem *P, int32_t Q);

/*
 * Algorithm 1 for Q query points at once (independent solves, one particle cloud
 * each).  Query q uses the Philox stream of solve index solve_index0 + q.  The Brownian
 * path of each particle (Eq. 2.7 with mu = 0, so X_k = x0 + sigma W(t_k)) is drawn
 * backwards from its end point by the Brownian bridge: W(T) = sqrt(T) xi_N and, for
 * k = N-1..1, W(t_k) = (k/(k+1)) W(t_{k+1}) + sqrt(dt k/(k+1)) xi_k, W(0) = 0.  Its
 * increments are independent N(0, dt I), the law Eq. 2.7 gives them; the forward sweep
 * needs one normal per coordinate and the backward sweep one per level.
 *   x0        device [Q][d]  query points
 *   seed      Philox4x32-10 key of the Brownian increments
 *   u0        device [Q]     output u(0, x0_q)
 *   grad_u0   device [Q][d]  output grad u(0, x0_q) (alpha_x of level 0), or NULL
 *   trace     optional per-level outputs, or NULL
 *   workspace device, >= fbsde_workspace_bytes(P, Q) bytes, 256-byte aligned
 * Returns FBSDE_OK when the work was enqueued.
 */
FBSDE_API int fbsde_solve(const fbsde_problem *P, int32_t Q, const double *x0, uint64_t seed,
                uint32_t solve_index0, double *u0, double *grad_u0, const fbsde_trace *trace,
                void *workspace, size_t workspace_bytes, fbsde_stream_t stream);

/*
 * Algorithm 1 as fbsde_solve, with the query points and results in HOST memory: copies x0 to
 * the device, solves, copies u0 and grad_u0 back and synchronises the stream.
 * theta (if the kind needs it) is read from P->theta as a HOST pointer here.
 * grad_u0 may be NULL.  Returns the solve's device status as well (blocking call).
 */
FBSDE_API int fbsde_solve_host(const fbsde_problem *P, int32_t Q, const double *x0_host, uint64_t seed,
                     uint32_t solve_index0, double *u0_host, double *grad_u0_host,
                     void *workspace, size_t workspace_bytes, fbsde_stream_t stream);

/*
 * fbsde_solve without a caller-supplied workspace, for callers that cannot allocate
 * device memory: a host application whose allocator owns the whole device, a plugin
 * that runs on another framework's stream and must not call cudaMalloc (which can
 * synchronise the device), or code that must not grow its memory after start-up.
 * The paper has no counterpart; this is a deployment convenience.
 *
 * The workspace is a fixed array of FBSDE_NOALLOC_MAX_BYTES in the library's device
 * module.  Every GPU that loads the library holds that array until the process exits.
 * Problems with fbsde_workspace_bytes(P, Q) > FBSDE_NOALLOC_MAX_BYTES are rejected with
 * FBSDE_ERR_WORKSPACE before any work is enqueued.  The call allocates nothing: no
 * cudaMalloc, no cudaFree, no allocating library routine.
 *   x0, u0, grad_u0 and P->theta are device pointers, as for fbsde_solve; grad_u0 may
 *   be NULL.  There is no trace output.
 * The first call on each device looks up the array's device address (with that
 * device current) and caches it; make that first call before any stream capture.  The
 * cached address is not refreshed, so calls on a device after cudaDeviceReset are not
 * supported.
 * All calls share the one array, which keeps the last call's contents.  Each solve
 * rewrites every byte of it that it later reads, so nothing needs clearing between
 * calls, but calls whose GPU work may overlap in time (other streams, other host
 * threads) race on the array and must be serialised by the caller.
 */
#define FBSDE_NOALLOC_MAX_BYTES (64u << 20)
FBSDE_API int fbsde_solve_noalloc(const fbsde_problem *P, int32_t Q, const double *x0,
                                  uint64_t seed, uint32_t solve_index0, double *u0,
                                  double *grad_u0, fbsde_stream_t stream);

/*
 * Algorithm 1 in its literal form: one regression per particle anchor.  At level k the
 * anchor of particle m is its own position X_k^m (Algorithm 1's backward loop over m, the
 * local linear approximation (2.9) centred at X_k^m): D_j^m = X_{k+1}^j - X_k^m, Gaussian
 * weights (2.11) with eps_k^2 = h^2 sigma^2 d (t_k + t_{k+1}), the ridge regression of
 * Lemma 3.7 / Remark 2.2 per anchor, Z_k^m = sigma alpha_x^m, and Newton (2.16)-(2.17)
 * with the anchor's own intercept alpha^m and Z_k^m.  u(0,x0) = mean_m Y_0^m; grad_u0 is
 * alpha_x at k = 0 (all anchors are x0 there).  Cost O(M^2 d) per level and CG pass: the
 * M regressions share two M x M x d contractions per pass.  With FP32 and M >= 1024 these
 * run on the tensor cores with the FP32 operands split into TF32 hi and lo parts (about
 * 1e-6 relative per product); FP64 and smaller M use FP32/FP64 SIMT products.  With uniform
 * weights (h <= 0 or inf) the result equals fbsde_solve's up to rounding.
 *   Same arguments as fbsde_solve (no trace); M <= 32768; theta (if the kind needs it)
 *   is a device pointer in P->theta; workspace >= fbsde_anchored_workspace_bytes(P)
 *   bytes, 256-byte aligned, reused for the Q queries one after the other.
 * Asynchronous on the stream like fbsde_solve: the call is captured once into a CUDA graph
 * (each level's CG passes a conditional while node that repeats while some anchor iterates
 * on), cached per device and argument list, and launched; a stream that is itself being
 * captured receives the work directly.  Returns FBSDE_OK, an argument error
 * (FBSDE_ERR_ARG, FBSDE_ERR_WORKSPACE) or FBSDE_ERR_CUDA; the device status (FBSDE_ERR_CG,
 * FBSDE_ERR_NEWTON, FBSDE_ERR_NONFINITE, or FBSDE_ERR_TIMEOUT when a tensor-core pipeline
 * wait ran out) is read after the work with fbsde_anchored_diagnostics.
 */
FBSDE_API size_t fbsde_anchored_workspace_bytes(const fbsde_problem *P);
FBSDE_API int fbsde_solve_anchored(const fbsde_problem *P, int32_t Q, const double *x0, uint64_t seed,
                                   uint32_t solve_index0, double *u0, double *grad_u0,
                                   void *workspace, size_t workspace_bytes, fbsde_stream_t stream);

/* Status of the last fbsde_solve_anchored / fbsde_solve_batch call on this workspace:
 * copies its status word on `stream` and waits for the stream (host-synchronising).
 * out->status: the first device status of any query; out->cg_iters_total: CG passes over
 * all levels and queries (each pass serves every anchor still iterating); the other fields
 * are 0.  Returns FBSDE_ERR_ARG for an invalid P or a NULL pointer, FBSDE_ERR_CUDA if the
 * copy fails. */
FBSDE_API int fbsde_anchored_diagnostics(const fbsde_problem *P, const void *workspace,
                                         fbsde_diag *out, fbsde_stream_t stream);

/* Algorithm 1 per particle anchor, each anchor's regression over a batch of K particles
 * (the batch reading of Remark 2.1): for anchor m the batch is the cyclic window
 * j = (m + q) mod M, q = 0..K-1, a window that contains the anchor's own path (q = 0)
 * and K - 1 other paths.  The window does not depend on the positions; since the other
 * paths are independent and identically distributed, those K - 1 particles are a random
 * sample of the cloud, but the anchor's own path is always in its batch.  The
 * Gaussian weights, the moments and the ridge are those of fbsde_solve_anchored restricted
 * to the batch (weights normalised over it); K = M is fbsde_solve_anchored.
 *   2 <= K <= M, else FBSDE_ERR_ARG; every other argument, the workspace
 *   (fbsde_anchored_workspace_bytes), the asynchronous launch and the return codes are
 *   those of fbsde_solve_anchored (status through fbsde_anchored_diagnostics).  The weights outside the window are zero, and the products
 *   skip the tiles and K-splits that lie wholly outside the band of the windows, so a CG
 *   pass costs O(M (K + 128) d) in its contractions; the results equal those of the
 *   products over all M particles.
 */
FBSDE_API int fbsde_solve_batch(const fbsde_problem *P, int64_t K, int32_t Q, const double *x0,
                                uint64_t seed, uint32_t solve_index0, double *u0, double *grad_u0,
                                void *workspace, size_t workspace_bytes, fbsde_stream_t stream);

/* The batch reading of fbsde_solve_batch with each anchor's regression solved directly
 * instead of by CG passes, so that its cost no longer grows with the CG's pass count: per
 * level and anchor, one block forms the weighted second moment of the anchor's window of
 * K particles (sum over the window of w D D^T, D = X_{k+1}^j - X_k^m), the CG form's
 * operator Gamma_m + lambda_m I from it (the same S_m, lambda_m and right-hand side),
 * factorises it as L D L^T and solves with the two triangular factors, all in the stream
 * precision.  Rows as in fbsde_solve_batch; the result is the same regression up to
 * rounding (the CG stops at cg_tol, this solve is exact up to its rounding).
 *   1 <= d <= FBSDE_BATCH_DIRECT_MAX_D and ridge_rel > 0 (the ridge keeps every pivot of
 *   the factorisation at least lambda_m), else FBSDE_ERR_ARG.  K, Q, the buffers, the
 *   workspace (fbsde_anchored_workspace_bytes), the asynchronous launch and the return codes
 *   are those of fbsde_solve_batch.  A pivot that rounding still leaves not positive and
 *   finite leaves that anchor's slope at 0 and sets the device status FBSDE_ERR_CG;
 *   fbsde_anchored_diagnostics reads it and counts no CG passes.
 */
#define FBSDE_BATCH_DIRECT_MAX_D 128
FBSDE_API int fbsde_solve_batch_direct(const fbsde_problem *P, int64_t K, int32_t Q,
                                       const double *x0, uint64_t seed, uint32_t solve_index0,
                                       double *u0, double *grad_u0, void *workspace,
                                       size_t workspace_bytes, fbsde_stream_t stream);

/* Bytes of device workspace that fbsde_adjoint needs (the solve's workspace plus a tape
   of N (M + 2 d) values per query).  0 when the arguments are invalid. */
FBSDE_API size_t fbsde_adjoint_workspace_bytes(const fbsde_problem *P, int32_t Q);

/*
 * Derivative of the estimator u(0, x0) of Algorithm 1 with respect to the query points
 * and to theta, for the same random increments (seed, solve indices), by a reverse sweep
 * over the levels.  The solve is re-run with a tape of its per-level regressions
 * (weights, first moments, ridge, alpha, alpha_x, Y_k); the reverse sweep regenerates
 * the particle paths from the Philox streams instead of storing them.  Per level it
 * needs one extra solve with the same SPD operator as the regression (Lemma 3.7).
 *   u0_bar    device [Q]    dL/du0 of each query (the cotangent)
 *   u0        device [Q]    output: u(0, x0) (the re-run solve)
 *   grad_u0   device [Q][d] output: alpha_x of level 0 (the method's grad u), or NULL
 *   x0_bar    device [Q][d] output: u0_bar_q * d u(0, x0_q) / d x0_q
 *   theta_bar device [d]    output: sum_q u0_bar_q * d u(0, x0_q) / d theta, or NULL;
 *                           only for HJB_LOGQUAD and AFFINE_TEST
 *   workspace device, >= fbsde_adjoint_workspace_bytes(P, Q) bytes, 256-byte aligned
 * Asynchronous like fbsde_solve; device errors via fbsde_diagnostics.
 */
FBSDE_API int fbsde_adjoint(const fbsde_problem *P, int32_t Q, const double *x0, uint64_t seed,
                            uint32_t solve_index0, const double *u0_bar, double *u0,
                            double *grad_u0, double *x0_bar, double *theta_bar, void *workspace,
                            size_t workspace_bytes, fbsde_stream_t stream);

/* Extra workspace bytes fbsde_solve_host needs on top of fbsde_workspace_bytes (device
   staging of x0, u0 and grad u0; no counterpart in the paper). */
FBSDE_API size_t fbsde_host_staging_bytes(const fbsde_problem *P, int32_t Q);

/* Synchronises the stream and reads the device-side status of the last solve that
   used this workspace: CG exhaustion of the regression solves (Eqs. 3.19-3.20), the
   largest Newton iteration count (Eqs. 2.16-2.17), non-finite results, timeouts. */
FBSDE_API int fbsde_diagnostics(const fbsde_problem *P, int32_t Q, const void *workspace,
                      fbsde_diag *out, fbsde_stream_t stream);

/* Philox4x32-10 (Salmon et al., SC'11) on n counters: ctr device [n][4],
   key device [2], out device [n][4].  Used to test the generator bit for bit. */
FBSDE_API int fbsde_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n,
                        fbsde_stream_t stream);

/* The standard normals xi_{s,k,j,i} of the Brownian paths of Eq. (2.7), exactly as
   the solver draws them (k = N: the end point W(T); 1 <= k < N: the bridge step to
   level k): particles j0..j0+nj-1 of level k of solve s, dimensions 0..d-1.  out: device [nj][d] of float (FBSDE_FP32) or
   double (FBSDE_FP64). */
FBSDE_API int fbsde_normals(uint64_t seed, uint32_t s, uint32_t k, uint32_t j0, int32_t nj, int32_t d,
                  int32_t precision, void *out, fbsde_stream_t stream);

/*
 * Plans: a solve, or a batch of heterogeneous solves (each Algorithm 1 on its own problem,
 * query points and cloud; the batching itself has no counterpart in the paper), captured
 * once into a CUDA graph and replayed with one launch.  Each CG loop is a conditional while node whose body
 * (product, reduction, CG step, convergence check) repeats on the device until every
 * query of that instance has converged, so no empty iterations are launched.  Instances
 * are spread over parallel graph branches and run concurrently on the GPU.  The
 * pointers of every instance are bound at creation: refill x0 in place and launch again.
 */
typedef struct fbsde_plan fbsde_plan;

typedef struct {
    fbsde_problem problem;   /* the instance's problem (theta: device pointer)          */
    int32_t Q;               /* query points of the instance                            */
    uint32_t solve_index0;   /* Philox solve index of its first query                   */
    uint64_t seed;           /* Philox key                                              */
    const double *x0;        /* device [Q][d]                                           */
    double *u0;              /* device [Q]                                              */
    double *grad_u0;         /* device [Q][d] or NULL                                   */
} fbsde_instance;

/* Device workspace bytes of a plan over n instances (their workspaces, 256-aligned). */
FBSDE_API size_t fbsde_plan_workspace_bytes(int32_t n, const fbsde_instance *inst);

/* Captures the instances into a graph (branches <= 0: min(n, 32) parallel branches) and
   instantiates it.  The workspace must stay allocated while the plan exists.  Returns
   FBSDE_ERR_ARG / FBSDE_ERR_WORKSPACE for bad arguments, FBSDE_ERR_CUDA if capture or
   instantiation fails; *plan is NULL on error. */
FBSDE_API int fbsde_plan_create(fbsde_plan **plan, int32_t n, const fbsde_instance *inst,
                                int32_t branches, void *workspace, size_t workspace_bytes);
/* One graph launch on the stream (asynchronous). */
FBSDE_API int fbsde_plan_launch(fbsde_plan *plan, fbsde_stream_t stream);
/* Synchronises the stream and reads the device status of every instance of the plan. */
FBSDE_API int fbsde_plan_diagnostics(fbsde_plan *plan, fbsde_diag *out, fbsde_stream_t stream);
/* The same for instance `index` (0-based, in creation order) alone. */
FBSDE_API int fbsde_plan_instance_diagnostics(fbsde_plan *plan, int32_t index, fbsde_diag *out,
                                              fbsde_stream_t stream);
FBSDE_API void fbsde_plan_destroy(fbsde_plan *plan);

/* Kernel families of the solve, for the profiler below. */
typedef enum {
    FBSDE_K_SETUP = 0,      /* per-query set-up                                          */
    FBSDE_K_FORWARD = 1,    /* forward sweep (2.7) of the particle rows                  */
    FBSDE_K_UPDATE = 2,     /* level update: reverse step of the particle rows           */
    FBSDE_K_MATVEC = 3,     /* matrix-free product of the regression (Sec. 2.4, Steps 1-2)*/
    FBSDE_K_MOMENTS = 4,    /* weighted moments of the regression (streaming)            */
    FBSDE_K_REDUCE = 5,     /* fixed-order FP64 sum of per-CTA partial vectors           */
    FBSDE_K_CG_STEP = 6,    /* per-query CG vector update                                */
    FBSDE_K_CG_POST = 7,    /* intercept, Z, outputs                                     */
    FBSDE_K_TRACE = 8,      /* trace copies                                              */
    FBSDE_K_PARTICLES = 9,  /* per-particle terminal value / prediction + Newton, weights*/
    FBSDE_K_FINALIZE = 10,  /* per-query regression set-up from the moments              */
    FBSDE_K_ADJOINT = 11,   /* reverse-sweep kernels other than the shared ones above    */
    FBSDE_K_STEP = 12,      /* fused level step of the FP32 path (d <= 10240): reverse step
                               of the rows, Newton (2.16)-(2.17), weights and moments in
                               one pass; the forward sweep's end point at k = N          */
    FBSDE_NUM_KERNELS = 13
} fbsde_kernel_family;

typedef struct {
    int64_t launches;  /* kernel launches of this family since fbsde_profile_start    */
    int64_t timed;     /* launches bracketed by CUDA events                           */
    double total_ms;   /* summed event time of the timed launches                     */
} fbsde_kernel_stats;

/* Process-wide launch profiler (measurement of the kernels above; no counterpart in the
   paper; off by default; not for concurrent solves from several host threads).  After fbsde_profile_start(n), every launch is counted and the first
   n launches are bracketed by CUDA events recorded on the launching stream.
   fbsde_profile_stop() waits for the recorded events, fills out[FBSDE_NUM_KERNELS]
   and switches the profiler off.  fbsde_profile_select(mask) restricts the timing to
   the families whose bit (1u << family) is set (all of them by default, and again after
   each fbsde_profile_stop); launches of the other families are still counted.  Each
   timed launch adds two event records to its stream, so timing only the family of
   interest keeps the profiler's own cost out of the rest of the step.  ERR_ARG for a
   mask with no valid family bit. */
/* How the eager entry points (fbsde_solve, fbsde_solve_host, fbsde_adjoint) launch the
   passes of a CG loop (fbsde_solve_noalloc always launches every pass, up to cg_max_iter,
   one by one on the stream, so that it creates no CUDA graph): while the profiler times the product
   family, the first FBSDE_PROFILED_EAGER_PASSES passes of every loop are launched one by
   one (each product launch bracketed by events; kernels of converged queries exit at
   once) and any further passes run in a cached CUDA graph whose conditional while loop
   stops when every query has converged.  Otherwise every pass runs in that graph.  On a
   stream that is being captured every pass is launched one by one, up to cg_max_iter.
   The results are the same bit for bit in every case. */
#define FBSDE_PROFILED_EAGER_PASSES 48
FBSDE_API int fbsde_profile_start(int32_t max_timed_launches);
FBSDE_API int fbsde_profile_select(uint32_t family_mask);
FBSDE_API int fbsde_profile_stop(fbsde_kernel_stats *out);
/* Name of a kernel family ("matvec", ...); "unknown" outside the enum. */
FBSDE_API const char *fbsde_kernel_name(int family);

/* Utilities without a counterpart in the paper: a static description of a status code
   (never NULL), and FBSDE_ABI_VERSION of the loaded library. */
FBSDE_API const char *fbsde_status_string(int status);
/* Check of the library's bounded device waits (no counterpart in the paper): every wait of
 * the kernels on an mbarrier gives up after a time limit, records FBSDE_ERR_TIMEOUT in the
 * solve's status and lets the kernel finish, so that a broken pipeline never hangs the
 * device.  This launches one warp that waits, with limit_ns, on an mbarrier that nothing
 * arrives on, and synchronises the stream.
 *   limit_ns   1 .. 10^9 nanoseconds, else FBSDE_ERR_ARG
 *   scratch    device, 16 bytes, 8-byte aligned, caller-owned (NULL: FBSDE_ERR_ARG)
 *   waited_ns  host, may be NULL: the time the wait took
 * Returns FBSDE_ERR_TIMEOUT when the wait gave up as designed (the expected result),
 * FBSDE_OK if it did not, FBSDE_ERR_CUDA if the launch or the copy failed. */
FBSDE_API int fbsde_check_bounded_wait(int64_t limit_ns, void *scratch, int64_t *waited_ns,
                                       fbsde_stream_t stream);

FBSDE_API int fbsde_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FBSDE_H */
