/*
 * fbsde_oracle.c -- FP64 CPU oracle of the localized stochastic FBSDE scheme of
 * Fang, Sheng, Su and Zhou, "A derivative-free localized stochastic method for
 * very high dimensional semilinear parabolic PDEs" (arXiv 2510.02635).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference for the CUDA
 * library.  Only the tests, the smoke check and the benchmark's CPU-baseline arm
 * may build, load or call it; the product path never does, and it shares no code,
 * header, table or helper with the CUDA sources.
 *
 * Style: plain and slow on purpose.  FP64 everywhere.  Every sum over particles
 * runs over j = 0..M-1 in order and every sum over dimensions over i = 0..d-1 in
 * order.  OpenMP only splits independent outputs (particles, or output elements)
 * between threads, so the results do not depend on the number of threads.
 *
 * What it computes (one solve = one query point x0):
 *   problem  (2.1): d_t u + 1/2 sigma^2 Lap u + f(t,x,u,sigma grad u) = 0, u(T,.) = g,
 *            with drift mu = 0 and a constant scalar diffusion sigma (all problems
 *            below), so the anchor of every regression is a_k = x0.
 *   grid     (Sec. 2.2): dt = T/N, t_k = k dt.
 *   forward  (2.7), Algorithm 1: X_0^j = x0, X_{k+1}^j = X_k^j + sigma dW_k^j, so with
 *            mu = 0 the increments telescope to X_N^j = x0 + sigma W^j(T);
 *            Y_N^j = g(X_N^j).  The Brownian path W^j at the grid times is drawn
 *            backwards from its end point by the Brownian bridge (Levy's construction;
 *            Glasserman, Monte Carlo Methods in Financial Engineering, 2004, Sec. 3.1):
 *              W(T) = sqrt(T) xi_{s,N,j},
 *              W(t_k) = (t_k/t_{k+1}) W(t_{k+1}) + sqrt(t_k dt / t_{k+1}) xi_{s,k,j},
 *            k = N-1..1, W(0) = 0.  Its increments W(t_{k+1}) - W(t_k) are independent
 *            N(0, dt I), the law (2.7) gives dW_k, so the estimator is the same random
 *            variable in law as with increments drawn in forward order.
 *   backward (2.6)/(2.8), Algorithm 1, for k = N-1..0:
 *            weighted local linear regression (2.10)-(2.15) of Y_{k+1}^j on
 *            D_j = X_{k+1}^j - a_k with Gaussian kernel weights (2.11), Remark 2.3,
 *            and the ridge of Remark 2.2, solved by conjugate gradients on the
 *            Schur complement of (2.15) (Lemma 3.7, Eqs. 3.19-3.20);
 *            Z_k = sigma^T alpha_x (Algorithm 1);
 *            E_hat_j = alpha + alpha_x . (X_k^j - a_k) (local affine model (2.9));
 *            Newton (2.16)-(2.17) on F(Y) = Y - E_hat_j - dt f(t_k, X_k^j, Y, Z_k).
 *   output   u(0,x0) = (1/M) sum_j Y_0^j, grad u(0,x0) = alpha_x at k = 0.
 *
 * Readings where the paper is silent or inconsistent (kept identical on the GPU):
 *   - one anchor per solve and level (the drift path of x0), so a level costs
 *     O(M d) as the paper states for its per-step cost;
 *   - D_j = X_{k+1}^j - a_k (next-level position minus the anchor) and the
 *     conditional expectation for particle j is the local affine prediction;
 *   - F(Y) = Y - E_hat - dt f (the sign that makes F = 0 the update of (2.8));
 *   - Newton starts at E_hat, stops when |dY| <= newton_tol * max(1,|Y|);
 *   - kernel K(r) = exp(-r^2) with eps_k^2 = h^2 E||D||^2, E||D||^2 = sigma^2 d t_{k+1},
 *     weights normalised to sum 1 and shifted by E||D||^2 (the shift cancels in the
 *     normalisation); h <= 0 or h = inf gives uniform weights;
 *   - ridge lambda = ridge_rel * tr(Gamma_c)/d on the slope only;
 *   - unpreconditioned CG from zero, stopping at ||r|| <= cg_tol ||rhs||;
 *   - X_0^j = x0 exactly at k = 0 (Algorithm 1 starts every path at x);
 *   - the backward sweep recovers X_k from X_{k+1} by the bridge step above,
 *     X_k = x0 + (t_k/t_{k+1}) (X_{k+1} - x0) + sigma sqrt(t_k dt / t_{k+1}) xi_{s,k,j}:
 *     nothing per level is stored, and the forward sweep draws one normal per
 *     dimension instead of N.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11) with counter (q, j, k, s), key (seed lo,
 * seed hi); each 32-bit word x gives u = ((x >> 9) + 0.5) 2^-23 in (0,1); the
 * Box-Muller transform (Box and Muller, 1958) turns word pairs (0,1) and (2,3) into
 * the normals of dimensions 4q..4q+3.
 */
#define _POSIX_C_SOURCE 199309L
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

enum {
    ORC_OK = 0,
    ORC_ERR_ARG = 1,
    ORC_ERR_NEWTON = 4,
    ORC_ERR_CG = 5,
    ORC_ERR_NONFINITE = 7,
    ORC_ERR_NOMEM = 8
};

/* Problem kinds (all with mu = 0 and constant scalar sigma). */
enum {
    ORC_AC_MANUFACTURED = 0, /* f = y - y^3 + q(t,x), u* = e^{t-T} (1/d) sum cos x_i       */
    ORC_LOGISTIC_GRAD = 1,   /* f = (y - (2+d)/(2d)) sum_i z_i, g = logistic(T + sum x/d)   */
    ORC_HJB_LOGQUAD = 2,     /* f = -|z|^2/2, g = log((1 + sum theta_i x_i^2)/2)            */
    ORC_AFFINE_TEST = 3,     /* f = c0 + c1 y + c2 sum z_i + c3 t, g = A + sum theta_i x_i  */
    ORC_CUBIC_TEST = 4,      /* f = y - y^3, g = A                                          */
    ORC_AC_DOUBLEWELL = 5,   /* f = y - y^3, g = 1/(2 + 0.4 |x|^2)  (Sec. 4.1, case 1)      */
    ORC_COS_LINEAR_TEST = 6  /* f = c0 + c1 y, g = (1/d) sum cos x_i                        */
};

typedef struct {
    int32_t kind;
    int32_t d;
    double sigma;
    double T;
    int32_t N;
    int32_t cg_max_iter;
    int64_t M;
    const double *theta; /* d coefficients for kinds 2 and 3, else NULL */
    double A, c0, c1, c2, c3; /* scalar parameters of the test kinds */
    double h;            /* kernel bandwidth factor; <= 0 or inf: uniform weights */
    double ridge_rel;
    double cg_tol;
    double newton_tol;
    int32_t newton_max_iter;
    int32_t pad_;
} orc_problem;

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (SC'11): round = two 32x32->64 products, xor with the other   */
/* two words and the key; key bumped by the Weyl constants between rounds.    */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* 32-bit word -> uniform on (0,1): ((x >> 9) + 1/2) * 2^-23 (exact in binary32). */
double orc_uniform(uint32_t x)
{
    return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Standard normals xi_{s,k,j,i}, i = 0..d-1, of particle j at level k of solve s. */
void orc_normals(uint64_t seed, uint32_t s, uint32_t k, uint32_t j, int32_t d, double *xi)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int32_t q = 0; 4 * q < d; ++q) {
        uint32_t ctr[4] = {(uint32_t)q, j, k, s}, w[4];
        orc_philox4x32_10(ctr, key, w);
        double r0 = sqrt(-2.0 * log(orc_uniform(w[0])));
        double a0 = 2.0 * M_PI * orc_uniform(w[1]);
        double r1 = sqrt(-2.0 * log(orc_uniform(w[2])));
        double a1 = 2.0 * M_PI * orc_uniform(w[3]);
        double z[4] = {r0 * cos(a0), r0 * sin(a0), r1 * cos(a1), r1 * sin(a1)};
        for (int m = 0; m < 4 && 4 * q + m < d; ++m)
            xi[4 * q + m] = z[m];
    }
}

/*
 * Particle positions of the Brownian path of (2.7) with mu = 0, drawn backwards by the
 * Brownian bridge (Levy's construction; Glasserman 2004, Sec. 3.1).  With W(0) = 0 the
 * conditional law of W(t_k) given W(t_{k+1}) is
 *   N((t_k/t_{k+1}) W(t_{k+1}), t_k (t_{k+1} - t_k)/t_{k+1} I),
 * so on positions X = x0 + sigma W:
 *   path_end:  X_N = x0 + sigma sqrt(T) xi_{s,N,j};
 *   path_step: X_k = x0 + (k/(k+1)) (X_{k+1} - x0) + sigma sqrt(dt k/(k+1)) xi_{s,k,j},
 *              1 <= k < N, and X_0 = x0 (k = 0).
 * xi is scratch of d doubles; Xk may alias Xn.
 */
static void path_end(const orc_problem *P, const double *x0, uint64_t seed, uint32_t s,
                     int64_t j, double *XN, double *xi)
{
    const int d = P->d;
    const double sT = P->sigma * sqrt(P->T);
    orc_normals(seed, s, (uint32_t)P->N, (uint32_t)j, d, xi);
    for (int i = 0; i < d; ++i) XN[i] = x0[i] + sT * xi[i];
}

static void path_step(const orc_problem *P, int k, const double *x0, uint64_t seed, uint32_t s,
                      int64_t j, const double *Xn, double *Xk, double *xi)
{
    const int d = P->d;
    if (k == 0) {
        for (int i = 0; i < d; ++i) Xk[i] = x0[i];
        return;
    }
    const double dt = P->T / P->N;
    const double ca = (double)k / (double)(k + 1);
    const double cb = P->sigma * sqrt(dt * (double)k / (double)(k + 1));
    orc_normals(seed, s, (uint32_t)k, (uint32_t)j, d, xi);
    for (int i = 0; i < d; ++i) Xk[i] = x0[i] + ca * (Xn[i] - x0[i]) + cb * xi[i];
}

/* The whole path X_0..X_N of particle j (out[(N+1) d], level-major), by the two steps
 * that orc_solve and orc_adjoint use. */
int orc_path(const orc_problem *P, const double *x0, uint64_t seed, uint32_t s, int64_t j,
             double *out)
{
    const int d = P->d, N = P->N;
    if (d < 1 || N < 1 || !(P->T > 0.0) || !(P->sigma > 0.0) || j < 0) return ORC_ERR_ARG;
    double *xi = (double *)malloc(sizeof(double) * d);
    if (!xi) return ORC_ERR_NOMEM;
    path_end(P, x0, seed, s, j, out + (size_t)N * d, xi);
    for (int k = N - 1; k >= 0; --k)
        path_step(P, k, x0, seed, s, j, out + (size_t)(k + 1) * d, out + (size_t)k * d, xi);
    free(xi);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Problem table: terminal condition g and driver f of (2.1).                 */
/* ------------------------------------------------------------------------- */
double orc_g(const orc_problem *P, const double *x)
{
    const int d = P->d;
    double s = 0.0;
    switch (P->kind) {
    case ORC_AC_MANUFACTURED:
    case ORC_COS_LINEAR_TEST:
        for (int i = 0; i < d; ++i) s += cos(x[i]);
        return s / d;
    case ORC_LOGISTIC_GRAD:
        for (int i = 0; i < d; ++i) s += x[i];
        return 1.0 / (1.0 + exp(-(P->T + s / d)));
    case ORC_HJB_LOGQUAD:
        for (int i = 0; i < d; ++i) s += P->theta[i] * x[i] * x[i];
        return log(0.5 * (1.0 + s));
    case ORC_AFFINE_TEST:
        for (int i = 0; i < d; ++i) s += P->theta[i] * x[i];
        return P->A + s;
    case ORC_CUBIC_TEST:
        return P->A;
    case ORC_AC_DOUBLEWELL:
        for (int i = 0; i < d; ++i) s += x[i] * x[i];
        return 1.0 / (2.0 + 0.4 * s);
    }
    return NAN;
}

/* The part of f that depends on (t, x, z) and not on y, as one scalar:
 *   AC_MANUFACTURED: q(t,x) = u*^3 - (2 - sigma^2/2) u*,  u* = e^{t-T} (1/d) sum cos x_i
 *   LOGISTIC_GRAD:   sum_i z_i
 *   HJB_LOGQUAD:     |z|^2
 *   AFFINE_TEST:     c2 sum_i z_i + c3 t
 *   others:          0                                                        */
double orc_f_feature(const orc_problem *P, double t, const double *x, const double *z)
{
    const int d = P->d;
    double s = 0.0;
    switch (P->kind) {
    case ORC_AC_MANUFACTURED: {
        for (int i = 0; i < d; ++i) s += cos(x[i]);
        double us = exp(t - P->T) * s / d;
        return us * us * us - (2.0 - 0.5 * P->sigma * P->sigma) * us;
    }
    case ORC_LOGISTIC_GRAD:
        for (int i = 0; i < d; ++i) s += z[i];
        return s;
    case ORC_HJB_LOGQUAD:
        for (int i = 0; i < d; ++i) s += z[i] * z[i];
        return s;
    case ORC_AFFINE_TEST:
        for (int i = 0; i < d; ++i) s += z[i];
        return P->c2 * s + P->c3 * t;
    }
    return 0.0;
}

/* f(t,x,y,z) given the feature above; *dfdy receives the partial derivative in y. */
double orc_f_scalar(const orc_problem *P, double feature, double y, double *dfdy)
{
    switch (P->kind) {
    case ORC_AC_MANUFACTURED:
        *dfdy = 1.0 - 3.0 * y * y;
        return y - y * y * y + feature;
    case ORC_LOGISTIC_GRAD:
        *dfdy = feature;
        return (y - (2.0 + P->d) / (2.0 * P->d)) * feature;
    case ORC_HJB_LOGQUAD:
        *dfdy = 0.0;
        return -0.5 * feature;
    case ORC_AFFINE_TEST:
        *dfdy = P->c1;
        return P->c0 + P->c1 * y + feature;
    case ORC_COS_LINEAR_TEST:
        *dfdy = P->c1;
        return P->c0 + P->c1 * y;
    case ORC_CUBIC_TEST:
    case ORC_AC_DOUBLEWELL:
        *dfdy = 1.0 - 3.0 * y * y;
        return y - y * y * y;
    }
    *dfdy = NAN;
    return NAN;
}

double orc_f(const orc_problem *P, double t, const double *x, double y, const double *z, double *dfdy)
{
    return orc_f_scalar(P, orc_f_feature(P, t, x, z), y, dfdy);
}

/* Newton iteration (2.17) on F(Y) = Y - E_hat - dt f (2.16), started at E_hat.
 * Returns the root; *iters = iterations used, or -1 when newton_max_iter ran out. */
double orc_newton(const orc_problem *P, double E_hat, double dt, double feature, int *iters)
{
    double y = E_hat;
    for (int n = 1; n <= P->newton_max_iter; ++n) {
        double dfdy, f = orc_f_scalar(P, feature, y, &dfdy);
        double F = y - E_hat - dt * f;
        double dF = 1.0 - dt * dfdy;
        double dy = F / dF;
        y -= dy;
        if (fabs(dy) <= P->newton_tol * fmax(1.0, fabs(y))) {
            *iters = n;
            return y;
        }
    }
    *iters = -1;
    return y;
}

/* ------------------------------------------------------------------------- */
/* One weighted local linear regression (2.10)-(2.15) with ridge (Remark 2.2).  */
/* ------------------------------------------------------------------------- */

/* q = (Gamma_c + lambda I) v,  Gamma_c v = sum_j w_j (D_j . v) D_j - S (S . v):
 * the two matrix-free products of Sec. 2.4 (Step 1: t_j = D_j . v; Step 2:
 * sum_j w_j t_j D_j) on the centred (Schur-complement) operator. */
static void gamma_c_apply(int d, int64_t M, const double *D, const double *w, const double *S,
                          double lambda, const double *v, double *t, double *q)
{
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < M; ++j) {
        const double *Dj = D + j * (int64_t)d;
        double s = 0.0;
        for (int i = 0; i < d; ++i) s += Dj[i] * v[i];
        t[j] = s;
    }
    double sv = 0.0;
    for (int i = 0; i < d; ++i) sv += S[i] * v[i];
#pragma omp parallel
    {
        int nt = 1, id = 0;
#ifdef _OPENMP
        nt = omp_get_num_threads();
        id = omp_get_thread_num();
#endif
        int i0 = (int)((int64_t)d * id / nt), i1 = (int)((int64_t)d * (id + 1) / nt);
        for (int i = i0; i < i1; ++i) q[i] = 0.0;
        /* for every output element q_i the terms are added in particle order j */
        for (int64_t j = 0; j < M; ++j) {
            const double *Dj = D + j * (int64_t)d;
            double c = w[j] * t[j];
            for (int i = i0; i < i1; ++i) q[i] += c * Dj[i];
        }
        for (int i = i0; i < i1; ++i) q[i] += -S[i] * sv + lambda * v[i];
    }
}

static double dotd(int d, const double *a, const double *b)
{
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += a[i] * b[i];
    return s;
}

/* sum_j c_j D_j (a d-vector) with each element summed in particle order. */
static void weighted_row_sum(int d, int64_t M, const double *D, const double *c, double *out)
{
#pragma omp parallel
    {
        int nt = 1, id = 0;
#ifdef _OPENMP
        nt = omp_get_num_threads();
        id = omp_get_thread_num();
#endif
        int i0 = (int)((int64_t)d * id / nt), i1 = (int)((int64_t)d * (id + 1) / nt);
        for (int i = i0; i < i1; ++i) out[i] = 0.0;
        for (int64_t j = 0; j < M; ++j) {
            const double *Dj = D + j * (int64_t)d;
            for (int i = i0; i < i1; ++i) out[i] += c[j] * Dj[i];
        }
    }
}

/*
 * Weighted local linear regression of Y_{k+1}^j on D_j.
 *   rho_j = |D_j|^2, w_j = exp(-(rho_j - rho_ref)/(h^2 rho_ref)) / sum  (2.11), Remark 2.3
 *   c = sum w_j Y_j, S = sum w_j D_j, b = sum w_j Y_j D_j        (moments of Lemma 3.7)
 *   (Gamma - S S^T + lambda I) alpha_x = b - c S                  (3.19) with ridge
 *   alpha = c - S . alpha_x                                        (3.20), S_0 = 1
 * Outputs alpha, alpha_x (d), optionally w (M) and the CG iteration count.
 * Returns ORC_OK, or ORC_ERR_CG when cg_max_iter ran out (alpha_x is then the last
 * iterate).
 */
int orc_llr(int32_t d, int64_t M, const double *D, const double *Y, double rho_ref, double h,
            double ridge_rel, double cg_tol, int32_t cg_max_iter, double *alpha, double *alpha_x,
            double *w_out, int32_t *cg_iters)
{
    if (d < 1 || M < 2) return ORC_ERR_ARG;
    double *w = (double *)malloc(sizeof(double) * M);
    double *wy = (double *)malloc(sizeof(double) * M);
    double *t = (double *)malloc(sizeof(double) * M);
    double *vec = (double *)malloc(sizeof(double) * 6 * (size_t)d);
    if (!w || !wy || !t || !vec) {
        free(w); free(wy); free(t); free(vec);
        return ORC_ERR_NOMEM;
    }
    double *S = vec, *b = vec + d, *r = vec + 2 * d, *p = vec + 3 * d, *q = vec + 4 * d,
           *rhs = vec + 5 * d;
    const int uniform = !(h > 0.0) || isinf(h);
    const double eps2 = h * h * rho_ref;

#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < M; ++j) {
        const double *Dj = D + j * (int64_t)d;
        double rho = 0.0;
        for (int i = 0; i < d; ++i) rho += Dj[i] * Dj[i];
        w[j] = uniform ? 1.0 : exp(-(rho - rho_ref) / eps2);
        t[j] = rho;
    }
    double W = 0.0;
    for (int64_t j = 0; j < M; ++j) W += w[j];
    for (int64_t j = 0; j < M; ++j) w[j] /= W;
    double c = 0.0, wrho = 0.0;
    for (int64_t j = 0; j < M; ++j) {
        c += w[j] * Y[j];
        wrho += w[j] * t[j];
    }
    for (int64_t j = 0; j < M; ++j) wy[j] = w[j] * Y[j];
    weighted_row_sum(d, M, D, w, S);
    weighted_row_sum(d, M, D, wy, b);
    const double trace = wrho - dotd(d, S, S);
    const double lambda = ridge_rel * trace / d;
    for (int i = 0; i < d; ++i) rhs[i] = b[i] - c * S[i];

    /* conjugate gradients from alpha_x = 0 */
    for (int i = 0; i < d; ++i) {
        alpha_x[i] = 0.0;
        r[i] = rhs[i];
        p[i] = rhs[i];
    }
    double rr = dotd(d, r, r);
    const double stop = cg_tol * sqrt(dotd(d, rhs, rhs));
    int it = 0, status = ORC_OK;
    while (sqrt(rr) > stop) {
        if (it >= cg_max_iter) {
            status = ORC_ERR_CG;
            break;
        }
        gamma_c_apply(d, M, D, w, S, lambda, p, t, q);
        double a = rr / dotd(d, p, q);
        for (int i = 0; i < d; ++i) {
            alpha_x[i] += a * p[i];
            r[i] -= a * q[i];
        }
        double rr_new = dotd(d, r, r);
        double beta = rr_new / rr;
        for (int i = 0; i < d; ++i) p[i] = r[i] + beta * p[i];
        rr = rr_new;
        ++it;
    }
    *alpha = c - dotd(d, S, alpha_x);
    if (cg_iters) *cg_iters = it;
    if (w_out) memcpy(w_out, w, sizeof(double) * M);
    free(w); free(wy); free(t); free(vec);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1 for one query point.                                           */
/* ------------------------------------------------------------------------- */

/*
 * Runs the forward sweep and the backward levels k = N-1, ..., N-max_levels
 * (max_levels = N: the whole method).  Outputs (any may be NULL):
 *   u0, grad_u0[d]     u(0,x0) and grad u(0,x0) (only when max_levels == N)
 *   alpha_lv[N]        intercept alpha of the regression at level k (index k)
 *   alphax_lv[N*d]     slope alpha_x at level k (row k)
 *   cg_iters_lv[N]     CG iterations at level k
 *   newton_lv[N]       most Newton iterations any particle needed at level k
 *   xN[M*d], yN[M]     X_N^j and Y_N^j = g(X_N^j) after the forward sweep
 *   y_lv[(N+1)*M]      Y_k^j for every level reached (row k)
 *   phase_s[2]         wall seconds of the forward sweep and of the backward levels run
 * Returns ORC_OK or the first error met (NEWTON, CG, NONFINITE); on NEWTON/CG the
 * sweep still runs to the end with the last iterates.
 */
int orc_solve(const orc_problem *P, const double *x0, uint64_t seed, uint32_t solve_index,
              int32_t max_levels, double *u0, double *grad_u0, double *alpha_lv,
              double *alphax_lv, int32_t *cg_iters_lv, int32_t *newton_lv, double *xN,
              double *yN, double *y_lv, double *phase_s)
{
    const int d = P->d, N = P->N;
    const int64_t M = P->M;
    if (d < 1 || N < 1 || M < 2 || !(P->T > 0.0) || !(P->sigma > 0.0) || max_levels < 0 ||
        max_levels > N)
        return ORC_ERR_ARG;
    if ((P->kind == ORC_HJB_LOGQUAD || P->kind == ORC_AFFINE_TEST) && !P->theta)
        return ORC_ERR_ARG;
    const double dt = P->T / N;
    const size_t Md = (size_t)M * (size_t)d;

    double *X = (double *)malloc(sizeof(double) * Md);
    double *D = (double *)malloc(sizeof(double) * Md);
    double *Y = (double *)malloc(sizeof(double) * M);
    double *ax = (double *)malloc(sizeof(double) * d);
    double *z = (double *)malloc(sizeof(double) * d);
    int *nit = (int *)malloc(sizeof(int) * M);
    int nthreads = 1;
#ifdef _OPENMP
    nthreads = omp_get_max_threads();
#endif
    double *xi_all = (double *)malloc(sizeof(double) * (size_t)d * nthreads);
    if (!X || !D || !Y || !ax || !z || !nit || !xi_all) {
        free(X); free(D); free(Y); free(ax); free(z); free(nit); free(xi_all);
        return ORC_ERR_NOMEM;
    }
    int status = ORC_OK;
    struct timespec tw0, tw1, tw2;
    clock_gettime(CLOCK_MONOTONIC, &tw0);

    /* forward sweep (2.7) with mu = 0: X_N = x0 + sigma W(T), W(T) = sqrt(T) xi_N */
#pragma omp parallel
    {
        int id = 0;
#ifdef _OPENMP
        id = omp_get_thread_num();
#endif
        double *xi = xi_all + (size_t)id * d;
#pragma omp for schedule(static)
        for (int64_t j = 0; j < M; ++j) {
            double *Xj = X + j * (int64_t)d;
            path_end(P, x0, seed, solve_index, j, Xj, xi);
            Y[j] = orc_g(P, Xj); /* terminal condition, Algorithm 1 */
        }
    }
    if (xN) memcpy(xN, X, sizeof(double) * Md);
    if (yN) memcpy(yN, Y, sizeof(double) * M);
    if (y_lv) memcpy(y_lv + (size_t)N * M, Y, sizeof(double) * M);
    clock_gettime(CLOCK_MONOTONIC, &tw1);

    for (int k = N - 1; k >= N - max_levels; --k) {
        const double t_k = k * dt, t_k1 = (k + 1) * dt;
        /* regression at level k on D_j = X_{k+1}^j - a_k, a_k = x0 */
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < M; ++j)
            for (int i = 0; i < d; ++i) D[j * (int64_t)d + i] = X[j * (int64_t)d + i] - x0[i];
        const double rho_ref = P->sigma * P->sigma * d * t_k1; /* E|D_j|^2 */
        double alpha;
        int cg_it = 0;
        int st = orc_llr(d, M, D, Y, rho_ref, P->h, P->ridge_rel, P->cg_tol, P->cg_max_iter,
                         &alpha, ax, NULL, &cg_it);
        if (st == ORC_ERR_NOMEM || st == ORC_ERR_ARG) {
            status = st;
            break;
        }
        if (st != ORC_OK && status == ORC_OK) status = st;
        for (int i = 0; i < d; ++i) z[i] = P->sigma * ax[i]; /* Z_k = sigma^T alpha_x */
        if (alpha_lv) alpha_lv[k] = alpha;
        if (alphax_lv) memcpy(alphax_lv + (size_t)k * d, ax, sizeof(double) * d);
        if (cg_iters_lv) cg_iters_lv[k] = cg_it;

        /* particles back to level k, local affine prediction, Newton (2.16)-(2.17) */
#pragma omp parallel
        {
            int id = 0;
#ifdef _OPENMP
            id = omp_get_thread_num();
#endif
            double *xi = xi_all + (size_t)id * d;
#pragma omp for schedule(static)
            for (int64_t j = 0; j < M; ++j) {
                double *Xj = X + j * (int64_t)d;
                path_step(P, k, x0, seed, solve_index, j, Xj, Xj, xi); /* X_k from X_{k+1} */
                double pred = alpha;
                for (int i = 0; i < d; ++i) pred += ax[i] * (Xj[i] - x0[i]);
                double feat = orc_f_feature(P, t_k, Xj, z);
                Y[j] = orc_newton(P, pred, dt, feat, &nit[j]);
            }
        }
        int nmax = 0;
        for (int64_t j = 0; j < M; ++j) {
            if (nit[j] < 0) {
                if (status == ORC_OK) status = ORC_ERR_NEWTON;
                nmax = P->newton_max_iter;
            } else if (nit[j] > nmax) {
                nmax = nit[j];
            }
        }
        if (newton_lv) newton_lv[k] = nmax;
        if (y_lv) memcpy(y_lv + (size_t)k * M, Y, sizeof(double) * M);
    }

    clock_gettime(CLOCK_MONOTONIC, &tw2);
    if (phase_s) {
        phase_s[0] = (tw1.tv_sec - tw0.tv_sec) + 1e-9 * (tw1.tv_nsec - tw0.tv_nsec);
        phase_s[1] = (tw2.tv_sec - tw1.tv_sec) + 1e-9 * (tw2.tv_nsec - tw1.tv_nsec);
    }
    if (max_levels == N && status != ORC_ERR_NOMEM && status != ORC_ERR_ARG) {
        double s = 0.0;
        for (int64_t j = 0; j < M; ++j) s += Y[j];
        if (u0) *u0 = s / M; /* Y_0 = (1/M) sum_m Y_0^m, Algorithm 1 */
        if (grad_u0) memcpy(grad_u0, ax, sizeof(double) * d);
        if (!isfinite(s / M) && status == ORC_OK) status = ORC_ERR_NONFINITE;
    } else {
        if (u0) *u0 = NAN;
    }
    free(X); free(D); free(Y); free(ax); free(z); free(nit); free(xi_all);
    return status;
}

/*
 * Algorithm 1 in its literal form: one regression per particle anchor.  At level k the
 * anchor of particle m is its own position X_k^m (Algorithm 1's backward loop over m;
 * the local linear approximation (2.9) centred at X_k^m), and
 *   D_j^m = X_{k+1}^j - X_k^m   (next-level positions minus the anchor, as in R2),
 *   Gaussian weights (2.11), Remark 2.3, with eps_k^2 = h^2 E|D^m|^2,
 *     E|D^m|^2 = sigma^2 d (t_k + t_{k+1})   (two independent paths from x0),
 *   the ridge regression of Y_{k+1}^j on D^m (Eqs. 3.19-3.20, Remark 2.2) -> alpha^m,
 *   alpha_x^m; Z_k^m = sigma alpha_x^m; the local model at the anchor, E_hat_m = alpha^m;
 *   Newton (2.16)-(2.17): Y_k^m = alpha^m + dt f(t_k, X_k^m, Y_k^m, Z_k^m).
 * u(0,x0) = (1/M) sum_m Y_0^m; at k = 0 every anchor is x0, so every regression is the
 * same and grad u(0,x0) = alpha_x^1 of level 0.  With uniform weights (h = inf) the
 * regressions differ only by a shift of D, which leaves alpha_x unchanged and moves
 * alpha^m to alpha + alpha_x . (X_k^m - x0): the result is orc_solve's.
 * The particle paths are those of orc_solve (path_end, path_step).  Cost O(M^2 d) per
 * level (M regressions over M particles).  Outputs u0, grad_u0[d] (may be NULL).
 */
int orc_solve_anchored(const orc_problem *P, const double *x0, uint64_t seed,
                       uint32_t solve_index, double *u0, double *grad_u0)
{
    const int d = P->d, N = P->N;
    const int64_t M = P->M;
    if (d < 1 || N < 1 || M < 2 || !(P->T > 0.0) || !(P->sigma > 0.0)) return ORC_ERR_ARG;
    if ((P->kind == ORC_HJB_LOGQUAD || P->kind == ORC_AFFINE_TEST) && !P->theta)
        return ORC_ERR_ARG;
    const double dt = P->T / N;
    const size_t Md = (size_t)M * (size_t)d;
    double *Xn = (double *)malloc(sizeof(double) * Md);   /* X_{k+1} */
    double *Xk = (double *)malloc(sizeof(double) * Md);   /* X_k (the anchors) */
    double *D = (double *)malloc(sizeof(double) * Md);
    double *Y = (double *)malloc(sizeof(double) * M);
    double *Yk = (double *)malloc(sizeof(double) * M);
    double *ax = (double *)malloc(sizeof(double) * d);
    double *z = (double *)malloc(sizeof(double) * d);
    double *xi = (double *)malloc(sizeof(double) * d);
    int status = ORC_OK;
    if (!Xn || !Xk || !D || !Y || !Yk || !ax || !z || !xi) {
        status = ORC_ERR_NOMEM;
        goto done;
    }
    for (int64_t j = 0; j < M; ++j) {
        path_end(P, x0, seed, solve_index, j, Xn + j * (int64_t)d, xi);
        Y[j] = orc_g(P, Xn + j * (int64_t)d);   /* terminal condition, Algorithm 1 */
    }
    for (int k = N - 1; k >= 0; --k) {
        const double t_k = k * dt;
        for (int64_t j = 0; j < M; ++j)
            path_step(P, k, x0, seed, solve_index, j, Xn + j * (int64_t)d, Xk + j * (int64_t)d, xi);
        const double rho_ref = P->sigma * P->sigma * d * (t_k + (k + 1) * dt);
        for (int64_t m = 0; m < M; ++m) {
            const double *a = Xk + m * (int64_t)d;
            for (int64_t j = 0; j < M; ++j)
                for (int i = 0; i < d; ++i) D[j * (int64_t)d + i] = Xn[j * (int64_t)d + i] - a[i];
            double alpha;
            int cg_it = 0;
            const int st = orc_llr(d, M, D, Y, rho_ref, P->h, P->ridge_rel, P->cg_tol,
                                   P->cg_max_iter, &alpha, ax, NULL, &cg_it);
            if (st == ORC_ERR_NOMEM || st == ORC_ERR_ARG) {
                status = st;
                goto done;
            }
            if (st != ORC_OK && status == ORC_OK) status = st;
            for (int i = 0; i < d; ++i) z[i] = P->sigma * ax[i];   /* Z_k^m = sigma alpha_x^m */
            const double feat = orc_f_feature(P, t_k, a, z);
            int it;
            Yk[m] = orc_newton(P, alpha, dt, feat, &it);
            if (it < 0 && status == ORC_OK) status = ORC_ERR_NEWTON;
            if (k == 0 && m == 0 && grad_u0) memcpy(grad_u0, ax, sizeof(double) * d);
        }
        memcpy(Y, Yk, sizeof(double) * M);
        double *tmp = Xn;   /* level k's positions are the cloud of level k-1 */
        Xn = Xk;
        Xk = tmp;
    }
    {
        double s = 0.0;
        for (int64_t m = 0; m < M; ++m) s += Y[m];
        if (u0) *u0 = s / M;   /* Y_0 = (1/M) sum_m Y_0^m, Algorithm 1 */
        if (!isfinite(s / M) && status == ORC_OK) status = ORC_ERR_NONFINITE;
    }
done:
    free(Xn); free(Xk); free(D); free(Y); free(Yk); free(ax); free(z); free(xi);
    return status;
}

/*
 * Algorithm 1 with one regression per particle anchor over the anchor's K nearest
 * particles only (Remark 2.1: a small subset of the nearest particles instead of all of
 * them; the random-batch reading keeps the cost O(M K d) per level).  As
 * orc_solve_anchored, except that for anchor m the regression runs over the K indices j
 * with the smallest |X_{k+1}^j - X_k^m|^2, ties broken by the smaller j, with the Gaussian
 * weights normalised over that subset.  K = M is orc_solve_anchored.
 */
typedef struct {
    double rho;
    int64_t j;
} orc_nb;

static int nb_cmp(const void *a, const void *b)
{
    const orc_nb *x = (const orc_nb *)a, *y = (const orc_nb *)b;
    if (x->rho < y->rho) return -1;
    if (x->rho > y->rho) return 1;
    return x->j < y->j ? -1 : (x->j > y->j ? 1 : 0);
}

int orc_solve_neighbours(const orc_problem *P, int64_t K, const double *x0, uint64_t seed,
                         uint32_t solve_index, double *u0, double *grad_u0)
{
    const int d = P->d, N = P->N;
    const int64_t M = P->M;
    if (d < 1 || N < 1 || M < 2 || K < 2 || K > M || !(P->T > 0.0) || !(P->sigma > 0.0))
        return ORC_ERR_ARG;
    if ((P->kind == ORC_HJB_LOGQUAD || P->kind == ORC_AFFINE_TEST) && !P->theta)
        return ORC_ERR_ARG;
    const double dt = P->T / N;
    const size_t Md = (size_t)M * (size_t)d;
    double *Xn = (double *)malloc(sizeof(double) * Md);
    double *Xk = (double *)malloc(sizeof(double) * Md);
    double *D = (double *)malloc(sizeof(double) * (size_t)K * d);
    double *Ys = (double *)malloc(sizeof(double) * K);
    double *Y = (double *)malloc(sizeof(double) * M);
    double *Yk = (double *)malloc(sizeof(double) * M);
    double *ax = (double *)malloc(sizeof(double) * d);
    double *z = (double *)malloc(sizeof(double) * d);
    double *xi = (double *)malloc(sizeof(double) * d);
    orc_nb *nb = (orc_nb *)malloc(sizeof(orc_nb) * M);
    int status = ORC_OK;
    if (!Xn || !Xk || !D || !Ys || !Y || !Yk || !ax || !z || !xi || !nb) {
        status = ORC_ERR_NOMEM;
        goto done;
    }
    for (int64_t j = 0; j < M; ++j) {
        path_end(P, x0, seed, solve_index, j, Xn + j * (int64_t)d, xi);
        Y[j] = orc_g(P, Xn + j * (int64_t)d);
    }
    for (int k = N - 1; k >= 0; --k) {
        const double t_k = k * dt;
        for (int64_t j = 0; j < M; ++j)
            path_step(P, k, x0, seed, solve_index, j, Xn + j * (int64_t)d, Xk + j * (int64_t)d, xi);
        const double rho_ref = P->sigma * P->sigma * d * (t_k + (k + 1) * dt);
        for (int64_t m = 0; m < M; ++m) {
            const double *a = Xk + m * (int64_t)d;
            for (int64_t j = 0; j < M; ++j) {
                double rho = 0.0;
                for (int i = 0; i < d; ++i) {
                    const double e = Xn[j * (int64_t)d + i] - a[i];
                    rho += e * e;
                }
                nb[j].rho = rho;
                nb[j].j = j;
            }
            qsort(nb, (size_t)M, sizeof(orc_nb), nb_cmp);
            for (int64_t q = 0; q < K; ++q) {
                const int64_t j = nb[q].j;
                for (int i = 0; i < d; ++i) D[q * (int64_t)d + i] = Xn[j * (int64_t)d + i] - a[i];
                Ys[q] = Y[j];
            }
            double alpha;
            int cg_it = 0;
            const int st = orc_llr(d, K, D, Ys, rho_ref, P->h, P->ridge_rel, P->cg_tol,
                                   P->cg_max_iter, &alpha, ax, NULL, &cg_it);
            if (st == ORC_ERR_NOMEM || st == ORC_ERR_ARG) {
                status = st;
                goto done;
            }
            if (st != ORC_OK && status == ORC_OK) status = st;
            for (int i = 0; i < d; ++i) z[i] = P->sigma * ax[i];
            const double feat = orc_f_feature(P, t_k, a, z);
            int it;
            Yk[m] = orc_newton(P, alpha, dt, feat, &it);
            if (it < 0 && status == ORC_OK) status = ORC_ERR_NEWTON;
            if (k == 0 && m == 0 && grad_u0) memcpy(grad_u0, ax, sizeof(double) * d);
        }
        memcpy(Y, Yk, sizeof(double) * M);
        double *tmp = Xn;
        Xn = Xk;
        Xk = tmp;
    }
    {
        double s = 0.0;
        for (int64_t m = 0; m < M; ++m) s += Y[m];
        if (u0) *u0 = s / M;
        if (!isfinite(s / M) && status == ORC_OK) status = ORC_ERR_NONFINITE;
    }
done:
    free(Xn); free(Xk); free(D); free(Ys); free(Y); free(Yk); free(ax); free(z); free(xi);
    free(nb);
    return status;
}

/*
 * Algorithm 1 with one regression per particle anchor over a batch of K particles (the
 * random-batch reading of Remark 2.1, after Jin, Li and Liu 2020): for anchor m the batch
 * is the cyclic window j = (m + q) mod M, q = 0..K-1.  The window does not depend on the
 * positions, and the particle paths are independent and identically distributed, so its
 * K - 1 particles other than the anchor's own path (q = 0, always in the batch) are a
 * random sample of the cloud; the Gaussian weights are normalised over the batch.  K = M
 * is orc_solve_anchored up to the order of the sums.
 */
int orc_solve_batch(const orc_problem *P, int64_t K, const double *x0, uint64_t seed,
                    uint32_t solve_index, double *u0, double *grad_u0)
{
    const int d = P->d, N = P->N;
    const int64_t M = P->M;
    if (d < 1 || N < 1 || M < 2 || K < 2 || K > M || !(P->T > 0.0) || !(P->sigma > 0.0))
        return ORC_ERR_ARG;
    if ((P->kind == ORC_HJB_LOGQUAD || P->kind == ORC_AFFINE_TEST) && !P->theta)
        return ORC_ERR_ARG;
    const double dt = P->T / N;
    const size_t Md = (size_t)M * (size_t)d;
    double *Xn = (double *)malloc(sizeof(double) * Md);
    double *Xk = (double *)malloc(sizeof(double) * Md);
    double *D = (double *)malloc(sizeof(double) * (size_t)K * d);
    double *Ys = (double *)malloc(sizeof(double) * K);
    double *Y = (double *)malloc(sizeof(double) * M);
    double *Yk = (double *)malloc(sizeof(double) * M);
    double *ax = (double *)malloc(sizeof(double) * d);
    double *z = (double *)malloc(sizeof(double) * d);
    double *xi = (double *)malloc(sizeof(double) * d);
    int status = ORC_OK;
    if (!Xn || !Xk || !D || !Ys || !Y || !Yk || !ax || !z || !xi) {
        status = ORC_ERR_NOMEM;
        goto done;
    }
    for (int64_t j = 0; j < M; ++j) {
        path_end(P, x0, seed, solve_index, j, Xn + j * (int64_t)d, xi);
        Y[j] = orc_g(P, Xn + j * (int64_t)d);
    }
    for (int k = N - 1; k >= 0; --k) {
        const double t_k = k * dt;
        for (int64_t j = 0; j < M; ++j)
            path_step(P, k, x0, seed, solve_index, j, Xn + j * (int64_t)d, Xk + j * (int64_t)d, xi);
        const double rho_ref = P->sigma * P->sigma * d * (t_k + (k + 1) * dt);
        for (int64_t m = 0; m < M; ++m) {
            const double *a = Xk + m * (int64_t)d;
            for (int64_t q = 0; q < K; ++q) {
                const int64_t j = (m + q) % M;
                for (int i = 0; i < d; ++i) D[q * (int64_t)d + i] = Xn[j * (int64_t)d + i] - a[i];
                Ys[q] = Y[j];
            }
            double alpha;
            int cg_it = 0;
            const int st = orc_llr(d, K, D, Ys, rho_ref, P->h, P->ridge_rel, P->cg_tol,
                                   P->cg_max_iter, &alpha, ax, NULL, &cg_it);
            if (st == ORC_ERR_NOMEM || st == ORC_ERR_ARG) {
                status = st;
                goto done;
            }
            if (st != ORC_OK && status == ORC_OK) status = st;
            for (int i = 0; i < d; ++i) z[i] = P->sigma * ax[i];
            const double feat = orc_f_feature(P, t_k, a, z);
            int it;
            Yk[m] = orc_newton(P, alpha, dt, feat, &it);
            if (it < 0 && status == ORC_OK) status = ORC_ERR_NEWTON;
            if (k == 0 && m == 0 && grad_u0) memcpy(grad_u0, ax, sizeof(double) * d);
        }
        memcpy(Y, Yk, sizeof(double) * M);
        double *tmp = Xn;
        Xn = Xk;
        Xk = tmp;
    }
    {
        double s = 0.0;
        for (int64_t m = 0; m < M; ++m) s += Y[m];
        if (u0) *u0 = s / M;
        if (!isfinite(s / M) && status == ORC_OK) status = ORC_ERR_NONFINITE;
    }
done:
    free(Xn); free(Xk); free(D); free(Ys); free(Y); free(Yk); free(ax); free(z); free(xi);
    return status;
}

/* ------------------------------------------------------------------------- */
/* Derivatives of the problem table used by the adjoint.                      */
/* ------------------------------------------------------------------------- */

/* gx[i] = dg/dx_i at x; gtheta[i] = dg/dtheta_i (zero for kinds without theta). */
void orc_g_grad(const orc_problem *P, const double *x, double *gx, double *gtheta)
{
    const int d = P->d;
    double s = 0.0;
    for (int i = 0; i < d; ++i) gx[i] = gtheta[i] = 0.0;
    switch (P->kind) {
    case ORC_AC_MANUFACTURED:
    case ORC_COS_LINEAR_TEST:
        for (int i = 0; i < d; ++i) gx[i] = -sin(x[i]) / d;
        break;
    case ORC_LOGISTIC_GRAD: {
        const double g = orc_g(P, x);
        for (int i = 0; i < d; ++i) gx[i] = g * (1.0 - g) / d;
        break;
    }
    case ORC_HJB_LOGQUAD:
        for (int i = 0; i < d; ++i) s += P->theta[i] * x[i] * x[i];
        for (int i = 0; i < d; ++i) {
            gx[i] = 2.0 * P->theta[i] * x[i] / (1.0 + s);
            gtheta[i] = x[i] * x[i] / (1.0 + s);
        }
        break;
    case ORC_AFFINE_TEST:
        for (int i = 0; i < d; ++i) {
            gx[i] = P->theta[i];
            gtheta[i] = x[i];
        }
        break;
    case ORC_AC_DOUBLEWELL: {
        const double g = orc_g(P, x);
        for (int i = 0; i < d; ++i) gx[i] = -0.8 * x[i] * g * g;
        break;
    }
    }
}

/* fx[i] = df/dx_i and fz[i] = df/dz_i at (t, x, y, z). */
void orc_f_grads(const orc_problem *P, double t, const double *x, double y, const double *z,
                 double *fx, double *fz)
{
    const int d = P->d;
    for (int i = 0; i < d; ++i) fx[i] = fz[i] = 0.0;
    switch (P->kind) {
    case ORC_AC_MANUFACTURED: {
        double s = 0.0;
        for (int i = 0; i < d; ++i) s += cos(x[i]);
        const double e = exp(t - P->T), us = e * s / d;
        const double dq = 3.0 * us * us - (2.0 - 0.5 * P->sigma * P->sigma);
        for (int i = 0; i < d; ++i) fx[i] = dq * (-e * sin(x[i]) / d);
        break;
    }
    case ORC_LOGISTIC_GRAD:
        for (int i = 0; i < d; ++i) fz[i] = y - (2.0 + d) / (2.0 * d);
        break;
    case ORC_HJB_LOGQUAD:
        for (int i = 0; i < d; ++i) fz[i] = -z[i];
        break;
    case ORC_AFFINE_TEST:
        for (int i = 0; i < d; ++i) fz[i] = P->c2;
        break;
    }
}

/* CG on (Gamma_c + lambda I) v = rhs with the stored cloud D, normalised weights w and
   first moment S (the operator of Eq. 3.19 with the ridge). */
static int gamma_c_solve(int d, int64_t M, const double *D, const double *w, const double *S,
                         double lambda, const double *rhs, double tol, int max_iter, double *v,
                         double *t)
{
    double *r = (double *)malloc(sizeof(double) * 3 * (size_t)d);
    if (!r) return ORC_ERR_NOMEM;
    double *p = r + d, *q = r + 2 * d;
    for (int i = 0; i < d; ++i) {
        v[i] = 0.0;
        r[i] = p[i] = rhs[i];
    }
    double rr = dotd(d, r, r);
    const double stop = tol * sqrt(rr);
    int it = 0, status = ORC_OK;
    while (sqrt(rr) > stop) {
        if (it >= max_iter) {
            status = ORC_ERR_CG;
            break;
        }
        gamma_c_apply(d, M, D, w, S, lambda, p, t, q);
        const double a = rr / dotd(d, p, q);
        for (int i = 0; i < d; ++i) {
            v[i] += a * p[i];
            r[i] -= a * q[i];
        }
        const double rr_new = dotd(d, r, r);
        const double beta = rr_new / rr;
        for (int i = 0; i < d; ++i) p[i] = r[i] + beta * p[i];
        rr = rr_new;
        ++it;
    }
    free(r);
    return status;
}

/*
 * Reverse-mode derivative of the estimator u(0,x0) of Algorithm 1 with respect to x0
 * and to theta (the terminal coefficients), for the same random increments.  A plain
 * tape: the forward pass stores X_k for every level, the weights, the first moments,
 * the ridge and Y_k with F'(Y_k); the reverse pass runs k = 0..N-1:
 *   gamma_j   = Ybar_k^j / F'_j                      (implicit function of (2.16))
 *   alphabar  = sum_j gamma_j,
 *   alphaxbar = sum_j gamma_j (X_k^j - x0) + sigma Zbar,  Zbar = dt sum_j gamma_j f_z
 *   x0bar    += dt sum_j gamma_j f_x(t_k, X_k^j)
 *   v         = (Gamma_c + lambda I)^-1 (alphaxbar - alphabar S_k)      (Eqs. 3.19-3.20)
 *   Ybar_{k+1}^j = w_j (alphabar + (D_j - S_k) . v),  D_j = X_{k+1}^j - x0,
 * then x0bar += sum_j Ybar_N^j grad g(X_N^j), thetabar = sum_j Ybar_N^j d_theta g(X_N^j).
 * The kernel weights and the ridge depend only on D_j, which does not move with x0.
 * Outputs u0, du_dx0[d], du_dtheta[d] (may be NULL), and v_levels[N][d] (may be NULL):
 * the solution v of level k's adjoint regression solve, a trace for tests.
 */
int orc_adjoint(const orc_problem *P, const double *x0, uint64_t seed, uint32_t solve_index,
                double *u0, double *du_dx0, double *du_dtheta, double *v_levels)
{
    const int d = P->d, N = P->N;
    const int64_t M = P->M;
    if (d < 1 || N < 1 || M < 2 || !(P->T > 0.0) || !(P->sigma > 0.0)) return ORC_ERR_ARG;
    if ((P->kind == ORC_HJB_LOGQUAD || P->kind == ORC_AFFINE_TEST) && !P->theta) return ORC_ERR_ARG;
    const double dt = P->T / N;
    const size_t Md = (size_t)M * d;
    double *X = (double *)malloc(sizeof(double) * Md * (N + 1));     /* X_k, k = 0..N */
    double *Yl = (double *)malloc(sizeof(double) * (size_t)M * (N + 1)); /* Y_k        */
    double *Fp = (double *)malloc(sizeof(double) * (size_t)M * (N + 1)); /* F'(Y_k)    */
    double *W = (double *)malloc(sizeof(double) * (size_t)M * N);        /* w of level k */
    double *Sl = (double *)malloc(sizeof(double) * (size_t)d * N);       /* S of level k */
    double *AX = (double *)malloc(sizeof(double) * (size_t)d * N);       /* alpha_x      */
    double *lam = (double *)malloc(sizeof(double) * N);
    double *D = (double *)malloc(sizeof(double) * Md);
    double *tmpM = (double *)malloc(sizeof(double) * M);
    double *Yb = (double *)malloc(sizeof(double) * M);
    double *gam = (double *)malloc(sizeof(double) * M);
    double *vec = (double *)malloc(sizeof(double) * 8 * (size_t)d);
    int *nit = (int *)malloc(sizeof(int) * M);
    int status = ORC_OK;
    if (!X || !Yl || !Fp || !W || !Sl || !AX || !lam || !D || !tmpM || !Yb || !gam || !vec || !nit) {
        status = ORC_ERR_NOMEM;
        goto done;
    }
    double *z = vec, *ab = vec + d, *rhs = vec + 2 * d, *v = vec + 3 * d, *fx = vec + 4 * d,
           *fz = vec + 5 * d, *xb = vec + 6 * d, *tb = vec + 7 * d;

    /* ---- the particle paths of every level (the same bridge as orc_solve) */
#pragma omp parallel
    {
        double *xi = (double *)malloc(sizeof(double) * d);
#pragma omp for schedule(static)
        for (int64_t j = 0; j < M; ++j) {
            double *XN = X + (size_t)N * Md + j * (int64_t)d;
            path_end(P, x0, seed, solve_index, j, XN, xi);
            for (int k = N - 1; k >= 0; --k)
                path_step(P, k, x0, seed, solve_index, j, X + (size_t)(k + 1) * Md + j * (int64_t)d,
                          X + (size_t)k * Md + j * (int64_t)d, xi);
            Yl[(size_t)N * M + j] = orc_g(P, XN);
        }
        free(xi);
    }
    /* ---- backward sweep (Algorithm 1), recording the tape */
    for (int k = N - 1; k >= 0; --k) {
        const double t_k = k * dt;
        const double *Xn = X + (size_t)(k + 1) * Md, *Xk = X + (size_t)k * Md;
        for (size_t e = 0; e < Md; ++e) D[e] = Xn[e] - x0[e % d];
        double alpha;
        int it;
        int st = orc_llr(d, M, D, Yl + (size_t)(k + 1) * M, P->sigma * P->sigma * d * (k + 1) * dt,
                         P->h, P->ridge_rel, P->cg_tol, P->cg_max_iter, &alpha, AX + (size_t)k * d,
                         W + (size_t)k * M, &it);
        if (st == ORC_ERR_NOMEM || st == ORC_ERR_ARG) {
            status = st;
            goto done;
        }
        if (st != ORC_OK && status == ORC_OK) status = st;
        /* S_k and lambda_k of this regression (as inside orc_llr) */
        double *S = Sl + (size_t)k * d;
        weighted_row_sum(d, M, D, W + (size_t)k * M, S);
        double wrho = 0.0;
        for (int64_t j = 0; j < M; ++j) {
            double rho = 0.0;
            for (int i = 0; i < d; ++i) rho += D[j * (int64_t)d + i] * D[j * (int64_t)d + i];
            wrho += W[(size_t)k * M + j] * rho;
        }
        lam[k] = P->ridge_rel * (wrho - dotd(d, S, S)) / d;
        const double *ax = AX + (size_t)k * d;
        for (int i = 0; i < d; ++i) z[i] = P->sigma * ax[i];
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < M; ++j) {
            const double *xj = Xk + j * (int64_t)d;
            double pred = alpha;
            for (int i = 0; i < d; ++i) pred += ax[i] * (xj[i] - x0[i]);
            const double feat = orc_f_feature(P, t_k, xj, z);
            const double y = orc_newton(P, pred, dt, feat, &nit[j]);
            double dfdy;
            (void)orc_f_scalar(P, feat, y, &dfdy);
            Yl[(size_t)k * M + j] = y;
            Fp[(size_t)k * M + j] = 1.0 - dt * dfdy;
        }
        for (int64_t j = 0; j < M; ++j)
            if (nit[j] < 0 && status == ORC_OK) status = ORC_ERR_NEWTON;
    }
    {
        double s = 0.0;
        for (int64_t j = 0; j < M; ++j) s += Yl[j];
        if (u0) *u0 = s / M;
    }
    /* ---- reverse sweep */
    for (int i = 0; i < d; ++i) xb[i] = tb[i] = 0.0;
    for (int64_t j = 0; j < M; ++j) Yb[j] = 1.0 / M; /* u = (1/M) sum_j Y_0^j */
    for (int k = 0; k < N; ++k) {
        const double t_k = k * dt;
        const double *Xk = X + (size_t)k * Md, *Xn = X + (size_t)(k + 1) * Md;
        const double *ax = AX + (size_t)k * d, *S = Sl + (size_t)k * d;
        for (int i = 0; i < d; ++i) z[i] = P->sigma * ax[i];
        double abar = 0.0;
        for (int64_t j = 0; j < M; ++j) {
            gam[j] = Yb[j] / Fp[(size_t)k * M + j];
            abar += gam[j];
        }
        for (int i = 0; i < d; ++i) ab[i] = 0.0;
        for (int64_t j = 0; j < M; ++j) {
            const double *xj = Xk + j * (int64_t)d;
            orc_f_grads(P, t_k, xj, Yl[(size_t)k * M + j], z, fx, fz);
            for (int i = 0; i < d; ++i) {
                ab[i] += gam[j] * (xj[i] - x0[i]) + P->sigma * dt * gam[j] * fz[i];
                xb[i] += dt * gam[j] * fx[i];
            }
        }
        for (int i = 0; i < d; ++i) rhs[i] = ab[i] - abar * S[i];
        for (size_t e = 0; e < Md; ++e) D[e] = Xn[e] - x0[e % d];
        int st = gamma_c_solve(d, M, D, W + (size_t)k * M, S, lam[k], rhs, P->cg_tol,
                               P->cg_max_iter, v, tmpM);
        if (st == ORC_ERR_NOMEM) {
            status = st;
            goto done;
        }
        if (st != ORC_OK && status == ORC_OK) status = st;
        if (v_levels)
            for (int i = 0; i < d; ++i) v_levels[(size_t)k * d + i] = v[i];
        const double sv = dotd(d, S, v);
        for (int64_t j = 0; j < M; ++j) {
            double dv = 0.0;
            for (int i = 0; i < d; ++i) dv += D[j * (int64_t)d + i] * v[i];
            Yb[j] = W[(size_t)k * M + j] * (abar + dv - sv);
        }
    }
    /* terminal condition Y_N = g(X_N) */
    for (int64_t j = 0; j < M; ++j) {
        orc_g_grad(P, X + (size_t)N * Md + j * (int64_t)d, fx, fz);
        for (int i = 0; i < d; ++i) {
            xb[i] += Yb[j] * fx[i];
            tb[i] += Yb[j] * fz[i];
        }
    }
    if (du_dx0) memcpy(du_dx0, xb, sizeof(double) * d);
    if (du_dtheta) memcpy(du_dtheta, tb, sizeof(double) * d);
done:
    free(X); free(Yl); free(Fp); free(W); free(Sl); free(AX); free(lam); free(D); free(tmpM);
    free(Yb); free(gam); free(vec); free(nit);
    return status;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
