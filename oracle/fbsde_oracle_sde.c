/*
 * fbsde_oracle_sde.c -- FP64 CPU oracle of the scheme with a drift and a state-dependent
 * diffusion (the forward SDE of Sec. 2.1, dX = mu(t,X) dt + sigma(t,X) dW, in its general
 * form), for the componentwise affine coefficients
 *     mu_i(x) = mu0 + mu1 x_i,      sigma(x) = diag(sig0 + sig1 x_i)
 * (Ornstein-Uhlenbeck for mu1 < 0, sig1 = 0; geometric Brownian motion for mu0 = sig0 = 0).
 *
 * TEST INFRASTRUCTURE ONLY, like fbsde_oracle.c (it is linked into the same library and
 * uses that file's Philox normals, problem table, Newton and regression).
 *
 * What it computes (one solve = one query point x0), in the order of Algorithm 1:
 *   anchor   a_0 = x0, a_{k+1} = a_k + mu(t_k, a_k) dt: the drift path of x0 (the anchor of
 *            the level-k regression, as in the scheme with mu = 0 where a_k = x0);
 *   forward  Euler-Maruyama (2.7): X_0^j = x0,
 *              X_{k+1}^j = X_k^j + mu(t_k, X_k^j) dt + sigma(t_k, X_k^j) sqrt(dt) xi_{s,k,j},
 *            k = 0..N-1, every level kept; Y_N^j = g(X_N^j);
 *   backward for k = N-1..0: the weighted ridge regression of Y_{k+1}^j on
 *            D_j = X_{k+1}^j - a_k (orc_llr: Eqs. 2.10-2.15, Remark 2.2, Lemma 3.7), with
 *            the kernel scale eps_k^2 = h^2 rho_k, rho_k = (1/M) sum_j |D_j|^2 the cloud's
 *            mean squared distance (its expectation sigma^2 d t_{k+1} when mu = 0 and sigma
 *            is constant, the value the driftless scheme uses);
 *            per particle Z_k^j = sigma(t_k, X_k^j)^T alpha_x (Algorithm 1's Z = sigma^T
 *            grad u with the diffusion at the particle), the local affine prediction at the
 *            particle's drifted position
 *              E_j = alpha + alpha_x . (X_k^j + mu(t_k, X_k^j) dt - a_k),
 *            and Newton (2.16)-(2.17) on F(Y) = Y - E_j - dt f(t_k, X_k^j, Y, Z_k^j);
 *   output   u(0,x0) = (1/M) sum_j Y_0^j, grad u(0,x0) = alpha_x at k = 0.
 * The normals xi_{s,k,j} are those of orc_normals with counter level k = 0..N-1 (the
 * increment of step k).
 *
 * Kinds beyond the driftless table (manufactured sources that make u* exact for these
 * coefficients; with s_i = sig0 + sig1 x_i and m_i = mu0 + mu1 x_i):
 *   DRIFT_AC (7):   g = (1/d) sum cos x_i, f = y - y^3 + q,
 *                   q = u*^3 - 2 u* + e^{t-T} (1/d) sum_i [s_i^2 cos x_i / 2 + m_i sin x_i],
 *                   u* = e^{t-T} (1/d) sum_i cos x_i;
 *   DRIFT_QUAD (8): g = (1/d) sum x_i^2, f = y - y^3 + q,
 *                   q = u*^3 - 2 u* - e^{t-T} (1/d) sum_i [s_i^2 + 2 m_i x_i],
 *                   u* = e^{t-T} (1/d) sum_i x_i^2.
 * The driftless kinds 0-6 keep their g and f (without a closed form under a drift, except
 * AFFINE_TEST, whose discrete scheme stays exactly affine).  HJB_LOGQUAD (|z|^2) needs the
 * per-particle |z|^2 and is accepted only with sig1 = 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { SDE_OK = 0, SDE_ERR_ARG = 1, SDE_ERR_NEWTON = 4, SDE_ERR_CG = 5,
       SDE_ERR_NONFINITE = 7, SDE_ERR_NOMEM = 8 };
enum { SDE_HJB_LOGQUAD = 2, SDE_DRIFT_AC = 7, SDE_DRIFT_QUAD = 8 };

/* the driftless problem record of fbsde_oracle.c (same layout) */
typedef struct {
    int32_t kind;
    int32_t d;
    double sigma;
    double T;
    int32_t N;
    int32_t cg_max_iter;
    int64_t M;
    const double *theta;
    double A, c0, c1, c2, c3;
    double h;
    double ridge_rel;
    double cg_tol;
    double newton_tol;
    int32_t newton_max_iter;
    int32_t pad_;
} orc_problem;

void orc_normals(uint64_t seed, uint32_t s, uint32_t k, uint32_t j, int32_t d, double *xi);
double orc_g(const orc_problem *P, const double *x);
double orc_f_feature(const orc_problem *P, double t, const double *x, const double *z);
double orc_f_scalar(const orc_problem *P, double feature, double y, double *dfdy);
int orc_llr(int32_t d, int64_t M, const double *D, const double *Y, double rho_ref, double h,
            double ridge_rel, double cg_tol, int32_t cg_max_iter, double *alpha, double *alpha_x,
            double *w_out, int32_t *cg_iters);

/* coefficients of the forward SDE; P->sigma is sig0 */
typedef struct {
    double mu0, mu1, sig1;
} orc_sde_coef;

static double drift(const orc_sde_coef *C, double x) { return C->mu0 + C->mu1 * x; }
static double diffusion(const orc_problem *P, const orc_sde_coef *C, double x)
{
    return P->sigma + C->sig1 * x;
}

/* g of the drift kinds, else the driftless table */
static double sde_g(const orc_problem *P, const double *x)
{
    const int d = P->d;
    double s = 0.0;
    if (P->kind == SDE_DRIFT_AC) {
        for (int i = 0; i < d; ++i) s += cos(x[i]);
        return s / d;
    }
    if (P->kind == SDE_DRIFT_QUAD) {
        for (int i = 0; i < d; ++i) s += x[i] * x[i];
        return s / d;
    }
    return orc_g(P, x);
}

/* y-independent part of f at (t, x, z) for the drift kinds (the source q), else the
 * driftless table's feature */
static double sde_feature(const orc_problem *P, const orc_sde_coef *C, double t, const double *x,
                          const double *z)
{
    const int d = P->d;
    const double e = exp(t - P->T);
    if (P->kind == SDE_DRIFT_AC) {
        double phi = 0.0, psi = 0.0;
        for (int i = 0; i < d; ++i) {
            const double s = diffusion(P, C, x[i]), m = drift(C, x[i]);
            phi += cos(x[i]);
            psi += 0.5 * s * s * cos(x[i]) + m * sin(x[i]);
        }
        const double us = e * phi / d;
        return us * us * us - 2.0 * us + e * psi / d;
    }
    if (P->kind == SDE_DRIFT_QUAD) {
        double phi = 0.0, psi = 0.0;
        for (int i = 0; i < d; ++i) {
            const double s = diffusion(P, C, x[i]), m = drift(C, x[i]);
            phi += x[i] * x[i];
            psi += s * s + 2.0 * m * x[i];
        }
        const double us = e * phi / d;
        return us * us * us - 2.0 * us - e * psi / d;
    }
    return orc_f_feature(P, t, x, z);
}

static double sde_f_scalar(const orc_problem *P, double feature, double y, double *dfdy)
{
    if (P->kind == SDE_DRIFT_AC || P->kind == SDE_DRIFT_QUAD) {
        *dfdy = 1.0 - 3.0 * y * y;
        return y - y * y * y + feature;
    }
    return orc_f_scalar(P, feature, y, dfdy);
}

/* Newton (2.17) on F(Y) = Y - E - dt f (2.16) from Y = E (the driftless rule) */
static double sde_newton(const orc_problem *P, double E, double dt, double feature, int *iters)
{
    double y = E;
    for (int n = 1; n <= P->newton_max_iter; ++n) {
        double dfdy, f = sde_f_scalar(P, feature, y, &dfdy);
        double dy = (y - E - dt * f) / (1.0 - dt * dfdy);
        y -= dy;
        if (fabs(dy) <= P->newton_tol * fmax(1.0, fabs(y))) {
            *iters = n;
            return y;
        }
    }
    *iters = -1;
    return y;
}

/*
 * Algorithm 1 with the coefficients C (see the header).  Outputs (may be NULL): u0,
 * grad_u0[d]; alpha_lv[N], alphax_lv[N d], cg_lv[N] per level; x_lv[(N+1) M d] the paths
 * (level-major).  Returns SDE_OK or the first error (NEWTON, CG, NONFINITE).
 */
int orc_solve_sde(const orc_problem *P, const orc_sde_coef *C, const double *x0, uint64_t seed,
                  uint32_t solve_index, double *u0, double *grad_u0, double *alpha_lv,
                  double *alphax_lv, int32_t *cg_lv, double *x_lv)
{
    const int d = P->d, N = P->N;
    const int64_t M = P->M;
    if (!C || d < 1 || N < 1 || M < 2 || !(P->T > 0.0)) return SDE_ERR_ARG;
    if ((P->kind == 2 || P->kind == 3) && !P->theta) return SDE_ERR_ARG;
    if (P->kind == SDE_HJB_LOGQUAD && C->sig1 != 0.0) return SDE_ERR_ARG;
    const double dt = P->T / N, sdt = sqrt(dt);
    const size_t Md = (size_t)M * d;
    double *X = (double *)malloc(sizeof(double) * (size_t)(N + 1) * Md);
    double *a = (double *)malloc(sizeof(double) * (size_t)(N + 1) * d);
    double *D = (double *)malloc(sizeof(double) * Md);
    double *Y = (double *)malloc(sizeof(double) * M);
    double *ax = (double *)malloc(sizeof(double) * d);
    double *z = (double *)malloc(sizeof(double) * d);
    double *xi = (double *)malloc(sizeof(double) * d);
    if (!X || !a || !D || !Y || !ax || !z || !xi) {
        free(X); free(a); free(D); free(Y); free(ax); free(z); free(xi);
        return SDE_ERR_NOMEM;
    }
    int status = SDE_OK;
    /* anchor: the drift path of x0 */
    memcpy(a, x0, sizeof(double) * d);
    for (int k = 0; k < N; ++k)
        for (int i = 0; i < d; ++i)
            a[(size_t)(k + 1) * d + i] = a[(size_t)k * d + i] + drift(C, a[(size_t)k * d + i]) * dt;
    /* forward Euler-Maruyama sweep (2.7), every level kept */
    for (int64_t j = 0; j < M; ++j) memcpy(X + (size_t)j * d, x0, sizeof(double) * d);
    for (int k = 0; k < N; ++k) {
        const double *Xk = X + (size_t)k * Md;
        double *Xn = X + (size_t)(k + 1) * Md;
        for (int64_t j = 0; j < M; ++j) {
            orc_normals(seed, solve_index, (uint32_t)k, (uint32_t)j, d, xi);
            for (int i = 0; i < d; ++i) {
                const double x = Xk[(size_t)j * d + i];
                Xn[(size_t)j * d + i] = x + drift(C, x) * dt + diffusion(P, C, x) * sdt * xi[i];
            }
        }
    }
    for (int64_t j = 0; j < M; ++j) Y[j] = sde_g(P, X + (size_t)N * Md + (size_t)j * d);
    if (x_lv) memcpy(x_lv, X, sizeof(double) * (size_t)(N + 1) * Md);

    for (int k = N - 1; k >= 0; --k) {
        const double t_k = k * dt;
        const double *Xn = X + (size_t)(k + 1) * Md, *Xk = X + (size_t)k * Md;
        const double *ak = a + (size_t)k * d;
        double rho = 0.0;   /* the cloud's mean squared distance to the anchor */
        for (int64_t j = 0; j < M; ++j) {
            double r = 0.0;
            for (int i = 0; i < d; ++i) {
                const double v = Xn[(size_t)j * d + i] - ak[i];
                D[(size_t)j * d + i] = v;
                r += v * v;
            }
            rho += r;
        }
        rho /= (double)M;
        double alpha;
        int32_t it = 0;
        int st = orc_llr(d, M, D, Y, rho, P->h, P->ridge_rel, P->cg_tol, P->cg_max_iter, &alpha,
                         ax, NULL, &it);
        if (st == SDE_ERR_NOMEM || st == SDE_ERR_ARG) {
            status = st;
            break;
        }
        if (st != SDE_OK && status == SDE_OK) status = st;
        if (alpha_lv) alpha_lv[k] = alpha;
        if (alphax_lv) memcpy(alphax_lv + (size_t)k * d, ax, sizeof(double) * d);
        if (cg_lv) cg_lv[k] = it;
        for (int64_t j = 0; j < M; ++j) {
            const double *x = Xk + (size_t)j * d;
            double E = alpha;
            for (int i = 0; i < d; ++i) {
                E += ax[i] * (x[i] + drift(C, x[i]) * dt - ak[i]);
                z[i] = diffusion(P, C, x[i]) * ax[i];   /* Z = sigma(t_k, X)^T alpha_x */
            }
            int n;
            Y[j] = sde_newton(P, E, dt, sde_feature(P, C, t_k, x, z), &n);
            if (n < 0 && status == SDE_OK) status = SDE_ERR_NEWTON;
        }
    }
    if (status != SDE_ERR_NOMEM && status != SDE_ERR_ARG) {
        double s = 0.0;
        for (int64_t j = 0; j < M; ++j) s += Y[j];
        if (u0) *u0 = s / M;
        if (grad_u0) memcpy(grad_u0, ax, sizeof(double) * d);
        if (!isfinite(s / M) && status == SDE_OK) status = SDE_ERR_NONFINITE;
    }
    free(X); free(a); free(D); free(Y); free(ax); free(z); free(xi);
    return status;
}

/* The problem table of this file as seen by the tests: g(x) and f(t, x, y, z) with
 * df/dy (z = sigma(t, x)^T grad u). */
double orc_sde_g(const orc_problem *P, const double *x) { return sde_g(P, x); }

double orc_sde_f(const orc_problem *P, const orc_sde_coef *C, double t, const double *x, double y,
                 const double *z, double *dfdy)
{
    return sde_f_scalar(P, sde_feature(P, C, t, x, z), y, dfdy);
}
