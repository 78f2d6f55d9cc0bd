// fbsde_adjoint.cuh -- kernels of the reverse sweep: the derivative of the estimator
// u(0,x0) of Algorithm 1 with respect to x0 and the terminal coefficients theta, for the
// same random increments.  Included after fbsde_kernels.cuh.
//
// With Ybar_k^j the adjoint of Y_k^j (Ybar_0^j = ubar / M), each level k = 0..N-1 runs:
//   Newton adjoint at level k (implicit function of Eq. 2.16):
//     gamma_j = Ybar_k^j / F'_j,  F' = 1 - dt df/dy,
//     alphabar   = sum_j gamma_j,
//     alphaxbar  = sum_j gamma_j Delta_k^j + sigma dt sum_j gamma_j df/dz_j   (Z = sigma alpha_x)
//     x0bar     += dt sum_j gamma_j df/dx_j
//   regression adjoint (Eqs. 3.19-3.20, one solve with the same SPD operator):
//     v = (Gamma_c + lambda I)^-1 (alphaxbar - alphabar S),
//     Ybar_{k+1}^j = (w_j / W) (alphabar - S.v + Delta_{k+1}^j . v),
// and finally x0bar += sum_j Ybar_N^j grad g(X_N^j), thetabar = sum_j Ybar_N^j d_theta g.
// The kernel weights, S and lambda depend only on Delta, which does not move with x0.
// In the code the Newton adjoint of level k+1 is fused with the regression adjoint of
// level k (both use the rows Delta_{k+1}).
#pragma once
#include "fbsde_kernels.cuh"

namespace fbsde {
namespace dev {

// Tape accessors (written by the primal when p.tape_w is set).
struct Tape {
    const Params &p;
    __device__ __forceinline__ explicit Tape(const Params &pp) : p(pp) {}
    template <typename Real> __device__ __forceinline__ Real *w(int lvl, int s) const
    {
        return reinterpret_cast<Real *>(p.tape_w) + ((size_t)lvl * p.Q + s) * p.M;
    }
    __device__ __forceinline__ double *Y(int lvl, int s) const
    {
        return p.tape_Y + ((size_t)lvl * p.Q + s) * p.M;
    }
    __device__ __forceinline__ double *S(int s, int lvl) const
    {
        return p.tape_v + (((size_t)s * p.N + lvl) * 2 + 0) * p.ld;
    }
    __device__ __forceinline__ double *ax(int s, int lvl) const
    {
        return p.tape_v + (((size_t)s * p.N + lvl) * 2 + 1) * p.ld;
    }
    // [0] lambda, [1] 1/W, [2] alpha
    __device__ __forceinline__ double *scal(int s, int lvl) const
    {
        return p.tape_s + ((size_t)s * p.N + lvl) * 4;
    }
    // adjoint vectors: 0 alphaxbar, 1 x0bar, 2 thetabar
    __device__ __forceinline__ double *av(int s, int which) const
    {
        return p.adj_v + ((size_t)s * 3 + which) * p.ld;
    }
};

// Level-0 start: all Y_0^j are equal (X_0 = x0), so Ybar_0^j = ubar/M gives
// gamma summed over particles = ubar / F'_0.  Sets alphabar, alphaxbar and the
// x-derivative of f at x0; zeroes thetabar.
template <typename Real>
__global__ void __launch_bounds__(kFinThreads) k_adj_init(Params p, const double *ubar)
{
    __shared__ double sm[32 * 4];
    const int s = blockIdx.x;
    const WS<Real> ws(p);
    const Tape tp(p);
    SolveState &st = p.st[s];
    const double *x0 = ws.v64(s, 6);
    const double *ax0 = tp.ax(s, 0);
    const double alpha0 = tp.scal(s, 0)[2];
    double a[2] = {0.0, 0.0};  // sum alpha_x, |alpha_x|^2 at level 0
    #pragma unroll 4
    for (int i = threadIdx.x; i < p.ld; i += blockDim.x) {
        a[0] += ax0[i];
        a[1] += ax0[i] * ax0[i];
    }
    block_sum(a, sm);
    const double sumz = p.sigma * a[0], zz = p.sigma * p.sigma * a[1];
    const double feat = f_feature(p, 0.0, st.phi0, sumz, zz);
    int it;
    const double y0 = newton(p, alpha0, feat, it);
    double dfdy;
    (void)f_scalar(p, feat, y0, dfdy);
    const double gsum = ubar[s] / (1.0 - p.dt * dfdy);
    // sigma dt gamma-weighted df/dz and dt gamma-weighted df/dx at x0
    const double e = exp(-p.T);
    const double us = e * st.phi0 / p.d;
    const double dq = 3.0 * us * us - (2.0 - 0.5 * p.sigma * p.sigma);
    #pragma unroll 4
    for (int i = threadIdx.x; i < p.ld; i += blockDim.x) {
        double zb = 0.0, xb = 0.0;
        if (i < p.d) {
            switch (p.kind) {
            case FBSDE_LOGISTIC_GRAD: zb = p.sigma * p.dt * gsum * (y0 - (2.0 + p.d) / (2.0 * p.d)); break;
            case FBSDE_HJB_LOGQUAD: zb = -p.sigma * p.sigma * p.dt * gsum * ax0[i]; break;
            case FBSDE_AFFINE_TEST: zb = p.sigma * p.dt * gsum * p.c2; break;
            case FBSDE_AC_MANUFACTURED: xb = p.dt * gsum * dq * (-e * sin(x0[i]) / p.d); break;
            }
        }
        tp.av(s, 0)[i] = zb;   // sum_j gamma_j Delta_0^j = 0
        tp.av(s, 1)[i] = xb;
        tp.av(s, 2)[i] = 0.0;
    }
    if (threadIdx.x == 0) st.abar = gsum;
}

// Starting guess of the adjoint solve of level k >= 1: the previous level's solution v
// (still in slot 0; the level-to-level change of v is small), rounded for the product
// k_matvec forms next (Gamma_c x needs sum_j w_j (D_j . x) D_j), and S . x.
template <typename Real>
__global__ void __launch_bounds__(kFinThreads) k_adj_warm(Params p)
{
    __shared__ double sm[32 * 4];
    const int s = blockIdx.x, k = p.level;
    const WS<Real> ws(p);
    const Tape tp(p);
    SolveState &st = p.st[s];
    const double *Sk = tp.S(s, k), *x = ws.v64(s, 0);
    Real *pR = ws.vR(s, 0);
    double a[1] = {0.0};
    #pragma unroll 4
    for (int i = threadIdx.x; i < p.ld; i += blockDim.x) {
        pR[i] = (Real)x[i];
        a[0] += Sk[i] * x[i];
    }
    block_sum(a, sm);
    if (threadIdx.x == 0) {
        st.sx = a[0];
        st.done = 0;   // the product runs for every query
    }
}

// Adjoint CG set-up at level k: operator of the level-k regression (tape: S, lambda,
// 1/W; weights via p.w), right-hand side alphaxbar - alphabar S.  Start from 0, or with
// warm = 1 from the guess of k_adj_warm, whose unnormalised product sum_j w_j (D_j . x) D_j
// is in slot 5: r = rhs - (Gamma_c + lambda I) x.
template <typename Real>
__global__ void __launch_bounds__(kFinThreads) k_adj_setup(Params p, int warm)
{
    __shared__ double sm[32 * 4];
    const int s = blockIdx.x, k = p.level;
    const WS<Real> ws(p);
    const Tape tp(p);
    SolveState &st = p.st[s];
    const double *Sk = tp.S(s, k), *ab = tp.av(s, 0);
    double *x = ws.v64(s, 0), *r = ws.v64(s, 1), *pp = ws.v64(s, 2), *S = ws.v64(s, 3);
    const double *Gx = ws.v64(s, 5);
    Real *pR = ws.vR(s, 0);
    const double abar = st.abar;
    const double *sc = tp.scal(s, k);
    const double lam = sc[0], invW = sc[1], sx = st.sx;
    double a[3] = {0.0, 0.0, 0.0};  // |rhs|^2, |r|^2, S.r
    #pragma unroll 4
    for (int i = threadIdx.x; i < p.ld; i += blockDim.x) {
        S[i] = Sk[i];
        const double rhs = ab[i] - abar * Sk[i];
        double ri = rhs;
        if (warm) ri -= Gx[i] * invW - Sk[i] * sx + lam * x[i];
        else x[i] = 0.0;
        r[i] = ri;
        pp[i] = ri;
        pR[i] = (Real)ri;
        a[0] += rhs * rhs;
        a[1] += ri * ri;
        a[2] += Sk[i] * ri;
    }
    block_sum(a, sm);
    if (threadIdx.x == 0) {
        st.lambda = lam;
        st.invW = invW;
        st.rr = a[1];
        st.rhs2 = a[0];
        st.sp = a[2];
        st.iters = 0;
        st.done = (a[1] <= p.cg_tol2 * a[0]) ? 1 : 0;
    }
}

// After the adjoint CG: v in the stream precision for the row pass, S.v.
template <typename Real>
__global__ void __launch_bounds__(kFinThreads) k_adj_post(Params p)
{
    __shared__ double sm[32 * 4];
    const int s = blockIdx.x;
    const WS<Real> ws(p);
    const double *x = ws.v64(s, 0), *S = ws.v64(s, 3);
    Real *xR = ws.vR(s, 1);
    double a[1] = {0.0};
    #pragma unroll 4
    for (int i = threadIdx.x; i < p.ld; i += blockDim.x) {
        xR[i] = (Real)x[i];
        a[0] += S[i] * x[i];
    }
    block_sum(a, sm);
    if (threadIdx.x == 0) p.st[s].sv = a[0];
}

// Row pass on Delta_{k+1}: per-segment sums of (Delta . v, sum_i cos(x0_i + Delta_i)).
template <typename Real, int VPT>
__global__ void __launch_bounds__(256) k_adj_rows(Params p)
{
    constexpr int E = Chunk<Real>::E;
    const WS<Real> ws(p);
    const int lane = threadIdx.x & 31;
    const int nch = p.ld / E;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const bool cos_feature = p.kind == FBSDE_AC_MANUFACTURED;
    for (RowItems w(p, (((unsigned long long)blockIdx.x * blockDim.x) + threadIdx.x) >> 5,
                    (unsigned long long)nwarps);
         w.s < (uint32_t)p.Q; w.next()) {
        const int seg = (int)w.seg, s = (int)w.s;
        const long long j = w.j;
        const Real *vr = ws.vR(s, 1), *x0r = ws.vR(s, 2);
        const Real *drow = ws.row(s, j);
        Real acc[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int c = seg * 32 * VPT + lane + 32 * v;
            if (c < nch) {
                const Chunk<Real> dl = ld_chunk(drow + c * E);
                const Chunk<Real> vc = ldg_chunk(vr + c * E);
#pragma unroll
                for (int e = 0; e < E; ++e) acc[0] += dl.v[e] * vc.v[e];
                if (cos_feature) {
                    const Chunk<Real> xc = ldg_chunk(x0r + c * E);
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (c * E + e < p.d) acc[1] += cos(xc.v[e] + dl.v[e]);
                }
            }
        }
        warp_sum(acc);
        if (lane == 0) {
            Real *o = ws.segp(s, j, seg);
            o[0] = acc[0];
            o[1] = acc[1];
            o[2] = Real(0);
        }
    }
}

// Per particle at level L = k+1 (one thread each): Ybar_L^j from the regression adjoint,
// then either the Newton adjoint of level L (L < N) or the terminal derivatives (L = N).
// Column-sum coefficients (coef[0..2]) and block scalars (spart[0..3]):
//   L < N:  coef = (gamma, dt gamma df/dx scale, 0), scalars (sum gamma, sum gamma (Y - c_L), 0, 0)
//   L = N:  coef per kind for grad g / d_theta g, scalars (sum Ybar, sum Ybar g(1-g)/d, 0, 0).
template <typename Real>
__global__ void __launch_bounds__(256) k_adj_particles(Params p)
{
    __shared__ double sm[32 * 4];
    const int s = blockIdx.y;
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const WS<Real> ws(p);
    const Tape tp(p);
    const SolveState &st = p.st[s];
    const int k = p.level, L = k + 1;
    const bool terminal = L == p.N;
    double sums[4] = {0.0, 0.0, 0.0, 0.0};
    if (j < p.M) {
        double tdot = 0.0, phi = 0.0;
        for (int seg = 0; seg < p.nseg; ++seg) {
            const Real *sp = ws.segp(s, j, seg);
            tdot += (double)sp[0];
            phi += (double)sp[1];
        }
        const double wn = (double)tp.w<Real>(k, s)[j] * tp.scal(s, k)[1];
        const double yb = wn * (st.abar - st.sv + tdot);
        const double yL = tp.Y(L, s)[j];
        Real *cf = ws.coef(s, j);
        if (!terminal) {
            const double t = L * p.dt;
            const double *axL = tp.ax(s, L);
            (void)axL;
            double feat;
            if (p.kind == FBSDE_AC_MANUFACTURED) feat = f_feature(p, t, phi, 0.0, 0.0);
            else feat = f_feature(p, t, 0.0, st.sumz_l, st.zz_l);
            double dfdy;
            (void)f_scalar(p, feat, yL, dfdy);
            const double gam = yb / (1.0 - p.dt * dfdy);
            double bsin = 0.0;
            if (p.kind == FBSDE_AC_MANUFACTURED) {
                const double e = exp(t - p.T);
                const double us = e * phi / p.d;
                bsin = p.dt * gam * (3.0 * us * us - (2.0 - 0.5 * p.sigma * p.sigma)) * (-e / p.d);
            }
            cf[0] = (Real)gam;
            cf[1] = (Real)bsin;
            cf[2] = Real(0);
            sums[0] = gam;
            sums[1] = gam * (yL - (2.0 + p.d) / (2.0 * p.d));
        } else {
            double b = 0.0, c = 0.0;
            switch (p.kind) {
            case FBSDE_AC_MANUFACTURED:
            case FBSDE_COS_LINEAR_TEST: b = -yb / p.d; break;                 // x sin
            case FBSDE_HJB_LOGQUAD: {                                        // 1 + s = 2 e^g
                const double one_s = 2.0 * exp(yL);
                b = 2.0 * yb / one_s;                                        // x theta x
                c = yb / one_s;                                              // x x^2
                break;
            }
            case FBSDE_AFFINE_TEST: c = yb; break;                           // x x
            case FBSDE_AC_DOUBLEWELL: b = -0.8 * yb * yL * yL; break;        // x x
            }
            cf[0] = Real(0);
            cf[1] = (Real)b;
            cf[2] = (Real)c;
            sums[0] = yb;
            sums[1] = p.kind == FBSDE_LOGISTIC_GRAD ? yb * yL * (1.0 - yL) / p.d : 0.0;
        }
    }
    block_sum(sums, sm);
    if (threadIdx.x == 0) {
        double *o = ws.spart(s, blockIdx.x);
        for (int i = 0; i < 4; ++i) o[i] = sums[i];
    }
}

// Column sums over the rows Delta_L with the coefficients of k_adj_particles:
//   part 0: sum coef0 Delta;  part 1: sum coef1 phi_B(x);  part 2: sum coef2 phi_C(x),
// x = x0 + Delta.  phi_B = sin (Allen-Cahn kinds) or x (theta-weighted later);
// phi_C = x^2 (log-quadratic terminal) or x (affine terminal).
template <typename Real, int VM>
__global__ void __launch_bounds__(256) k_adj_colsum(Params p, int mode_b, int mode_c)
{
    constexpr int E = Chunk<Real>::E;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int tile = blockIdx.x, g = blockIdx.y, s = blockIdx.z;
    const WS<Real> ws(p);
    const int nch = p.ld / E;
    const int c0 = tile * 256 * VM;
    const int tile_nch = min(nch - c0, 256 * VM);
    const int tpr = min(256, (tile_nch + VM - 1) / VM);
    const int R = 256 / tpr;
    const int rg = threadIdx.x / tpr, tc = threadIdx.x - rg * tpr;
    const Real *x0r = ws.vR(s, 2);
    long long r0, r1;
    row_range(p.M, p.G, g, r0, r1);
    Chunk<Real> acc[3][VM];
#pragma unroll
    for (int v = 0; v < VM; ++v) {
        zero(acc[0][v]);
        zero(acc[1][v]);
        zero(acc[2][v]);
    }
    if (rg < R) {
        for (long long j = r0 + rg; j < r1; j += R) {
            const Real *cf = ws.coef(s, j);
            const Real w0 = cf[0], w1 = cf[1], w2 = cf[2];
            const Real *drow = ws.row(s, j);
#pragma unroll
            for (int v = 0; v < VM; ++v) {
                const int c = c0 + tc + tpr * v;
                if (c - c0 < tile_nch) {
                    const Chunk<Real> dl = ld_chunk(drow + c * E);
                    const Chunk<Real> xc = ldg_chunk(x0r + c * E);
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const Real x = xc.v[e] + dl.v[e];
                        const bool in = c * E + e < p.d;
                        acc[0][v].v[e] += w0 * dl.v[e];
                        const Real fb = mode_b == 1 ? sin(x) : (mode_b == 2 ? x : Real(0));
                        const Real fc = mode_c == 1 ? x * x : (mode_c == 2 ? x : Real(0));
                        if (in) {
                            acc[1][v].v[e] += w1 * fb;
                            acc[2][v].v[e] += w2 * fc;
                        }
                    }
                }
            }
        }
    }
    if (R == 1) {
        if (rg >= R) return;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Real *dst = ws.part(s, g, a);
#pragma unroll
            for (int v = 0; v < VM; ++v) {
                const int c = c0 + tc + tpr * v;
                if (c - c0 < tile_nch) st_chunk(dst + c * E, acc[a][v]);
            }
        }
        return;
    }
    Real *red = reinterpret_cast<Real *>(smem_raw);
    if (rg < R) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int v = 0; v < VM; ++v) {
                const int cl = tc + tpr * v;
                if (cl < tile_nch)
                    st_chunk(red + (((size_t)rg * 3 + a) * tile_nch + cl) * E, acc[a][v]);
            }
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 3 * tile_nch; idx += blockDim.x) {
        const int a = idx / tile_nch, cl = idx - a * tile_nch;
        Chunk<Real> sum = ld_chunk(red + ((size_t)a * tile_nch + cl) * E);
        for (int r = 1; r < R; ++r) {
            const Chunk<Real> o = ld_chunk(red + (((size_t)r * 3 + a) * tile_nch + cl) * E);
#pragma unroll
            for (int e = 0; e < E; ++e) sum.v[e] += o.v[e];
        }
        st_chunk(ws.part(s, g, a) + (c0 + cl) * E, sum);
    }
}

// Per query after the column sums of level L = k+1 (reduced into v64 slots 3..5):
//   L < N: alphabar = sum gamma, alphaxbar = sum gamma Delta_L + sigma dt sum gamma df/dz,
//          x0bar += sum (dt gamma df/dx);
//   L = N: x0bar += grad g terms, thetabar += d_theta g terms.
// Also loads the level-L quantities of z for the next particle pass.
template <typename Real>
__global__ void __launch_bounds__(kFinThreads) k_adj_finalize(Params p)
{
    __shared__ double sm[32 * 4];
    const int s = blockIdx.x, L = p.level + 1;
    const WS<Real> ws(p);
    const Tape tp(p);
    SolveState &st = p.st[s];
    double sc[2] = {0.0, 0.0};
    for (int b = 0; b < p.GP; ++b) {
        sc[0] += ws.spart(s, b)[0];
        sc[1] += ws.spart(s, b)[1];
    }
    const double *A = ws.v64(s, 3), *B = ws.v64(s, 4), *C = ws.v64(s, 5);
    const double *theta = p.theta;
    double *ab = tp.av(s, 0), *xb = tp.av(s, 1), *tb = tp.av(s, 2);
    if (L < p.N) {
        const double *axL = tp.ax(s, L);
        #pragma unroll 4
        for (int i = threadIdx.x; i < p.ld; i += blockDim.x) {
            double zb = 0.0;
            if (i < p.d) {
                switch (p.kind) {
                case FBSDE_LOGISTIC_GRAD: zb = p.sigma * p.dt * sc[1]; break;
                case FBSDE_HJB_LOGQUAD: zb = -p.sigma * p.sigma * p.dt * sc[0] * axL[i]; break;
                case FBSDE_AFFINE_TEST: zb = p.sigma * p.dt * p.c2 * sc[0]; break;
                }
            }
            ab[i] = A[i] + zb;
            xb[i] += B[i];
        }
        if (threadIdx.x == 0) st.abar = sc[0];
    } else {
        for (int i = threadIdx.x; i < p.d; i += blockDim.x) {
            const double th = theta ? theta[i] : 0.0;
            switch (p.kind) {
            case FBSDE_AC_MANUFACTURED:
            case FBSDE_COS_LINEAR_TEST:
            case FBSDE_AC_DOUBLEWELL: xb[i] += B[i]; break;
            case FBSDE_LOGISTIC_GRAD: xb[i] += sc[1]; break;
            case FBSDE_HJB_LOGQUAD:
                xb[i] += th * B[i];
                tb[i] += C[i];
                break;
            case FBSDE_AFFINE_TEST:
                xb[i] += th * sc[0];
                tb[i] += C[i];
                break;
            }
        }
    }
    (void)sm;
}

// Per query: level-L z quantities (sum alpha_x, |alpha_x|^2) for the next Newton adjoint.
template <typename Real>
__global__ void __launch_bounds__(kFinThreads) k_adj_zlevel(Params p)
{
    __shared__ double sm[32 * 4];
    const int s = blockIdx.x, L = p.level + 1;
    const Tape tp(p);
    double a[2] = {0.0, 0.0};
    if (L < p.N) {
        const double *ax = tp.ax(s, L);
        #pragma unroll 4
        for (int i = threadIdx.x; i < p.ld; i += blockDim.x) {
            a[0] += ax[i];
            a[1] += ax[i] * ax[i];
        }
    }
    block_sum(a, sm);
    if (threadIdx.x == 0) {
        p.st[s].sumz_l = p.sigma * a[0];
        p.st[s].zz_l = p.sigma * p.sigma * a[1];
    }
}

// Outputs: x0bar [Q][d]; thetabar [d] = sum over queries (in query order).
template <typename Real>
__global__ void k_adj_output(Params p, double *x0bar, double *thetabar)
{
    const Tape tp(p);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < p.Q * p.d;
         idx += gridDim.x * blockDim.x) {
        const int s = idx / p.d, i = idx - s * p.d;
        x0bar[idx] = tp.av(s, 1)[i];
    }
    if (thetabar) {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p.d; i += gridDim.x * blockDim.x) {
            double a = 0.0;
            for (int s = 0; s < p.Q; ++s) a += tp.av(s, 2)[i];
            thetabar[i] = a;
        }
    }
}

}  // namespace dev
}  // namespace fbsde
