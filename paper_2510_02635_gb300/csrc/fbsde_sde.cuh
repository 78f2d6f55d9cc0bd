// fbsde_sde.cuh -- kernels of the scheme with a drift and a state-dependent diffusion: the
// forward SDE of Sec. 2.1, dX = mu(t,X) dt + sigma(t,X) dW, with the componentwise affine
// coefficients mu_i(x) = mu0 + mu1 x_i and sigma(x) = diag(sigma + sig1 x_i).  Included
// after fbsde_kernels.cuh.
//
//   k_sde_anchor   the drift path of x0, a_{k+1} = a_k + mu(a_k) dt (the anchor of the
//                  level-k regression), kept as offsets c_k = a_k - x0;
//   k_sde_forward  one Euler-Maruyama step (2.7) of the rows, out of place:
//                  Delta_{k+1} = Delta_k + mu(x) dt + sigma(x) sqrt(dt) xi_k, x = x0 + Delta_k;
//   k_sde_rows     per row segment of level k: alpha_x . Delta, |Delta|^2, |Delta - c|^2 (c
//                  the anchor of the regression that level k's values feed), g . Delta (the
//                  next solve's starting guess) and the two feature sums of f (of g at k = N);
//   k_sde_rho      the cloud's mean squared distance to that anchor, the kernel scale.
// Rows hold Delta = X - x0; the regression on Delta equals the regression on X - a_k up to
// its intercept, which is then the value at Delta = 0 (the slope and the centred operator
// do not move with the anchor).
#pragma once
#include "fbsde_kernels.cuh"

namespace fbsde {
namespace dev {

// c_0 = 0, c_{k+1} = c_k + (mu0 + mu1 (x0 + c_k)) dt per coordinate, in FP64, for
// k = 0..N (grid-stride over (query, coordinate); padding stays zero).
template <typename Real>
__global__ void __launch_bounds__(256) k_sde_anchor(Params p)
{
    const WS<Real> ws(p);
    const long long n = (long long)p.Q * p.ld;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < n;
         it += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(it / p.ld), i = (int)(it - (long long)s * p.ld);
        const double x0 = ws.v64(s, 6)[i];
        double c = 0.0;
        for (int k = 0; k <= p.N; ++k) {
            ws.anchor(s, k)[i] = i < p.d ? (Real)c : Real(0);
            c += (p.mu0 + p.mu1 * (x0 + c)) * p.dt;
        }
    }
}

// Euler-Maruyama step k -> k + 1 of every row; from == nullptr: level 0 (Delta_0 = 0).
// One warp per (query, particle, row segment), the walk of k_update (no integer division
// per item); padding (i >= d) stays zero.
template <typename Real, int VPT>
__global__ void __launch_bounds__(256) k_sde_forward(Params p, int k, const Real *from, Real *to)
{
    constexpr int E = Chunk<Real>::E;
    const WS<Real> ws(p);
    const int lane = threadIdx.x & 31;
    const int nch = p.ld / E;
    const Real sdt = (Real)sqrt(p.dt), dt = (Real)p.dt;
    const Real mu0 = (Real)p.mu0, mu1 = (Real)p.mu1, sg0 = (Real)p.sigma, sg1 = (Real)p.sig1;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (RowItems w(p, (((unsigned long long)blockIdx.x * blockDim.x) + threadIdx.x) >> 5,
                    (unsigned long long)nwarps);
         w.s < (uint32_t)p.Q; w.next()) {
        const int seg = (int)w.seg, s = (int)w.s;
        const size_t row = (size_t)s * p.M + w.j;
        const Real *src = from ? from + row * p.ld : nullptr;
        Real *dst = to + row * p.ld;
        const Real *x0r = ws.vR(s, 2);
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int c = seg * 32 * VPT + lane + 32 * v;
            if (c < nch) {
                Chunk<Real> dl;
                if (src) dl = ld_chunk(src + c * E);
                else zero(dl);
                const Chunk<Real> xc = ldg_chunk(x0r + c * E);
                const Chunk<Real> z = normal_chunk((Chunk<Real> *)nullptr, c, w.j, (uint32_t)k,
                                                   p.solve0 + (uint32_t)s, p.key0, p.key1, p.d);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const Real x = xc.v[e] + dl.v[e];
                    const Real v2 = dl.v[e] + (mu0 + mu1 * x) * dt + (sg0 + sg1 * x) * sdt * z.v[e];
                    dl.v[e] = c * E + e < p.d ? v2 : Real(0);
                }
                st_chunk(dst + c * E, dl);
            }
        }
    }
}

// Per-element terms of the two feature sums of level k (k < N: f's; k = N: g's) at
// x = x0 + Delta (sines and cosines in the stream precision, as cos_stream):
//   kind 0:   cos x (the Allen-Cahn source);
//   kind 7:   cos x and s^2 cos x / 2 + m sin x  (s = sigma + sig1 x, m = mu0 + mu1 x);
//   kind 8:   x^2 and s^2 + 2 m x;
//   k = N:    the terminal feature of g (g_term of the driftless kinds; cos x for kind 7,
//             x^2 for kind 8).
template <typename Real>
__device__ __forceinline__ void sde_terms(const Params &p, bool terminal, Real x, Real th,
                                          Real &t4, Real &t5)
{
    const Real m = (Real)p.mu0 + (Real)p.mu1 * x, sg = (Real)p.sigma + (Real)p.sig1 * x;
    t5 = Real(0);
    if (terminal) {
        t4 = p.kind == FBSDE_DRIFT_AC ? cos_stream(x)
             : p.kind == FBSDE_DRIFT_QUAD ? x * x
                                          : g_term(p.kind, x, th);
        return;
    }
    switch (p.kind) {
    case FBSDE_AC_MANUFACTURED:
        t4 = cos_stream(x);
        break;
    case FBSDE_DRIFT_AC: {
        const Real cx = cos_stream(x), sx = sin_stream(x);
        t4 = cx;
        t5 = Real(0.5) * sg * sg * cx + m * sx;
        break;
    }
    case FBSDE_DRIFT_QUAD:
        t4 = x * x;
        t5 = sg * sg + Real(2) * m * x;
        break;
    default:
        t4 = Real(0);
    }
}

// Row sums of level k (one warp per (query, particle, row segment), the layout of
// k_update): [0] alpha_x . Delta, [1] |Delta|^2, [2] |Delta - c|^2 with c the anchor offset
// of level k - 1 (the regression level k's values feed), [3] g . Delta (g the starting
// guess of that regression's solve), [4], [5] the feature sums (sde_terms; padding
// excluded).
// src != nullptr: the rows of level k are read from src (a stored level) and copied into
// the row buffer on the way.
template <typename Real, int VPT>
__global__ void __launch_bounds__(256) k_sde_rows(Params p, int k, const Real *src)
{
    constexpr int E = Chunk<Real>::E;
    const WS<Real> ws(p);
    const int lane = threadIdx.x & 31;
    const int nch = p.ld / E;
    const bool terminal = k == p.N;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (RowItems w(p, (((unsigned long long)blockIdx.x * blockDim.x) + threadIdx.x) >> 5,
                    (unsigned long long)nwarps);
         w.s < (uint32_t)p.Q; w.next()) {
        const int seg = (int)w.seg, s = (int)w.s;
        const long long j = w.j;
        Real *drow = ws.row(s, j);
        const Real *srow = src ? src + ((size_t)s * p.M + j) * p.ld : nullptr;
        const Real *ar = ws.anchor(s, k - 1);
        Real acc[kSegSums] = {Real(0), Real(0), Real(0), Real(0), Real(0), Real(0)};
#pragma unroll
        for (int v = 0; v < VPT; ++v) {
            const int c = seg * 32 * VPT + lane + 32 * v;
            if (c < nch) {
                Chunk<Real> dl;
                if (srow) {
                    dl = ld_chunk(srow + c * E);
                    st_chunk(drow + c * E, dl);
                } else {
                    dl = ld_chunk(drow + c * E);
                }
                const Chunk<Real> xc = ldg_chunk(ws.vR(s, 1) + c * E);   // alpha_x
                const Chunk<Real> x0c = ldg_chunk(ws.vR(s, 2) + c * E);
                const Chunk<Real> gc = ldg_chunk(ws.vR(s, 3) + c * E);
                const Chunk<Real> cc = ldg_chunk(ar + c * E);
                const Chunk<Real> th = ldg_chunk(ws.thetaR() + c * E);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const Real dv = dl.v[e];
                    acc[0] += xc.v[e] * dv;
                    acc[1] += dv * dv;
                    acc[2] += (dv - cc.v[e]) * (dv - cc.v[e]);
                    acc[3] += gc.v[e] * dv;
                    if (c * E + e < p.d) {
                        Real t4, t5;
                        sde_terms(p, terminal, x0c.v[e] + dv, th.v[e], t4, t5);
                        acc[4] += t4;
                        acc[5] += t5;
                    }
                }
            }
        }
        warp_sum(acc);
        if (lane == 0) {
            Real *o = ws.segp(s, j, seg);
#pragma unroll
            for (int a = 0; a < kSegSums; ++a) o[a] = acc[a];
        }
    }
}

// One CTA per query: rho_ref = (1/M) sum_j |Delta_j - c|^2, the kernel scale of the
// regression level k's values feed (strided over the particles, then the block tree).
template <typename Real>
__global__ void __launch_bounds__(kFinThreads) k_sde_rho(Params p)
{
    __shared__ double sm[32 * 4];
    const int s = blockIdx.x;
    const WS<Real> ws(p);
    double acc[1] = {0.0};
    for (long long j = threadIdx.x; j < p.M; j += blockDim.x) {
        double r = 0.0;
        for (int seg = 0; seg < p.nseg; ++seg) r += (double)ws.segp(s, j, seg)[2];
        acc[0] += r;
    }
    block_sum(acc, sm);
    if (threadIdx.x == 0) p.st[s].rho_ref = acc[0] / (double)p.M;
}

}  // namespace dev
}  // namespace fbsde
