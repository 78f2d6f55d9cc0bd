// fbsde_anchored.cu -- Algorithm 1 in its literal form: one regression per particle
// anchor (the backward loop over m of Algorithm 1, the local linear approximation (2.9)
// centred at each particle's own position X_k^m).  For a query x0, at level k:
//   D_j^m = X_{k+1}^j - X_k^m, rho_jm = |D_j^m|^2 = |P_j|^2 + |A_m|^2 - 2 P_j . A_m with
//   P = X_{k+1} - x0 and A = X_k - x0 (the particle rows of both levels),
//   w_jm = K(rho_jm) (Gaussian, eps_k^2 = h^2 sigma^2 d (t_k + t_{k+1})),
//   W_m = sum_j w_jm, c_m = sum_j w_jm Y_j / W_m, S_m = (sum_j w_jm P_j) / W_m - A_m,
//   rhs_m = (sum_j w_jm Y_j P_j - c_m sum_j w_jm P_j) / W_m        (Eq. 3.19),
//   lambda_m = ridge_rel (sum_j w_jm rho_jm / W_m - |S_m|^2) / d    (Remark 2.2),
// then for every anchor at once the CG on (Gamma_m + lambda_m I) x_m = rhs_m with
//   Gamma_m v = sum_j w_jm (D_j^m . v) D_j^m / W_m - S_m (S_m . v),
//   D_j^m . v_m = P_j . v_m - A_m . v_m,
// i.e. per CG pass the two contractions U = P V^T (M x M x d) and G = T^T P
// (M x d x M, T_jm = w_jm (U_jm - A_m . v_m) / W_m): Gamma_m v_m = G_m - (sum_j T_jm) A_m
// - S_m (S_m . v_m).  Finally alpha_m = c_m - S_m . x_m (Eq. 3.20), Z_k^m = sigma x_m and
// Newton (2.16)-(2.17) Y_k^m = alpha_m + dt f(t_k, X_k^m, Y_k^m, Z_k^m).  u(0,x0) is the
// mean of Y_0^m; grad u(0,x0) = x of anchor 0 at k = 0 (every anchor is x0 there).
// The particle paths are the solve's own (Brownian bridge, Philox normals).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fbsde_kernels.cuh"

namespace fbsde {
namespace anchored {

using dev::Chunk;

// Per-anchor scalars of the regression and its CG.
struct Anchor {
    double W, c, lam, rr, rhs2, sp, ap, alpha;
    int32_t done, iters, status, pad;
};

// ---------------------------------------------------------------------------
// Tiled SIMT matrix product, 64 x 64 tile per block, 256 threads of 4 x 4 outputs.
//   TN = false: C[r][c] = sum_k A[r][k] B[c][k]   (A: Mr x K, B: Nc x K, row-major)
//   TN = true:  C[r][c] = sum_k A[k][r] B[k][c]   (A: K x Mr, B: K x Nc, row-major)
// The sum over k runs in tile order and, inside a tile, in k order (fixed per layout).
// Split K: block z sums k in [z kc, (z+1) kc) into its own output C + z Mr ldc; the
// consumers add the splits in z order.
// ---------------------------------------------------------------------------
template <typename Real, bool TN>
__global__ void __launch_bounds__(256) k_gemm(int Mr, int Nc, int K, int kc,
                                              const Real *__restrict__ A, int lda,
                                              const Real *__restrict__ B, int ldb,
                                              Real *__restrict__ C, int ldc)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ Real As[BK][BM + 1];
    __shared__ Real Bs[BK][BN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
    const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
    C += (size_t)blockIdx.z * Mr * ldc;
    Real acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = Real(0);
    for (int k0 = kb; k0 < ke; k0 += BK) {
        for (int e = threadIdx.x; e < BM * BK; e += 256) {
            int kk, rr;
            if (TN) { kk = e / BM; rr = e - kk * BM; }
            else { rr = e / BK; kk = e - rr * BK; }
            const int gr = r0 + rr, gk = k0 + kk;
            Real v = Real(0);
            if (gr < Mr && gk < ke) v = TN ? A[(size_t)gk * lda + gr] : A[(size_t)gr * lda + gk];
            As[kk][rr] = v;
        }
        for (int e = threadIdx.x; e < BN * BK; e += 256) {
            int kk, cc;
            if (TN) { kk = e / BN; cc = e - kk * BN; }
            else { cc = e / BK; kk = e - cc * BK; }
            const int gc = c0 + cc, gk = k0 + kk;
            Real v = Real(0);
            if (gc < Nc && gk < ke) v = TN ? B[(size_t)gk * ldb + gc] : B[(size_t)gc * ldb + gk];
            Bs[kk][cc] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            Real a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + ty + 16 * i;
        if (r >= Mr) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = c0 + tx + 16 * j;
            if (c < Nc) C[(size_t)r * ldc + c] = acc[i][j];
        }
    }
}

// FP32 variant with a 128 x 128 tile per block: 256 threads, each owning an 8 x 8 block
// of outputs (rows 4 ty .. 4 ty + 3 and 64 + 4 ty .., columns likewise with tx), read from
// shared memory four at a time.  Same layouts, split K and summation order rules as k_gemm.
template <bool TN>
__global__ void __launch_bounds__(256) k_gemm128(int Mr, int Nc, int K, int kc,
                                                 const float *__restrict__ A, int lda,
                                                 const float *__restrict__ B, int ldb,
                                                 float *__restrict__ C, int ldc)
{
    constexpr int BM = 128, BN = 128, BK = 8, PAD = 4;
    __shared__ __align__(16) float As[BK][BM + PAD];
    __shared__ __align__(16) float Bs[BK][BN + PAD];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int r0 = blockIdx.y * BM, c0 = blockIdx.x * BN;
    const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
    C += (size_t)blockIdx.z * Mr * ldc;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
    for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = threadIdx.x + 256 * u;
            int kk, rr;
            if (TN) { kk = e / BM; rr = e - kk * BM; }
            else { rr = e / BK; kk = e - rr * BK; }
            const int gr = r0 + rr, gk = k0 + kk;
            float v = 0.0f;
            if (gr < Mr && gk < ke) v = TN ? A[(size_t)gk * lda + gr] : A[(size_t)gr * lda + gk];
            As[kk][rr] = v;
            int cc;
            if (TN) { kk = e / BN; cc = e - kk * BN; }
            else { cc = e / BK; kk = e - cc * BK; }
            const int gc = c0 + cc, gk2 = k0 + kk;
            float w = 0.0f;
            if (gc < Nc && gk2 < ke) w = TN ? B[(size_t)gk2 * ldb + gc] : B[(size_t)gc * ldb + gk2];
            Bs[kk][cc] = w;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[kk][4 * ty]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[kk][64 + 4 * ty]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[kk][4 * tx]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[kk][64 + 4 * tx]);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = r0 + (i < 4 ? 4 * ty + i : 64 + 4 * ty + i - 4);
        if (r >= Mr) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = c0 + (j < 4 ? 4 * tx + j : 64 + 4 * tx + j - 4);
            if (c < Nc) C[(size_t)r * ldc + c] = acc[i][j];
        }
    }
}

// Fixed-order block sum of NV doubles (blockDim.x a multiple of 32, <= 1024).
template <int NV> __device__ __forceinline__ void bsum(double (&v)[NV], double *sm)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i)
#pragma unroll
        for (int o = 16; o; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sm[warp * NV + i] = v[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double a = 0.0;
        for (int w = 0; w < nw; ++w) a += sm[w * NV + i];
        v[i] = a;
    }
    __syncthreads();
}

// Terminal level: P_j = sigma sqrt(T) xi_{N,j} (end point of the Brownian path) and
// Y_j = g(x0 + P_j).  One block per particle.
template <typename Real>
__global__ void __launch_bounds__(128) k_anc_terminal(Params p, const double *x0, uint32_t sidx,
                                                      Real *P, double *Y)
{
    constexpr int E = Chunk<Real>::E;
    __shared__ double sm[32];
    const int j = blockIdx.x;
    const int nch = p.ld / E;
    const Real wb = (Real)(p.sigma * sqrt(p.T));
    double acc[1] = {0.0};
    for (int c = threadIdx.x; c < nch; c += blockDim.x) {
        Chunk<Real> z = dev::normal_chunk((Chunk<Real> *)nullptr, c, (uint32_t)j, (uint32_t)p.N,
                                          sidx, p.key0, p.key1, p.d);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int i = c * E + e;
            const Real v = wb * z.v[e];
            P[(size_t)j * p.ld + i] = v;
            if (i < p.d) {
                const Real th = p.theta ? (Real)p.theta[i] : Real(0);
                acc[0] += (double)dev::g_term(p.kind, (Real)x0[i] + v, th);
            }
        }
    }
    bsum(acc, sm);
    if (threadIdx.x == 0) Y[j] = dev::g_value(p, acc[0]);
}

// Brownian-bridge step to level k (1 <= k < N): A_j = a P_j + b xi_{k,j}; level 0: A = 0.
template <typename Real>
__global__ void k_anc_step(Params p, int k, uint32_t sidx, double a, double b, const Real *P, Real *A)
{
    constexpr int E = Chunk<Real>::E;
    const int nch = p.ld / E;
    const long long n = (long long)p.M * nch;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < n;
         it += (long long)gridDim.x * blockDim.x) {
        const long long j = it / nch;
        const int c = (int)(it - j * nch);
        Chunk<Real> o;
        if (k == 0) {
            dev::zero(o);
        } else {
            const Chunk<Real> z = dev::normal_chunk((Chunk<Real> *)nullptr, c, (uint32_t)j,
                                                    (uint32_t)k, sidx, p.key0, p.key1, p.d);
            const Chunk<Real> x = dev::ld_chunk(P + (size_t)j * p.ld + c * E);
#pragma unroll
            for (int e = 0; e < E; ++e) o.v[e] = (Real)a * x.v[e] + (Real)b * z.v[e];
        }
        dev::st_chunk(A + (size_t)j * p.ld + c * E, o);
    }
}

// Row norms |X_j|^2 and, with Y, the rows Y_j P_j.  One block per row.
template <typename Real>
__global__ void __launch_bounds__(128) k_anc_rows(Params p, const Real *P, const Real *A,
                                                  const double *Y, double *pn, double *an, Real *YP)
{
    __shared__ double sm[32 * 2];
    const int j = blockIdx.x;
    double acc[2] = {0.0, 0.0};
    const double y = Y[j];
    for (int i = threadIdx.x; i < p.ld; i += blockDim.x) {
        const Real x = P[(size_t)j * p.ld + i], a = A[(size_t)j * p.ld + i];
        acc[0] += (double)x * x;
        acc[1] += (double)a * a;
        YP[(size_t)j * p.ld + i] = (Real)(y * (double)x);
    }
    bsum(acc, sm);
    if (threadIdx.x == 0) {
        pn[j] = acc[0];
        an[j] = acc[1];
    }
}

// Column pass over the rows j of chunk blockIdx.y (kRowChunk rows, in order) for every
// anchor m (thread per anchor); per-chunk partial sums go to part[chunk][m][.] and the
// consumers add the chunks in order.
//   mode 0: w_jm from rho_jm = pn_j + an_m - 2 G_jm, stored in W; sums w, w Y, w rho.
//   mode 1: T_jm = w_jm (G_jm - A_m . v_m) / W_m stored in T; sum T.
constexpr int kRowChunk = 64;
template <typename Real>
__global__ void k_anc_columns(Params p, int mode, double rho_ref, const Real *G, const double *pn,
                              const double *an, const double *Y, Real *W, Real *T,
                              const Anchor *st, double *part)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= p.M) return;
    const long long j0 = (long long)blockIdx.y * kRowChunk;
    const long long j1 = min((long long)p.M, j0 + kRowChunk);
    double *o = part + ((size_t)blockIdx.y * p.M + m) * 3;
    // arithmetic in the stream precision (the FP64 pipe is a small fraction of the FP32
    // one on this part); the chunk sums are widened to FP64
    if (mode == 0) {
        Real sw = 0, swy = 0, swr = 0;
        const Real am = (Real)an[m], ref = (Real)rho_ref;
        const Real scale = p.uniform ? Real(0) : (Real)(-1.0 / (p.h2 * rho_ref));
        for (long long j = j0; j < j1; ++j) {
            const Real rho = max((Real)pn[j] + am - Real(2) * G[(size_t)j * p.M + m], Real(0));
            const Real w = exp((rho - ref) * scale);
            W[(size_t)j * p.M + m] = w;
            sw += w;
            swy += w * (Real)Y[j];
            swr += w * rho;
        }
        o[0] = (double)sw;
        o[1] = (double)swy;
        o[2] = (double)swr;
    } else {
        const Anchor &a = st[m];
        if (a.done) return;
        const Real inv = (Real)(1.0 / a.W), ap = (Real)a.ap;
        Real sum = 0;
        for (long long j = j0; j < j1; ++j) {
            const size_t ix = (size_t)j * p.M + m;
            const Real t = W[ix] * (G[ix] - ap) * inv;
            T[ix] = t;
            sum += t;
        }
        o[0] = (double)sum;
    }
}

// Per anchor (one block): S, rhs, lambda, and the CG start x = 0, r = p = rhs.
template <typename Real>
__global__ void __launch_bounds__(256) k_anc_setup(Params p, int nrc, int nsplit, const Real *A,
                                                   const Real *G2, const Real *G3,
                                                   const double *part, Anchor *st, double *S,
                                                   double *rhs, double *x, double *r, double *pv,
                                                   Real *V)
{
    __shared__ double sm[32 * 4];
    __shared__ double sw_sh[3];
    const int m = blockIdx.x;
    Anchor &a = st[m];
    if (threadIdx.x == 0) {   // the column sums of the weights, chunks in order
        double sw = 0.0, swy = 0.0, swr = 0.0;
        for (int c = 0; c < nrc; ++c) {
            const double *o = part + ((size_t)c * p.M + m) * 3;
            sw += o[0];
            swy += o[1];
            swr += o[2];
        }
        sw_sh[0] = sw;
        sw_sh[1] = swy / sw;
        sw_sh[2] = swr / sw;
    }
    __syncthreads();
    const double invW = 1.0 / sw_sh[0], c = sw_sh[1];
    const size_t o = (size_t)m * p.ld, split = (size_t)p.M * p.ld;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};   // |S|^2, |rhs|^2, S . rhs, A . rhs
    for (int i = threadIdx.x; i < p.ld; i += blockDim.x) {
        double g2 = 0.0, g3 = 0.0;
        for (int z = 0; z < nsplit; ++z) {
            g2 += (double)G2[z * split + o + i];
            g3 += (double)G3[z * split + o + i];
        }
        g2 *= invW;
        const double s = g2 - (double)A[o + i];
        const double b = g3 * invW - c * g2;
        S[o + i] = s;
        rhs[o + i] = b;
        x[o + i] = 0.0;
        r[o + i] = b;
        pv[o + i] = b;
        V[o + i] = (Real)b;
        acc[0] += s * s;
        acc[1] += b * b;
        acc[2] += s * b;
        acc[3] += (double)A[o + i] * b;
    }
    bsum(acc, sm);
    if (threadIdx.x == 0) {
        a.W = sw_sh[0];
        a.c = c;
        a.lam = p.ridge_rel * (sw_sh[2] - acc[0]) / p.d;
        a.rr = acc[1];
        a.rhs2 = acc[1];
        a.sp = acc[2];
        a.ap = acc[3];
        a.iters = 0;
        a.status = 0;
        a.done = acc[1] == 0.0 ? 1 : 0;
    }
}

// One CG pass per anchor (one warp per anchor, kAncWarps anchors per block):
// q = G_m - colsum_m A_m - S_m (S_m . p_m) + lambda p, a = rr / (p . q), x += a p,
// r -= a q, p = r + (rr'/rr) p; counts the anchors still active.
constexpr int kAncWarps = 8;
__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <typename Real>
__global__ void __launch_bounds__(32 * kAncWarps) k_anc_cg(Params p, int nrc, int nsplit,
                                                           const Real *A, const Real *G,
                                                           const double *part, const double *S,
                                                           Anchor *st, double *x, double *r,
                                                           double *pv, double *q, Real *V,
                                                           int *active)
{
    const int lane = threadIdx.x & 31;
    const int m = blockIdx.x * kAncWarps + (threadIdx.x >> 5);
    if (m >= p.M) return;
    Anchor &a = st[m];
    if (a.done) return;
    double cs = 0.0;   // sum_j T_jm, row chunks in order (lane 0's sum is used)
    for (int c = lane; c < nrc; c += 32) cs += part[((size_t)c * p.M + m) * 3];
    cs = __shfl_sync(0xffffffffu, wsum(cs), 0);
    const size_t o = (size_t)m * p.ld, split = (size_t)p.M * p.ld;
    const double sp = a.sp, lam = a.lam, rr = a.rr;
    double pq = 0.0;
    for (int i = lane; i < p.ld; i += 32) {
        double g = 0.0;
        for (int z = 0; z < nsplit; ++z) g += (double)G[z * split + o + i];
        const double qi = g - cs * (double)A[o + i] - S[o + i] * sp + lam * pv[o + i];
        q[o + i] = qi;
        pq += pv[o + i] * qi;
    }
    pq = __shfl_sync(0xffffffffu, wsum(pq), 0);
    if (!(pq > 0.0) || !isfinite(pq)) {
        if (lane == 0) {
            a.done = 1;
            if (!(rr <= p.cg_tol2 * a.rhs2)) a.status = FBSDE_ERR_CG;
        }
        return;
    }
    const double step = rr / pq;
    double rn = 0.0;
    for (int i = lane; i < p.ld; i += 32) {
        x[o + i] += step * pv[o + i];
        const double ri = r[o + i] - step * q[o + i];
        r[o + i] = ri;
        rn += ri * ri;
    }
    const double rr_new = __shfl_sync(0xffffffffu, wsum(rn), 0), beta = rr_new / rr;
    double b0 = 0.0, b1 = 0.0;
    for (int i = lane; i < p.ld; i += 32) {
        const double pi = r[o + i] + beta * pv[o + i];
        pv[o + i] = pi;
        V[o + i] = (Real)pi;
        b0 += S[o + i] * pi;
        b1 += (double)A[o + i] * pi;
    }
    b0 = wsum(b0);
    b1 = wsum(b1);
    if (lane == 0) {
        a.rr = rr_new;
        a.sp = b0;
        a.ap = b1;
        a.iters += 1;
        if (rr_new <= p.cg_tol2 * a.rhs2) {
            a.done = 1;
        } else if (a.iters >= p.cg_max_iter) {
            a.done = 1;
            a.status = FBSDE_ERR_CG;
        } else {
            atomicAdd(active, 1);
        }
    }
}

// Per anchor (one block): alpha = c - S . x (Eq. 3.20), Z = sigma x, the features of f at
// (t_k, X_k^m, Z) and Newton (2.16)-(2.17) for Y_k^m.
template <typename Real>
__global__ void __launch_bounds__(256) k_anc_newton(Params p, double t_k, const double *x0,
                                                    const Real *A, const double *S,
                                                    const double *x, Anchor *st, double *Ynew,
                                                    int *status)
{
    __shared__ double sm[32 * 4];
    const int m = blockIdx.x;
    Anchor &a = st[m];
    const size_t o = (size_t)m * p.ld;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};   // S . x, sum cos(x0 + A), sum x, |x|^2
    for (int i = threadIdx.x; i < p.ld; i += blockDim.x) {
        const double xi = x[o + i];
        acc[0] += S[o + i] * xi;
        if (i < p.d) acc[1] += cos(x0[i] + (double)A[o + i]);
        acc[2] += xi;
        acc[3] += xi * xi;
    }
    bsum(acc, sm);
    if (threadIdx.x == 0) {
        const double alpha = a.c - acc[0];
        a.alpha = alpha;
        const double feat = dev::f_feature(p, t_k, acc[1], p.sigma * acc[2],
                                           p.sigma * p.sigma * acc[3]);
        int it;
        const double y = dev::newton(p, alpha, feat, it);
        Ynew[m] = y;
        int s = a.status;
        if (it < 0 && s == 0) s = FBSDE_ERR_NEWTON;
        if (!isfinite(y) && s == 0) s = FBSDE_ERR_NONFINITE;
        if (s) atomicCAS(status, 0, s);
    }
}

// u(0,x0) = mean of Y_0^m (fixed order) and grad u(0,x0) = x of anchor 0.
__global__ void __launch_bounds__(256) k_anc_output(int M, int d, const double *Y, const double *x,
                                                    double *u0, double *grad)
{
    __shared__ double sm[32];
    double acc[1] = {0.0};
    for (int m = threadIdx.x; m < M; m += blockDim.x) acc[0] += Y[m];
    bsum(acc, sm);
    if (threadIdx.x == 0) *u0 = acc[0] / M;
    if (grad)
        for (int i = threadIdx.x; i < d; i += blockDim.x) grad[i] = x[i];
}

}  // namespace anchored
}  // namespace fbsde

// ---------------------------------------------------------------------------
// Host driver.
// ---------------------------------------------------------------------------
namespace fbsde {
namespace anchored {
namespace {

constexpr size_t kAl = 256;
inline size_t up(size_t x) { return (x + kAl - 1) / kAl * kAl; }
constexpr int64_t kMaxM = 32768;   // three M x M matrices per call
constexpr int kCheckEvery = 4;     // CG passes between host checks of the active count

struct Lay {
    int d, ld, N;
    int64_t M;
    size_t rs;   // bytes of one stream-precision value
    int nrc, nsplit, kc;   // row chunks of the column pass; K splits (kc rows each) of the
                           // tall contractions
    size_t P, A, YP, V, G1, W, T, G2, G3, S, rhs, x, r, pv, q, Y, Yn, pn, an, cs, st, cnt, total;
};

bool lay(const fbsde_problem *P, Lay &L)
{
    if (!P || P->d < 1 || P->N < 1 || P->M < 2 || P->M > kMaxM) return false;
    if (P->kind < FBSDE_AC_MANUFACTURED || P->kind > FBSDE_COS_LINEAR_TEST) return false;
    if (P->precision != FBSDE_FP32 && P->precision != FBSDE_FP64) return false;
    if (P->d > (P->precision == FBSDE_FP64 ? FBSDE_MAX_D_FP64 : FBSDE_MAX_D)) return false;
    if (!(P->sigma > 0.0) || !(P->T > 0.0) || !(P->cg_tol > 0.0) || !(P->ridge_rel >= 0.0))
        return false;
    if (P->cg_max_iter < 0 || P->newton_max_iter < 0) return false;
    L.d = P->d;
    L.ld = (P->d + 3) / 4 * 4;
    L.N = P->N;
    L.M = P->M;
    L.rs = P->precision == FBSDE_FP32 ? 4 : 8;
    const size_t M = (size_t)L.M, ld = (size_t)L.ld;
    L.nrc = (int)((L.M + kRowChunk - 1) / kRowChunk);
    {   // enough blocks for about two waves of the 152 SMs, at least 256 rows per split
        const long long tiles = ((long long)(ld + 63) / 64) * ((L.M + 63) / 64);
        const long long want = std::max(1ll, (2ll * 152 * 4 + tiles - 1) / tiles);
        const long long ns = std::max(1ll, std::min(want, (long long)(L.M / 256)));
        L.kc = (int)(((L.M + ns - 1) / ns + 15) / 16 * 16);
        L.nsplit = (int)((L.M + L.kc - 1) / L.kc);   // every split holds rows
    }
    size_t o = 0;
    auto take = [&](size_t b) { const size_t r = o; o = up(o + b); return r; };
    L.P = take(M * ld * L.rs);
    L.A = take(M * ld * L.rs);
    L.YP = take(M * ld * L.rs);
    L.V = take(M * ld * L.rs);
    L.G1 = take(M * M * L.rs);
    L.W = take(M * M * L.rs);
    L.T = take(M * M * L.rs);
    L.G2 = take((size_t)L.nsplit * M * ld * L.rs);
    L.G3 = take((size_t)L.nsplit * M * ld * L.rs);
    L.S = take(M * ld * 8);
    L.rhs = take(M * ld * 8);
    L.x = take(M * ld * 8);
    L.r = take(M * ld * 8);
    L.pv = take(M * ld * 8);
    L.q = take(M * ld * 8);
    L.Y = take(M * 8);
    L.Yn = take(M * 8);
    L.pn = take(M * 8);
    L.an = take(M * 8);
    L.cs = take((size_t)L.nrc * M * 3 * 8);
    L.st = take(M * sizeof(Anchor));
    L.cnt = take(2 * sizeof(int));
    L.total = o;
    return true;
}

Params params_of(const fbsde_problem *P, const Lay &L, uint64_t seed)
{
    Params p{};
    p.kind = P->kind;
    p.d = P->d;
    p.ld = L.ld;
    p.N = P->N;
    p.M = P->M;
    p.Q = 1;
    p.sigma = P->sigma;
    p.T = P->T;
    p.dt = P->T / P->N;
    p.sdt = P->sigma * std::sqrt(p.dt);
    p.A = P->A;
    p.c0 = P->c0;
    p.c1 = P->c1;
    p.c2 = P->c2;
    p.c3 = P->c3;
    p.uniform = !(P->h > 0.0) || std::isinf(P->h);
    p.h2 = p.uniform ? 1.0 : P->h * P->h;
    p.ridge_rel = P->ridge_rel;
    p.cg_tol2 = P->cg_tol * P->cg_tol;
    p.cg_max_iter = P->cg_max_iter > 0 ? P->cg_max_iter : 200;
    p.newton_max_iter = P->newton_max_iter > 0 ? P->newton_max_iter : 50;
    p.newton_tol = P->newton_tol > 0.0 ? P->newton_tol : 1e-13;
    p.theta = P->theta;
    p.key0 = (uint32_t)seed;
    p.key1 = (uint32_t)(seed >> 32);
    return p;
}

template <typename Real, bool TN>
cudaError_t gemm(int Mr, int Nc, int K, int kc, const Real *A, int lda, const Real *B, int ldb,
                 Real *C, int ldc, cudaStream_t s)
{
    if constexpr (sizeof(Real) == 4) {
        if (Mr >= 1024 && Nc >= 64) {   // large enough to fill the GPU with 128 x 128 tiles
            const dim3 grid((Nc + 127) / 128, (Mr + 127) / 128, (K + kc - 1) / kc);
            k_gemm128<TN><<<grid, 256, 0, s>>>(Mr, Nc, K, kc, A, lda, B, ldb, C, ldc);
            return cudaGetLastError();
        }
    }
    const dim3 grid((Nc + 63) / 64, (Mr + 63) / 64, (K + kc - 1) / kc);
    k_gemm<Real, TN><<<grid, 256, 0, s>>>(Mr, Nc, K, kc, A, lda, B, ldb, C, ldc);
    return cudaGetLastError();
}

#define ANC_TRY(call)                                                                       \
    do {                                                                                     \
        if ((e = (call)) != cudaSuccess) return e;                                           \
    } while (0)

// One query: the forward sweep, then the levels k = N-1..0.  *status gets the first
// device status (CG or Newton failure); the call synchronises on s for the CG checks.
template <typename Real>
cudaError_t solve_one(const fbsde_problem *Pb, const Lay &L, const double *x0, uint64_t seed,
                      uint32_t sidx, double *u0, double *grad, char *ws, cudaStream_t s,
                      int *status, int *host_cnt)
{
    cudaError_t e;
    Params p = params_of(Pb, L, seed);
    const int M = (int)L.M, ld = L.ld;
    Real *P = reinterpret_cast<Real *>(ws + L.P), *A = reinterpret_cast<Real *>(ws + L.A);
    Real *YP = reinterpret_cast<Real *>(ws + L.YP), *V = reinterpret_cast<Real *>(ws + L.V);
    Real *G1 = reinterpret_cast<Real *>(ws + L.G1), *W = reinterpret_cast<Real *>(ws + L.W);
    Real *T = reinterpret_cast<Real *>(ws + L.T);
    Real *G2 = reinterpret_cast<Real *>(ws + L.G2), *G3 = reinterpret_cast<Real *>(ws + L.G3);
    double *S = reinterpret_cast<double *>(ws + L.S), *rhs = reinterpret_cast<double *>(ws + L.rhs);
    double *x = reinterpret_cast<double *>(ws + L.x), *r = reinterpret_cast<double *>(ws + L.r);
    double *pv = reinterpret_cast<double *>(ws + L.pv), *q = reinterpret_cast<double *>(ws + L.q);
    double *Y = reinterpret_cast<double *>(ws + L.Y), *Yn = reinterpret_cast<double *>(ws + L.Yn);
    double *pn = reinterpret_cast<double *>(ws + L.pn), *an = reinterpret_cast<double *>(ws + L.an);
    double *cs = reinterpret_cast<double *>(ws + L.cs);
    Anchor *st = reinterpret_cast<Anchor *>(ws + L.st);
    int *cnt = reinterpret_cast<int *>(ws + L.cnt);   // [0] active anchors, [1] status
    ANC_TRY(cudaMemsetAsync(cnt, 0, 2 * sizeof(int), s));
    k_anc_terminal<Real><<<M, 128, 0, s>>>(p, x0, sidx, P, Y);
    ANC_TRY(cudaGetLastError());
    const dim3 cgrid((M + 127) / 128, L.nrc);
    for (int k = L.N - 1; k >= 0; --k) {
        const double t_k = k * p.dt;
        const double a = (double)k / (double)(k + 1), b = p.sigma * std::sqrt(p.dt * a);
        k_anc_step<Real><<<152 * 8, 256, 0, s>>>(p, k, sidx, a, b, P, A);
        ANC_TRY(cudaGetLastError());
        k_anc_rows<Real><<<M, 128, 0, s>>>(p, P, A, Y, pn, an, YP);
        ANC_TRY(cudaGetLastError());
        ANC_TRY((gemm<Real, false>(M, M, ld, ld, P, ld, A, ld, G1, M, s)));   // P A^T
        const double rho_ref = p.sigma * p.sigma * p.d * (t_k + (k + 1) * p.dt);
        k_anc_columns<Real><<<cgrid, 128, 0, s>>>(p, 0, rho_ref, G1, pn, an, Y, W, T, st, cs);
        ANC_TRY(cudaGetLastError());
        ANC_TRY((gemm<Real, true>(M, ld, M, L.kc, W, M, P, ld, G2, ld, s)));    // W^T P
        ANC_TRY((gemm<Real, true>(M, ld, M, L.kc, W, M, YP, ld, G3, ld, s)));   // W^T (Y P)
        k_anc_setup<Real><<<M, 256, 0, s>>>(p, L.nrc, L.nsplit, A, G2, G3, cs, st, S, rhs, x, r,
                                           pv, V);
        ANC_TRY(cudaGetLastError());
        for (int it = 0; it < p.cg_max_iter; ++it) {
            const bool check = it % kCheckEvery == kCheckEvery - 1 || it + 1 == p.cg_max_iter;
            if (check) ANC_TRY(cudaMemsetAsync(cnt, 0, sizeof(int), s));   // counts this pass
            ANC_TRY((gemm<Real, false>(M, M, ld, ld, P, ld, V, ld, G1, M, s)));   // U = P V^T
            k_anc_columns<Real><<<cgrid, 128, 0, s>>>(p, 1, 0.0, G1, pn, an, Y, W, T, st, cs);
            ANC_TRY(cudaGetLastError());
            ANC_TRY((gemm<Real, true>(M, ld, M, L.kc, T, M, P, ld, G2, ld, s)));   // T^T P
            k_anc_cg<Real><<<(M + kAncWarps - 1) / kAncWarps, 32 * kAncWarps, 0, s>>>(
                p, L.nrc, L.nsplit, A, G2, cs, S, st, x, r, pv, q, V, cnt);
            ANC_TRY(cudaGetLastError());
            if (check) {
                ANC_TRY(cudaMemcpyAsync(host_cnt, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
                ANC_TRY(cudaStreamSynchronize(s));
                if (*host_cnt == 0) break;   // every anchor converged (or failed)
            }
        }
        k_anc_newton<Real><<<M, 256, 0, s>>>(p, t_k, x0, A, S, x, st, Yn, cnt + 1);
        ANC_TRY(cudaGetLastError());
        std::swap(P, A);   // level k's rows are the cloud of level k-1
        std::swap(Y, Yn);
    }
    k_anc_output<<<1, 256, 0, s>>>(M, L.d, Y, x, u0, grad);
    ANC_TRY(cudaGetLastError());
    ANC_TRY(cudaMemcpyAsync(host_cnt, cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    ANC_TRY(cudaStreamSynchronize(s));
    if (*host_cnt && !*status) *status = *host_cnt;
    return cudaSuccess;
}

}  // namespace
}  // namespace anchored
}  // namespace fbsde

using namespace fbsde::anchored;

extern "C" {

size_t fbsde_anchored_workspace_bytes(const fbsde_problem *P)
{
    Lay L;
    return lay(P, L) ? L.total : 0;
}

int fbsde_solve_anchored(const fbsde_problem *P, int32_t Q, const double *x0, uint64_t seed,
                         uint32_t solve_index0, double *u0, double *grad_u0, void *workspace,
                         size_t workspace_bytes, fbsde_stream_t stream)
{
    Lay L;
    if (!lay(P, L) || Q < 1 || !x0 || !u0) return FBSDE_ERR_ARG;
    if ((P->kind == FBSDE_HJB_LOGQUAD || P->kind == FBSDE_AFFINE_TEST) && !P->theta)
        return FBSDE_ERR_ARG;
    if (!workspace || workspace_bytes < L.total || (reinterpret_cast<uintptr_t>(workspace) % kAl))
        return FBSDE_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    char *ws = static_cast<char *>(workspace);
    int status = FBSDE_OK, host_cnt = 0;
    for (int q = 0; q < Q; ++q) {
        const double *xq = x0 + (size_t)q * P->d;
        double *gq = grad_u0 ? grad_u0 + (size_t)q * P->d : nullptr;
        const cudaError_t e =
            P->precision == FBSDE_FP32
                ? solve_one<float>(P, L, xq, seed, solve_index0 + q, u0 + q, gq, ws, s, &status,
                                   &host_cnt)
                : solve_one<double>(P, L, xq, seed, solve_index0 + q, u0 + q, gq, ws, s, &status,
                                    &host_cnt);
        if (e != cudaSuccess) return FBSDE_ERR_CUDA;
    }
    return status;
}

}  // extern "C"
